"""f3 on the GPU: the spin-exchange and pair-hopping terms (H_nd of Eq. Ham1)
in the product, the ground state, the Green's function chains (one chain at
a time and the batched chains of small sectors), the interaction energy and
(in test_zz_no_alloc.py) the allocation-free residual, against the oracle (oracle/fock.py H_nd,
pinned by tests/test_oracle_kanamori.py).

Tolerances as in the density-density tests: FP64 products <= 1e-13 x the
elementwise bound sum_k |H_ik||v_k|, FP32 <= 4e-6 x the bound; E0 <= 1e-10
relative; G from FP64 chains <= 1e-8; the interaction energy on the same
vector <= 1e-12 (FP64 vectors) or 1e-6 (FP32 vectors, whose H_nd dot is
summed in FP32)."""
import numpy as np
import pytest
import torch

from oracle import fock, gf, lanczos, observables
from workloads import (ImpurityModel, make_model, with_exchange, workload_full_norb3_ns15,
                       workload_full_norb5_ns15, workload_full_ns18)

pytestmark = pytest.mark.gpu


def kanamori(norb, nbath, U, J, Jx, Jp, seed):
    """Spin-dependent levels and hybridisations (no spin-rotation symmetry,
    so no degenerate multiplets within a sector)."""
    b = make_model(norb, nbath, U=U, Jh=J, seed=seed)
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=norb, nbath=nbath, U=b.U, Ust=b.Ust, Jh=b.Jh,
                         e_imp=b.e_imp + r.normal(0, .2, (2, norb)),
                         e_bath=b.e_bath + r.normal(0, .2, b.e_bath.shape),
                         v_bath=b.v_bath * r.uniform(.5, 1.5, b.v_bath.shape), Jx=Jx, Jp=Jp)


CASES = {
    "norb4_ns8": (kanamori(4, 1, 2.4, 0.4, 0.35, 0.3, 41), 3, 4),      # D = 3,920
    "norb3_ns9": (kanamori(3, 2, 2.6, 0.4, 0.35, 0.3, 31), 4, 5),      # D = 15,876
    "norb2_ns10": (kanamori(2, 4, 3.0, 0.5, 0.5, 0.45, 32), 5, 4),     # D = 52,920
    "norb5_ns10": (kanamori(5, 1, 3.0, 0.5, 0.4, 0.5, 33), 5, 4),      # D = 52,920, 20 moves
    "norb3_ns12": (kanamori(3, 3, 2.5, 0.4, 0.4, 0.3, 34), 6, 5),      # D = 731,808
    "norb3_up0": (kanamori(3, 2, 2.6, 0.4, 0.35, 0.3, 35), 0, 5),      # no up electron
    "pair_only": (kanamori(3, 2, 2.6, 0.4, 0.0, 0.45, 36), 4, 4),      # J_X = 0
    "exch_only": (kanamori(3, 2, 2.6, 0.4, 0.45, 0.0, 37), 5, 4),      # J_P = 0
}


def _bound(ref, v):
    V = np.abs(v).reshape(ref.dim_dw, ref.dim_up)
    B = np.abs(ref.diagonal()) * V + (abs(ref.H_up) @ V.T).T + abs(ref.H_dw) @ V
    return B.reshape(-1) + abs(ref.H_nd) @ np.abs(v)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nd_matvec_elementwise(ed, case, prec):
    m, nup, ndw = CASES[case]
    ref = fock.Sector(m, nup, ndw)
    s = ed.Sector(m, nup, ndw)
    rng = np.random.default_rng(7)
    dt = torch.float64 if prec == "fp64" else torch.float32
    vt = torch.tensor(rng.uniform(-1, 1, ref.dim), dtype=dt, device="cuda")
    wt = torch.full_like(vt, float("nan"))
    ed.matvec(s, vt, wt, prec)
    torch.cuda.synchronize()
    v = vt.double().cpu().numpy()
    want = ref.matvec(v)
    got = wt.double().cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 4e-6
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - want) <= tol * _bound(ref, v))
    # the H_nd part is not negligible in these products
    assert np.abs(ref.H_nd @ v).max() > 0.05 or nup == 0
    s.free()


@pytest.mark.parametrize("case", ["norb3_ns9", "norb5_ns10", "norb3_ns12"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["tiled", "elementwise"])
def test_nd_block_major_product(ed, case, prec, kernel):
    """The block-major product (the Lanczos vectors' layout) with either
    product kernel pinned equals the sector-order product up to rounding."""
    m, nup, ndw = CASES[case]
    ref = fock.Sector(m, nup, ndw)
    s = ed.Sector(m, nup, ndw)
    s.set_kernel(kernel, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(3)
    v = torch.rand(s.dim, device="cuda", dtype=dt, generator=g) * 2 - 1
    vb = torch.empty(s.blocked_dim, device="cuda", dtype=dt)
    ed.permute(s, v, vb, True, prec)
    wb = torch.zeros_like(vb)
    ed.matvec_blocked(s, vb, wb, prec)
    w = torch.empty_like(v)
    ed.permute(s, wb, w, False, prec)
    # no kernel writes the padding columns: they keep their zeros
    assert int((wb != 0).sum()) <= s.dim
    vh = v.double().cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 4e-6
    assert np.all(np.abs(w.double().cpu().numpy() - ref.matvec(vh)) <= tol * _bound(ref, vh))
    s.free()


@pytest.mark.parametrize("case", ["norb4_ns8", "norb3_ns9", "norb5_ns10", "norb3_ns12",
                                  "pair_only", "exch_only"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_polish"])
def test_nd_ground_state(ed, case, prec):
    m, nup, ndw = CASES[case]
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, prec, psi=psi)
    assert abs(r["e0"] - ro["e0"]) <= 1e-10 * abs(ro["e0"])
    p = psi.cpu().numpy()
    ov = abs(float(p @ ro["psi"])) / (np.linalg.norm(p) * np.linalg.norm(ro["psi"]))
    assert ov > 1 - 1e-9
    # the polished FP32 vector keeps an FP32-size residual (E0 converges as its square)
    assert r["residual"] < (1e-8 if prec == "fp64" else 1e-5)
    s.free()


@pytest.mark.parametrize("case", ["norb4_ns8", "norb3_ns9", "norb3_ns12"])
def test_nd_gf_against_oracle(ed, case):
    """G(i w_n) of every orbital and spin from FP64 chains: through
    ed_gf_lanczos (one chain at a time) and through ed_solve (small sectors:
    the batched chains, one CTA per chain, H_nd inside the chain kernel)."""
    m, nup, ndw = CASES[case]
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    out, Gall = ed.solve(m, nup, ndw, precision="fp64", gf_precision="fp64", nmats=128,
                         beta=50.0)
    assert abs(out["e0"] - ro["e0"]) <= 1e-10 * abs(ro["e0"])
    for spin in (0, 1):
        for orb in range(m.norb):
            Go = gf.impurity_gf(m, nup, ndw, ro["psi"], ro["e0"], orb, spin, beta=50.0, nmats=128)
            G, _ = ed.gf_lanczos(s, psi, r["e0"], orb, spin, "fp64", beta=50.0, nmats=128)
            assert np.abs(G - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max()), (orb, spin)
            Gs = Gall[spin, orb]
            assert np.abs(Gs - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max()), (orb, spin)
    s.free()


@pytest.mark.parametrize("case", ["norb3_ns9", "norb5_ns10"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nd_interaction_energy(ed, case, prec):
    m, nup, ndw = CASES[case]
    s = ed.Sector(m, nup, ndw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    psi = torch.empty(s.dim, dtype=dt, device="cuda")
    ed.lanczos_ground(s, prec, psi=psi)
    ob = ed.observables(s, psi, prec)
    p = psi.double().cpu().numpy()
    dens, nn, e_int = observables.local_observables(m, nup, ndw, p)
    assert np.abs(ob["dens"] - dens).max() <= 1e-12
    # FP32 vectors: <psi|H_nd|psi> is summed in FP32 (coefficients rounded to
    # FP32, at most Norb^2 terms per element) before the FP64 partials
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(ob["e_int"] - e_int) <= tol * max(1.0, abs(e_int))
    ref = fock.get_sector(m, nup, ndw)
    e_nd = float(p @ (ref.H_nd @ p)) / float(p @ p)
    assert abs(e_nd) > 1e-3
    s.free()


def _row_reference(m, map_up, map_dw, ref_lite, vf, r, c):
    """(H v) at (r, c) from the oracle: the factorised part entry by entry
    (Eq. Hbuild) plus the H_nd terms of the state (fock.nondiagonal_row)."""
    d = ref_lite.E_up[c] + ref_lite.E_dw[r] + ref_lite.W[ref_lite.m_up[c], ref_lite.m_dw[r]]
    acc = d * vf(r, c)
    hu, hd = ref_lite.H_up, ref_lite.H_dw
    for k in range(hu.indptr[c], hu.indptr[c + 1]):
        acc += hu.data[k] * vf(r, hu.indices[k])
    for k in range(hd.indptr[r], hd.indptr[r + 1]):
        acc += hd.data[k] * vf(hd.indices[k], c)
    for el, Ju, Jd in fock.nondiagonal_row(m, int(map_up[c]), int(map_dw[r])):
        acc += el * vf(int(np.searchsorted(map_dw, Jd)), int(np.searchsorted(map_up, Ju)))
    return acc


@pytest.mark.parametrize("maker", [workload_full_norb3_ns15, workload_full_norb5_ns15,
                                   workload_full_ns18])
def test_nd_full_size_sampled(ed, maker):
    """The FP32 product with H_nd at the full sizes (Ns = 15 three and five
    orbitals, Ns = 18), on sampled outputs; the input is a closed-form
    function of the index so that the oracle can evaluate any entry."""
    wl = maker(0)
    m = wl.model
    s = ed.Sector(m, wl.nup, wl.ndw)
    dup, ddw, n = s.dim_up, s.dim_dw, s.dim
    v = torch.empty(n, device="cuda", dtype=torch.float32)
    step = 1 << 27
    for o in range(0, n, step):
        idx = torch.arange(o, min(n, o + step), device="cuda", dtype=torch.float64)
        v[o:o + len(idx)] = (torch.sin(0.37 * idx) + torch.cos(0.011 * idx)).float()
    del idx
    w = torch.empty_like(v)
    ed.matvec(s, v, w, "fp32")
    torch.cuda.synchronize()

    class Lite:
        pass
    L = Lite()
    L.map_up = fock.build_sector_map(m.ns, wl.nup)
    L.map_dw = fock.build_sector_map(m.ns, wl.ndw)
    L.H_up = fock.spin_hopping_matrix(m, 0, wl.nup, L.map_up)
    L.H_dw = fock.spin_hopping_matrix(m, 1, wl.ndw, L.map_dw)
    L.E_up, L.m_up = fock.spin_diagonal(m, 0, wl.nup, L.map_up)
    L.E_dw, L.m_dw = fock.spin_diagonal(m, 1, wl.ndw, L.map_dw)
    L.W = fock.interaction_table(m)

    def vf(r, c):
        i = int(r) * int(dup) + int(c)
        return float(np.float32(np.sin(0.37 * i) + np.cos(0.011 * i)))
    rng = np.random.default_rng(6)
    rows = np.concatenate([[0, ddw - 1, ddw // 2], rng.integers(0, ddw, 60)])
    cols = np.concatenate([[0, dup - 1, dup // 3], rng.integers(0, dup, 60)])
    want = np.array([_row_reference(m, L.map_up, L.map_dw, L, vf, r, c)
                     for r, c in zip(rows, cols)])
    n_nd = sum(len(fock.nondiagonal_row(m, int(L.map_up[c]), int(L.map_dw[r])))
               for r, c in zip(rows, cols))
    assert n_nd > 20                                  # the samples exercise H_nd
    flat = torch.tensor(rows.astype(np.int64) * dup + cols.astype(np.int64), device="cuda")
    got = w[flat].double().cpu().numpy()
    assert np.abs(got - want).max() <= 2e-5 * max(1.0, np.abs(want).max())
    s.free()
