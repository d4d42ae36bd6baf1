"""f4 on the GPU: the electron-phonon (Holstein) extension of Sec. 4 through
ed_eph_matvec / ed_eph_lanczos_ground / ed_eph_gf_lanczos_z, against the
oracle (oracle/eph.py, pinned by tests/test_oracle_eph.py) and the closed
forms of the atomic limit.

Tolerances: products FP64 <= 1e-13 and FP32 <= 4e-6 times the elementwise
bound sum_k |H_ik| |v_k|; E0 <= 1e-10 relative (FP64 and FP32 + polish); G
from FP64 chains <= 1e-8."""
import math

import numpy as np
import pytest
import torch

from oracle import eph, fock, lanczos
from workloads import ImpurityModel, make_model, workload_eph_ns12

pytestmark = pytest.mark.gpu


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


CASES = {
    "norb1_ns6": (make_model(1, 5, U=2.0, e_d=-1.0, seed=91), 3, 3, 0.6, [0.4], 6),
    "norb2_ns8": (_asym(make_model(2, 3, U=2.5, Jh=0.4, seed=92), 92), 4, 3, 0.7, [0.3, 0.5], 4),
    "norb3_ns9": (_asym(make_model(3, 2, U=2.2, Jh=0.3, seed=93), 93), 4, 5, 0.5,
                  [0.2, 0.3, 0.25], 3),
    "nph0": (make_model(2, 3, U=2.5, Jh=0.4, seed=94), 4, 4, 0.6, [0.3, 0.3], 0),
}


def _phonons(case):
    m, nup, ndw, w0, g, nph = CASES[case]
    return m, nup, ndw, eph.Phonon(w0=w0, g=np.array(g), nph=nph)


def _bound(m, ph, nup, ndw, v):
    """Elementwise sum_k |H_ik| |v_k| of the coupled product."""
    el = fock.get_sector(m, nup, ndw)
    A = np.abs(v).reshape(ph.dph, el.dim)
    out = np.empty_like(A)
    ng = np.abs(eph.coupling_diagonal(m, ph, nup, ndw))
    for p in range(ph.dph):
        V = A[p].reshape(el.dim_dw, el.dim_up)
        B = np.abs(el.diagonal()) * V + (abs(el.H_up) @ V.T).T + abs(el.H_dw) @ V
        out[p] = B.reshape(-1) + abs(ph.w0) * p * A[p]
        if p > 0:
            out[p] += ng * math.sqrt(p) * A[p - 1]
        if p < ph.nph:
            out[p] += ng * math.sqrt(p + 1) * A[p + 1]
    return out.reshape(-1)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eph_matvec_elementwise(ed, case, prec):
    m, nup, ndw, ph = _phonons(case)
    s = ed.Sector(m, nup, ndw)
    ref = eph.Sector(m, ph, nup, ndw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(11)
    vt = torch.tensor(rng.uniform(-1, 1, ref.dim), dtype=dt, device="cuda")
    wt = torch.full_like(vt, float("nan"))
    ed.eph_matvec(s, ed.phonon(ph.w0, ph.g, ph.nph), vt, wt, prec)
    torch.cuda.synchronize()
    v = vt.double().cpu().numpy()
    got = wt.double().cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 4e-6
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref.matvec(v)) <= tol * _bound(m, ph, nup, ndw, v))
    s.free()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32_polish"])
def test_eph_ground_state(ed, case, prec):
    m, nup, ndw, ph = _phonons(case)
    ref = eph.Sector(m, ph, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(ref.dim, dtype=torch.float64, device="cuda")
    r = ed.eph_lanczos_ground(s, ed.phonon(ph.w0, ph.g, ph.nph), prec, psi=psi)
    assert abs(r["e0"] - ro["e0"]) <= 1e-10 * abs(ro["e0"])
    p = psi.cpu().numpy()
    assert abs(abs(float(p @ ro["psi"])) - 1.0) < 1e-9
    assert r["residual"] < (1e-8 if prec == "fp64" else 1e-5)
    s.free()


@pytest.mark.parametrize("n", [(1, 0), (1, 1)])
def test_eph_polaron_levels(ed, n):
    """One level, no bath: the lowest coupled energy is the displaced
    oscillator's e n + U n_up n_dw - g^2 n^2 / w0."""
    U, e, w0, g = 1.7, -0.4, 0.8, 0.5
    m = ImpurityModel(norb=1, nbath=0, U=U, Ust=U, Jh=0.0, e_imp=np.array([e]),
                      e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))
    nup, ndw = n
    s = ed.Sector(m, nup, ndw)
    r = ed.eph_lanczos_ground(s, ed.phonon(w0, [g], 40), "fp64")
    ne = nup + ndw
    assert abs(r["e0"] - (e * ne + U * nup * ndw - g * g * ne * ne / w0)) < 1e-10
    s.free()


def test_eph_franck_condon_gf(ed):
    e, w0, g = 0.9, 0.6, 0.45
    m = ImpurityModel(norb=1, nbath=0, U=2.0, Ust=2.0, Jh=0.0, e_imp=np.array([e]),
                      e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))
    ph = ed.phonon(w0, [g], 30)
    s = ed.Sector(m, 0, 0)
    psi = torch.empty(31, dtype=torch.float64, device="cuda")
    r = ed.eph_lanczos_ground(s, ph, "fp64", psi=psi)
    z = np.concatenate([1j * (2 * np.arange(64) + 1) * np.pi / 20.0,
                        np.linspace(-2, 4, 50) + 0.1j])
    G, info = ed.eph_gf_lanczos_z(s, ph, psi, r["e0"], 0, 0, z, "fp64", nsteps=31)
    lam = (g / w0) ** 2
    want = sum(math.exp(-lam) * lam ** k / math.factorial(k) / (z - (e - g * g / w0 + k * w0))
               for k in range(31))
    assert np.abs(G - want).max() < 1e-10
    assert info["weight_hole"] == 0.0 and abs(info["weight_particle"] - 1.0) < 1e-12
    s.free()


@pytest.mark.parametrize("case", ["norb1_ns6", "norb2_ns8", "norb3_ns9"])
def test_eph_gf_against_oracle(ed, case):
    m, nup, ndw, ph = _phonons(case)
    ref = eph.Sector(m, ph, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(ref.dim, dtype=torch.float64, device="cuda")
    pp = ed.phonon(ph.w0, ph.g, ph.nph)
    r = ed.eph_lanczos_ground(s, pp, "fp64", psi=psi)
    # Matsubara axis and the real axis at eta = 0.5: closer to the axis the two
    # implementations' chains differ in their rounding-dependent part (after
    # orthogonality is lost), by 2e-8 at eta = 0.3 here
    z = np.concatenate([1j * (2 * np.arange(64) + 1) * np.pi / 50.0,
                        np.linspace(-6, 6, 121) + 0.5j])
    for spin in (0, 1):
        for orb in range(m.norb):
            Go = eph.impurity_gf_z(m, ph, nup, ndw, ro["psi"], ro["e0"], orb, spin, z,
                                   nsteps=120)
            G, _ = ed.eph_gf_lanczos_z(s, pp, psi, r["e0"], orb, spin, z, "fp64", nsteps=120)
            assert np.abs(G - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max()), (orb, spin)
    # FP32 chains from the polished state
    psi2 = torch.empty(ref.dim, dtype=torch.float64, device="cuda")
    r2 = ed.eph_lanczos_ground(s, pp, "fp32_polish", psi=psi2)
    Go = eph.impurity_gf_z(m, ph, nup, ndw, ro["psi"], ro["e0"], 0, 0, z, nsteps=120)
    G2, _ = ed.eph_gf_lanczos_z(s, pp, psi2, r2["e0"], 0, 0, z, "fp32_polish", nsteps=120)
    assert np.abs(G2 - Go).max() <= 1e-5
    s.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eph_full_size_product(ed, prec):
    """The product at the phonon benchmark's size (Ns = 12, (6,6), N_ph = 10,
    D = 9,391,536) element by element against the oracle's slice product."""
    wl = workload_eph_ns12(0, 10)
    m, x = wl.model, wl.extra
    ph = eph.Phonon(w0=x["w0"], g=np.array(x["g"]), nph=x["nph"])
    s = ed.Sector(m, wl.nup, wl.ndw)
    ref = eph.Sector(m, ph, wl.nup, wl.ndw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(5)
    vt = (torch.rand(ref.dim, dtype=torch.float64, device="cuda", generator=g) - 0.5).to(dt)
    wt = torch.empty_like(vt)
    ed.eph_matvec(s, ed.phonon(ph.w0, ph.g, ph.nph), vt, wt, prec)
    torch.cuda.synchronize()
    v = vt.double().cpu().numpy()
    got = wt.double().cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 4e-6
    assert np.all(np.abs(got - ref.matvec(v)) <= tol * _bound(m, ph, wl.nup, wl.ndw, v))
    s.free()
