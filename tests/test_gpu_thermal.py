"""f2 on the GPU: several low-lying states (ed_lanczos_states, shift-deflated
Lanczos), the annealing truncation (ed_espace_truncate) and the
finite-temperature Green's function (ed_gf_thermal_z), against the oracle
(oracle/thermal.py, pinned by tests/test_oracle_thermal.py).

Tolerances: energies <= 1e-10 relative (FP64 and FP32 + polish); states
orthonormal and spanning the oracle's eigenvectors to 1e-6 (an FP64 Lanczos
vector at tolerance 1e-12 carries a residual of order 1e-7), 1e-4 after the
FP32 + polish path; weights equal to 1e-15;
thermal G <= 1e-8 against the exact Lehmann sum."""
import numpy as np
import pytest
import torch

from oracle import fock, thermal
from workloads import ImpurityModel, make_model, workload_ns8

pytestmark = pytest.mark.gpu


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape),
                         Jx=model.Jx, Jp=model.Jp)


CASES = {
    "ns8": (workload_ns8().model, 4, 4, 6),
    "norb2_ns8_asym": (_asym(make_model(2, 3, U=2.4, Jh=0.4, seed=71), 71), 4, 3, 6),
    "norb2_ns10_asym": (_asym(make_model(2, 4, U=3.0, Jh=0.5, seed=72), 72), 5, 4, 5),
}


def _check_states(E, psis, Eo, Vo, tol_e, tol_v=1e-6):
    assert np.abs(E - Eo).max() <= tol_e * max(1.0, np.abs(Eo).max())
    P = psis.double().cpu().numpy().T                 # D x k
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < tol_v
    # the GPU states span the oracle's eigenvectors (degenerate sets included)
    assert np.abs(Vo @ (Vo.T @ P) - P).max() < tol_v


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32_polish"])
def test_lowest_states_against_oracle(ed, case, prec):
    m, nup, ndw, k = CASES[case]
    fock._SECTOR_CACHE.clear()
    Eo, Vo = thermal.lowest_states(m, nup, ndw, k + 2, dense_below=0)
    s = ed.Sector(m, nup, ndw)
    psis = torch.empty((k, s.dim), dtype=torch.float64, device="cuda")
    E, res = ed.lanczos_states(s, k, prec, psis=psis)
    # FP32 + polish: a few FP64 steps converge the energy (error ~ residual^2)
    # but leave the vector an error of order residual / gap
    _check_states(E, psis, Eo[:k], Vo[:, :k + 2], 1e-10, 1e-6 if prec == "fp64" else 1e-4)
    assert all(r["residual"] < (1e-6 if prec == "fp64" else 1e-5) for r in res)
    s.free()


def test_degenerate_kanamori_atom_states(ed):
    """Two-orbital Kanamori atom with one bath level per orbital, sector
    (2, 2): orbital-symmetric, so several levels are degenerate; all
    states of the lowest 10 with their multiplicities."""
    b = make_model(2, 1, U=3.0, Jh=0.5, seed=73)
    m = ImpurityModel(norb=2, nbath=1, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=b.e_imp,
                      e_bath=np.full((2, 2, 1), 0.3), v_bath=np.full((2, 2, 1), 0.4),
                      Jx=0.5, Jp=0.5)
    fock._SECTOR_CACHE.clear()
    Ed, Vd = np.linalg.eigh(fock.Sector(m, 2, 2).hamiltonian().toarray())
    assert np.min(np.diff(Ed[:10])) < 1e-9          # the case has degenerate levels
    s = ed.Sector(m, 2, 2)
    psis = torch.empty((10, s.dim), dtype=torch.float64, device="cuda")
    E, _ = ed.lanczos_states(s, 10, "fp64", psis=psis)
    # the degenerate set at the 10th level may be cut: compare with all
    # eigenvectors whose energy is within the found range
    top = np.searchsorted(Ed, E.max() + 1e-8)
    _check_states(np.sort(E), psis, Ed[:10], Vd[:, :top], 1e-10)
    s.free()


def test_espace_truncate_matches_oracle(ed):
    rng = np.random.default_rng(9)
    Es = [np.sort(rng.uniform(0, 3, n)) for n in (5, 3, 7, 1)]
    for beta, cutoff, ntotal, step in [(2.0, 1e-3, 0, 2), (10.0, 1e-9, 6, 3), (0.5, 0.0, 0, 1)]:
        w, nxt, nk = ed.espace_truncate(Es, beta, cutoff, ntotal, step)
        wo, nxo = thermal.espace_truncate(Es, beta, cutoff, ntotal or (1 << 30), step)
        for a, b in zip(w, wo):
            assert np.abs(a - b).max() < 1e-15
        assert nxt == nxo
        assert nk == sum(int(np.count_nonzero(x)) for x in wo)


def test_thermal_gf_against_lehmann_sum(ed):
    """All states of four small sectors (every state from the deflated
    solver) against the exact finite-T Lehmann sum."""
    m = _asym(make_model(1, 3, U=2.2, e_d=-0.9, seed=3), 3)
    fock._SECTOR_CACHE.clear()
    sectors = [(2, 2), (2, 1), (1, 2), (3, 2)]
    z = np.concatenate([1j * (2 * np.arange(40) + 1) * np.pi / 8.0, np.linspace(-5, 5, 41) + 0.2j])
    secs, psis, energies, keep = [], [], [], []
    for nu, nd in sectors:
        s = ed.Sector(m, nu, nd)
        p = torch.empty((s.dim, s.dim), dtype=torch.float64, device="cuda")
        E, _ = ed.lanczos_states(s, s.dim, "fp64", psis=p)
        for i in range(s.dim):
            secs.append(s)
            psis.append(p[i])
            energies.append(E[i])
        keep.append((s, p))
    for beta in (0.7, 3.0):
        G, w = ed.gf_thermal_z(secs, psis, energies, beta, 0.0, 0, 0, z, "fp64", nsteps=64)
        Gx = thermal.lehmann_thermal_z(m, sectors, beta, 0, 0, z)
        assert np.abs(G - Gx).max() < 1e-8
        assert abs(w.sum() - 1.0) < 1e-14
    for s, _ in keep:
        s.free()


def test_thermal_gf_truncated_against_oracle(ed):
    """Five states per sector of three Ns = 8 sectors, beta = 4 with the
    truncation, against the oracle's ARPACK states and chains."""
    m = CASES["norb2_ns8_asym"][0]
    fock._SECTOR_CACHE.clear()
    sectors = [(4, 3), (3, 4), (4, 4)]
    z = 1j * (2 * np.arange(64) + 1) * np.pi / 4.0
    secs, psis, energies, orc = [], [], [], []
    for nu, nd in sectors:
        s = ed.Sector(m, nu, nd)
        p = torch.empty((5, s.dim), dtype=torch.float64, device="cuda")
        E, _ = ed.lanczos_states(s, 5, "fp64", psis=p)
        Eo, Vo = thermal.lowest_states(m, nu, nd, 5, dense_below=0)
        for i in range(5):
            secs.append(s)
            psis.append(p[i])
            energies.append(E[i])
            orc.append((nu, nd, Vo[:, i], Eo[i]))
    G, w = ed.gf_thermal_z(secs, psis, energies, 4.0, 1e-6, 0, 0, z, "fp64", nsteps=200)
    wo, _ = thermal.espace_truncate([np.array([e for (a, b, _, e) in orc if (a, b) == sec])
                                     for sec in sectors], 4.0, 1e-6)
    wflat = np.concatenate(wo)
    assert np.abs(w - wflat).max() < 1e-9
    states = [(wflat[i],) + orc[i][:2] + (orc[i][2], orc[i][3]) for i in range(len(orc))]
    Go = thermal.thermal_gf_z(m, states, 0, 0, z, nsteps=200)
    assert np.abs(G - Go).max() < 1e-8
    for s in set(secs):
        s.free()
