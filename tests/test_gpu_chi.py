"""f1 susceptibilities on the GPU (ed_chi_z): spin, charge and s-wave pair
functions against the oracle (oracle/chi.py, pinned by
tests/test_oracle_chi.py): the same two-chain algorithm, FP64 <= 1e-8 on the
Matsubara axis and the real axis at eta = 0.5; FP32 chains on the polished
state <= 1e-5 (relative); the empty-atom pair function 1/(z - (2e + U));
inter-orbital spin and charge functions (ed_chi_ab_z) against the oracle's
auxiliary-operator construction, C_aa = ed_chi_z, C_ab = C_ba, and C_ab = 0
at U = 0 with each orbital on its own bath; the excitonic function against
the oracle (FP64 1e-8, FP32 + polish 1e-5) and, at U = 0, against the closed
form from the one-body eigenvectors; C(tau) in imaginary time (ed_chi_tau)
against the oracle's poles-and-weights evaluation (FP64 1e-8, FP32 + polish
1e-5, relative) and C(tau) = C(beta - tau) for spin and charge."""
import numpy as np
import pytest
import torch

from oracle import chi, fock, lanczos
from workloads import ImpurityModel, make_model, with_exchange

pytestmark = pytest.mark.gpu


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape),
                         Jx=model.Jx, Jp=model.Jp)


CASES = {
    "norb1_ns8": (_asym(make_model(1, 7, U=2.0, e_d=-1.0, seed=51), 51), 4, 4),
    "norb2_ns8": (_asym(make_model(2, 3, U=2.5, Jh=0.4, seed=52), 52), 4, 3),
    "norb2_ns10": (_asym(make_model(2, 4, U=3.0, Jh=0.5, seed=53), 53), 5, 5),
    "kanamori_ns9": (_asym(with_exchange(make_model(3, 2, U=2.6, Jh=0.4, seed=54)), 54), 4, 5),
}
Z = np.concatenate([1j * 2 * np.pi * np.arange(1, 40) / 20.0, np.linspace(-6, 6, 61) + 0.5j])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kind", chi.KINDS)
def test_chi_against_oracle(ed, case, kind):
    m, nup, ndw = CASES[case]
    fock._SECTOR_CACHE.clear()
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    for orb in range(m.norb):
        Co, parts = chi.chi_z(m, nup, ndw, ro["psi"], ro["e0"], kind, orb, Z, nsteps=150,
                              return_parts=True)
        C, w = ed.chi_z(s, psi, r["e0"], kind, orb, Z, "fp64", nsteps=150)
        assert np.abs(C - Co).max() <= 1e-8 * max(1.0, np.abs(Co).max()), (orb, kind)
        assert abs(w[0] - parts.get(1, 0.0)) < 1e-10 and abs(w[1] - parts.get(-1, 0.0)) < 1e-10
    # FP32 chains from the polished state
    psi2 = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r2 = ed.lanczos_ground(s, "fp32_polish", psi=psi2)
    Co = chi.chi_z(m, nup, ndw, ro["psi"], ro["e0"], kind, 0, Z, nsteps=150)
    C2, _ = ed.chi_z(s, psi2, r2["e0"], kind, 0, Z, "fp32_polish", nsteps=150)
    assert np.abs(C2 - Co).max() <= 1e-5 * max(1.0, np.abs(Co).max())
    s.free()


def test_pair_function_of_the_empty_atom(ed):
    e, U = 0.7, 1.3
    m = ImpurityModel(norb=1, nbath=0, U=U, Ust=U, Jh=0.0, e_imp=np.array([e]),
                      e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))
    s = ed.Sector(m, 0, 0)
    psi = torch.ones(1, dtype=torch.float64, device="cuda")
    C, w = ed.chi_z(s, psi, 0.0, "pair", 0, Z, "fp64", nsteps=4)
    assert np.abs(C - 1.0 / (Z - (2 * e + U))).max() < 1e-14
    assert w == (1.0, 0.0)
    s.free()


@pytest.mark.parametrize("case", ["norb2_ns8", "norb2_ns10", "kanamori_ns9"])
@pytest.mark.parametrize("kind", ("spin", "charge"))
def test_inter_orbital_chi_against_oracle(ed, case, kind):
    m, nup, ndw = CASES[case]
    fock._SECTOR_CACHE.clear()
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    Co = chi.chi_ab_z(m, nup, ndw, ro["psi"], ro["e0"], kind, 0, 1, Z, nsteps=150)
    C01 = ed.chi_ab_z(s, psi, r["e0"], kind, 0, 1, Z, "fp64", nsteps=150)
    C10 = ed.chi_ab_z(s, psi, r["e0"], kind, 1, 0, Z, "fp64", nsteps=150)
    scale = max(1.0, np.abs(Co).max())
    assert np.abs(C01 - Co).max() <= 1e-8 * scale
    assert np.abs(C01 - C10).max() <= 1e-10 * scale
    C11 = ed.chi_ab_z(s, psi, r["e0"], kind, 1, 1, Z, "fp64", nsteps=150)
    C1, _ = ed.chi_z(s, psi, r["e0"], kind, 1, Z, "fp64", nsteps=150)
    assert np.abs(C11 - C1).max() <= 1e-10 * max(1.0, np.abs(C1).max())
    # FP32 chains from the polished state
    psi2 = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r2 = ed.lanczos_ground(s, "fp32_polish", psi=psi2)
    C2 = ed.chi_ab_z(s, psi2, r2["e0"], kind, 0, 1, Z, "fp32_polish", nsteps=150)
    assert np.abs(C2 - Co).max() <= 1e-5 * scale
    with pytest.raises(ed.EDError):
        ed.chi_ab_z(s, psi, r["e0"], "pair", 0, 1, Z, "fp64")
    s.free()


@pytest.mark.parametrize("kind", ("spin", "charge"))
def test_inter_orbital_chi_vanishes_at_u0(ed, kind):
    b = make_model(2, 3, U=0.0, Jh=0.0, seed=45)
    m = _asym(ImpurityModel(norb=2, nbath=3, U=0.0, Ust=0.0, Jh=0.0, e_imp=b.e_imp,
                            e_bath=b.e_bath, v_bath=b.v_bath), 45)
    s = ed.Sector(m, 4, 3)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    C01 = ed.chi_ab_z(s, psi, r["e0"], kind, 0, 1, Z, "fp64", nsteps=200)
    C0, _ = ed.chi_z(s, psi, r["e0"], kind, 0, Z, "fp64", nsteps=200)
    assert np.abs(C0).max() > 1e-2
    assert np.abs(C01).max() < 1e-8
    s.free()


@pytest.mark.parametrize("case", ["norb3_ns9", "kanamori_ns9"])
@pytest.mark.parametrize("pair", [(0, 2), (1, 2)])
def test_exciton_chi_against_oracle(ed, case, pair):
    a, b = pair
    if case == "norb3_ns9":
        m, nup, ndw = _asym(make_model(3, 2, U=2.3, Jh=0.35, seed=55), 55), 5, 4
    else:
        m, nup, ndw = CASES[case]
    fock._SECTOR_CACHE.clear()
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    Co = chi.chi_exciton_z(m, nup, ndw, ro["psi"], ro["e0"], a, b, Z, nsteps=150)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    C = ed.chi_ab_z(s, psi, r["e0"], "exciton", a, b, Z, "fp64", nsteps=150)
    scale = max(1.0, np.abs(Co).max())
    assert np.abs(Co).max() > 1e-3
    assert np.abs(C - Co).max() <= 1e-8 * scale
    Cba = ed.chi_ab_z(s, psi, r["e0"], "exciton", b, a, Z, "fp64", nsteps=150)
    assert np.abs(Cba - C).max() <= 1e-10 * scale       # the same operator
    psi2 = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r2 = ed.lanczos_ground(s, "fp32_polish", psi=psi2)
    C2 = ed.chi_ab_z(s, psi2, r2["e0"], "exciton", a, b, Z, "fp32_polish", nsteps=150)
    assert np.abs(C2 - Co).max() <= 1e-5 * scale
    with pytest.raises(ed.EDError):
        ed.chi_ab_z(s, psi, r["e0"], "exciton", a, a, Z, "fp64")
    s.free()


def test_exciton_chi_u0_closed_form(ed):
    base = make_model(3, 2, U=0.0, Jh=0.0, seed=47)
    m = _asym(ImpurityModel(norb=3, nbath=2, U=0.0, Ust=0.0, Jh=0.0, e_imp=base.e_imp,
                            e_bath=base.e_bath, v_bath=base.v_bath), 47)
    nup, ndw, a, b = 4, 5, 0, 2
    want = np.zeros(Z.shape, dtype=np.complex128)
    for spin, n in ((0, nup), (1, ndw)):
        h = np.diag(fock.level_energies(m, spin))
        for o in range(3):
            for nu in range(2):
                i, j = fock.level_of_impurity(m, o), fock.level_of_bath(m, o, nu)
                h[i, j] = h[j, i] = m.v_bath[spin, o, nu]
        e, U = np.linalg.eigh(h)
        op = np.zeros_like(h)
        op[a, b] = op[b, a] = 1.0
        M = U.T @ op @ U
        for k in range(n):
            for l in range(n, len(e)):
                d = e[l] - e[k]
                want += M[l, k] ** 2 * (1 / (Z - d) - 1 / (Z + d))
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    C = ed.chi_ab_z(s, psi, r["e0"], "exciton", a, b, Z, "fp64", nsteps=300)
    assert np.abs(C - want).max() <= 1e-8 * max(1.0, np.abs(want).max())
    s.free()


@pytest.mark.parametrize("case", ["norb2_ns8", "kanamori_ns9"])
@pytest.mark.parametrize("kind", chi.KINDS)
def test_chi_tau_against_oracle(ed, case, kind):
    m, nup, ndw = CASES[case]
    beta = 30.0
    tau = np.linspace(0.0, beta, 301)
    fock._SECTOR_CACHE.clear()
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    Co = chi.chi_tau(m, nup, ndw, ro["psi"], ro["e0"], kind, 0, tau, beta, nsteps=120)
    s = ed.Sector(m, nup, ndw)
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(s, "fp64", psi=psi)
    C = ed.chi_tau(s, psi, r["e0"], kind, 0, tau, beta, "fp64", nsteps=120)
    scale = max(1.0, np.abs(Co).max())
    assert np.abs(C - Co).max() <= 1e-8 * scale
    if kind != "pair":
        assert np.abs(C - C[::-1]).max() <= 1e-10 * scale
    psi2 = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    r2 = ed.lanczos_ground(s, "fp32_polish", psi=psi2)
    C2 = ed.chi_tau(s, psi2, r2["e0"], kind, 0, tau, beta, "fp32_polish", nsteps=120)
    assert np.abs(C2 - Co).max() <= 1e-5 * scale
    with pytest.raises(ed.EDError):
        ed.chi_tau(s, psi, r["e0"], kind, 0, np.array([beta + 1.0]), beta, "fp64")
    s.free()
