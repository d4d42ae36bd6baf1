"""Pins of the susceptibility oracle (oracle/chi.py), no GPU.

* chains = the exact Lehmann sum of Eq. KLgf with the bosonic sign (every
  kind, chains long enough to be exact);
* U = 0 closed forms from the one-body eigenvectors (an independent route:
  the ground state is a Slater determinant per spin):
  - spin / charge: sum_sigma c_sigma^2 sum_{k occ, l empty} (u_l u_k)^2
    [1/(z - (e_l - e_k)) - 1/(z + (e_l - e_k))], c = (1/2, -1/2) or (1, 1);
  - pair: sum_{l, m empty} (u_l u_m)^2 / (z - (e_l + e_m))
    - sum_{k, q occ} (u_k u_q)^2 / (z - (e_k + e_q));
* the atom: an empty level e with interaction U has the pair function
  1 / (z - (2e + U));
* C(i nu) of a hermitian operator is real, even in nu and negative;
* inter-orbital C_ab (spin, charge) from the chains of O_a + O_b, O_a, O_b
  = the exact off-diagonal Lehmann sum; C_ab = C_ba; C_aa = the one-orbital
  function; C_ab = 0 at U = 0 with each orbital on its own bath (the
  particle-hole excitations of the two orbitals never mix), while each
  orbital's own function does not vanish;
* excitonic function (singlet inter-orbital particle-hole operator) = the
  exact Lehmann sum, and at U = 0 = the closed form from the one-body
  eigenvectors (Wick: sum over particle-hole pairs of |<l|o|k>|^2, o the
  one-body matrix of the operator), for a pair with a level between them
  (the fermionic sign matters) and an adjacent pair;
* imaginary time: C(tau) from the chains' poles and weights = the exact
  Lehmann sum in tau; its bosonic Fourier transform = -C(i nu_n) of chi_z (an
  independent route: the continued fraction); C(tau) = C(beta - tau) for the
  hermitian spin and charge operators.
"""
import numpy as np
import pytest

from oracle import chi, fock, lanczos
from workloads import ImpurityModel, make_model


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


Z = np.concatenate([1j * 2 * np.pi * np.arange(1, 30) / 10.0, np.linspace(-4, 4, 33) + 0.25j])


@pytest.mark.parametrize("kind", chi.KINDS)
def test_chains_equal_lehmann_sum(kind):
    m = _asym(make_model(2, 1, U=2.4, Jh=0.4, seed=41), 41)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 2, 1)
    r = lanczos.ground_state(s.matvec, s.dim)
    for orb in range(2):
        C = chi.chi_z(m, 2, 1, r["psi"], r["e0"], kind, orb, Z, nsteps=64)
        Cx, e0 = chi.lehmann_chi_z(m, 2, 1, kind, orb, Z)
        assert abs(e0 - r["e0"]) < 1e-12
        assert np.abs(C - Cx).max() < 1e-10, (kind, orb)


def _one_body(m, spin):
    h = np.diag(fock.level_energies(m, spin))
    for a in range(m.norb):
        for nu in range(m.nbath):
            i, j = fock.level_of_impurity(m, a), fock.level_of_bath(m, a, nu)
            h[i, j] = h[j, i] = m.v_bath[spin, a, nu]
    return np.linalg.eigh(h)


@pytest.mark.parametrize("kind", chi.KINDS)
def test_u0_closed_forms(kind):
    b = make_model(1, 5, U=0.0, Jh=0.0, e_d=0.1, seed=42)
    m = _asym(ImpurityModel(norb=1, nbath=5, U=0.0, Ust=0.0, Jh=0.0, e_imp=b.e_imp,
                            e_bath=b.e_bath, v_bath=b.v_bath), 42)
    nup, ndw = 3, 2
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    C = chi.chi_z(m, nup, ndw, r["psi"], r["e0"], kind, 0, Z, nsteps=300)
    (eu, Uu), (ed, Ud) = _one_body(m, 0), _one_body(m, 1)
    uu, ud = Uu[0, :], Ud[0, :]
    want = np.zeros(Z.shape, dtype=np.complex128)
    if kind in ("spin", "charge"):
        cs = (0.5, -0.5) if kind == "spin" else (1.0, 1.0)
        for c, e, u, n in ((cs[0], eu, uu, nup), (cs[1], ed, ud, ndw)):
            for k in range(n):
                for l in range(n, len(e)):
                    d = e[l] - e[k]
                    want += c * c * (u[l] * u[k]) ** 2 * (1 / (Z - d) - 1 / (Z + d))
    else:
        for l in range(nup, len(eu)):
            for q in range(ndw, len(ed)):
                want += (uu[l] * ud[q]) ** 2 / (Z - (eu[l] + ed[q]))
        for k in range(nup):
            for q in range(ndw):
                want -= (uu[k] * ud[q]) ** 2 / (Z - (eu[k] + ed[q]))
    assert np.abs(C - want).max() < 1e-9


def test_pair_function_of_the_empty_atom():
    e, U = 0.7, 1.3
    m = ImpurityModel(norb=1, nbath=0, U=U, Ust=U, Jh=0.0, e_imp=np.array([e]),
                      e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))
    fock._SECTOR_CACHE.clear()
    C = chi.chi_z(m, 0, 0, np.array([1.0]), 0.0, "pair", 0, Z, nsteps=4)
    assert np.abs(C - 1.0 / (Z - (2 * e + U))).max() < 1e-14


@pytest.mark.parametrize("kind", ("spin", "charge"))
def test_hermitian_functions_real_even_negative(kind):
    m = _asym(make_model(1, 5, U=2.0, e_d=-1.0, seed=43), 43)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 3)
    r = lanczos.ground_state(s.matvec, s.dim)
    nu = 2 * np.pi * np.arange(1, 20) / 10.0
    Cp = chi.chi_z(m, 3, 3, r["psi"], r["e0"], kind, 0, 1j * nu, nsteps=200)
    Cm = chi.chi_z(m, 3, 3, r["psi"], r["e0"], kind, 0, -1j * nu, nsteps=200)
    assert np.abs(Cp.imag).max() < 1e-12
    assert np.abs(Cp - Cm).max() < 1e-12
    assert np.all(Cp.real < 0)


@pytest.mark.parametrize("kind", ("spin", "charge"))
def test_inter_orbital_chains_equal_lehmann_sum(kind):
    m = _asym(make_model(2, 2, U=2.4, Jh=0.4, seed=44), 44)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    C01 = chi.chi_ab_z(m, 3, 2, r["psi"], r["e0"], kind, 0, 1, Z, nsteps=120)
    C10 = chi.chi_ab_z(m, 3, 2, r["psi"], r["e0"], kind, 1, 0, Z, nsteps=120)
    Cx = chi.lehmann_chi_ab_z(m, 3, 2, kind, 0, 1, Z)
    assert np.abs(Cx).max() > 1e-3                 # a non-trivial function here
    assert np.abs(C01 - Cx).max() < 1e-10
    assert np.abs(C01 - C10).max() < 1e-12
    Caa = chi.chi_ab_z(m, 3, 2, r["psi"], r["e0"], kind, 1, 1, Z, nsteps=120)
    C1 = chi.chi_z(m, 3, 2, r["psi"], r["e0"], kind, 1, Z, nsteps=120)
    assert np.abs(Caa - C1).max() < 1e-10


@pytest.mark.parametrize("kind", ("spin", "charge"))
def test_inter_orbital_function_vanishes_at_u0(kind):
    b = make_model(2, 3, U=0.0, Jh=0.0, seed=45)
    m = _asym(ImpurityModel(norb=2, nbath=3, U=0.0, Ust=0.0, Jh=0.0, e_imp=b.e_imp,
                            e_bath=b.e_bath, v_bath=b.v_bath), 45)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 4, 3)
    r = lanczos.ground_state(s.matvec, s.dim)
    C01 = chi.chi_ab_z(m, 4, 3, r["psi"], r["e0"], kind, 0, 1, Z, nsteps=200)
    C0 = chi.chi_z(m, 4, 3, r["psi"], r["e0"], kind, 0, Z, nsteps=200)
    assert np.abs(C0).max() > 1e-2
    assert np.abs(C01).max() < 1e-9


def _exciton_u0_closed_form(m, nup, ndw, a, b, z):
    """sum_sigma sum_{k occupied, l empty} |(U^T o U)_{lk}|^2
    [1/(z - (e_l - e_k)) - 1/(z + (e_l - e_k))] with o the one-body matrix of
    c^+_a c_b + c^+_b c_a (levels a, b are the impurity orbitals)."""
    want = np.zeros(z.shape, dtype=np.complex128)
    for spin, n in ((0, nup), (1, ndw)):
        e, U = _one_body(m, spin)
        o = np.zeros((len(e), len(e)))
        la, lb = fock.level_of_impurity(m, a), fock.level_of_impurity(m, b)
        o[la, lb] = o[lb, la] = 1.0
        M = U.T @ o @ U
        for k in range(n):
            for l in range(n, len(e)):
                d = e[l] - e[k]
                want += M[l, k] ** 2 * (1 / (z - d) - 1 / (z + d))
    return want


@pytest.mark.parametrize("pair", [(0, 2), (0, 1)])
def test_exciton_chains_equal_lehmann_sum(pair):
    a, b = pair
    m = _asym(make_model(3, 1, U=2.2, Jh=0.3, seed=46), 46)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    C = chi.chi_exciton_z(m, 3, 2, r["psi"], r["e0"], a, b, Z, nsteps=150)
    Cx = chi.lehmann_chi_exciton_z(m, 3, 2, a, b, Z)
    assert np.abs(Cx).max() > 1e-3
    assert np.abs(C - Cx).max() < 1e-10


@pytest.mark.parametrize("pair", [(0, 2), (1, 2)])
def test_exciton_u0_closed_form(pair):
    a, b = pair
    base = make_model(3, 2, U=0.0, Jh=0.0, seed=47)
    m = _asym(ImpurityModel(norb=3, nbath=2, U=0.0, Ust=0.0, Jh=0.0, e_imp=base.e_imp,
                            e_bath=base.e_bath, v_bath=base.v_bath), 47)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 4, 5)
    r = lanczos.ground_state(s.matvec, s.dim)
    C = chi.chi_exciton_z(m, 4, 5, r["psi"], r["e0"], a, b, Z, nsteps=300)
    want = _exciton_u0_closed_form(m, 4, 5, a, b, Z)
    assert np.abs(want).max() > 1e-3
    assert np.abs(C - want).max() < 1e-9


TAU_BETA = 40.0
TAU = np.linspace(0.0, TAU_BETA, 8001)


@pytest.mark.parametrize("kind", chi.KINDS)
def test_chi_tau_lehmann_and_fourier(kind):
    m = _asym(make_model(2, 2, U=2.4, Jh=0.4, seed=44), 44)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    C = chi.chi_tau(m, 3, 2, r["psi"], r["e0"], kind, 1, TAU, TAU_BETA, nsteps=120)
    Cx = chi.lehmann_chi_tau(m, 3, 2, kind, 1, TAU, TAU_BETA)
    assert np.abs(C - Cx).max() < 1e-10 * max(1.0, np.abs(Cx).max())
    nu = 2 * np.pi * np.arange(1, 8) / TAU_BETA
    ft = np.array([np.trapezoid(np.exp(1j * v * TAU) * C, TAU) for v in nu])
    Cz = chi.chi_z(m, 3, 2, r["psi"], r["e0"], kind, 1, 1j * nu, nsteps=120)
    assert np.abs(ft + Cz).max() < 2e-5
    if kind in ("spin", "charge"):
        assert np.abs(C - C[::-1]).max() < 1e-12
