"""Pins of the oracle's spin-exchange and pair-hopping terms (H_nd of
Eq. Ham1, J_X and J_P), no GPU.

* every sector block of the whole-Fock-space Hamiltonian built from
  Jordan-Wigner matrices, and the state-by-state walk, equal the oracle's
  sector matrix;
* matrix elements between two-electron atomic states worked out by hand
  from the anticommutation relations: <b up, a dw|H|a up, b dw> = +J_X and
  <a up a dw|H|b up b dw> = +J_P;
* the atomic multiplets of the rotationally invariant Kanamori interaction
  (U' = U - 2J, J_X = J_P = J; e.g. Georges, de' Medici and Mravlje, Annu.
  Rev. Condens. Matter Phys. 4, 137 (2013)): two orbitals with two
  electrons: U - 3J (3 states), U - J (2), U + J (1); three orbitals with two
  electrons: U - 3J (9), U - J (5), U + 2J (1); three orbitals with three
  electrons: 3U - 9J (4), 3U - 6J (10), 3U - 4J (6);
* spin-rotation invariance with a bath: with J_X = J the sector
  (n + 1, n - 1) spectrum lies inside the (n, n) spectrum (S^+ maps one
  onto the other); with J_X = 0 it does not;
* the interaction energy includes <H_nd> (E0 - E_free = E_int) and the
  Hartree tail of Sigma is unchanged by H_nd.
"""
import numpy as np
import pytest

from oracle import fock, fullfock, gf, lanczos, observables
from workloads import ImpurityModel, make_model


def kanamori(norb, nbath, U, J, Jx=None, Jp=None, Ust=None, seed=0, asym=None, e_d=None):
    """Model with spin exchange and pair hopping (default J_X = J_P = J,
    U' = U - 2J); asym: seed of a spin-dependent perturbation of the levels
    and hybridisations."""
    b = make_model(norb, nbath, U=U, Jh=J, Ust=Ust, seed=seed, e_d=e_d)
    e_imp, e_bath, v_bath = b.e_imp, b.e_bath, b.v_bath
    if asym is not None:
        r = np.random.default_rng(asym)
        e_imp = e_imp + r.normal(0, .2, (2, norb))
        e_bath = e_bath + r.normal(0, .2, e_bath.shape)
        v_bath = v_bath * r.uniform(.5, 1.5, v_bath.shape)
    return ImpurityModel(norb=norb, nbath=nbath, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=e_imp,
                         e_bath=e_bath, v_bath=v_bath, Jx=J if Jx is None else Jx,
                         Jp=J if Jp is None else Jp)


def _dense(m, nup, ndw):
    fock._SECTOR_CACHE.clear()
    return fock.Sector(m, nup, ndw).hamiltonian().toarray()


@pytest.mark.parametrize("norb,nbath", [(2, 1), (3, 1), (2, 2)])
def test_kanamori_sector_blocks_equal_jordan_wigner(norb, nbath):
    m = kanamori(norb, nbath, U=2.9, J=0.45, Jx=0.35, Jp=0.27, seed=70 + norb, asym=norb)
    H = fullfock.fock_space_hamiltonian(m)
    assert abs(H - H.T).max() < 1e-14
    ns = m.ns
    for nup in range(ns + 1):
        for ndw in range(ns + 1):
            idx = fullfock.sector_indices(ns, nup, ndw)
            B = H[idx][:, idx].toarray()
            A = _dense(m, nup, ndw)
            assert np.abs(A - B).max() < 1e-13, (nup, ndw)
    n_up = np.array([bin(I & ((1 << ns) - 1)).count("1") for I in range(1 << 2 * ns)])
    n_dw = np.array([bin(I >> ns).count("1") for I in range(1 << 2 * ns)])
    Hc = H.tocoo()
    assert np.all(n_up[Hc.row] == n_up[Hc.col]) and np.all(n_dw[Hc.row] == n_dw[Hc.col])


@pytest.mark.parametrize("norb,nbath,sectors", [(2, 3, [(4, 4), (3, 5), (5, 2)]),
                                                (4, 1, [(4, 4), (3, 4), (2, 5)])])
def test_kanamori_statewise_sector_matrix(norb, nbath, sectors):
    m = kanamori(norb, nbath, U=2.2, J=0.3, Jx=0.25, Jp=0.4, seed=80 + norb, asym=norb)
    for (nu, nd) in sectors:
        fock._SECTOR_CACHE.clear()
        s = fock.Sector(m, nu, nd)
        A = s.hamiltonian()
        B = fullfock.sector_hamiltonian_statewise(m, nu, nd)
        assert abs(A - B).max() < 1e-13
        assert abs(s.H_nd - s.H_nd.T).max() == 0.0
        v = np.random.default_rng(nu + 7 * nd).normal(size=s.dim)
        assert np.abs(s.matvec(v) - B @ v).max() < 1e-12


def test_two_electron_matrix_elements_by_hand():
    """Atom with two orbitals, sector (1, 1), sector order (up index
    fastest): states (u0,d0), (u1,d0), (u0,d1), (u1,d1).  With the basis
    state d+_{a up} d+_{b dw}|0> (up modes before down modes):
    -J_X d+_{b up} d_{b dw} d+_{a dw} d_{a up} d+_{a up} d+_{b dw}|0>
    = +J_X d+_{b up} d+_{a dw}|0>, and
    J_P d+_{a up} d+_{a dw} d_{b dw} d_{b up} d+_{b up} d+_{b dw}|0>
    = +J_P d+_{a up} d+_{a dw}|0>."""
    Jx, Jp, U, Ust, Jh = 0.31, 0.17, 2.0, 1.3, 0.4
    m = ImpurityModel(norb=2, nbath=0, U=U, Ust=Ust, Jh=Jh, e_imp=np.zeros(2),
                      e_bath=np.zeros((2, 0)), v_bath=np.zeros((2, 0)), Jx=Jx, Jp=Jp)
    H = _dense(m, 1, 1)
    want = np.array([[U, 0, 0, Jp],
                     [0, Ust, Jx, 0],
                     [0, Jx, Ust, 0],
                     [Jp, 0, 0, U]])
    assert np.abs(H - want).max() < 1e-15


def _n_electron_spectrum(m, n):
    ev = []
    for nup in range(n + 1):
        ndw = n - nup
        if nup <= m.ns and ndw <= m.ns:
            ev.extend(np.linalg.eigvalsh(_dense(m, nup, ndw)))
    return np.sort(np.array(ev))


@pytest.mark.parametrize("norb,n,levels", [
    (2, 2, [(-3, 3), (-1, 2), (1, 1)]),           # U + k J
    (3, 2, [(-3, 9), (-1, 5), (2, 1)]),
    (3, 3, [(-9, 4), (-6, 10), (-4, 6)]),         # 3U + k J
])
def test_kanamori_atomic_multiplets(norb, n, levels):
    U, J = 3.0, 0.55
    m = ImpurityModel(norb=norb, nbath=0, U=U, Ust=U - 2 * J, Jh=J, e_imp=np.zeros(norb),
                      e_bath=np.zeros((norb, 0)), v_bath=np.zeros((norb, 0)), Jx=J, Jp=J)
    base = U if n == 2 else 3 * U
    want = np.sort(np.concatenate([np.full(c, base + k * J) for k, c in levels]))
    assert np.abs(_n_electron_spectrum(m, n) - want).max() < 1e-12


def _contained(small, big, tol=1e-9):
    return max(np.abs(big - e).min() for e in small) < tol


def test_spin_rotation_invariance_with_bath():
    m = kanamori(2, 2, U=2.6, J=0.5, Jx=0.5, Jp=0.3, Ust=1.9, seed=91)
    e33 = np.linalg.eigvalsh(_dense(m, 3, 3))
    e42 = np.linalg.eigvalsh(_dense(m, 4, 2))
    e51 = np.linalg.eigvalsh(_dense(m, 5, 1))
    assert _contained(e42, e33) and _contained(e51, e42)
    # without the spin exchange the density-density part breaks the symmetry
    m0 = kanamori(2, 2, U=2.6, J=0.5, Jx=0.0, Jp=0.3, Ust=1.9, seed=91)
    assert not _contained(np.linalg.eigvalsh(_dense(m0, 4, 2)),
                          np.linalg.eigvalsh(_dense(m0, 3, 3)), 1e-3)


def _u0(m):
    return ImpurityModel(norb=m.norb, nbath=m.nbath, U=0.0, Ust=0.0, Jh=0.0, e_imp=m.e_imp,
                         e_bath=m.e_bath, v_bath=m.v_bath)


def test_interaction_energy_includes_nondiagonal_terms():
    m = kanamori(2, 3, U=2.6, J=0.4, Jx=0.45, Jp=0.35, seed=64, asym=64)
    nup, ndw = 4, 3
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    _, _, e_int = observables.local_observables(m, nup, ndw, r["psi"])
    e_free = float(r["psi"] @ fock.Sector(_u0(m), nup, ndw).matvec(r["psi"]))
    assert abs(r["e0"] - e_free - e_int) < 1e-10 * max(1.0, abs(r["e0"]))
    e_nd = float(r["psi"] @ (s.H_nd @ r["psi"]))
    assert abs(e_nd) > 1e-3            # the terms matter in this state


def test_hartree_tail_unchanged_by_nondiagonal_terms():
    m = kanamori(2, 3, U=2.6, J=0.4, Jx=0.45, Jp=0.35, seed=63, asym=63)
    nup, ndw = 4, 3
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    dens, _, _ = observables.local_observables(m, nup, ndw, r["psi"])
    z = np.array([1e4j, 2e4j])
    for spin in (0, 1):
        for orb in range(m.norb):
            G = gf.impurity_gf_z(m, nup, ndw, r["psi"], r["e0"], orb, spin, z)
            S = observables.self_energy(m, orb, spin, z, G)
            err = np.abs(S - observables.hartree(m, dens, orb, spin))
            assert err[0] < 2e-3 and err[1] < 0.6 * err[0] + 1e-9, (orb, spin, err)


def test_row_terms_equal_matrix_row():
    m = kanamori(3, 1, U=2.4, J=0.35, Jx=0.3, Jp=0.2, seed=5, asym=5)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 3)
    H = s.H_nd.tocsr()
    rng = np.random.default_rng(3)
    for i in rng.integers(0, s.dim, 40):
        iu, idw = i % s.dim_up, i // s.dim_up
        terms = fock.nondiagonal_row(m, int(s.map_up[iu]), int(s.map_dw[idw]))
        got = {}
        for el, Ju, Jd in terms:
            j = int(np.searchsorted(s.map_dw, Jd)) * s.dim_up + int(np.searchsorted(s.map_up, Ju))
            got[j] = got.get(j, 0.0) + el
        row = H.getrow(int(i))
        assert dict(zip(row.indices.tolist(), row.data.tolist())) == got
