"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case patches one oracle function with a plausible error (a dropped sign,
a dropped interaction term, a swapped index, a wrong sign in the hole part of
G) and checks that the corresponding independent pin no longer holds.
"""
import numpy as np
import pytest

from oracle import fock, fullfock, gf, lanczos
from workloads import make_model


def _jw_mismatch(m, nup, ndw):
    fock._SECTOR_CACHE.clear()
    A = fock.Sector(m, nup, ndw).hamiltonian().toarray()
    B = fullfock.fock_sector_block(m, nup, ndw)
    return np.abs(A - B).max()


MODEL = make_model(2, 2, U=3.1, Jh=0.6, seed=12)


def test_dropped_fermion_sign_is_caught(monkeypatch):
    assert _jw_mismatch(MODEL, 3, 2) < 1e-13
    monkeypatch.setattr(fock, "sign_before", lambda I, pos: 1)
    assert _jw_mismatch(MODEL, 3, 2) > 1e-3


def test_dropped_same_spin_term_is_caught(monkeypatch):
    orig = fock.spin_diagonal

    def bad(model, spin, n, smap=None):
        E, mask = orig(model, spin, n, smap)
        both = np.array([bin(int(x)).count("1") == 2 for x in mask])
        return E - both * (model.Ust - model.Jh), mask
    monkeypatch.setattr(fock, "spin_diagonal", bad)
    assert _jw_mismatch(MODEL, 3, 2) > 1e-3


def test_swapped_interaction_index_is_caught(monkeypatch):
    orig = fock.interaction_table
    monkeypatch.setattr(fock, "interaction_table", lambda m: orig(m).T[:, ::-1])
    assert _jw_mismatch(MODEL, 3, 2) > 1e-3


def test_wrong_hole_sign_in_gf_is_caught(monkeypatch):
    m = make_model(1, 5, U=0.0, e_d=0.05, seed=51)
    s = fock.Sector(m, 3, 3)
    r = lanczos.ground_state(s.matvec, s.dim)
    wn = gf.matsubara(100.0, 16)
    h = np.diag(fock.level_energies(m, 0))
    for nu in range(m.nbath):
        h[0, 1 + nu] = h[1 + nu, 0] = m.v_bath[0, 0, nu]
    ref = np.array([np.linalg.inv(1j * w * np.eye(m.ns) - h)[0, 0] for w in wn])
    G = gf.impurity_gf(m, 3, 3, r["psi"], r["e0"], 0, 0, nmats=16)
    assert np.abs(G - ref).max() < 1e-9
    orig = gf.continued_fraction
    calls = {"n": 0}

    def bad(a, b, z):
        calls["n"] += 1
        out = orig(a, b, z)
        return -out if calls["n"] % 2 == 0 else out   # flips the hole term
    monkeypatch.setattr(gf, "continued_fraction", bad)
    G2 = gf.impurity_gf(m, 3, 3, r["psi"], r["e0"], 0, 0, nmats=16)
    assert np.abs(G2 - ref).max() > 1e-3


def _two_orbital_case():
    from workloads import ImpurityModel
    r = np.random.default_rng(64)
    base = make_model(2, 3, U=2.6, Jh=0.4, seed=64)
    m = ImpurityModel(norb=2, nbath=3, U=base.U, Ust=base.Ust, Jh=base.Jh,
                      e_imp=base.e_imp + r.normal(0, .2, (2, 2)),
                      e_bath=base.e_bath + r.normal(0, .2, base.e_bath.shape),
                      v_bath=base.v_bath * r.uniform(.5, 1.5, base.v_bath.shape))
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 4, 3)
    return m, s, lanczos.ground_state(s.matvec, s.dim)


def _e_int_mismatch(m, s, r):
    from oracle import observables
    from workloads import ImpurityModel
    m0 = ImpurityModel(norb=m.norb, nbath=m.nbath, U=0.0, Ust=0.0, Jh=0.0, e_imp=m.e_imp,
                       e_bath=m.e_bath, v_bath=m.v_bath)
    e_free = float(r["psi"] @ fock.Sector(m0, 4, 3).matvec(r["psi"]))
    _, _, e_int = observables.local_observables(m, 4, 3, r["psi"])
    return abs(r["e0"] - e_free - e_int)


def test_dropped_same_spin_term_in_interaction_energy_is_caught(monkeypatch):
    from oracle import observables
    m, s, r = _two_orbital_case()
    assert _e_int_mismatch(m, s, r) < 1e-10
    orig = observables.local_observables

    def bad(model, nup, ndw, psi):
        dens, nn, e_int = orig(model, nup, ndw, psi)
        return dens, nn, e_int - (model.Ust - model.Jh) * (nn[0, 0, 0, 1] + nn[1, 1, 0, 1])
    monkeypatch.setattr(observables, "local_observables", bad)
    assert _e_int_mismatch(m, s, r) > 1e-3


def test_wrong_spin_in_hartree_term_is_caught(monkeypatch):
    from oracle import observables
    m, s, r = _two_orbital_case()
    dens, _, _ = observables.local_observables(m, 4, 3, r["psi"])
    z = np.array([1e4j])

    def tail_err():
        G = gf.impurity_gf_z(m, 4, 3, r["psi"], r["e0"], 0, 0, z)
        S = observables.self_energy(m, 0, 0, z, G)
        return abs(S[0] - observables.hartree(m, dens, 0, 0))
    assert tail_err() < 2e-3

    def bad(model, d, orb, spin):   # the same-spin density where the other spin's belongs
        h = model.U * d[spin, orb]
        for b in range(model.norb):
            if b != orb:
                h += model.Ust * d[1 - spin, b] + (model.Ust - model.Jh) * d[spin, b]
        return h
    monkeypatch.setattr(observables, "hartree", bad)
    assert tail_err() > 1e-2


def test_wrong_sign_in_hybridisation_is_caught(monkeypatch):
    from oracle import observables
    m, s, r = _two_orbital_case()
    z = 1j * gf.matsubara(50.0, 32)

    def sigma_max():
        G = gf.impurity_gf_z(m, 4, 3, r["psi"], r["e0"], 0, 0, z)
        return np.abs(observables.self_energy(m, 0, 0, z, G)).max()
    from workloads import ImpurityModel
    m0 = ImpurityModel(norb=2, nbath=3, U=0.0, Ust=0.0, Jh=0.0, e_imp=m.e_imp, e_bath=m.e_bath,
                       v_bath=m.v_bath)
    fock._SECTOR_CACHE.clear()
    s0 = fock.Sector(m0, 4, 3)
    r0 = lanczos.ground_state(s0.matvec, s0.dim)
    G0 = gf.impurity_gf_z(m0, 4, 3, r0["psi"], r0["e0"], 0, 0, z)
    assert np.abs(observables.self_energy(m0, 0, 0, z, G0)).max() < 1e-7
    orig = observables.hybridisation
    monkeypatch.setattr(observables, "hybridisation", lambda mm, o, sp, zz: -orig(mm, o, sp, zz))
    assert np.abs(observables.self_energy(m0, 0, 0, z, G0)).max() > 1e-2


# ------------------------------------------------ spin exchange and pair hopping

def _atom_multiplet_error():
    """Largest distance of the oracle's two- and three-electron spectra of a
    three-orbital atom from the Kanamori multiplets U - 3J (9), U - J (5),
    U + 2J (1) and 3U - 9J (4), 3U - 6J (10), 3U - 4J (6).  (The sign of
    J_X shows only with three electrons: with two, U' + J_X and U' - J_X
    merely trade eigenvectors.)"""
    from workloads import ImpurityModel
    U, J = 3.0, 0.55
    m = ImpurityModel(norb=3, nbath=0, U=U, Ust=U - 2 * J, Jh=J, e_imp=np.zeros(3),
                      e_bath=np.zeros((3, 0)), v_bath=np.zeros((3, 0)), Jx=J, Jp=J)
    wants = {2: [(U - 3 * J, 9), (U - J, 5), (U + 2 * J, 1)],
             3: [(3 * U - 9 * J, 4), (3 * U - 6 * J, 10), (3 * U - 4 * J, 6)]}
    err = 0.0
    for n, levels in wants.items():
        ev = []
        for nup in range(n + 1):
            fock._SECTOR_CACHE.clear()
            ev.extend(np.linalg.eigvalsh(fock.Sector(m, nup, n - nup).hamiltonian().toarray()))
        want = np.sort(np.concatenate([np.full(c, e) for e, c in levels]))
        err = max(err, np.abs(np.sort(ev) - want).max())
    return err


def _mutate_terms(monkeypatch, edit):
    orig = fock.nondiagonal_terms
    monkeypatch.setattr(fock, "nondiagonal_terms", lambda m: edit(m, orig(m)))


def test_wrong_sign_of_spin_exchange_is_caught(monkeypatch):
    assert _atom_multiplet_error() < 1e-12
    _mutate_terms(monkeypatch, lambda m, ts: [(-c if o[1] == (o[0][0], 1, 0) else c, o)
                                              for c, o in ts])
    assert _atom_multiplet_error() > 1e-3


def test_dropped_pair_hopping_is_caught(monkeypatch):
    _mutate_terms(monkeypatch, lambda m, ts: [(c, o) for c, o in ts if o[1] != (o[0][0], 1, 1)])
    assert _atom_multiplet_error() > 1e-3


def test_swapped_pair_annihilators_are_caught(monkeypatch):
    """d_{b up} d_{b dw} in place of d_{b dw} d_{b up}: the pair hopping
    changes sign; the Jordan-Wigner blocks and the multiplets see it."""
    from workloads import ImpurityModel
    _mutate_terms(monkeypatch, lambda m, ts: [(c, o[:2] + [o[3], o[2]]) if o[1][2] == 1 else (c, o)
                                              for c, o in ts])
    assert _atom_multiplet_error() > 1e-3
    b = make_model(2, 1, U=2.9, Jh=0.45, seed=72)
    m = ImpurityModel(norb=2, nbath=1, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=b.e_imp,
                      e_bath=b.e_bath, v_bath=b.v_bath, Jx=0.35, Jp=0.27)
    assert _jw_mismatch(m, 2, 2) > 1e-3


def test_interaction_energy_without_nondiagonal_terms_is_caught(monkeypatch):
    from oracle import observables
    from workloads import ImpurityModel
    b = make_model(2, 3, U=2.6, Jh=0.4, seed=64)
    m = ImpurityModel(norb=2, nbath=3, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=b.e_imp,
                      e_bath=b.e_bath, v_bath=b.v_bath, Jx=0.45, Jp=0.35)
    m0 = ImpurityModel(norb=2, nbath=3, U=0.0, Ust=0.0, Jh=0.0, e_imp=b.e_imp,
                       e_bath=b.e_bath, v_bath=b.v_bath)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 4, 3)
    r = lanczos.ground_state(s.matvec, s.dim)
    e_free = float(r["psi"] @ fock.Sector(m0, 4, 3).matvec(r["psi"]))

    def gap():
        return abs(r["e0"] - e_free - observables.local_observables(m, 4, 3, r["psi"])[2])
    assert gap() < 1e-10
    orig = observables.local_observables

    def bad(model, nup, ndw, psi):
        d, nn, e = orig(model, nup, ndw, psi)
        sec = fock.get_sector(model, nup, ndw)
        p = np.asarray(psi) / np.linalg.norm(psi)
        return d, nn, e - float(p @ (sec.H_nd @ p))
    monkeypatch.setattr(observables, "local_observables", bad)
    assert gap() > 1e-3


# ------------------------------------------------------------ electron-phonon

def _polaron_error():
    """Distance of the coupled atom's lowest level (two electrons) from the
    displaced-oscillator value e n + U - g^2 n^2 / w0."""
    from oracle import eph
    from workloads import ImpurityModel
    U, e, w0, g = 1.7, -0.4, 0.8, 0.5
    m = ImpurityModel(norb=1, nbath=0, U=U, Ust=U, Jh=0.0, e_imp=np.array([e]),
                      e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))
    ph = eph.Phonon(w0=w0, g=np.array([g]), nph=40)
    fock._SECTOR_CACHE.clear()
    ev = np.linalg.eigvalsh(eph.hamiltonian(m, ph, 1, 1).toarray())
    return abs(ev[0] - (2 * e + U - 4 * g * g / w0))


def test_wrong_displacement_matrix_is_caught(monkeypatch):
    import scipy.sparse as sp
    from oracle import eph
    assert _polaron_error() < 1e-10

    def bad(nph):   # sqrt(p) in place of sqrt(p + 1)
        off = np.sqrt(np.arange(0, nph, dtype=np.float64))
        return sp.csr_matrix(sp.diags([off, off], [-1, 1], shape=(nph + 1, nph + 1)))
    monkeypatch.setattr(eph, "displacement", bad)
    assert _polaron_error() > 1e-3


def test_coupling_to_n_minus_one_is_caught(monkeypatch):
    from oracle import eph
    orig = eph.coupling_diagonal
    monkeypatch.setattr(eph, "coupling_diagonal",
                        lambda m, ph, nu, nd: orig(m, ph, nu, nd) - float(np.sum(ph.g)))
    assert _polaron_error() > 1e-3


# ------------------------------------------------------------ finite temperature

def _thermal_mismatch():
    from oracle import thermal
    from workloads import ImpurityModel
    b = make_model(1, 3, U=2.2, e_d=-0.9, seed=3)
    r = np.random.default_rng(3)
    m = ImpurityModel(norb=1, nbath=3, U=b.U, Ust=b.Ust, Jh=b.Jh,
                      e_imp=b.e_imp + r.normal(0, .2, (2, 1)),
                      e_bath=b.e_bath + r.normal(0, .2, b.e_bath.shape),
                      v_bath=b.v_bath * r.uniform(.5, 1.5, b.v_bath.shape))
    fock._SECTOR_CACHE.clear()
    sectors = [(2, 2), (2, 1), (1, 2)]
    per = [np.linalg.eigh(fock.get_sector(m, nu, nd).hamiltonian().toarray()) for nu, nd in sectors]
    w, _ = thermal.espace_truncate([e for e, _ in per], 0.7, 0.0)
    states = [(ws[i], nu, nd, V[:, i], E[i]) for (nu, nd), (E, V), ws in zip(sectors, per, w)
              for i in range(len(E))]
    z = 1j * (2 * np.arange(20) + 1) * np.pi / 0.7
    G = thermal.thermal_gf_z(m, states, 0, 0, z, nsteps=64)
    return np.abs(G - thermal.lehmann_thermal_z(m, sectors, 0.7, 0, 0, z)).max()


def test_wrong_boltzmann_sign_is_caught(monkeypatch):
    from oracle import thermal
    assert _thermal_mismatch() < 1e-11
    orig = thermal.espace_truncate
    monkeypatch.setattr(thermal, "espace_truncate",
                        lambda Es, beta, cutoff, *a, **k: orig(Es, -beta, cutoff, *a, **k))
    assert _thermal_mismatch() > 1e-3


def test_unnormalised_weights_are_caught(monkeypatch):
    from oracle import thermal
    orig = thermal.espace_truncate

    def bad(*a, **k):
        w, n = orig(*a, **k)
        return [x * 2.0 for x in w], n
    monkeypatch.setattr(thermal, "espace_truncate", bad)
    assert _thermal_mismatch() > 1e-3


# ------------------------------------------------------------ susceptibilities

def test_fermionic_sign_in_susceptibility_is_caught(monkeypatch):
    """The O|gs> chain entered with the fermionic sign: the U = 0 charge
    function no longer matches its closed form from the one-body
    eigenvectors."""
    from oracle import chi
    from workloads import ImpurityModel
    m0 = make_model(1, 5, U=0.0, Jh=0.0, e_d=0.1, seed=42)
    m = ImpurityModel(norb=1, nbath=5, U=0.0, Ust=0.0, Jh=0.0, e_imp=m0.e_imp,
                      e_bath=m0.e_bath, v_bath=m0.v_bath)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    z = 1j * 2 * np.pi * np.arange(1, 20) / 10.0
    want = np.zeros(z.shape, dtype=np.complex128)
    for spin, n in ((0, 3), (1, 2)):
        h = np.diag(fock.level_energies(m, spin))
        for nu in range(5):
            h[0, 1 + nu] = h[1 + nu, 0] = m.v_bath[spin, 0, nu]
        e, U = np.linalg.eigh(h)
        u = U[0, :]
        for k in range(n):
            for l in range(n, 6):
                d = e[l] - e[k]
                want += (u[l] * u[k]) ** 2 * (1 / (z - d) - 1 / (z + d))

    def err():
        return np.abs(chi.chi_z(m, 3, 2, r["psi"], r["e0"], "charge", 0, z, nsteps=300) - want).max()
    assert err() < 1e-9
    monkeypatch.setattr(chi, "HOLE_TERM_SIGN", -1.0)
    assert err() > 1e-3


def test_wrong_inter_orbital_combination_is_caught(monkeypatch):
    """The auxiliary-operator combination of the inter-orbital function with
    its 1/2 dropped no longer matches the exact off-diagonal Lehmann sum, and
    with the sign of C_bb flipped it no longer vanishes at U = 0 (orbitals on
    their own baths)."""
    from oracle import chi
    from workloads import ImpurityModel
    z = 1j * 2 * np.pi * np.arange(1, 20) / 10.0
    m = make_model(2, 2, U=2.4, Jh=0.4, seed=44)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    want = chi.lehmann_chi_ab_z(m, 3, 2, "spin", 0, 1, z)

    def err_lehmann():
        return np.abs(chi.chi_ab_z(m, 3, 2, r["psi"], r["e0"], "spin", 0, 1, z, nsteps=120)
                      - want).max()
    b = make_model(2, 3, U=0.0, Jh=0.0, seed=45)
    m0 = ImpurityModel(norb=2, nbath=3, U=0.0, Ust=0.0, Jh=0.0, e_imp=b.e_imp,
                       e_bath=b.e_bath, v_bath=b.v_bath)
    fock._SECTOR_CACHE.clear()
    s0 = fock.Sector(m0, 4, 3)
    r0 = lanczos.ground_state(s0.matvec, s0.dim)

    def size_u0():
        return np.abs(chi.chi_ab_z(m0, 4, 3, r0["psi"], r0["e0"], "charge", 0, 1, z,
                                   nsteps=200)).max()
    assert err_lehmann() < 1e-10 and size_u0() < 1e-9
    monkeypatch.setattr(chi, "AB_COEFFS", (1.0, -1.0, -1.0))
    assert err_lehmann() > 1e-3
    monkeypatch.setattr(chi, "AB_COEFFS", (0.5, -0.5, 0.5))
    assert size_u0() > 1e-3


def test_dropped_sign_of_exciton_move_is_caught(monkeypatch):
    """The excitonic operator built without the fermionic sign of moving an
    electron past occupied levels no longer matches the U = 0 closed form
    from the one-body eigenvectors for orbitals 0 and 2 (level 1 between)."""
    from oracle import chi
    from workloads import ImpurityModel
    z = 1j * 2 * np.pi * np.arange(1, 20) / 10.0
    base = make_model(3, 2, U=0.0, Jh=0.0, seed=47)
    m = ImpurityModel(norb=3, nbath=2, U=0.0, Ust=0.0, Jh=0.0, e_imp=base.e_imp,
                      e_bath=base.e_bath, v_bath=base.v_bath)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 4, 5)
    r = lanczos.ground_state(s.matvec, s.dim)
    want = np.zeros(z.shape, dtype=np.complex128)
    for spin, n in ((0, 4), (1, 5)):
        h = np.diag(fock.level_energies(m, spin))
        for a in range(3):
            for nu in range(2):
                i, j = fock.level_of_impurity(m, a), fock.level_of_bath(m, a, nu)
                h[i, j] = h[j, i] = m.v_bath[spin, a, nu]
        e, U = np.linalg.eigh(h)
        o = np.zeros_like(h)
        o[0, 2] = o[2, 0] = 1.0
        M = U.T @ o @ U
        for k in range(n):
            for l in range(n, len(e)):
                d = e[l] - e[k]
                want += M[l, k] ** 2 * (1 / (z - d) - 1 / (z + d))

    def err():
        return np.abs(chi.chi_exciton_z(m, 4, 5, r["psi"], r["e0"], 0, 2, z, nsteps=300)
                      - want).max()
    assert err() < 1e-9
    monkeypatch.setattr(chi, "move_sign", lambda I, between: 1.0)
    assert err() > 1e-3


def test_swapped_imaginary_time_terms_are_caught(monkeypatch):
    """C(tau) with the O^+|gs> and O|gs> chains decaying over the wrong
    times: its Fourier transform no longer equals -C(i nu_n) of the continued
    fraction (pair function, whose two terms differ)."""
    from oracle import chi
    beta = 40.0
    tau = np.linspace(0.0, beta, 8001)
    m = make_model(2, 2, U=2.4, Jh=0.4, seed=44)
    fock._SECTOR_CACHE.clear()
    s = fock.Sector(m, 3, 2)
    r = lanczos.ground_state(s.matvec, s.dim)
    nu = 2 * np.pi * np.arange(1, 8) / beta
    Cz = chi.chi_z(m, 3, 2, r["psi"], r["e0"], "pair", 1, 1j * nu, nsteps=120)

    def err():
        C = chi.chi_tau(m, 3, 2, r["psi"], r["e0"], "pair", 1, tau, beta, nsteps=120)
        ft = np.array([np.trapezoid(np.exp(1j * v * tau) * C, tau) for v in nu])
        return np.abs(ft + Cz).max()
    assert err() < 2e-5
    monkeypatch.setattr(chi, "tau_argument",
                        lambda t, b, create: b - t if create > 0 else t)
    assert err() > 1e-3
