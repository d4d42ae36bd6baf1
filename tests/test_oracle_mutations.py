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
