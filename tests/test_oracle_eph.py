"""Pins of the electron-phonon oracle (oracle/eph.py, Sec. 4), no GPU.

* every coupled sector block of the whole space (electronic Fock space from
  Jordan-Wigner matrices x the truncated phonon space, phonon index slowest)
  equals the oracle's Eq. HephBuild matrix, and its product equals the
  slice-by-slice matvec;
* g = 0: the spectrum is {E_e + w0 p};
* the atomic limit (one level, no bath) is the displaced oscillator:
  w0 b^+b + g n (b + b^+) = w0 (b + g n / w0)^+ (b + g n / w0) - g^2 n^2 / w0,
  so the lowest energy of n electrons is e n + U n_up n_dw - g^2 n^2 / w0,
  with levels w0 apart above it (polaron shift; the effective U is
  U - 2 g^2 / w0);
* the Green's function of the empty level is the independent-boson
  (Franck-Condon) result G(z) = sum_k e^{-l} l^k / k! / (z - (e - g^2/w0 + k w0)),
  l = (g / w0)^2.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import eph, fock, fullfock, lanczos
from workloads import ImpurityModel, make_model


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


def _atom(U, e):
    return ImpurityModel(norb=1, nbath=0, U=U, Ust=U, Jh=0.0, e_imp=np.array([e]),
                         e_bath=np.zeros((1, 0)), v_bath=np.zeros((1, 0)))


@pytest.mark.parametrize("norb,nbath", [(1, 2), (2, 1)])
def test_coupled_blocks_equal_jordan_wigner_times_phonons(norb, nbath):
    m = _asym(make_model(norb, nbath, U=2.3, Jh=0.3, seed=81 + norb), norb)
    ph = eph.Phonon(w0=0.7, g=np.linspace(0.4, 0.6, norb), nph=3)
    ns = m.ns
    He = fullfock.fock_space_hamiltonian(m)
    c = fullfock.jordan_wigner_annihilators(2 * ns)
    ng = sp.csr_matrix(He.shape)
    for a in range(norb):
        for s in range(2):
            ng = ng + ph.g[a] * (c[a + s * ns].T @ c[a + s * ns])
    dF = He.shape[0]
    X = eph.displacement(ph.nph)
    H = (sp.kron(sp.identity(ph.dph), He) + sp.kron(sp.diags(ph.w0 * np.arange(ph.dph)),
                                                   sp.identity(dF)) + sp.kron(X, ng)).tocsr()
    for nup in range(ns + 1):
        for ndw in range(ns + 1):
            idx_e = fullfock.sector_indices(ns, nup, ndw)
            idx = np.concatenate([idx_e + p * dF for p in range(ph.dph)])
            B = H[idx][:, idx].toarray()
            fock._SECTOR_CACHE.clear()
            A = eph.hamiltonian(m, ph, nup, ndw).toarray()
            assert np.abs(A - B).max() < 1e-13, (nup, ndw)
            v = np.random.default_rng(nup + 5 * ndw).normal(size=A.shape[0])
            assert np.abs(eph.Sector(m, ph, nup, ndw).matvec(v) - A @ v).max() < 1e-12


def test_zero_coupling_spectrum():
    m = _asym(make_model(2, 1, U=2.0, Jh=0.3, seed=5), 5)
    ph = eph.Phonon(w0=0.45, g=np.zeros(2), nph=4)
    fock._SECTOR_CACHE.clear()
    ee = np.linalg.eigvalsh(fock.Sector(m, 2, 1).hamiltonian().toarray())
    want = np.sort((ee[None, :] + ph.w0 * np.arange(ph.dph)[:, None]).ravel())
    got = np.linalg.eigvalsh(eph.hamiltonian(m, ph, 2, 1).toarray())
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("nup,ndw", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_displaced_oscillator(nup, ndw):
    U, e, w0, g = 1.7, -0.4, 0.8, 0.5
    m = _atom(U, e)
    ph = eph.Phonon(w0=w0, g=np.array([g]), nph=40)
    fock._SECTOR_CACHE.clear()
    ev = np.linalg.eigvalsh(eph.hamiltonian(m, ph, nup, ndw).toarray())
    n = nup + ndw
    base = e * n + U * nup * ndw - g * g * n * n / w0
    assert np.abs(ev[:6] - (base + w0 * np.arange(6))).max() < 1e-10
    # the Lanczos ground state of the coupled sector
    s = eph.Sector(m, ph, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    assert abs(r["e0"] - base) < 1e-10


def test_franck_condon_green_function():
    e, w0, g = 0.9, 0.6, 0.45
    m = _atom(2.0, e)
    ph = eph.Phonon(w0=w0, g=np.array([g]), nph=30)
    fock._SECTOR_CACHE.clear()
    s = eph.Sector(m, ph, 0, 0)
    r = lanczos.ground_state(s.matvec, s.dim)
    assert abs(r["e0"]) < 1e-12                  # empty level, phonon vacuum
    z = 1j * (2 * np.arange(64) + 1) * np.pi / 20.0
    z = np.concatenate([z, np.linspace(-2, 4, 50) + 0.1j])
    G = eph.impurity_gf_z(m, ph, 0, 0, r["psi"], r["e0"], 0, 0, z, nsteps=ph.dph)
    lam = (g / w0) ** 2
    want = sum(math.exp(-lam) * lam ** k / math.factorial(k) / (z - (e - g * g / w0 + k * w0))
               for k in range(ph.dph))
    assert np.abs(G - want).max() < 1e-10
