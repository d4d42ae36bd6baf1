"""Pins of the several-states and finite-temperature oracle
(oracle/thermal.py), no GPU.

* ARPACK's lowest states of a sector equal the dense eigh ones;
* the Boltzmann-weighted sum of per-state chain Green's functions with every
  state of the chosen sectors kept equals the exact finite-temperature
  Lehmann sum from dense spectra (chains long enough to be exact);
* T -> 0: only the ground state survives the truncation and the thermal G
  is the T = 0 G; the weights sum to one and z G(z) -> 1 (each state's
  particle and hole weights add to one);
* the truncation and the per-sector state counts of Sec. 6.2 on worked
  examples.
"""
import math

import numpy as np
import pytest

from oracle import fock, gf, lanczos, thermal
from workloads import ImpurityModel, make_model, workload_ns8


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


def test_arpack_states_equal_dense():
    m = workload_ns8().model
    fock._SECTOR_CACHE.clear()
    E, V = thermal.lowest_states(m, 4, 4, 6, dense_below=0)
    Ed, Vd = np.linalg.eigh(fock.Sector(m, 4, 4).hamiltonian().toarray())
    assert np.abs(E - Ed[:6]).max() < 1e-10
    # the same invariant subspace (degenerate pairs allowed)
    P = Vd[:, :6] @ (Vd[:, :6].T @ V)
    assert np.abs(P - V).max() < 1e-7


def _states(m, sectors, beta, cutoff, nsteps):
    per = [np.linalg.eigh(fock.get_sector(m, nu, nd).hamiltonian().toarray()) for nu, nd in sectors]
    w, _ = thermal.espace_truncate([e for e, _ in per], beta, cutoff)
    out = []
    for (nu, nd), (E, V), ws in zip(sectors, per, w):
        for i in range(len(E)):
            out.append((ws[i], nu, nd, V[:, i], E[i]))
    return out


def test_thermal_gf_equals_lehmann_sum():
    m = _asym(make_model(1, 3, U=2.2, e_d=-0.9, seed=3), 3)
    fock._SECTOR_CACHE.clear()
    sectors = [(2, 2), (2, 1), (1, 2), (3, 2)]
    z = np.concatenate([1j * (2 * np.arange(40) + 1) * np.pi / 8.0, np.linspace(-5, 5, 41) + 0.2j])
    for beta in (0.7, 3.0):
        states = _states(m, sectors, beta, 0.0, 64)
        G = thermal.thermal_gf_z(m, states, 0, 0, z, nsteps=64)
        Gx = thermal.lehmann_thermal_z(m, sectors, beta, 0, 0, z)
        assert np.abs(G - Gx).max() < 1e-11
        assert abs(sum(s[0] for s in states) - 1.0) < 1e-14
        zz = np.array([1e6j])
        assert abs(zz[0] * thermal.thermal_gf_z(m, states, 0, 0, zz, nsteps=64)[0] - 1.0) < 1e-5


def test_zero_temperature_limit():
    m = _asym(make_model(2, 1, U=2.5, Jh=0.4, seed=8), 8)
    fock._SECTOR_CACHE.clear()
    sectors = [(2, 2), (2, 1), (1, 2)]
    states = _states(m, sectors, 1e3, 1e-9, 64)
    kept = [s for s in states if s[0] > 0]
    assert len(kept) == 1 and abs(kept[0][0] - 1.0) < 1e-15
    w, nu, nd, psi, e = kept[0]
    z = 1j * (2 * np.arange(30) + 1) * np.pi / 1e3
    G = thermal.thermal_gf_z(m, states, 1, 0, z, nsteps=64)
    G0 = gf.impurity_gf_z(m, nu, nd, psi, e, 1, 0, z, nsteps=64)
    assert np.abs(G - G0).max() < 1e-13


def test_truncation_worked_examples():
    Es = [np.array([0.0, 0.1, 5.0]), np.array([0.05, 3.0])]
    w, nxt = thermal.espace_truncate(Es, beta=10.0, cutoff=1e-3, step=2)
    f = [1.0, math.exp(-1.0), math.exp(-0.5)]
    Z = sum(f)
    assert np.allclose(w[0], [1.0 / Z, math.exp(-1.0) / Z, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(w[1], [math.exp(-0.5) / Z, 0.0], rtol=0, atol=1e-15)
    assert nxt == [3, 2]       # tops dropped: one more than kept
    # every computed state of the second sector kept: it asks for `step` more
    w, nxt = thermal.espace_truncate([np.array([0.0, 0.2]), np.array([0.1])], beta=1.0,
                                     cutoff=1e-3, step=3)
    assert nxt == [5, 4]
    # the total cap keeps the lowest states
    w, _ = thermal.espace_truncate(Es, beta=10.0, cutoff=1e-3, ntotal=2)
    assert np.count_nonzero(w[0]) == 1 and np.count_nonzero(w[1]) == 1
