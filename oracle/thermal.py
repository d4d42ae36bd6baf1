"""Several low-lying states and finite temperature (oracle, test only).

* the lowest states of a sector: the eigenpairs of the oracle's sector
  operator from ARPACK (scipy's eigsh, implicitly restarted Lanczos), the
  library the paper uses for several states (Sec. 5, P-ARPACK);
* the eigenspace list with the annealing truncation of Sec. 6.2: the states
  of several sectors sorted by energy; E0 the lowest; a state is kept when its
  Boltzmann factor e^{-beta (E_i - E0)} is at least `cutoff` (reading: the
  printed "<" is the condition for dropping a state), at most `ntotal`
  states; weights w_i = e^{-beta (E_i - E0)} / Z over the kept states.  The
  next number of states per sector: a sector whose highest computed state
  was kept may hold more states under the threshold and asks for `step` more,
  any other sector asks for one more than it kept;
* the finite-temperature Green's function (App. A, the thermal average over
  the eigenstates of Eq. KLgf): G(z) = sum_i w_i G_i(z), G_i the T = 0 form
  of state i with its own energy E_i;
* the exact Lehmann sum at finite temperature from dense spectra of a sector
  and its neighbours, for pins.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as sla

from . import fock, gf


def lowest_states(model, nup, ndw, nstates, dense_below=2000):
    """(E[nstates] ascending, V[:, nstates]) of the sector: dense eigh for
    small sectors, ARPACK on the sector's product otherwise."""
    s = fock.get_sector(model, nup, ndw)
    k = min(nstates, s.dim)
    if s.dim <= dense_below:
        E, V = np.linalg.eigh(s.hamiltonian().toarray())
        return E[:k], V[:, :k]
    op = sla.LinearOperator((s.dim, s.dim), matvec=s.matvec, dtype=np.float64)
    E, V = sla.eigsh(op, k=k, which="SA", tol=1e-13, ncv=max(2 * k + 10, 30))
    order = np.argsort(E)
    return E[order], V[:, order]


def espace_truncate(energies_per_sector, beta, cutoff, ntotal=1 << 30, step=2):
    """Annealing truncation (Sec. 6.2).  energies_per_sector: list of
    ascending energy arrays, one per sector.  Returns (weights per sector,
    next state counts per sector)."""
    allE = [(e, si, i) for si, es in enumerate(energies_per_sector) for i, e in enumerate(es)]
    allE.sort()
    e0 = allE[0][0]
    kept = []
    for e, si, i in allE:
        if len(kept) >= ntotal:
            break
        if math.exp(-beta * (e - e0)) >= cutoff:
            kept.append((e, si, i))
    z = sum(math.exp(-beta * (e - e0)) for e, _, _ in kept)
    weights = [np.zeros(len(es)) for es in energies_per_sector]
    for e, si, i in kept:
        weights[si][i] = math.exp(-beta * (e - e0)) / z
    nxt = []
    for si, es in enumerate(energies_per_sector):
        nk = int(np.count_nonzero(weights[si]))
        top_kept = len(es) > 0 and weights[si][len(es) - 1] > 0
        nxt.append(len(es) + step if top_kept else nk + 1)
    return weights, nxt


def thermal_gf_z(model, states, orb, spin, z, nsteps=200):
    """G(z) = sum_i w_i G_i(z); states: list of (w_i, nup, ndw, psi_i, E_i)."""
    z = np.asarray(z, dtype=np.complex128)
    G = np.zeros(z.shape, dtype=np.complex128)
    for w, nup, ndw, psi, e in states:
        if w == 0.0:
            continue
        G += w * gf.impurity_gf_z(model, nup, ndw, psi, e, orb, spin, z, nsteps=nsteps)
    return G


def lehmann_thermal_z(model, sectors, beta, orb, spin, z):
    """Exact finite-T Lehmann sum over every state of the given sectors (the
    initial states) and all states of their neighbours:
    G(z) = (1/Z) sum_n e^{-beta E_n} [sum_m |<m|c^+|n>|^2 / (z - (E_m - E_n))
                                     + |<m|c|n>|^2 / (z + (E_m - E_n))]."""
    z = np.asarray(z, dtype=np.complex128)
    spec = {}

    def eig(nu, nd):
        if (nu, nd) not in spec:
            s = fock.get_sector(model, nu, nd)
            spec[(nu, nd)] = np.linalg.eigh(s.hamiltonian().toarray())
        return spec[(nu, nd)]
    e0 = min(eig(nu, nd)[0][0] for nu, nd in sectors)
    G = np.zeros(z.shape, dtype=np.complex128)
    Z = 0.0
    for nu, nd in sectors:
        E, V = eig(nu, nd)
        for n in range(len(E)):
            wn = math.exp(-beta * (E[n] - e0))
            Z += wn
            for create in (+1, -1):
                phi, (n2u, n2d) = gf._apply(model, V[:, n], nu, nd, orb, spin, create)
                if phi is None or not np.any(phi):
                    continue
                E1, U1 = eig(n2u, n2d)
                amp = (U1.T @ phi) ** 2
                if create > 0:
                    G += wn * (amp[None, :] / (z[:, None] - (E1 - E[n])[None, :])).sum(1)
                else:
                    G += wn * (amp[None, :] / (z[:, None] + (E1 - E[n])[None, :])).sum(1)
    return G / Z
