"""Electron-phonon (Holstein) impurity model (oracle, test only).

Sec. 4: one phonon mode at the impurity, H = H_e + H_e-ph + H_ph with
H_ph = w0 b^+ b and H_e-ph = sum_{alpha sigma} g_alpha d^+_{alpha sigma}
d_{alpha sigma} (b + b^+); the phonon number is cut off at N_ph, so the local
phonon space is |0>, ..., |N_ph> (D_ph = N_ph + 1).

Sector S[N_up, N_dw] of the coupled system is the electronic sector times the
phonon space, with the phonon index slowest (Eq. Vdecomp2):
i = i_e + i_ph * D_e, i_e the electronic sector index (i_up + i_dw D_up).
The sector matrix is Eq. HephBuild:
H_S = 1_ph (x) H_e + H_ph (x) 1_e + X (x) N_g,
X = b + b^+ (<p|X|p+1> = <p+1|X|p> = sqrt(p+1)) and N_g the diagonal matrix
of sum_alpha g_alpha (n_{alpha up} + n_{alpha dw}) over the electronic basis.

c and c^+ act on the electronic part of every phonon slice (Sec. 4.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fock, gf
from .lanczos import lanczos_chain


@dataclass
class Phonon:
    """One phonon mode: frequency w0, couplings g[alpha], cut-off N_ph."""
    w0: float
    g: np.ndarray
    nph: int

    @property
    def dph(self) -> int:
        return self.nph + 1


def displacement(nph: int) -> sp.csr_matrix:
    """X = b + b^+ on |0>..|N_ph>."""
    off = np.sqrt(np.arange(1, nph + 1, dtype=np.float64))
    return sp.csr_matrix(sp.diags([off, off], [-1, 1], shape=(nph + 1, nph + 1)))


def coupling_diagonal(model, ph: Phonon, nup: int, ndw: int) -> np.ndarray:
    """N_g[i_e] = sum_alpha g_alpha (n_{alpha up} + n_{alpha dw}) of every
    electronic basis state, sector order ([D_dw][D_up] flattened)."""
    s = fock.get_sector(model, nup, ndw)
    nu = np.array([[(int(I) >> a) & 1 for a in range(model.norb)] for I in s.map_up], float)
    nd = np.array([[(int(I) >> a) & 1 for a in range(model.norb)] for I in s.map_dw], float)
    g = np.asarray(ph.g, dtype=np.float64)
    return ((nd @ g)[:, None] + (nu @ g)[None, :]).reshape(-1)


def hamiltonian(model, ph: Phonon, nup: int, ndw: int) -> sp.csr_matrix:
    """Eq. HephBuild as an explicit sparse matrix (small sectors)."""
    He = fock.get_sector(model, nup, ndw).hamiltonian()
    Ie = sp.identity(He.shape[0], format="csr")
    Iph = sp.identity(ph.dph, format="csr")
    Hph = sp.diags(ph.w0 * np.arange(ph.dph, dtype=np.float64))
    Ng = sp.diags(coupling_diagonal(model, ph, nup, ndw))
    H = sp.kron(Iph, He) + sp.kron(Hph, Ie) + sp.kron(displacement(ph.nph), Ng)
    return sp.csr_matrix(H)


class Sector:
    """The coupled sector: matvec applies Eq. HephBuild slice by slice."""

    def __init__(self, model, ph: Phonon, nup: int, ndw: int):
        self.model, self.ph = model, ph
        self.nup, self.ndw = nup, ndw
        self.el = fock.get_sector(model, nup, ndw)
        self.de = self.el.dim
        self.dim = self.de * ph.dph
        self.ng = coupling_diagonal(model, ph, nup, ndw)

    def matvec(self, v: np.ndarray) -> np.ndarray:
        """w[p] = H_e v[p] + w0 p v[p] + N_g (sqrt(p) v[p-1] + sqrt(p+1) v[p+1])."""
        V = v.reshape(self.ph.dph, self.de)
        W = np.empty_like(V)
        for p in range(self.ph.dph):
            W[p] = self.el.matvec(V[p]) + self.ph.w0 * p * V[p]
            x = np.zeros(self.de)
            if p > 0:
                x += np.sqrt(p) * V[p - 1]
            if p < self.ph.nph:
                x += np.sqrt(p + 1) * V[p + 1]
            W[p] += self.ng * x
        return W.reshape(-1)


def apply_op(model, ph: Phonon, psi, nup, ndw, orb, spin, create):
    """c^+ (create = +1) or c (-1) of (orb, spin) on every phonon slice of a
    coupled-sector vector; returns (phi, (nup2, ndw2)) or (None, ...)."""
    de = fock.get_sector(model, nup, ndw).dim
    P = np.asarray(psi).reshape(ph.dph, de)
    out = []
    target = None
    for p in range(ph.dph):
        phi, target = gf._apply(model, P[p], nup, ndw, orb, spin, create)
        if phi is None:
            return None, target
        out.append(phi)
    return np.concatenate(out), target


def impurity_gf_z(model, ph: Phonon, nup, ndw, psi, e0, orb, spin, z, nsteps=200):
    """G(z) of the coupled model at T = 0 (Eq. KLgf with the coupled H):
    n+ [(E0 + z - T+)^-1]_00 - n- [(E0 - z - T-)^-1]_00 from Lanczos chains
    on the N +- 1 coupled sectors."""
    z = np.asarray(z, dtype=np.complex128)
    G = np.zeros(z.shape, dtype=np.complex128)
    for create in (+1, -1):
        phi, (n2u, n2d) = apply_op(model, ph, psi, nup, ndw, orb, spin, create)
        if phi is None:
            continue
        nrm2 = float(phi @ phi)
        if nrm2 == 0.0:
            continue
        sec = Sector(model, ph, n2u, n2d)
        a, b = lanczos_chain(sec.matvec, phi, nsteps)
        if create > 0:
            G += nrm2 * gf.continued_fraction(a, b, e0 + z)
        else:
            G -= nrm2 * gf.continued_fraction(a, b, e0 - z)
    return G
