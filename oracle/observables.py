"""Self-energy, non-interacting impurity function and local observables
(oracle, test only).

Sec. 6.8 and App. B (the impurity self-energy on the Matsubara axis, the
Green's functions on the real axis, the impurity observables):

* G0(z) of the normal bath: G0_{alpha sigma}(z)^-1 = z - e_{alpha sigma}
  - Delta_{alpha sigma}(z), with the hybridisation function
  Delta(z) = sum_nu V_{nu alpha sigma}^2 / (z - eps_{nu alpha sigma})
  (Eq. Ham1 with a diagonal H^loc and bath h);
* Dyson: Sigma(z) = G0(z)^-1 - G(z)^-1;
* from the ground state psi of a sector (sector order, Eq. Vmatrix):
  densities <n_{alpha sigma}>, the density-density correlators
  <n_{alpha sigma} n_{beta sigma'}> (double occupancy d_alpha =
  <n_{alpha up} n_{alpha dw}>) and the interaction energy <H_int> of Eq. Ham1:
  U sum_alpha n_{a up} n_{a dw} + U' sum_{a != b} n_{a up} n_{b dw}
  + (U' - J) sum_{a < b, sigma} n_{a sigma} n_{b sigma}, plus <psi|H_nd|psi>
  for the spin exchange and pair hopping (J_X, J_P);
* the Hartree (first-moment) limit of Sigma at large |z|:
  U <n_{a, -s}> + U' sum_{b != a} <n_{b, -s}> + (U' - J) sum_{b != a} <n_{b, s}>.
  Reading: the spin exchange and pair hopping add nothing to the diagonal
  first moment <{[c_{a s}, H], c^+_{a s}}>: a term that holds c^+_{a s}
  leaves an odd operator without that mode, which anticommutes with
  c^+_{a s}; a term that holds c_{a s} commutes to zero.
"""
from __future__ import annotations

import numpy as np

from . import fock


def hybridisation(model, orb, spin, z):
    """Delta_{orb,spin}(z) = sum_nu V^2 / (z - eps_nu)."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(z.shape, dtype=np.complex128)
    for nu in range(model.nbath):
        out += model.v_bath[spin, orb, nu] ** 2 / (z - model.e_bath[spin, orb, nu])
    return out


def g0_inverse(model, orb, spin, z):
    """G0_{orb,spin}(z)^-1 = z - e_imp - Delta(z)."""
    z = np.asarray(z, dtype=np.complex128)
    return z - model.e_imp[spin, orb] - hybridisation(model, orb, spin, z)


def self_energy(model, orb, spin, z, G):
    """Dyson equation: Sigma(z) = G0(z)^-1 - G(z)^-1."""
    return g0_inverse(model, orb, spin, z) - 1.0 / np.asarray(G, dtype=np.complex128)


def local_observables(model, nup, ndw, psi):
    """(dens[2][norb], nn[2][2][norb][norb], e_int) of a sector-order vector
    psi (normalised here): dens[s][a] = <n_{a s}>,
    nn[s][t][a][b] = <n_{a s} n_{b t}>, e_int = <H_int>."""
    s = fock.get_sector(model, nup, ndw)
    P = np.abs(np.asarray(psi, dtype=np.float64)) ** 2
    P = (P / P.sum()).reshape(s.dim_dw, s.dim_up)
    no = model.norb
    occ_up = np.array([[(int(I) >> a) & 1 for a in range(no)] for I in s.map_up], dtype=np.float64)
    occ_dw = np.array([[(int(I) >> a) & 1 for a in range(no)] for I in s.map_dw], dtype=np.float64)
    # n[s] has shape [D_dw][D_up][norb]
    n = [np.broadcast_to(occ_up[None, :, :], (s.dim_dw, s.dim_up, no)),
         np.broadcast_to(occ_dw[:, None, :], (s.dim_dw, s.dim_up, no))]
    dens = np.zeros((2, no))
    nn = np.zeros((2, 2, no, no))
    for sg in range(2):
        dens[sg] = np.einsum("rc,rca->a", P, n[sg])
        for tg in range(2):
            nn[sg, tg] = np.einsum("rc,rca,rcb->ab", P, n[sg], n[tg])
    e_int = 0.0
    for a in range(no):
        e_int += model.U * nn[0, 1, a, a]
        for b in range(no):
            if a != b:
                e_int += model.Ust * nn[0, 1, a, b]
            if a < b:
                e_int += (model.Ust - model.Jh) * (nn[0, 0, a, b] + nn[1, 1, a, b])
    if s.H_nd is not None:
        p = np.asarray(psi, dtype=np.float64)
        e_int += float(p @ (s.H_nd @ p)) / float(p @ p)
    return dens, nn, float(e_int)


def hartree(model, dens, orb, spin):
    """First moment of Sigma_{orb,spin} (its limit at large |z|)."""
    o = 1 - spin
    h = model.U * dens[o, orb]
    for b in range(model.norb):
        if b != orb:
            h += model.Ust * dens[o, b] + (model.Ust - model.Jh) * dens[spin, b]
    return h
