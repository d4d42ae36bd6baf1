"""Impurity Green's function on the Matsubara axis (oracle, test only).

Sec. 6.8 / Eq. KLgf at T = 0 for the fermionic impurity function
G_{alpha sigma}(z) = <gs| c (z - (H - E0))^-1 c^+ |gs> + <gs| c^+ (z + (H - E0))^-1 c |gs>.
Reading: the printed "-/+" sign of the second term is taken as "+" for
fermions (standard Lehmann form; pinned by the U = 0 closed form).

Each term is evaluated with a Lanczos chain started from phi = c^+|gs> (or
c|gs>) and the continued fraction of its tridiagonal coefficients; the weight
is n = ||phi||^2.  Matsubara grid at T = 0: w_n = (2n+1) pi / beta.
"""
from __future__ import annotations

import numpy as np

from . import fock
from .lanczos import lanczos_chain


def matsubara(beta: float, nmats: int) -> np.ndarray:
    return (2 * np.arange(nmats) + 1) * np.pi / beta


def apply_cdag(model, psi, nup, ndw, orb, spin):
    """phi = c^+_{orb, spin} psi: S[nup,ndw] -> S[nup+1,ndw] (spin up) or
    S[nup,ndw+1] (spin down).  Sign (-1)**# with # the occupied modes before
    (orb, spin) in the order 1up..Ns up, 1dw..Ns dw (Sec. 2.3); for a down
    electron that includes all N_up up electrons."""
    return _apply(model, psi, nup, ndw, orb, spin, +1)


def apply_c(model, psi, nup, ndw, orb, spin):
    """phi = c_{orb, spin} psi into S[nup-1,ndw] or S[nup,ndw-1]."""
    return _apply(model, psi, nup, ndw, orb, spin, -1)


def _apply(model, psi, nup, ndw, orb, spin, create):
    ns = model.ns
    a = fock.level_of_impurity(model, orb)
    src = fock.get_sector(model, nup, ndw)
    nup2 = nup + create if spin == 0 else nup
    ndw2 = ndw + create if spin == 1 else ndw
    if not (0 <= nup2 <= ns and 0 <= ndw2 <= ns):
        return None, (nup2, ndw2)
    dst = fock.get_sector(model, nup2, ndw2)
    P = psi.reshape(src.dim_dw, src.dim_up)
    out = np.zeros((dst.dim_dw, dst.dim_up))
    smap = src.map_up if spin == 0 else src.map_dw
    tmap = dst.map_up if spin == 0 else dst.map_dw
    for i, I in enumerate(smap):
        I = int(I)
        occ = (I >> a) & 1
        if create > 0 and occ:
            continue
        if create < 0 and not occ:
            continue
        sgn = -1.0 if fock.popcount(I & ((1 << a) - 1)) & 1 else 1.0
        if spin == 1 and (nup & 1):
            sgn = -sgn
        J = I ^ (1 << a)
        j = fock.binary_search(tmap, J)
        if spin == 0:
            out[:, j] += sgn * P[:, i]
        else:
            out[j, :] += sgn * P[i, :]
    return out.reshape(-1), (nup2, ndw2)


def continued_fraction(a, b, z):
    """[(z - T)^-1]_{00} for the tridiagonal T(a, b), by the backward
    recurrence of the continued fraction (Sec. 6.8)."""
    z = np.asarray(z, dtype=np.complex128)
    n = len(a)
    f = z - a[n - 1]
    for j in range(n - 2, -1, -1):
        f = z - a[j] - (b[j + 1] ** 2) / f
    return 1.0 / f


def impurity_gf(model, nup, ndw, psi, e0, orb, spin, nsteps=200, beta=100.0,
                nmats=512, return_parts=False):
    """G_{orb,spin}(i w_n) from two Lanczos chains of ``nsteps`` steps."""
    return impurity_gf_z(model, nup, ndw, psi, e0, orb, spin, 1j * matsubara(beta, nmats),
                         nsteps=nsteps, return_parts=return_parts)


def impurity_gf_z(model, nup, ndw, psi, e0, orb, spin, z, nsteps=200, return_parts=False):
    """G_{orb,spin}(z) at arbitrary complex frequencies z (Eq. KLgf at T = 0):
    n+ [(E0 + z - T+)^-1]_00 - n- [(E0 - z - T-)^-1]_00 from the chains
    started at c^+|gs> and c|gs> (z = i w_n: the Matsubara axis; z = w + i eta:
    the real axis, retarded)."""
    z = np.asarray(z, dtype=np.complex128)
    G = np.zeros(z.shape, dtype=np.complex128)
    parts = {}
    for create in (+1, -1):
        phi, (n2u, n2d) = _apply(model, psi, nup, ndw, orb, spin, create)
        if phi is None:
            parts[create] = (0.0, np.array([]), np.array([0.0]))
            continue
        nrm2 = float(np.dot(phi, phi))
        if nrm2 == 0.0:
            parts[create] = (0.0, np.array([]), np.array([0.0]))
            continue
        sec = fock.get_sector(model, n2u, n2d)
        a, b = lanczos_chain(sec.matvec, phi, nsteps)
        parts[create] = (nrm2, a, b)
        if create > 0:
            G += nrm2 * continued_fraction(a, b, e0 + z)
        else:
            G -= nrm2 * continued_fraction(a, b, e0 - z)
    if return_parts:
        return G, parts
    return G


def lehmann_gf_dense(model, nup, ndw, orb, spin, beta=100.0, nmats=512):
    """Exact T = 0 Lehmann sum of Eq. KLgf from dense eigenvectors of the
    sector and its two neighbours (small sectors only)."""
    return lehmann_gf_dense_z(model, nup, ndw, orb, spin, 1j * matsubara(beta, nmats))


def lehmann_gf_dense_z(model, nup, ndw, orb, spin, z):
    """The exact Lehmann sum at arbitrary complex frequencies z: returns
    (G(z), E0)."""
    z = np.asarray(z, dtype=np.complex128)
    s0 = fock.get_sector(model, nup, ndw)
    E, U = np.linalg.eigh(s0.hamiltonian().toarray())
    e0, gs = E[0], U[:, 0]
    G = np.zeros(z.shape, dtype=np.complex128)
    for create in (+1, -1):
        phi, (n2u, n2d) = _apply(model, gs, nup, ndw, orb, spin, create)
        if phi is None or not np.any(phi):
            continue
        s1 = fock.get_sector(model, n2u, n2d)
        E1, U1 = np.linalg.eigh(s1.hamiltonian().toarray())
        w = (U1.T @ phi) ** 2
        if create > 0:
            G += (w[None, :] / (z[:, None] - (E1 - e0)[None, :])).sum(1)
        else:
            G += (w[None, :] / (z[:, None] + (E1 - e0)[None, :])).sum(1)
    return G, e0
