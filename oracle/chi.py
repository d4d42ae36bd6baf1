"""Impurity susceptibilities at T = 0 (oracle, test only).

Sec. 6.8, Eq. KLgf with the bosonic sign: for an operator O,
C_O(z) = <O (z - (H - E0))^-1 O^+> - <O^+ (z + (H - E0))^-1 O>,
evaluated with a Lanczos chain started from O^+|gs> (first term) and one
from O|gs> (second term):
C_O(z) = n+ [(E0 + z - T+)^-1]_00 + n- [(E0 - z - T-)^-1]_00
(the second term's 1/(z + E_m - E0) = -[(E0 - z) - E_m]^-1 and the bosonic
"-" in front give "+"); n+- are the squared norms of the start vectors.

Operators (orbital-diagonal):
* spin   O = S^z_a = (n_{a up} - n_{a dw}) / 2,
* charge O = n_a = n_{a up} + n_{a dw},
* pair   O = d_{a dw} d_{a up} (s-wave; O^+ = d^+_{a up} d^+_{a dw}).
Reading: the spin and charge functions use the connected operator
O - <O> (for a hermitian O both terms then start from (O - <O>)|gs>, and the
E_m = E0 component, which would make C(0) singular, is removed).

Imaginary time (Sec. 6.8 evaluates the susceptibilities on the
imaginary-time axis as well).  Reading: on [0, beta] at T = 0,
C(tau) = n+ sum_m |a+_m|^2 exp(-tau (E+_m - E0))
       + n- sum_m |a-_m|^2 exp(-(beta - tau)(E-_m - E0)),
the first term from the O^+|gs> chain, the second from the O|gs> chain, with
E_m and |a_m|^2 the eigenvalues of the chain's tridiagonal matrix and the
squared first components of its eigenvectors; its bosonic Fourier transform
int_0^beta exp(i nu_n tau) C(tau) dtau is -C(i nu_n) up to exp(-beta (E_m -
E0)) terms, and for a hermitian operator C(tau) = C(beta - tau).

Excitonic function (Sec. 6.8 names it among the susceptibilities).  Reading:
the singlet inter-orbital particle-hole operator of an orbital pair a != b,
O = sum_sigma (c^+_{a sigma} c_{b sigma} + c^+_{b sigma} c_{a sigma}),
hermitian and real, keeping (N_up, N_dw); its connected function from two
chains of (O - <O>)|gs> like the spin and charge functions.

Inter-orbital functions (Sec. 6.8, the auxiliary-operator construction of
non-diagonal correlation functions): C_ab(z) = <A (z - (H - E0))^-1 B> -
<B (z + (H - E0))^-1 A> for A = O_a, B = O_b from the chains of O_a + O_b,
O_a and O_b.  Reading: for the real diagonal spin and charge operators, a
real symmetric H and a real ground state, C_ab = C_ba, so the paper's second
auxiliary operator A - iB is not needed and
C_ab = [C(O_a + O_b) - C_aa - C_bb] / 2.
"""
from __future__ import annotations

import numpy as np

from . import fock, gf
from .lanczos import lanczos_chain

KINDS = ("spin", "charge", "pair")

# sign with which the O|gs> chain enters C_O (bosonic: +, see the module text)
HOLE_TERM_SIGN = +1.0

# C_ab = c0 C(O_a + O_b) + c1 C_aa + c2 C_bb (the auxiliary-operator
# construction, real form: see the module text)
AB_COEFFS = (0.5, -0.5, -0.5)


def diagonal_values(model, nup, ndw, kind, orb):
    """O of a diagonal operator on every basis state (sector order)."""
    s = fock.get_sector(model, nup, ndw)
    nu = np.array([(int(I) >> orb) & 1 for I in s.map_up], dtype=np.float64)
    nd = np.array([(int(I) >> orb) & 1 for I in s.map_dw], dtype=np.float64)
    if kind == "spin":
        return (0.5 * (nu[None, :] - nd[:, None])).reshape(-1)
    if kind == "charge":
        return (nu[None, :] + nd[:, None]).reshape(-1)
    raise ValueError(kind)


def diagonal_values_sum(model, nup, ndw, kind, orbs):
    """O_{a_1} + O_{a_2} + ... on every basis state (orbitals may repeat)."""
    return sum(diagonal_values(model, nup, ndw, kind, a) for a in orbs)


def start_vectors(model, nup, ndw, psi, kind, orb):
    """[(vector, (nup', ndw'), create)] for the two terms: create = +1 for
    O^+|gs>, -1 for O|gs>.  For spin and charge, `orb` may be a tuple of
    orbitals: O is then the sum of their operators."""
    if kind in ("spin", "charge"):
        orbs = orb if isinstance(orb, tuple) else (orb,)
        o = diagonal_values_sum(model, nup, ndw, kind, orbs)
        avg = float(psi @ (o * psi)) / float(psi @ psi)
        phi = (o - avg) * psi
        return [(phi, (nup, ndw), +1), (phi, (nup, ndw), -1)]
    out = []
    # O^+ = d^+_{a up} d^+_{a dw}: d^+_{a dw} first, then d^+_{a up}
    p1, s1 = gf._apply(model, psi, nup, ndw, orb, 1, +1)
    if p1 is not None:
        p2, s2 = gf._apply(model, p1, s1[0], s1[1], orb, 0, +1)
        if p2 is not None:
            out.append((p2, s2, +1))
    # O = d_{a dw} d_{a up}: d_{a up} first, then d_{a dw}
    q1, t1 = gf._apply(model, psi, nup, ndw, orb, 0, -1)
    if q1 is not None:
        q2, t2 = gf._apply(model, q1, t1[0], t1[1], orb, 1, -1)
        if q2 is not None:
            out.append((q2, t2, -1))
    return out


def chi_z(model, nup, ndw, psi, e0, kind, orb, z, nsteps=200, return_parts=False):
    """C_O(z) from the two chains."""
    z = np.asarray(z, dtype=np.complex128)
    C = np.zeros(z.shape, dtype=np.complex128)
    parts = {}
    for phi, (n2u, n2d), create in start_vectors(model, nup, ndw, psi, kind, orb):
        nrm2 = float(phi @ phi)
        parts[create] = nrm2
        if nrm2 == 0.0:
            continue
        sec = fock.get_sector(model, n2u, n2d)
        a, b = lanczos_chain(sec.matvec, phi, nsteps)
        if create > 0:
            C += nrm2 * gf.continued_fraction(a, b, e0 + z)
        else:
            C += HOLE_TERM_SIGN * nrm2 * gf.continued_fraction(a, b, e0 - z)
    if return_parts:
        return C, parts
    return C


def lehmann_chi_z(model, nup, ndw, kind, orb, z):
    """The exact T = 0 sum of Eq. KLgf (bosonic sign) from dense eigenvectors:
    sum_m |<m|O^+|0>|^2 / (z - (E_m - E0)) - |<m|O|0>|^2 / (z + (E_m - E0))."""
    z = np.asarray(z, dtype=np.complex128)
    s0 = fock.get_sector(model, nup, ndw)
    E, U = np.linalg.eigh(s0.hamiltonian().toarray())
    e0, gs = E[0], U[:, 0]
    C = np.zeros(z.shape, dtype=np.complex128)
    for phi, (n2u, n2d), create in start_vectors(model, nup, ndw, gs, kind, orb):
        if not np.any(phi):
            continue
        s1 = fock.get_sector(model, n2u, n2d)
        E1, U1 = np.linalg.eigh(s1.hamiltonian().toarray())
        w = (U1.T @ phi) ** 2
        if create > 0:
            C += (w[None, :] / (z[:, None] - (E1 - e0)[None, :])).sum(1)
        else:
            C -= (w[None, :] / (z[:, None] + (E1 - e0)[None, :])).sum(1)
    return C, e0


def chi_ab_z(model, nup, ndw, psi, e0, kind, a, b, z, nsteps=200):
    """Inter-orbital C_ab(z) for kind = spin or charge, from the chains of
    O_a + O_b, O_a and O_b (the auxiliary-operator construction, real form:
    see the module text)."""
    if kind not in ("spin", "charge"):
        raise ValueError(kind)
    cs = chi_z(model, nup, ndw, psi, e0, kind, (a, b), z, nsteps)
    ca = chi_z(model, nup, ndw, psi, e0, kind, a, z, nsteps)
    cb = chi_z(model, nup, ndw, psi, e0, kind, b, z, nsteps)
    c0, c1, c2 = AB_COEFFS
    return c0 * cs + c1 * ca + c2 * cb


def lehmann_chi_ab_z(model, nup, ndw, kind, a, b, z):
    """The exact T = 0 off-diagonal function from dense eigenvectors:
    sum_m <0|A|m><m|B|0> [1/(z - (E_m - E0)) - 1/(z + (E_m - E0))] with the
    connected A = O_a - <O_a>, B = O_b - <O_b>."""
    z = np.asarray(z, dtype=np.complex128)
    s0 = fock.get_sector(model, nup, ndw)
    E, U = np.linalg.eigh(s0.hamiltonian().toarray())
    gs = U[:, 0]
    oa = diagonal_values(model, nup, ndw, kind, a)
    ob = diagonal_values(model, nup, ndw, kind, b)
    pa = (oa - gs @ (oa * gs)) * gs
    pb = (ob - gs @ (ob * gs)) * gs
    wa, wb = U.T @ pa, U.T @ pb
    d = E - E[0]
    w = wa * wb
    return (w[None, :] * (1.0 / (z[:, None] - d[None, :]) - 1.0 / (z[:, None] + d[None, :]))).sum(1)


def move_sign(I, between):
    """(-1)^(occupied levels of string I in the mask `between`): the sign of
    moving one electron between the two levels that bound the mask."""
    return -1.0 if fock.popcount(I & between) & 1 else 1.0


def exciton_matrix(model, nup, ndw, a, b):
    """The excitonic operator O = sum_sigma (c^+_a c_b + c^+_b c_a) of the
    impurity orbitals a != b on the sector (sector order), built string by
    string: moving an electron between levels a and b of one spin string
    takes the sign (-1)^(occupied levels strictly between them); the dw
    operators' Jordan-Wigner signs from the up string cancel in pairs."""
    import scipy.sparse as sp
    s = fock.get_sector(model, nup, ndw)
    la, lb = fock.level_of_impurity(model, a), fock.level_of_impurity(model, b)
    lo, hi = min(la, lb), max(la, lb)
    between = ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)

    def moves(smap):
        out = []
        for i, I in enumerate(smap):
            I = int(I)
            for src, dst in ((lb, la), (la, lb)):
                if (I >> src) & 1 and not (I >> dst) & 1:
                    J = I ^ (1 << src) ^ (1 << dst)
                    out.append((fock.binary_search(smap, J), i, move_sign(I, between)))
        return out
    rows, cols, vals = [], [], []
    du, dd = s.dim_up, s.dim_dw
    for j, i, sgn in moves(s.map_up):          # up moves: same dw string
        for r in range(dd):
            rows.append(r * du + j); cols.append(r * du + i); vals.append(sgn)
    for j, i, sgn in moves(s.map_dw):          # dw moves: same up string
        for c in range(du):
            rows.append(j * du + c); cols.append(i * du + c); vals.append(sgn)
    return sp.csr_matrix((vals, (rows, cols)), shape=(s.dim, s.dim))


def chi_exciton_z(model, nup, ndw, psi, e0, a, b, z, nsteps=200):
    """Excitonic C_O(z) of the orbital pair (a, b) from the two chains of the
    connected (O - <O>)|gs> (bosonic sign, as chi_z)."""
    z = np.asarray(z, dtype=np.complex128)
    O = exciton_matrix(model, nup, ndw, a, b)
    avg = float(psi @ (O @ psi)) / float(psi @ psi)
    phi = O @ psi - avg * psi
    nrm2 = float(phi @ phi)
    if nrm2 == 0.0:
        return np.zeros(z.shape, dtype=np.complex128)
    sec = fock.get_sector(model, nup, ndw)
    al, be = lanczos_chain(sec.matvec, phi, nsteps)
    return nrm2 * gf.continued_fraction(al, be, e0 + z) + \
        HOLE_TERM_SIGN * nrm2 * gf.continued_fraction(al, be, e0 - z)


def lehmann_chi_exciton_z(model, nup, ndw, a, b, z):
    """The exact T = 0 excitonic function from dense eigenvectors."""
    z = np.asarray(z, dtype=np.complex128)
    s0 = fock.get_sector(model, nup, ndw)
    E, U = np.linalg.eigh(s0.hamiltonian().toarray())
    gs = U[:, 0]
    O = exciton_matrix(model, nup, ndw, a, b).toarray()
    phi = O @ gs - (gs @ O @ gs) * gs
    w = (U.T @ phi) ** 2
    d = E - E[0]
    return (w[None, :] * (1.0 / (z[:, None] - d[None, :]) - 1.0 / (z[:, None] + d[None, :]))).sum(1)


def tau_argument(tau, beta, create):
    """The time a term of C(tau) decays over: tau for the O^+|gs> chain,
    beta - tau for the O|gs> chain (see the module text)."""
    return tau if create > 0 else beta - tau


def chi_tau(model, nup, ndw, psi, e0, kind, orb, tau, beta, nsteps=200):
    """C(tau) for tau in [0, beta] (see the module text) from the chains of
    chi_z: each chain's poles and weights from the eigenvalues and first
    eigenvector components of its tridiagonal matrix (scipy's tridiagonal
    eigensolver)."""
    from scipy.linalg import eigh_tridiagonal
    tau = np.asarray(tau, dtype=np.float64)
    C = np.zeros(tau.shape)
    for phi, (n2u, n2d), create in start_vectors(model, nup, ndw, psi, kind, orb):
        nrm2 = float(phi @ phi)
        if nrm2 == 0.0:
            continue
        sec = fock.get_sector(model, n2u, n2d)
        a, b = lanczos_chain(sec.matvec, phi, nsteps)
        lam, Z = eigh_tridiagonal(a, b[1:len(a)])
        w = Z[0, :] ** 2
        d = lam - e0
        t = tau_argument(tau, beta, create)
        C += nrm2 * (w[None, :] * np.exp(-t[:, None] * d[None, :])).sum(1)
    return C


def lehmann_chi_tau(model, nup, ndw, kind, orb, tau, beta):
    """The exact C(tau) from dense eigenvectors: sum_m |<m|O^+|0>|^2
    exp(-tau (E_m - E0)) + |<m|O|0>|^2 exp(-(beta - tau)(E_m - E0))."""
    tau = np.asarray(tau, dtype=np.float64)
    s0 = fock.get_sector(model, nup, ndw)
    E, U = np.linalg.eigh(s0.hamiltonian().toarray())
    e0, gs = E[0], U[:, 0]
    C = np.zeros(tau.shape)
    for phi, (n2u, n2d), create in start_vectors(model, nup, ndw, gs, kind, orb):
        if not np.any(phi):
            continue
        s1 = fock.get_sector(model, n2u, n2d)
        E1, U1 = np.linalg.eigh(s1.hamiltonian().toarray())
        w = (U1.T @ phi) ** 2
        t = tau_argument(tau, beta, create)
        C += (w[None, :] * np.exp(-t[:, None] * (E1 - e0)[None, :])).sum(1)
    return C
