"""Sector basis, signs and the spin-factorised Hamiltonian (oracle, test only).

Conventions (readings of the paper, all 0-based):

* level a of one spin string is bit a of the integer I_sigma.  Impurity orbital
  alpha is level alpha (alpha < Norb); bath level nu of orbital alpha is level
  Norb + alpha*Nbath + nu.  Ns = Norb (Nbath + 1) (Sec. 2.1, normal bath).
* the full Fock state is I = I_up + 2**Ns * I_dw and the mode order for signs
  is 1up..Ns up, 1dw..Ns dw (Sec. 2.3).
* sector index i = i_up + i_dw * D_up (Eq. SectorIndxDecomp, 0-based): the
  vector is a row-major [D_dw][D_up] matrix (Eq. Vmatrix).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def popcount(x: int) -> int:
    return bin(x).count("1")


def level_of_impurity(model, alpha: int) -> int:
    return alpha


def level_of_bath(model, alpha: int, nu: int) -> int:
    return model.norb + alpha * model.nbath + nu


def build_sector_map(nbit: int, n: int) -> np.ndarray:
    """Sec. 6.3 (build_sector): scan all integers 0 .. 2**nbit - 1 in
    ascending order and keep those whose popcount equals the sector's
    electron number."""
    out = []
    for I in range(1 << nbit):
        if popcount(I) == n:
            out.append(I)
    return np.array(out, dtype=np.int64)


def binary_search(smap: np.ndarray, I: int) -> int:
    """Sec. 6.3: reverse look-up of a state in the ascending map by binary
    search; returns the 0-based index or -1."""
    lo, hi = 0, len(smap) - 1
    while lo <= hi:
        mid = (lo + hi) // 2
        x = int(smap[mid])
        if x == I:
            return mid
        if x < I:
            lo = mid + 1
        else:
            hi = mid - 1
    return -1


def sign_before(I: int, pos: int) -> int:
    """(-1)**#, # = number of occupied levels below ``pos`` in the string
    (Sec. 2.3, the sign rule of c and c^+)."""
    return -1 if popcount(I & ((1 << pos) - 1)) & 1 else 1


def apply_cdag_c(I: int, p: int, q: int):
    """c^+_p c_q |I> for one spin string: returns (sign, J) or (0, -1).

    Sec. 2.3: c_q first (sign from levels below q), then c^+_p on the new
    string (sign from levels below p).  The other spin's string contributes
    the same factor to both operators and cancels, so it is left out."""
    if not (I >> q) & 1:
        return 0, -1
    s1 = sign_before(I, q)
    I1 = I ^ (1 << q)
    if (I1 >> p) & 1:
        return 0, -1
    s2 = sign_before(I1, p)
    return s1 * s2, I1 | (1 << p)


def spin_hopping_matrix(model, spin: int, n: int, smap=None) -> sp.csr_matrix:
    """H_sigma of Eq. Hdecomp: the hybridisation part of Eq. Ham1,
    sum_{alpha,nu} V^nu_{alpha sigma} (d^+_alpha a_{nu alpha} + h.c.),
    on the per-spin basis of ``n`` electrons (Eq. Hbuild, second and third
    terms).  Built by applying the operators to every basis string."""
    ns = model.ns
    if smap is None:
        smap = build_sector_map(ns, n)
    dim = len(smap)
    rows, cols, vals = [], [], []
    for j in range(dim):
        J = int(smap[j])
        for a in range(model.norb):
            d = level_of_impurity(model, a)
            for nu in range(model.nbath):
                b = level_of_bath(model, a, nu)
                V = model.v_bath[spin, a, nu]
                for (p, q) in ((d, b), (b, d)):
                    s, I = apply_cdag_c(J, p, q)
                    if s == 0:
                        continue
                    i = binary_search(smap, I)
                    rows.append(i)
                    cols.append(j)
                    vals.append(s * V)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))
    H.sum_duplicates()
    H.sort_indices()
    return H


def level_energies(model, spin: int) -> np.ndarray:
    """One-body energies of the Ns levels of one spin (diagonal H^loc and
    diagonal bath h of Eq. Ham1)."""
    eps = np.zeros(model.ns)
    for a in range(model.norb):
        eps[level_of_impurity(model, a)] = model.e_imp[spin, a]
        for nu in range(model.nbath):
            eps[level_of_bath(model, a, nu)] = model.e_bath[spin, a, nu]
    return eps


def spin_diagonal(model, spin: int, n: int, smap=None):
    """Per-spin diagonal energy and impurity occupation mask.

    E_sigma[i] = sum_a eps_a n_a + (U' - J) sum_{alpha<beta} n_alpha n_beta
    (the one-body terms and the same-spin density-density term of Eq. Ham1);
    mask[i] = impurity bits of the string."""
    ns = model.ns
    if smap is None:
        smap = build_sector_map(ns, n)
    eps = level_energies(model, spin)
    E = np.zeros(len(smap))
    mask = np.zeros(len(smap), dtype=np.int64)
    for i, I in enumerate(smap):
        I = int(I)
        e = 0.0
        for a in range(ns):
            if (I >> a) & 1:
                e += eps[a]
        for al in range(model.norb):
            for be in range(al + 1, model.norb):
                if (I >> al) & 1 and (I >> be) & 1:
                    e += model.Ust - model.Jh
        E[i] = e
        mask[i] = I & ((1 << model.norb) - 1)
    return E, mask


def interaction_table(model) -> np.ndarray:
    """W[m_up][m_dw] = U sum_alpha n_{alpha up} n_{alpha dw}
    + U' sum_{alpha != beta} n_{alpha up} n_{beta dw} (Eq. Ham1), for impurity
    occupation masks m_up, m_dw."""
    no = model.norb
    W = np.zeros((1 << no, 1 << no))
    for mu in range(1 << no):
        for md in range(1 << no):
            w = 0.0
            for al in range(no):
                for be in range(no):
                    if (mu >> al) & 1 and (md >> be) & 1:
                        w += model.U if al == be else model.Ust
            W[mu, md] = w
    return W


def nondiagonal_terms(model):
    """H_nd of Eq. Ham1 as (coefficient, operator string) pairs, the string
    a list of (level, spin, create) read left to right as written:
    spin exchange  -J_X d^+_{a up} d_{a dw} d^+_{b dw} d_{b up} and
    pair hopping   +J_P d^+_{a up} d^+_{a dw} d_{b dw} d_{b up},
    for every ordered pair of impurity orbitals a != b (Sec. 3.2: the part of
    H that keeps N_up and N_dw but not the per-spin factorisation)."""
    terms = []
    for a in range(model.norb):
        for b in range(model.norb):
            if a == b:
                continue
            A, B = level_of_impurity(model, a), level_of_impurity(model, b)
            if model.Jx != 0.0:
                terms.append((-model.Jx, [(A, 0, 1), (A, 1, 0), (B, 1, 1), (B, 0, 0)]))
            if model.Jp != 0.0:
                terms.append((model.Jp, [(A, 0, 1), (A, 1, 1), (B, 1, 0), (B, 0, 0)]))
    return terms


def apply_operator_string(ns: int, I, ops):
    """Apply an operator string (rightmost operator first) to full Fock
    integers I = I_up + 2**Ns I_dw (an int64 array): mode of (level, spin) is
    level + spin Ns, and each c or c^+ contributes (-1)**(occupied modes below
    it) before it acts (Sec. 2.3).  Returns (sign, J): sign 0 where the
    string annihilates the state."""
    I = np.array(I, dtype=np.int64, copy=True)
    sign = np.ones(I.shape, dtype=np.int64)
    for (lev, spin, create) in reversed(ops):
        m = lev + spin * ns
        occ = (I >> m) & 1
        sign[occ == create] = 0
        below = np.zeros(I.shape, dtype=np.int64)
        for k in range(m):
            below += (I >> k) & 1
        sign = np.where(below & 1, -sign, sign)
        I = I ^ (np.int64(1) << m)
    return sign, I


def nondiagonal_matrix(model, map_up, map_dw) -> sp.csr_matrix:
    """H_nd on the sector of the two maps, built by applying every term of
    nondiagonal_terms to every basis state (column j = the image of state j)
    and locating the image by binary search in the maps (Sec. 6.3)."""
    ns = model.ns
    du, dd = len(map_up), len(map_dw)
    src = np.arange(du * dd, dtype=np.int64)
    I = map_up[src % du].astype(np.int64) + (map_dw[src // du].astype(np.int64) << ns)
    rows, cols, vals = [], [], []
    for coef, ops in nondiagonal_terms(model):
        sgn, J = apply_operator_string(ns, I, ops)
        k = sgn != 0
        Ju, Jd = J[k] & ((1 << ns) - 1), J[k] >> ns
        iu, idw = np.searchsorted(map_up, Ju), np.searchsorted(map_dw, Jd)
        assert np.all(map_up[iu] == Ju) and np.all(map_dw[idw] == Jd)
        rows.append(idw * du + iu)
        cols.append(src[k])
        vals.append(coef * sgn[k])
    n = du * dd
    if not rows:
        return sp.csr_matrix((n, n))
    H = sp.csr_matrix((np.concatenate(vals).astype(np.float64),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    H.sum_duplicates()
    return H


def nondiagonal_row(model, I_up: int, I_dw: int):
    """The terms of H_nd applied to one basis state: [(element, J_up, J_dw)].
    H_nd is real and symmetric (the adjoint of the (a, b) term of either kind
    is the (b, a) term), so these are also the entries of the state's row:
    (H_nd v)_i = sum of element * v_j over this list."""
    ns = model.ns
    out = []
    I = np.array([int(I_up) + (int(I_dw) << ns)], dtype=np.int64)
    for coef, ops in nondiagonal_terms(model):
        sgn, J = apply_operator_string(ns, I, ops)
        if sgn[0] != 0:
            out.append((coef * int(sgn[0]), int(J[0]) & ((1 << ns) - 1), int(J[0]) >> ns))
    return out


class Sector:
    """Per-spin pieces of the sector S[N_up, N_dw] (Sec. 2.2-2.4), and the
    non-factorisable part H_nd of Eq. Ham1 as an explicit sparse matrix when
    J_X or J_P is non-zero."""

    def __init__(self, model, nup: int, ndw: int):
        self.model = model
        self.nup, self.ndw = nup, ndw
        ns = model.ns
        self.map_up = build_sector_map(ns, nup)
        self.map_dw = build_sector_map(ns, ndw)
        self.dim_up, self.dim_dw = len(self.map_up), len(self.map_dw)
        self.dim = self.dim_up * self.dim_dw
        self.H_up = spin_hopping_matrix(model, 0, nup, self.map_up)
        self.H_dw = spin_hopping_matrix(model, 1, ndw, self.map_dw)
        self.E_up, self.m_up = spin_diagonal(model, 0, nup, self.map_up)
        self.E_dw, self.m_dw = spin_diagonal(model, 1, ndw, self.map_dw)
        self.W = interaction_table(model)
        self.H_nd = None
        if model.Jx != 0.0 or model.Jp != 0.0:
            self.H_nd = nondiagonal_matrix(model, self.map_up, self.map_dw)

    def diagonal(self) -> np.ndarray:
        """H_d of Eq. Hdecomp as a [D_dw][D_up] array."""
        return (self.E_up[None, :] + self.E_dw[:, None]
                + self.W[self.m_up[None, :], self.m_dw[:, None]])

    def matvec(self, v: np.ndarray) -> np.ndarray:
        """w = H_d v + (H_up x 1) v + (1 x H_dw) v + H_nd v, the serial
        product of Sec. 6.7 without MPI: the up part runs along each dw row
        (contiguous), the dw part along the strided axis, H_nd over the whole
        sector (Sec. 3.2)."""
        V = v.reshape(self.dim_dw, self.dim_up)
        Wm = self.diagonal() * V
        Wm += (self.H_up @ V.T).T
        Wm += self.H_dw @ V
        w = Wm.reshape(-1)
        if self.H_nd is not None:
            w = w + self.H_nd @ v
        return w

    def hamiltonian(self) -> sp.csr_matrix:
        """Explicit sparse sector matrix of Eq. Hbuild (small sectors)."""
        Iu = sp.identity(self.dim_up, format="csr")
        Id = sp.identity(self.dim_dw, format="csr")
        H = (sp.kron(Id, self.H_up) + sp.kron(self.H_dw, Iu)
             + sp.diags(self.diagonal().reshape(-1)))
        if self.H_nd is not None:
            H = H + self.H_nd
        return sp.csr_matrix(H)


def orbital_occupations(model, I: int) -> tuple:
    """Per-orbital electron numbers of one spin string: the impurity level of
    orbital alpha plus its Nbath bath levels (the per-orbital quantum numbers
    of Sec. 2.2, N_ud = Norb, conserved by a diagonal H^loc, a normal bath and
    the density-density interaction)."""
    out = []
    for a in range(model.norb):
        n = (I >> level_of_impurity(model, a)) & 1
        for nu in range(model.nbath):
            n += (I >> level_of_bath(model, a, nu)) & 1
        out.append(n)
    return tuple(out)


def orbital_sector_indices(model, nup, ndw, nup_orb, ndw_orb) -> np.ndarray:
    """Sector indices (i_up + i_dw D_up) of the states of S[nup, ndw] whose
    per-orbital occupations are nup_orb (up) and ndw_orb (dw): the finer
    sector of Sec. 2.2."""
    s = get_sector(model, nup, ndw)
    iu = [i for i, I in enumerate(s.map_up) if orbital_occupations(model, int(I)) == tuple(nup_orb)]
    idw = [i for i, I in enumerate(s.map_dw) if orbital_occupations(model, int(I)) == tuple(ndw_orb)]
    return np.array([u + d * s.dim_up for d in idw for u in iu], dtype=np.int64)


_SECTOR_CACHE: dict = {}


def get_sector(model, nup: int, ndw: int) -> Sector:
    key = (id(model), nup, ndw)
    s = _SECTOR_CACHE.get(key)
    if s is None or s.model is not model:
        s = Sector(model, nup, ndw)
        _SECTOR_CACHE[key] = s
    return s
