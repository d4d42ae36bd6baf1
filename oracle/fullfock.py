"""Independent checkers for the sector Hamiltonian (oracle, test only).

Neither function uses the per-spin factorisation or the helpers of
``oracle.fock``:

* ``fock_space_hamiltonian`` builds Eq. Ham1 on the whole Fock space from
  Jordan-Wigner matrices of the 2 Ns annihilation operators, mode m = a for
  (a, up) and m = Ns + a for (a, down) (the order of Sec. 2.3), the spin
  exchange and pair hopping as products of those matrices in the order
  written; only for Ns <= 6 (4**6 = 4096 states).
* ``sector_hamiltonian_statewise`` walks the sector states one by one,
  applies every term of Eq. Ham1 with the sign counted over all 2 Ns modes,
  and looks the result up in a dictionary (Ns <= 8).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _imp_level(model, a):
    return a


def _bath_level(model, a, nu):
    return model.norb + a * model.nbath + nu


def jordan_wigner_annihilators(nmodes: int):
    """c_m = Z x ... x Z x a x 1 x ... x 1 with Z on the modes below m.
    Kronecker factor order: the leftmost factor is the most significant bit,
    so bit m of the state integer is occupation of mode m."""
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |1> -> |0>
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    I2 = sp.identity(2, format="csr")
    ops = []
    for m in range(nmodes):
        M = None
        for p in range(nmodes - 1, -1, -1):
            f = I2 if p > m else (a if p == m else Z)
            M = f if M is None else sp.kron(M, f, format="csr")
        ops.append(M)
    return ops


def fock_space_hamiltonian(model):
    ns = model.ns
    if ns > 6:
        raise ValueError("full Fock space only for Ns <= 6")
    c = jordan_wigner_annihilators(2 * ns)

    def mode(level, spin):
        return level + spin * ns

    def n(m):
        return c[m].T @ c[m]

    dimF = 1 << (2 * ns)
    H = sp.csr_matrix((dimF, dimF))
    for s in range(2):
        for a in range(model.norb):
            H = H + model.e_imp[s, a] * n(mode(_imp_level(model, a), s))
            for nu in range(model.nbath):
                md = mode(_imp_level(model, a), s)
                mb = mode(_bath_level(model, a, nu), s)
                H = H + model.e_bath[s, a, nu] * n(mb)
                hop = c[md].T @ c[mb]
                H = H + model.v_bath[s, a, nu] * (hop + hop.T)
    for a in range(model.norb):
        H = H + model.U * (n(mode(a, 0)) @ n(mode(a, 1)))
        for b in range(model.norb):
            if a != b:
                H = H + model.Ust * (n(mode(a, 0)) @ n(mode(b, 1)))
    for s in range(2):
        for a in range(model.norb):
            for b in range(a + 1, model.norb):
                H = H + (model.Ust - model.Jh) * (n(mode(a, s)) @ n(mode(b, s)))
    # -J_X d+_{a up} d_{a dw} d+_{b dw} d_{b up} + J_P d+_{a up} d+_{a dw} d_{b dw} d_{b up}
    for a in range(model.norb):
        for b in range(model.norb):
            if a == b:
                continue
            au, ad = c[mode(_imp_level(model, a), 0)], c[mode(_imp_level(model, a), 1)]
            bu, bd = c[mode(_imp_level(model, b), 0)], c[mode(_imp_level(model, b), 1)]
            H = H - model.Jx * (au.T @ ad @ bd.T @ bu)
            H = H + model.Jp * (au.T @ ad.T @ bd @ bu)
    return sp.csr_matrix(H)


def sector_indices(ns: int, nup: int, ndw: int) -> np.ndarray:
    """Fock integers of S[nup, ndw] in sector order: up index fastest, both
    spin strings ascending (Eq. SectorIndxDecomp)."""
    ups = [I for I in range(1 << ns) if bin(I).count("1") == nup]
    dws = [I for I in range(1 << ns) if bin(I).count("1") == ndw]
    return np.array([u + (d << ns) for d in dws for u in ups], dtype=np.int64)


def fock_sector_block(model, nup: int, ndw: int) -> np.ndarray:
    H = fock_space_hamiltonian(model)
    idx = sector_indices(model.ns, nup, ndw)
    return H[idx][:, idx].toarray()


def sector_hamiltonian_statewise(model, nup: int, ndw: int) -> sp.csr_matrix:
    ns = model.ns
    if ns > 8:
        raise ValueError("state-by-state build only for Ns <= 8")
    idx = sector_indices(ns, nup, ndw)
    where = {int(I): k for k, I in enumerate(idx)}

    def occ(I, m):
        return (I >> m) & 1

    def hop(I, p, q):
        # c^+_p c_q on the full 2Ns-bit string, signs over all modes below
        if not occ(I, q):
            return 0, None
        s = -1 if bin(I & ((1 << q) - 1)).count("1") % 2 else 1
        I = I & ~(1 << q)
        if occ(I, p):
            return 0, None
        s *= -1 if bin(I & ((1 << p) - 1)).count("1") % 2 else 1
        return s, I | (1 << p)

    rows, cols, vals = [], [], []
    for j, J in enumerate(idx):
        J = int(J)
        diag = 0.0
        for s in range(2):
            for a in range(model.norb):
                md = _imp_level(model, a) + s * ns
                diag += model.e_imp[s, a] * occ(J, md)
                for nu in range(model.nbath):
                    mb = _bath_level(model, a, nu) + s * ns
                    diag += model.e_bath[s, a, nu] * occ(J, mb)
                    for (p, q) in ((md, mb), (mb, md)):
                        sg, I = hop(J, p, q)
                        if sg:
                            rows.append(where[I])
                            cols.append(j)
                            vals.append(sg * model.v_bath[s, a, nu])
        # spin exchange and pair hopping: one operator at a time, right to left
        for a in range(model.norb):
            for b in range(model.norb):
                if a == b:
                    continue
                for coef, ops in ((-model.Jx, ((a, 1), (a + ns, 0), (b + ns, 1), (b, 0))),
                                  (model.Jp, ((a, 1), (a + ns, 1), (b + ns, 0), (b, 0)))):
                    if coef == 0.0:
                        continue
                    I, sg = J, 1
                    for (m, create) in reversed(ops):
                        if occ(I, m) == create:
                            sg = 0
                            break
                        if bin(I & ((1 << m) - 1)).count("1") % 2:
                            sg = -sg
                        I ^= 1 << m
                    if sg:
                        rows.append(where[I])
                        cols.append(j)
                        vals.append(sg * coef)
        for a in range(model.norb):
            diag += model.U * occ(J, a) * occ(J, a + ns)
            for b in range(model.norb):
                if a != b:
                    diag += model.Ust * occ(J, a) * occ(J, b + ns)
            for b in range(a + 1, model.norb):
                for s in range(2):
                    diag += (model.Ust - model.Jh) * occ(J, a + s * ns) * occ(J, b + s * ns)
        rows.append(j)
        cols.append(j)
        vals.append(diag)
    n = len(idx)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    H.sum_duplicates()
    return H
