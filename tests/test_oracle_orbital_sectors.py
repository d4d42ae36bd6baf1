"""Pins of the per-orbital quantum numbers (Sec. 2.2, N_ud = Norb), no GPU.

* with the density-density interaction the sector matrix has no element
  between states of different per-orbital occupations (block diagonal over
  the finer sectors), and the finer sectors partition the sector;
* the spin exchange and pair hopping break the partition (elements between
  finer sectors exist);
* the sector's E0 is the lowest of the finer sectors' E0.
"""
import itertools

import numpy as np

from oracle import fock
from workloads import ImpurityModel, make_model


def _tuples(norb, g, n):
    return [t for t in itertools.product(range(g + 1), repeat=norb) if sum(t) == n]


def test_finer_sectors_partition_and_block_diagonal():
    m = make_model(2, 2, U=2.6, Jh=0.4, seed=61)
    fock._SECTOR_CACHE.clear()
    nup, ndw = 3, 2
    H = fock.Sector(m, nup, ndw).hamiltonian().tocsr()
    label = np.full(H.shape[0], -1)
    blocks = []
    for tu in _tuples(2, 3, nup):
        for td in _tuples(2, 3, ndw):
            idx = fock.orbital_sector_indices(m, nup, ndw, tu, td)
            if idx.size:
                assert np.all(label[idx] == -1)
                label[idx] = len(blocks)
                blocks.append(idx)
    assert np.all(label >= 0)
    Hc = H.tocoo()
    assert np.all(label[Hc.row] == label[Hc.col])
    e0 = np.linalg.eigvalsh(H.toarray())[0]
    e_blocks = [np.linalg.eigvalsh(H[b][:, b].toarray())[0] for b in blocks]
    assert abs(min(e_blocks) - e0) < 1e-12


def test_exchange_breaks_the_partition():
    b = make_model(2, 2, U=2.6, Jh=0.4, seed=61)
    m = ImpurityModel(norb=2, nbath=2, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=b.e_imp,
                      e_bath=b.e_bath, v_bath=b.v_bath, Jx=0.4, Jp=0.4)
    fock._SECTOR_CACHE.clear()
    H = fock.Sector(m, 3, 3).hamiltonian().tocoo()
    a = fock.orbital_sector_indices(m, 3, 3, (2, 1), (1, 2))
    c = fock.orbital_sector_indices(m, 3, 3, (1, 2), (2, 1))
    inside = set(a.tolist())
    other = set(c.tolist())
    assert any(r in inside and k in other for r, k in zip(H.row, H.col))
