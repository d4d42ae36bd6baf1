"""a1/a2 on the GPU: sector LUTs, CSR and diagonal tables against the oracle.

Integer tables (strings, row pointers, columns, impurity masks) must be
bit-exact; matrix values are +-V exactly; the FP64 diagonal sums agree to
rounding (the oracle adds the same terms in a different order)."""
import math

import numpy as np
import pytest

from oracle import fock
from workloads import make_model, workload_ns8, workload_ns14, workload_ns16, ImpurityModel

pytestmark = pytest.mark.gpu


def _asym(m, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=m.norb, nbath=m.nbath, U=m.U, Ust=m.Ust, Jh=m.Jh,
                         e_imp=m.e_imp + r.normal(0, .2, (2, m.norb)),
                         e_bath=m.e_bath + r.normal(0, .2, m.e_bath.shape),
                         v_bath=m.v_bath * r.uniform(.5, 1.5, m.v_bath.shape))


CASES = [
    (make_model(1, 0, U=1.0, seed=1), 1, 0),          # Ns=1, one state per spin
    (make_model(1, 3, U=2.0, seed=2), 0, 4),          # empty / full spin strings
    (make_model(2, 2, U=2.0, Jh=0.3, seed=3), 3, 2),
    (make_model(3, 1, U=2.0, Jh=0.3, seed=4), 2, 4),
    (make_model(3, 2, U=2.0, Jh=0.3, seed=5), 4, 5),  # Norb=3, Ns=9
    (workload_ns8().model, 4, 4),
    (make_model(2, 4, U=3.0, Jh=0.5, seed=6), 5, 4),  # Ns=10
]


def _check_spin(E_tables, ref_map, H, Ed, mask):
    t = E_tables
    assert np.array_equal(t["map"].astype(np.int64), ref_map)
    assert np.array_equal(t["imask"].astype(np.int64), mask)
    assert np.array_equal(t["rowptr"], H.indptr.astype(np.int32))
    assert np.array_equal(t["col"], H.indices.astype(np.int32))
    assert np.array_equal(t["val"], H.data)
    assert np.abs(t["ediag"] - Ed).max(initial=0) <= 1e-13 * max(1.0, np.abs(Ed).max(initial=0))


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_luts_and_csr_bit_exact(ed, ci):
    m, nup, ndw = CASES[ci]
    m = _asym(m, ci)
    s = ed.Sector(m, nup, ndw)
    ref = fock.Sector(m, nup, ndw)
    assert s.dim_up == math.comb(m.ns, nup) and s.dim_dw == math.comb(m.ns, ndw)
    _check_spin(s.tables(0), ref.map_up, ref.H_up, ref.E_up, ref.m_up)
    _check_spin(s.tables(1), ref.map_dw, ref.H_dw, ref.E_dw, ref.m_dw)
    assert np.abs(s.wtable() - ref.W).max() <= 1e-14 * max(1, abs(m.U))
    s.free()


@pytest.mark.parametrize("maker,n", [(workload_ns14, 7), (workload_ns16, 8)])
def test_large_spin_tables(ed, maker, n):
    """Full-size spin tables of the Ns=14 and Ns=16 workloads."""
    wl = maker(0)
    s = ed.Sector(wl.model, n, n)
    ref_map = fock.build_sector_map(wl.model.ns, n)
    H = fock.spin_hopping_matrix(wl.model, 0, n, ref_map)
    Ed, mask = fock.spin_diagonal(wl.model, 0, n, ref_map)
    _check_spin(s.tables(0), ref_map, H, Ed, mask)
    assert s.dim == wl.dim
    s.free()


def test_ns18_tables_properties(ed):
    """Ns=18 (D_sigma = 48,620): strings ascending with 9 bits, columns sorted
    and in range, H symmetric, nnz from the closed form."""
    from workloads import workload_ns18
    wl = workload_ns18(0)
    s = ed.Sector(wl.model, 9, 9)
    t = s.tables(0)
    mp = t["map"].astype(np.int64)
    assert len(mp) == 48620 and np.all(np.diff(mp) > 0)
    assert all(bin(int(x)).count("1") == 9 for x in mp[::97])
    nnz = 3 * 5 * 2 * math.comb(16, 8)
    assert len(t["col"]) == nnz and t["rowptr"][-1] == nnz
    import scipy.sparse as sp
    H = sp.csr_matrix((t["val"], t["col"], t["rowptr"]), shape=(48620, 48620))
    assert abs(H - H.T).max() == 0
    assert s.dim == 2363904400
    s.free()


def test_invalid_arguments(ed):
    m = make_model(1, 3, U=1.0, seed=1)
    with pytest.raises(ed.EDError) as e:
        ed.Sector(m, 5, 1)
    assert e.value.status == ed.ED_ERR_ARG
    m2 = make_model(1, 3, U=1.0, seed=1)
    m2.Jx = 0.1   # one orbital: no spin exchange term, the sector builds
    ed.Sector(m2, 2, 2).free()
    m3 = make_model(6, 1, U=1.0, seed=1)   # Norb above ED_MAX_NORB
    with pytest.raises(ed.EDError) as e:
        ed.Sector(m3, 2, 2)
    assert e.value.status == ed.ED_ERR_UNSUPPORTED
