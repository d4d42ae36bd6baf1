"""f3 per-orbital sectors on the GPU (ed_lanczos_ground_orbital): the ground
state of every finer sector of a two-orbital and a three-orbital sector
against the oracle's submatrix (E0 <= 1e-10 relative, psi up to its sign,
zero outside the finer sector); the lowest finer-sector E0 of the Ns = 16
benchmark sector equals the oracle's stored E0 of the whole sector."""
import itertools
import json
import os

import numpy as np
import pytest
import torch

from oracle import fock
from workloads import ImpurityModel, make_model, workload_ns16

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tuples(norb, g, n):
    return [t for t in itertools.product(range(g + 1), repeat=norb) if sum(t) == n]


def _asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


@pytest.mark.parametrize("norb,nbath,nup,ndw", [(2, 3, 4, 3), (3, 2, 4, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32_polish"])
def test_finer_sectors_against_oracle(ed, norb, nbath, nup, ndw, prec):
    m = _asym(make_model(norb, nbath, U=2.5, Jh=0.4, seed=60 + norb), 60 + norb)
    fock._SECTOR_CACHE.clear()
    H = fock.Sector(m, nup, ndw).hamiltonian().tocsr()
    s = ed.Sector(m, nup, ndw)
    e_all = []
    for tu in _tuples(norb, nbath + 1, nup):
        for td in _tuples(norb, nbath + 1, ndw):
            idx = fock.orbital_sector_indices(m, nup, ndw, tu, td)
            if idx.size == 0:
                with pytest.raises(ed.EDError):
                    ed.orbital_sector_dims(s, tu, td)
                continue
            du, dd = ed.orbital_sector_dims(s, tu, td)
            assert du * dd == idx.size
            E, V = np.linalg.eigh(H[idx][:, idx].toarray())
            psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
            r = ed.lanczos_ground_orbital(s, tu, td, prec, psi=psi)
            assert abs(r["e0"] - E[0]) <= 1e-10 * max(1.0, abs(E[0])), (tu, td)
            p = psi.cpu().numpy()
            mask = np.ones(s.dim, bool)
            mask[idx] = False
            assert np.all(p[mask] == 0.0)
            if idx.size > 1 and E[1] - E[0] > 1e-6:
                tol = 1e-8 if prec == "fp64" else 1e-4
                assert abs(abs(float(p[idx] @ V[:, 0])) - 1.0) < tol
            e_all.append(r["e0"])
    e0 = np.linalg.eigvalsh(H.toarray())[0]
    assert abs(min(e_all) - e0) <= 1e-10 * abs(e0)
    s.free()


def test_ns16_finer_sectors_reach_the_golden_e0(ed):
    with open(os.path.join(GOLD, "oracle_ns16.json")) as f:
        g = json.load(f)
    wl = workload_ns16(0)
    s = ed.Sector(wl.model, wl.nup, wl.ndw)
    best = np.inf
    for tu in _tuples(2, 8, 8):
        for td in _tuples(2, 8, 8):
            r = ed.lanczos_ground_orbital(s, tu, td, "fp32_polish")
            best = min(best, r["e0"])
    assert abs(best - g["e0"]) <= 1e-10 * abs(g["e0"])
    s.free()


def test_exchange_is_refused(ed):
    b = make_model(2, 2, U=2.5, Jh=0.4, seed=3)
    m = ImpurityModel(norb=2, nbath=2, U=b.U, Ust=b.Ust, Jh=b.Jh, e_imp=b.e_imp,
                      e_bath=b.e_bath, v_bath=b.v_bath, Jx=0.3, Jp=0.0)
    s = ed.Sector(m, 3, 3)
    with pytest.raises(ed.EDError) as e:
        ed.lanczos_ground_orbital(s, (2, 1), (1, 2))
    assert e.value.status == ed.ED_ERR_UNSUPPORTED
    s.free()
