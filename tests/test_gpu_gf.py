"""a7/a8 on the GPU: impurity G(i w_n) from c^+/c Lanczos chains and
continued fractions, against the oracle.

Tolerances (max |dG| over the grid): FP64 <= 1e-8; FP32 chains <= 1e-5."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import fock, gf, lanczos
from workloads import make_model, workload_ns8, workload_ns14, workload_norb2_ns14, workload_ns16

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        g = json.load(f)
    return g, np.array(g["G_re"]) + 1j * np.array(g["G_im"])


def _ground(ed, s, prec):
    psi = torch.empty(s.dim, dtype=torch.float32 if prec == "fp32" else torch.float64,
                      device="cuda")
    r = ed.lanczos_ground(s, prec, psi=psi)
    return r, psi


def test_ns8_gf_fp64(ed):
    g, Gref = _gold("oracle_ns8.json")
    s = ed.Sector(workload_ns8().model, 4, 4)
    r, psi = _ground(ed, s, "fp64")
    G, info = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=100.0, nmats=512)
    assert np.abs(G - Gref).max() <= 1e-8
    assert abs(info["weight_particle"] - g["weight_particle"]) < 1e-12
    assert abs(info["weight_hole"] - g["weight_hole"]) < 1e-12
    assert abs(info["weight_particle"] + info["weight_hole"] - 1) < 1e-12
    Gd, _ = ed.gf_lanczos(s, psi, r["e0"], 0, 1, "fp64", nsteps=200, beta=100.0, nmats=512)
    assert np.abs(Gd - G).max() <= 1e-10       # spin symmetry at N_up = N_dw
    assert np.abs(G.real).max() <= 1e-9        # particle-hole symmetric model
    s.free()


@pytest.mark.parametrize("prec", ["fp32", "fp32_polish"])
def test_ns8_gf_fp32(ed, prec):
    g, Gref = _gold("oracle_ns8.json")
    s = ed.Sector(workload_ns8().model, 4, 4)
    r, psi = _ground(ed, s, prec)
    G, _ = ed.gf_lanczos(s, psi, r["e0"], 0, 0, prec, nsteps=200, beta=100.0, nmats=512)
    assert np.abs(G - Gref).max() <= 1e-5
    s.free()


def test_ns14_gf(ed):
    g, Gref = _gold("oracle_ns14.json")
    wl = workload_ns14(0)
    s = ed.Sector(wl.model, 7, 7)
    r, psi = _ground(ed, s, "fp64")
    G, _ = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=100.0, nmats=512)
    assert np.abs(G - Gref).max() <= 1e-8
    rp, psip = _ground(ed, s, "fp32_polish")
    G2, _ = ed.gf_lanczos(s, psip, rp["e0"], 0, 0, "fp32_polish", nsteps=200, beta=100.0,
                          nmats=512)
    assert np.abs(G2 - Gref).max() <= 1e-5
    s.free()


def test_norb2_ns14_ground_and_gf(ed):
    """Two-orbital Kanamori sector (5,6), D = 6,012,006 (tiled product, many
    block pairs, N_up != N_dw): E0, psi samples and G_{0,up} against the
    oracle, FP64 and FP32 + polish."""
    g, Gref = _gold("oracle_norb2_ns14.json")
    wl = workload_norb2_ns14(0)
    s = ed.Sector(wl.model, wl.nup, wl.ndw)
    assert s.blocked_kernel() in ("tiled", "elementwise")  # chosen by the autotuner
    r, psi = _ground(ed, s, "fp64")
    assert abs(r["e0"] - g["e0"]) <= 1e-10 * abs(g["e0"])
    p = psi.cpu().numpy()
    p *= np.sign(p[np.argmax(np.abs(p))])
    idx = np.array(g["psi_index"])
    assert np.abs(p[idx] - np.array(g["psi_value"])).max() < 1e-8
    G, info = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=100.0, nmats=512)
    assert np.abs(G - Gref).max() <= 1e-8
    assert abs(info["weight_particle"] - g["weight_particle"]) < 1e-10
    assert abs(info["weight_hole"] - g["weight_hole"]) < 1e-10
    rp, psip = _ground(ed, s, "fp32_polish")
    assert abs(rp["e0"] - g["e0"]) <= 1e-10 * abs(g["e0"])
    G2, _ = ed.gf_lanczos(s, psip, rp["e0"], 0, 0, "fp32_polish", nsteps=200, beta=100.0,
                          nmats=512)
    assert np.abs(G2 - Gref).max() <= 1e-5
    s.free()


def test_ns16_benchmark_sector_against_golden(ed):
    """The Ns=16 two-orbital half-filled sector (D = 165,636,900) against the
    oracle's stored FP64 run (tests/golden/make_golden.py ns16): E0 of the
    FP64 path, of the raw FP32 Lanczos (1e-6) and of FP32 + polish (1e-10);
    256 samples of psi; G_{0,up}(i w_n) and the chain weights from FP64
    chains (1e-8) and from FP32 chains on the polished state (1e-5)."""
    g, Gref = _gold("oracle_ns16.json")
    wl = workload_ns16(0)
    s = ed.Sector(wl.model, wl.nup, wl.ndw)
    e = g["e0"]
    r, psi = _ground(ed, s, "fp64")
    assert abs(r["e0"] - e) <= 1e-10 * abs(e)
    sgn = float(torch.sign(psi[torch.argmax(psi.abs())]))
    idx = torch.tensor(g["psi_index"], device="cuda")
    assert np.abs(sgn * psi[idx].cpu().numpy() - np.array(g["psi_value"])).max() < 1e-8
    G, info = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=100.0, nmats=512)
    assert np.abs(G - Gref).max() <= 1e-8
    assert abs(info["weight_particle"] - g["weight_particle"]) < 1e-10
    assert abs(info["weight_hole"] - g["weight_hole"]) < 1e-10
    del psi
    rp, psip = _ground(ed, s, "fp32_polish")
    assert abs(rp["e0_raw"] - e) <= 1e-6 * abs(e)
    assert abs(rp["e0"] - e) <= 1e-10 * abs(e)
    G2, _ = ed.gf_lanczos(s, psip, rp["e0"], 0, 0, "fp32_polish", nsteps=200, beta=100.0,
                          nmats=512)
    # FP32 chains run on H - E0 (diagonal tables shifted before their FP32
    # rounding): 3.3e-7 here, against 1.3e-5 for chains on H itself, whose
    # diagonal entries of order |E0| = 22 round to 2^-24 |E0|
    assert np.abs(G2 - Gref).max() <= 1e-5
    s.free()


@pytest.mark.parametrize("spin", [0, 1])
def test_gf_multiorbital_asymmetric_sector(ed, spin):
    """Norb=2, N_up != N_dw, spin-dependent bath: every orbital and spin
    against the oracle chains (both chains, signs of down operators)."""
    m = make_model(2, 3, U=2.4, Jh=0.4, seed=23)
    m.e_bath[1] += 0.1
    nup, ndw = 4, 3
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s = ed.Sector(m, nup, ndw)
    r, psi = _ground(ed, s, "fp64")
    assert abs(r["e0"] - ro["e0"]) < 1e-10 * abs(ro["e0"])
    for orb in range(2):
        Go = gf.impurity_gf(m, nup, ndw, ro["psi"], ro["e0"], orb, spin, nsteps=120, nmats=64)
        G, _ = ed.gf_lanczos(s, psi, r["e0"], orb, spin, "fp64", nsteps=120, beta=100.0, nmats=64)
        assert np.abs(G - Go).max() <= 1e-8, (orb, spin)
    s.free()


@pytest.mark.parametrize("gprec", ["fp64", "fp32"])
def test_solve_batched_chains_against_oracle(ed, gprec):
    """ed_solve on small sectors runs every chain of the solve in one batched
    launch (one CTA per chain): Norb=2, N_up != N_dw, spin-dependent bath, so
    the eight chains live in four sectors of different dimension.  Every
    G_{orb,spin} against the oracle chains, and the same G twice."""
    m = make_model(2, 3, U=2.4, Jh=0.4, seed=23)
    m.e_bath[1] += 0.1
    nup, ndw = 4, 3
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    prec = "fp64" if gprec == "fp64" else "fp32_polish"
    res, G = ed.solve(m, nup, ndw, precision=prec, gf_precision=gprec, nmats=64, beta=100.0,
                      gf_steps=120)
    assert abs(res["e0"] - ro["e0"]) < 1e-10 * abs(ro["e0"])
    assert res["gf_chains"] == 8
    tol = 1e-8 if gprec == "fp64" else 1e-5
    for spin in range(2):
        for orb in range(2):
            Go = gf.impurity_gf(m, nup, ndw, ro["psi"], ro["e0"], orb, spin, nsteps=120, nmats=64)
            assert np.abs(G[spin, orb] - Go).max() <= tol, (orb, spin)
    _, G2 = ed.solve(m, nup, ndw, precision=prec, gf_precision=gprec, nmats=64, beta=100.0,
                     gf_steps=120)
    assert np.array_equal(G, G2)


def test_gf_u0_closed_form(ed):
    m = make_model(1, 5, U=0.0, e_d=0.07, seed=31)
    s = ed.Sector(m, 3, 3)
    r, psi = _ground(ed, s, "fp64")
    G, info = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=50.0, nmats=32)
    h = np.diag(fock.level_energies(m, 0))
    for nu in range(5):
        h[0, 1 + nu] = h[1 + nu, 0] = m.v_bath[0, 0, nu]
    wn = gf.matsubara(50.0, 32)
    ref = np.array([np.linalg.inv(1j * w * np.eye(6) - h)[0, 0] for w in wn])
    assert np.abs(G - ref).max() <= 1e-9
    s.free()


def test_solve_entry_point(ed):
    g, Gref = _gold("oracle_ns8.json")
    wl = workload_ns8()
    res, G = ed.solve(wl.model, 4, 4, precision="fp64", gf_precision="fp64", nmats=512)
    assert abs(res["e0"] - g["e0_dense"]) <= 1e-10 * abs(g["e0_dense"])
    assert np.abs(G[0, 0] - Gref).max() <= 1e-8
    assert np.abs(G[1, 0] - Gref).max() <= 1e-8
