"""f1 on the GPU: the impurity Green's function at arbitrary complex
frequencies (Matsubara axis and real axis), the Dyson self-energy and local
observables, through ed_gf_lanczos_z / ed_sigma / ed_observables, against the
oracle (oracle/gf.py, oracle/observables.py) and the oracle's pins.

Tolerances: G from FP64 chains <= 1e-8 (the same 200-step algorithm on both
sides); the Dyson and observable kernels against the oracle applied to the
same G or psi <= 1e-12 relative (FP64 arithmetic of a few terms)."""
import numpy as np
import pytest
import torch

from oracle import fock, gf, lanczos, observables
from workloads import ImpurityModel, make_model, workload_ns8

pytestmark = pytest.mark.gpu


def _asym():
    """Two orbitals, spin-dependent bath, N_up != N_dw."""
    r = np.random.default_rng(64)
    b = make_model(2, 3, U=2.6, Jh=0.4, seed=64)
    return ImpurityModel(norb=2, nbath=3, U=b.U, Ust=b.Ust, Jh=b.Jh,
                         e_imp=b.e_imp + r.normal(0, .2, (2, 2)),
                         e_bath=b.e_bath + r.normal(0, .2, b.e_bath.shape),
                         v_bath=b.v_bath * r.uniform(.5, 1.5, b.v_bath.shape)), 4, 3


CASES = {"ns8": lambda: (workload_ns8().model, 4, 4), "norb2_asym": _asym}


def _ground(ed, m, nup, ndw, prec="fp64"):
    s = ed.Sector(m, nup, ndw)
    dt = torch.float32 if prec == "fp32" else torch.float64
    psi = torch.empty(s.dim, dtype=dt, device="cuda")
    r = ed.lanczos_ground(s, prec, psi=psi)
    return s, r, psi


def test_gf_z_on_the_matsubara_axis_equals_gf_lanczos(ed):
    m, nup, ndw = CASES["ns8"]()
    s, r, psi = _ground(ed, m, nup, ndw)
    G, info = ed.gf_lanczos(s, psi, r["e0"], 0, 0, "fp64", nsteps=200, beta=100.0, nmats=512)
    Gz, info_z = ed.gf_lanczos_z(s, psi, r["e0"], 0, 0, 1j * gf.matsubara(100.0, 512), "fp64")
    assert info == info_z
    assert np.abs(Gz - G).max() <= 1e-13 * np.abs(G).max()
    s.free()


@pytest.mark.parametrize("case", sorted(CASES))
def test_real_axis_gf_against_oracle(ed, case):
    """Retarded G(w + i eta) from FP64 chains against the oracle's chains, in
    every orbital and spin, at eta = 0.3 (where a 200-step chain's continued
    fraction agrees with the exact Lehmann sum to rounding: the oracle pin;
    closer to the axis the two implementations' plain-Lanczos chains, equal
    in their well-determined moments, differ in the rounding-dependent part
    after orthogonality is lost, up to 2e-4 at eta = 0.05 here); causality
    and the spectral sum rule on the GPU's values at eta = 0.05; FP32 chains
    at eta = 0.3 within the FP32 bound."""
    m, nup, ndw = CASES[case]()
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    s, r, psi = _ground(ed, m, nup, ndw)
    assert abs(r["e0"] - ro["e0"]) <= 1e-10 * abs(ro["e0"])
    w = np.linspace(-8.0, 8.0, 801)
    for spin in (0, 1):
        for orb in range(m.norb):
            Go = gf.impurity_gf_z(m, nup, ndw, ro["psi"], ro["e0"], orb, spin, w + 0.3j)
            G, _ = ed.gf_lanczos_z(s, psi, r["e0"], orb, spin, w + 0.3j, "fp64")
            assert np.abs(G - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max()), (orb, spin)
            G, _ = ed.gf_lanczos_z(s, psi, r["e0"], orb, spin, w + 0.05j, "fp64")
            assert np.all(G.imag <= 0.0)
    wide = np.linspace(-40.0, 40.0, 16001)
    G, _ = ed.gf_lanczos_z(s, psi, r["e0"], 0, 0, wide + 0.05j, "fp64")
    assert abs(-np.trapezoid(G.imag, wide) / np.pi - 1.0) < 2 * 0.05 / (np.pi * 40.0) + 1e-3
    # FP32 chains from the FP32 + polish ground state
    sp, rp, psip = _ground(ed, m, nup, ndw, "fp32_polish")
    z3 = w + 0.3j
    Go = gf.impurity_gf_z(m, nup, ndw, ro["psi"], ro["e0"], 0, 0, z3)
    G3, _ = ed.gf_lanczos_z(sp, psip, rp["e0"], 0, 0, z3, "fp32_polish")
    assert np.abs(G3 - Go).max() <= 1e-5
    s.free()
    sp.free()


@pytest.mark.parametrize("case", sorted(CASES))
def test_sigma_against_oracle_and_pins(ed, case):
    """ed_sigma against the oracle's Dyson equation applied to the same G;
    the GPU self-energy of the particle-hole symmetric Ns=8 model has
    Re Sigma = U/2; its large-|z| limit is the Hartree term of the GPU
    densities."""
    m, nup, ndw = CASES[case]()
    s, r, psi = _ground(ed, m, nup, ndw)
    ob = ed.observables(s, psi)
    z = 1j * gf.matsubara(100.0, 64)
    for spin in (0, 1):
        for orb in range(m.norb):
            G, _ = ed.gf_lanczos_z(s, psi, r["e0"], orb, spin, z, "fp64")
            S = ed.sigma(m, orb, spin, z, G)
            So = observables.self_energy(m, orb, spin, z, G)
            assert np.abs(S - So).max() <= 1e-12 * max(1.0, np.abs(So).max()), (orb, spin)
            if case == "ns8":
                assert np.abs(S.real - m.U / 2).max() < 1e-6
            zt = np.array([1e4j])
            Gt, _ = ed.gf_lanczos_z(s, psi, r["e0"], orb, spin, zt, "fp64")
            St = ed.sigma(m, orb, spin, zt, Gt)
            assert abs(St[0] - observables.hartree(m, ob["dens"], orb, spin)) < 2e-3
    s.free()


@pytest.mark.parametrize("case,prec", [("ns8", "fp64"), ("ns8", "fp32"),
                                       ("norb2_asym", "fp64"), ("norb3", "fp32_polish")])
def test_observables_against_oracle(ed, case, prec):
    """Densities, correlators and the interaction energy of the GPU ground
    state against the oracle evaluated on the same vector (and on the
    oracle's own ground state); densities equal the hole weights of the
    chains."""
    if case == "norb3":
        m, nup, ndw = make_model(3, 1, U=2.2, Jh=0.4, seed=66), 3, 3
    else:
        m, nup, ndw = CASES[case]()
    s, r, psi = _ground(ed, m, nup, ndw, prec)
    ob = ed.observables(s, psi, prec)
    p = psi.double().cpu().numpy()
    dens, nn, e_int = observables.local_observables(m, nup, ndw, p)
    assert abs(ob["norm"] - float(p @ p)) <= 1e-12
    assert np.abs(ob["dens"] - dens).max() <= 1e-12
    assert np.abs(ob["nn"] - nn).max() <= 1e-12
    assert abs(ob["e_int"] - e_int) <= 1e-12 * max(1.0, abs(e_int))
    ref = fock.Sector(m, nup, ndw)
    ro = lanczos.ground_state(ref.matvec, ref.dim)
    d_o, nn_o, e_o = observables.local_observables(m, nup, ndw, ro["psi"])
    # the FP32 ground state, polished or not, carries a residual of order 1e-5
    tol = 1e-8 if prec == "fp64" else 1e-5
    assert np.abs(ob["dens"] - d_o).max() <= tol
    assert abs(ob["e_int"] - e_o) <= tol * max(1.0, abs(e_o))
    if prec == "fp64":
        for spin in (0, 1):
            _, info = ed.gf_lanczos(s, psi, r["e0"], 0, spin, "fp64", nsteps=20, beta=10.0,
                                    nmats=4)
            assert abs(info["weight_hole"] - ob["dens"][spin, 0]) <= 1e-12
    s.free()
