"""Pins of the CPU oracle against things other than itself (no GPU).

Each test ties one oracle function to brute force, a closed form, a symmetry
of the model or a library routine, so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fock, fullfock, gf, lanczos, observables
from workloads import (SplitMix64, make_model, splitmix64_uniform_array,
                       workload_ns8, ImpurityModel)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    want = [int(x[0]) for x in _golden_ints("splitmix64_seed1234567.txt")]
    r = SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == want
    u = splitmix64_uniform_array(1234567, 5)
    assert np.array_equal(u, np.array([(w >> 11) * 2.0 ** -53 for w in want]))


# ---------------------------------------------------------------- a1: LUTs

@pytest.mark.parametrize("ns", range(1, 15))
def test_sector_map_counts_and_order(ns):
    for n in range(ns + 1):
        m = fock.build_sector_map(ns, n)
        assert len(m) == math.comb(ns, n)
        assert np.all(np.diff(m) > 0)
        assert all(bin(int(x)).count("1") == n for x in m)


@pytest.mark.parametrize("ns,n", [(8, 4), (10, 3), (12, 6), (14, 7), (16, 8), (18, 9)])
def test_rank_is_colex_combinatorial_number(ns, n):
    """rank(I) = sum_k C(p_k, k) over the set bits p_1 < ... < p_n equals the
    position in the ascending map (Sec. 6.3); checked for every state."""
    m = fock.build_sector_map(ns, n)
    for idx in range(0, len(m), max(1, len(m) // 3000)):
        I = int(m[idx])
        pos = [p for p in range(ns) if (I >> p) & 1]
        r = sum(math.comb(p, k + 1) for k, p in enumerate(pos))
        assert r == idx
        assert fock.binary_search(m, I) == idx
    assert fock.binary_search(m, (1 << ns) - 1 if n != ns else 0) == -1 or n in (0, ns)


def test_rank_matches_itertools_colex_small():
    ns, n = 9, 4
    combos = sorted(itertools.combinations(range(ns), n), key=lambda c: sum(1 << p for p in c))
    m = fock.build_sector_map(ns, n)
    assert [sum(1 << p for p in c) for c in combos] == [int(x) for x in m]


def test_workload_sector_dimensions():
    rows = _golden_ints("sector_dimensions.txt")
    for ns, nup, ndw, d in rows:
        ns, nup, ndw, d = int(ns), int(nup), int(ndw), int(d)
        assert math.comb(ns, nup) * math.comb(ns, ndw) == d
    for ns, nup, ndw, d in rows[:2]:
        assert len(fock.build_sector_map(int(ns), int(nup))) ** 2 == int(d)


# ---------------------------------------------------------------- a2: H

def _small_models():
    return [
        make_model(1, 5, U=2.7, e_d=-1.1, seed=11),
        make_model(2, 2, U=3.1, Jh=0.6, seed=12),
        make_model(3, 1, U=2.2, Jh=0.3, seed=13),
    ]


def _spin_asym(model, seed):
    r = np.random.default_rng(seed)
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp + r.normal(0, .2, (2, model.norb)),
                         e_bath=model.e_bath + r.normal(0, .2, model.e_bath.shape),
                         v_bath=model.v_bath * r.uniform(.5, 1.5, model.v_bath.shape))


@pytest.mark.parametrize("mi", range(3))
def test_sector_blocks_equal_jordan_wigner_fock_space(mi):
    """Every sector block of the whole-Fock-space Hamiltonian built from
    Jordan-Wigner operators equals the spin-factorised sector matrix."""
    m = _spin_asym(_small_models()[mi], mi)
    H = fullfock.fock_space_hamiltonian(m)
    ns = m.ns
    for nup in range(ns + 1):
        for ndw in range(ns + 1):
            idx = fullfock.sector_indices(ns, nup, ndw)
            B = H[idx][:, idx].toarray()
            A = fock.Sector(m, nup, ndw).hamiltonian().toarray()
            assert np.abs(A - B).max() < 1e-13, (nup, ndw)
    # sectors do not couple
    n_up = np.array([bin(I & ((1 << ns) - 1)).count("1") for I in range(1 << 2 * ns)])
    n_dw = np.array([bin(I >> ns).count("1") for I in range(1 << 2 * ns)])
    Hc = H.tocoo()
    assert np.all(n_up[Hc.row] == n_up[Hc.col]) and np.all(n_dw[Hc.row] == n_dw[Hc.col])


def test_statewise_sector_matrix_ns8():
    wl = workload_ns8()
    m = _spin_asym(wl.model, 5)
    for (nu, nd) in [(4, 4), (3, 5), (5, 2)]:
        A = fock.Sector(m, nu, nd).hamiltonian()
        B = fullfock.sector_hamiltonian_statewise(m, nu, nd)
        assert abs(A - B).max() < 1e-13
        assert abs(A - A.T).max() == 0.0


def test_factorised_matvec_equals_explicit_matrix():
    m = _spin_asym(make_model(2, 3, U=2.0, Jh=0.3, seed=7), 1)
    s = fock.Sector(m, 3, 5)
    v = np.random.default_rng(0).normal(size=s.dim)
    B = fullfock.sector_hamiltonian_statewise(m, 3, 5)
    assert np.abs(s.matvec(v) - B @ v).max() < 1e-12


# ---------------------------------------------------------------- E0

def _lanczos_e0(m, nup, ndw, tol=1e-12):
    s = fock.Sector(m, nup, ndw)
    r = lanczos.lanczos_ground(s.matvec, lanczos.start_vector(0x5EED, s.dim), tol=tol)
    return r["e0"], s


def test_e0_equals_dense_eigh_ns8():
    wl = workload_ns8()
    e0, s = _lanczos_e0(wl.model, 4, 4)
    ex = np.linalg.eigvalsh(s.hamiltonian().toarray())[0]
    assert abs(e0 - ex) <= 1e-12 * abs(ex)


def _one_body(m, spin):
    ns = m.ns
    h = np.diag(fock.level_energies(m, spin))
    for a in range(m.norb):
        for nu in range(m.nbath):
            i, j = fock.level_of_impurity(m, a), fock.level_of_bath(m, a, nu)
            h[i, j] = h[j, i] = m.v_bath[spin, a, nu]
    return h


@pytest.mark.parametrize("norb,nbath,nup,ndw", [(1, 7, 4, 4), (1, 7, 3, 5), (2, 3, 4, 3), (3, 2, 4, 5)])
def test_e0_u0_closed_form(norb, nbath, nup, ndw):
    """U = U' = J = 0: E0 is the sum of the lowest N_up (N_dw) eigenvalues of
    the Ns x Ns one-body matrix of each spin."""
    m = _spin_asym(make_model(norb, nbath, U=0.0, Jh=0.0, e_d=0.13, seed=21), 3)
    e0, _ = _lanczos_e0(m, nup, ndw)
    eu = np.linalg.eigvalsh(_one_body(m, 0))
    ed = np.linalg.eigvalsh(_one_body(m, 1))
    ref = eu[:nup].sum() + ed[:ndw].sum()
    assert abs(e0 - ref) <= 1e-11 * max(1, abs(ref))


@pytest.mark.parametrize("norb,nbath,nup,ndw", [(1, 7, 4, 4), (2, 3, 4, 3), (3, 2, 5, 4)])
def test_e0_atomic_limit(norb, nbath, nup, ndw):
    """V = 0: minimise over impurity occupations the impurity energy plus the
    lowest remaining bath levels of each spin."""
    m0 = make_model(norb, nbath, U=2.5, Jh=0.4, seed=31)
    m = ImpurityModel(norb=norb, nbath=nbath, U=m0.U, Ust=m0.Ust, Jh=m0.Jh, e_imp=m0.e_imp,
                      e_bath=m0.e_bath, v_bath=np.zeros_like(m0.v_bath))
    s = fock.Sector(m, nup, ndw)
    e_min = np.inf
    for mu in range(1 << norb):
        for md in range(1 << norb):
            ku, kd = bin(mu).count("1"), bin(md).count("1")
            if ku > nup or kd > ndw or nup - ku > norb * nbath or ndw - kd > norb * nbath:
                continue
            e = 0.0
            for a in range(norb):
                nau, nad = (mu >> a) & 1, (md >> a) & 1
                e += m.e_imp[0, a] * nau + m.e_imp[1, a] * nad + m.U * nau * nad
                for b in range(norb):
                    if b != a:
                        e += m.Ust * nau * ((md >> b) & 1)
                for b in range(a + 1, norb):
                    e += (m.Ust - m.Jh) * (nau * ((mu >> b) & 1) + nad * ((md >> b) & 1))
            e += np.sort(m.e_bath[0].ravel())[:nup - ku].sum()
            e += np.sort(m.e_bath[1].ravel())[:ndw - kd].sum()
            e_min = min(e_min, e)
    assert abs(s.diagonal().min() - e_min) < 1e-12
    assert abs(s.H_up).max() == 0 and abs(s.H_dw).max() == 0


def test_twin_and_particle_hole_symmetry():
    """Spin-symmetric model: E(N_up,N_dw) = E(N_dw,N_up).  The Ns=8 workload
    is particle-hole symmetric (e_d = -U/2, bath grid symmetric about 0,
    equal V): E(N_up,N_dw) = E(Ns-N_up, Ns-N_dw)."""
    wl = workload_ns8()
    m = wl.model
    e35, _ = _lanczos_e0(m, 3, 5)
    e53, _ = _lanczos_e0(m, 5, 3)
    e53b, _ = _lanczos_e0(m, 5, 3)
    assert abs(e35 - e53) < 1e-11
    e34, _ = _lanczos_e0(m, 3, 4)
    e54, _ = _lanczos_e0(m, 5, 4)
    assert abs(e34 - e54) < 1e-11
    assert e53 == e53b


# ---------------------------------------------------------------- tridiagonal

@pytest.mark.parametrize("k", [1, 2, 7, 64, 300])
def test_tridiagonal_eigenpair_against_lapack(k):
    r = np.random.default_rng(k)
    a = r.normal(size=k)
    b = np.concatenate([[0.0], np.abs(r.normal(size=k - 1)) + 0.05])
    th = lanczos.tridiag_lowest(a, b)
    w, V = sla.eigh_tridiagonal(a, b[1:])
    assert abs(th - w[0]) <= 1e-13 * max(1, abs(w[0]))
    y = lanczos.tridiag_vector(a, b, th)
    ref = V[:, 0] * np.sign(V[int(np.argmax(np.abs(V[:, 0]))), 0])
    assert np.abs(y - ref).max() < 1e-9


def test_ground_vector_residual_and_dense_ns8():
    wl = workload_ns8()
    s = fock.Sector(wl.model, 4, 4)
    r = lanczos.ground_state(s.matvec, s.dim)
    e, res = lanczos.rayleigh_residual(s.matvec, r["psi"])
    assert res < 1e-10
    E, U = np.linalg.eigh(s.hamiltonian().toarray())
    assert abs(abs(U[:, 0] @ r["psi"]) - 1.0) < 1e-12


def test_alpha_by_linearity_matches_paige_form():
    """The CUDA path forms alpha_j = <v_j, H v_j> - beta_j <v_j, v_{j-1}>
    (with the computed <v_j, v_{j-1}>) and the vector update w = H v_j -
    beta_j v_{j-1} - alpha_j v_j; the oracle uses alpha_j = <v_j, H v_j -
    beta_j v_{j-1}>.  Both, written out here in FP64 on the Ns=8 sector,
    give the same coefficients to rounding over 40 steps (well past the
    loss of orthogonality of the plain recurrence), and the oracle's own
    routine gives the same first coefficients."""
    wl = workload_ns8()
    s = fock.Sector(wl.model, 4, 4)
    v0 = lanczos.start_vector(0x5EED, s.dim)
    steps = 40

    def run(linear):
        v = v0 / np.linalg.norm(v0)
        vp = np.zeros_like(v)
        a_s, b_s, c = [], [0.0], 0.0
        for j in range(steps):
            hv = s.matvec(v)
            if linear:
                a = float(v @ hv) - b_s[j] * c
                w = hv - b_s[j] * vp - a * v
            else:
                w = hv - b_s[j] * vp
                a = float(v @ w)
                w = w - a * v
            b = float(np.linalg.norm(w))
            c = float(w @ v) / b     # <v_{j+1}, v_j>
            a_s.append(a)
            b_s.append(b)
            vp, v = v, w / b
        return np.array(a_s), np.array(b_s[1:])

    a_lin, b_lin = run(True)
    a_pai, b_pai = run(False)
    scale = max(np.abs(a_pai).max(), b_pai.max())
    assert np.abs(a_lin - a_pai).max() <= 1e-12 * scale
    assert np.abs(b_lin - b_pai).max() <= 1e-12 * scale
    r = lanczos.lanczos_ground(s.matvec, v0, maxit=steps, tol=0.0)
    k = min(10, len(r["alpha"]))
    assert np.abs(r["alpha"][:k] - a_pai[:k]).max() <= 1e-12 * scale


# ---------------------------------------------------------------- a7: c, c^+

@pytest.mark.parametrize("spin", [0, 1])
@pytest.mark.parametrize("create", [+1, -1])
def test_creation_annihilation_against_jordan_wigner(spin, create):
    m = _spin_asym(make_model(2, 2, U=1.0, Jh=0.2, seed=41), 9)
    ns = m.ns
    nup, ndw = 3, 2
    src = fullfock.sector_indices(ns, nup, ndw)
    psi = np.random.default_rng(1).normal(size=len(src))
    c = fullfock.jordan_wigner_annihilators(2 * ns)
    full = np.zeros(1 << 2 * ns)
    full[src] = psi
    for orb in range(m.norb):
        mode = fock.level_of_impurity(m, orb) + spin * ns
        op = c[mode].T if create > 0 else c[mode]
        out_full = op @ full
        phi, (nu2, nd2) = gf._apply(m, psi, nup, ndw, orb, spin, create)
        dst = fullfock.sector_indices(ns, nu2, nd2)
        assert np.abs(out_full[dst] - phi).max() == 0.0
        assert np.abs(np.delete(out_full, dst)).max() == 0.0


# ---------------------------------------------------------------- a8: G(iw)

def test_gf_u0_closed_form():
    """U = 0: G_{dd}(i w) = [(i w - h)^-1]_{dd} with h the one-body matrix;
    the chain breaks down within Ns steps so the continued fraction is exact."""
    m = _spin_asym(make_model(1, 7, U=0.0, e_d=0.05, seed=51), 4)
    s = fock.Sector(m, 4, 4)
    r = lanczos.ground_state(s.matvec, s.dim)
    wn = gf.matsubara(100.0, 64)
    for spin in (0, 1):
        G = gf.impurity_gf(m, 4, 4, r["psi"], r["e0"], 0, spin, nmats=64)
        h = _one_body(m, spin)
        ref = np.array([np.linalg.inv(1j * w * np.eye(m.ns) - h)[0, 0] for w in wn])
        assert np.abs(G - ref).max() < 1e-9


def test_gf_lehmann_symmetry_and_sum_rule_ns8():
    wl = workload_ns8()
    m = wl.model
    s = fock.Sector(m, 4, 4)
    r = lanczos.ground_state(s.matvec, s.dim)
    G, parts = gf.impurity_gf(m, 4, 4, r["psi"], r["e0"], 0, 0, return_parts=True)
    Gx, e0x = gf.lehmann_gf_dense(m, 4, 4, 0, 0)
    assert abs(r["e0"] - e0x) < 1e-12 * abs(e0x)
    assert np.abs(G - Gx).max() < 1e-10
    assert np.abs(G.real).max() < 1e-10          # particle-hole symmetry
    assert abs(parts[1][0] + parts[-1][0] - 1.0) < 1e-12   # <c c^+ + c^+ c> = 1
    wn = gf.matsubara(0.01, 4)                   # far tail: i w G -> 1
    Gt = gf.impurity_gf(m, 4, 4, r["psi"], r["e0"], 0, 0, beta=0.01, nmats=4)
    assert np.abs(1j * wn * Gt - 1.0).max() < 1e-3
    Gd = gf.impurity_gf(m, 4, 4, r["psi"], r["e0"], 0, 1)
    assert np.abs(G - Gd).max() < 1e-10          # spin symmetry at N_up = N_dw


# ---------------------------------------------------------------- f1: Sigma, real axis, observables

def _u0(m):
    """The same model with every interaction switched off."""
    return ImpurityModel(norb=m.norb, nbath=m.nbath, U=0.0, Ust=0.0, Jh=0.0, e_imp=m.e_imp,
                         e_bath=m.e_bath, v_bath=m.v_bath)


def test_g0_inverse_is_schur_complement_of_one_body_matrix():
    """1 / G0^-1(z) of the normal bath equals [(z - h)^-1]_{dd} of the
    one-body matrix h (an independent route: a dense inverse)."""
    m = _spin_asym(make_model(2, 3, U=2.0, Jh=0.3, seed=61), 61)
    z = np.array([0.3j, 1.7j, 0.4 + 0.05j, -1.1 + 0.2j])
    for spin in (0, 1):
        h = _one_body(m, spin)
        for orb in range(m.norb):
            d = fock.level_of_impurity(m, orb)
            ref = np.array([np.linalg.inv(x * np.eye(m.ns) - h)[d, d] for x in z])
            got = 1.0 / observables.g0_inverse(m, orb, spin, z)
            assert np.abs(got - ref).max() < 1e-12


def test_sigma_vanishes_without_interaction():
    """U = U' = J = 0: the chains span their Krylov spaces exactly, so G = G0
    and the Dyson self-energy is zero."""
    m = _spin_asym(make_model(2, 3, U=0.0, Jh=0.0, Ust=0.0, seed=62), 62)
    s = fock.Sector(m, 4, 3)
    r = lanczos.ground_state(s.matvec, s.dim)
    z = 1j * gf.matsubara(50.0, 64)
    for spin in (0, 1):
        for orb in range(m.norb):
            G = gf.impurity_gf_z(m, 4, 3, r["psi"], r["e0"], orb, spin, z)
            S = observables.self_energy(m, orb, spin, z, G)
            assert np.abs(S).max() < 1e-7, (orb, spin)


def test_sigma_particle_hole_symmetry_ns8():
    """Particle-hole symmetric single-orbital model at half filling
    (e_d = -U/2, symmetric bath): Re Sigma(i w_n) = U / 2 at every n."""
    wl = workload_ns8()
    m = wl.model
    s = fock.Sector(m, 4, 4)
    r = lanczos.ground_state(s.matvec, s.dim)
    z = 1j * gf.matsubara(100.0, 128)
    G = gf.impurity_gf_z(m, 4, 4, r["psi"], r["e0"], 0, 0, z)
    S = observables.self_energy(m, 0, 0, z, G)
    assert np.abs(S.real - m.U / 2).max() < 1e-9
    assert np.all(S.imag <= 1e-12)              # causal: Im Sigma(i w) <= 0


@pytest.mark.parametrize("case", ["ns8", "norb2_asym"])
def test_sigma_hartree_tail(case):
    """At large |z| the self-energy tends to its first moment, the Hartree
    term U<n_{a,-s}> + U' sum <n_{b,-s}> + (U'-J) sum <n_{b,s}>; the next
    term falls as 1/|z|."""
    if case == "ns8":
        m, nup, ndw = workload_ns8().model, 4, 4
    else:
        m, nup, ndw = _spin_asym(make_model(2, 3, U=2.6, Jh=0.4, seed=63), 63), 4, 3
    s = fock.Sector(m, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    dens, _, _ = observables.local_observables(m, nup, ndw, r["psi"])
    z = np.array([1e4j, 2e4j])
    for spin in (0, 1):
        for orb in range(m.norb):
            G = gf.impurity_gf_z(m, nup, ndw, r["psi"], r["e0"], orb, spin, z)
            S = observables.self_energy(m, orb, spin, z, G)
            h = observables.hartree(m, dens, orb, spin)
            err = np.abs(S - h)
            assert err[0] < 2e-3 and err[1] < 0.6 * err[0] + 1e-9, (orb, spin, err)


def test_real_axis_gf_lehmann_causality_and_sum_rule():
    """The real-axis G(w + i eta) of the 200-step chains against the exact
    Lehmann sum (dense eigenvectors) on the Ns=8 sector: equal to rounding
    for eta = 0.3 (the continued fraction of a 200-step chain converges
    quickly a distance eta from the real axis; at eta = 0.05 the two differ
    by 6e-4 near the poles, as a 200-step chain does not span the 3920-state
    Krylov space: reading 15), Im G <= 0 everywhere, and the spectral sum rule
    -1/pi int Im G(w + i eta) dw = n+ + n- = 1 (the Lorentzian tails beyond
    |w| = 40 cut 2 eta / (pi 40) at most)."""
    wl = workload_ns8()
    m = wl.model
    s = fock.Sector(m, 4, 4)
    r = lanczos.ground_state(s.matvec, s.dim)
    w = np.linspace(-10.0, 10.0, 2001)
    G3 = gf.impurity_gf_z(m, 4, 4, r["psi"], r["e0"], 0, 0, w + 0.3j)
    Gx, _ = gf.lehmann_gf_dense_z(m, 4, 4, 0, 0, w + 0.3j)
    assert np.abs(G3 - Gx).max() < 1e-11
    eta = 0.05
    w = np.linspace(-40.0, 40.0, 16001)
    G = gf.impurity_gf_z(m, 4, 4, r["psi"], r["e0"], 0, 0, w + 1j * eta)
    assert np.all(G.imag <= 0.0)
    weight = -np.trapezoid(G.imag, w) / np.pi
    assert abs(weight - 1.0) < 2 * eta / (np.pi * 40.0) + 1e-3


def test_local_observables_pins():
    """Densities equal the hole weights ||c_{a s} psi||^2 of the chains (the
    operators of Sec. 2.3, an independent route); particle-hole symmetry
    gives n = 1/2; without interaction the two spins are uncorrelated,
    <n_up n_dw> = <n_up><n_dw>; the interaction energy equals E0 minus the
    energy of the same state under the model with every interaction
    switched off; in the atomic limit (V = 0) the double occupancy is 0 or
    1."""
    # densities vs chain weights, and E_int, on an asymmetric two-orbital sector
    m = _spin_asym(make_model(2, 3, U=2.6, Jh=0.4, seed=64), 64)
    nup, ndw = 4, 3
    s = fock.Sector(m, nup, ndw)
    r = lanczos.ground_state(s.matvec, s.dim)
    psi = r["psi"]
    dens, nn, e_int = observables.local_observables(m, nup, ndw, psi)
    for spin in (0, 1):
        for orb in range(m.norb):
            phi, _ = gf._apply(m, psi, nup, ndw, orb, spin, -1)
            assert abs(dens[spin, orb] - float(phi @ phi)) < 1e-12
            assert abs(nn[spin, spin, orb, orb] - dens[spin, orb]) < 1e-12   # n^2 = n
    s0 = fock.Sector(_u0(m), nup, ndw)
    e_free = float(psi @ s0.matvec(psi))
    assert abs(r["e0"] - e_free - e_int) < 1e-10 * max(1.0, abs(r["e0"]))
    # particle-hole symmetric single orbital at half filling
    wl = workload_ns8()
    s8 = fock.Sector(wl.model, 4, 4)
    r8 = lanczos.ground_state(s8.matvec, s8.dim)
    d8, nn8, _ = observables.local_observables(wl.model, 4, 4, r8["psi"])
    assert np.abs(d8 - 0.5).max() < 1e-10
    assert 0.0 < nn8[0, 1, 0, 0] < 0.25          # U > 0 suppresses double occupancy
    # no interaction: spins uncorrelated
    mu = _u0(m)
    su = fock.Sector(mu, nup, ndw)
    ru = lanczos.ground_state(su.matvec, su.dim)
    du, nnu, eu = observables.local_observables(mu, nup, ndw, ru["psi"])
    assert eu == 0.0
    for a in range(m.norb):
        for b in range(m.norb):
            assert abs(nnu[0, 1, a, b] - du[0, a] * du[1, b]) < 1e-9
    # atomic limit: integer double occupancy
    ma = ImpurityModel(norb=1, nbath=3, U=1.5, Ust=1.5, Jh=0.0, e_imp=np.array([-0.4]),
                       e_bath=np.array([[-0.9, 0.2, 0.8]]), v_bath=np.zeros((1, 3)))
    sa = fock.Sector(ma, 2, 1)
    E, U = np.linalg.eigh(sa.hamiltonian().toarray())
    assert E[1] - E[0] > 1e-6                    # a non-degenerate ground state
    _, nna, _ = observables.local_observables(ma, 2, 1, U[:, 0])
    assert min(abs(nna[0, 1, 0, 0]), abs(nna[0, 1, 0, 0] - 1.0)) < 1e-12
