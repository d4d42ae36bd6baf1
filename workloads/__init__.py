"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method (no Hamiltonian, no Lanczos, no
Green's function). It only draws numbers and packages model parameters:

* ``SplitMix64`` — the 64-bit generator of Steele, Lea and Flood ("Fast
  splittable pseudorandom number generators", OOPSLA 2014), in the form given
  by S. Vigna's public-domain ``splitmix64.c``: state += 0x9E3779B97F4A7C15,
  then the mixing function with multipliers 0xBF58476D1CE4E5B9 and
  0x94D049BB133111EB and shifts 30, 27, 31.  Uniform doubles are the top 53
  bits times 2**-53.
* ``ImpurityModel`` — the parameters of the density-density Anderson impurity
  Hamiltonian (Eq. Ham1 with J_X = J_P = 0, diagonal H^loc and h, "normal"
  bath: every impurity orbital has its own Nbath levels, Sec. 6.4).
* the benchmark recipes: the paper's protocol (random bath energies in
  [-2, 2], half filling, several bath realisations, Sec. 5) made concrete for
  the five workloads used here.

Bath draw order (one reading of the paper, which gives no generator): for
orbital alpha, for bath level nu: first the energy, then the hybridisation.
The bath is spin independent unless a caller builds a model by hand.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    """Output function of SplitMix64 applied to a 64-bit state value."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        return splitmix64_mix(self.state)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


def splitmix64_uniform_array(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Element i is the uniform double from output number (offset + i) of a
    SplitMix64 stream started at ``seed`` (counter-based form: the state
    before mixing is seed + (offset + i + 1) * gamma mod 2**64)."""
    i = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (i + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class ImpurityModel:
    """Density-density Anderson impurity model with a normal bath.

    Arrays are spin resolved: ``e_imp[s, a]``, ``e_bath[s, a, nu]``,
    ``v_bath[s, a, nu]`` with s = 0 (up), 1 (down).  ``Ust`` is U' and the
    same-spin inter-orbital coupling is ``Ust - Jh`` (Eq. Ham1).
    """

    norb: int
    nbath: int
    U: float
    Ust: float
    Jh: float
    e_imp: np.ndarray
    e_bath: np.ndarray
    v_bath: np.ndarray
    Jx: float = 0.0
    Jp: float = 0.0
    name: str = ""

    @property
    def ns(self) -> int:
        return self.norb * (self.nbath + 1)

    def __post_init__(self):
        self.e_imp = np.ascontiguousarray(np.broadcast_to(
            np.asarray(self.e_imp, dtype=np.float64), (2, self.norb)))
        self.e_bath = np.ascontiguousarray(np.broadcast_to(
            np.asarray(self.e_bath, dtype=np.float64), (2, self.norb, self.nbath)))
        self.v_bath = np.ascontiguousarray(np.broadcast_to(
            np.asarray(self.v_bath, dtype=np.float64), (2, self.norb, self.nbath)))


def half_filling_ed(norb: int, U: float, Ust: float, Jh: float) -> float:
    """Impurity level at the particle-hole symmetric point of the
    density-density interaction: -(U + (norb-1)(2U' - J)) / 2."""
    return -0.5 * (U + (norb - 1) * (2.0 * Ust - Jh))


def random_bath(norb: int, nbath: int, seed: int,
                e_range=(-2.0, 2.0), v_range=(0.2, 0.6)):
    """Spin-independent random bath: for alpha, for nu: energy then V."""
    rng = SplitMix64(seed)
    e = np.zeros((norb, nbath))
    v = np.zeros((norb, nbath))
    for a in range(norb):
        for nu in range(nbath):
            e[a, nu] = rng.uniform(*e_range)
            v[a, nu] = rng.uniform(*v_range)
    return e, v


def make_model(norb, nbath, U, Jh=0.0, Ust=None, e_d=None, e_bath=None,
               v_bath=None, seed=0, name=""):
    if Ust is None:
        Ust = U - 2.0 * Jh
    if e_d is None:
        e_d = half_filling_ed(norb, U, Ust, Jh)
    if e_bath is None or v_bath is None:
        e_r, v_r = random_bath(norb, nbath, seed)
        e_bath = e_r if e_bath is None else e_bath
        v_bath = v_r if v_bath is None else v_bath
    e_imp = np.full(norb, float(e_d))
    return ImpurityModel(norb=norb, nbath=nbath, U=U, Ust=Ust, Jh=Jh,
                         e_imp=e_imp, e_bath=e_bath, v_bath=v_bath, name=name)


@dataclass
class Workload:
    name: str
    model: ImpurityModel
    nup: int
    ndw: int
    gf_steps: int = 200
    nmats: int = 512
    beta: float = 100.0
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        ns = self.model.ns
        return math.comb(ns, self.nup) * math.comb(ns, self.ndw)


def workload_ns8(seed: int = 0) -> Workload:
    """Single-orbital AIM, Nbath=7 (Ns=8), sector (4,4), D=4,900; U=2,
    e_d=-U/2, bath energies evenly spaced in [-1,1], V=0.5."""
    nb = 7
    e = np.array([-1.0 + 2.0 * k / (nb - 1) for k in range(nb)])[None, :]
    v = np.full((1, nb), 0.5)
    m = make_model(1, nb, U=2.0, e_d=-1.0, e_bath=e, v_bath=v, name="aim_ns8")
    return Workload("aim_norb1_ns8_n4_4", m, 4, 4,
                    description="Norb=1 Nbath=7 Ns=8 sector (4,4) D=4900 U=2 e_d=-1 grid bath V=0.5")


def workload_ns14(seed: int = 0) -> Workload:
    """Single-orbital AIM, Nbath=13 (Ns=14), half filling (7,7),
    D=11,778,624; U=4, e_d=-2, e_k~U[-2,2], V_k~U[0.2,0.6]."""
    e, v = random_bath(1, 13, seed)
    m = make_model(1, 13, U=4.0, e_d=-2.0, e_bath=e, v_bath=v, name="aim_ns14")
    return Workload("aim_norb1_ns14_n7_7", m, 7, 7,
                    description=f"Norb=1 Nbath=13 Ns=14 sector (7,7) D=11778624 U=4 seed={seed}")


def workload_norb2_ns14(seed: int = 0) -> Workload:
    """Two-orbital density-density Kanamori AIM, Nbath=6 per orbital
    (Ns=14), off half filling (5,6), D=6,012,006; U=3, J=0.5, U'=2.  A
    parity case for the two-orbital product at a size the oracle solves in
    minutes."""
    e, v = random_bath(2, 6, seed)
    m = make_model(2, 6, U=3.0, Jh=0.5, Ust=2.0, e_bath=e, v_bath=v, name="kanamori2_ns14")
    return Workload("kanamori_norb2_ns14_n5_6", m, 5, 6,
                    description=f"Norb=2 Nbath=6 Ns=14 sector (5,6) D=6012006 U=3 J=0.5 seed={seed}")


def workload_ns16(seed: int = 0) -> Workload:
    """Two-orbital density-density Kanamori AIM, Nbath=7 per orbital (Ns=16),
    half filling (8,8), D=165,636,900; U=3, J=0.5, U'=2, e_d=-3.25."""
    e, v = random_bath(2, 7, seed)
    m = make_model(2, 7, U=3.0, Jh=0.5, Ust=2.0, e_bath=e, v_bath=v, name="kanamori2_ns16")
    return Workload("kanamori_norb2_ns16_n8_8", m, 8, 8,
                    description=f"Norb=2 Nbath=7 Ns=16 sector (8,8) D=165636900 U=3 J=0.5 seed={seed}")


def workload_ns18(seed: int = 0) -> Workload:
    """Three-orbital density-density Kanamori AIM, Nbath=5 per orbital
    (Ns=18), half filling (9,9), D=2,363,904,400; U=2.5, J=0.4, U'=1.7,
    e_d=-4.25."""
    e, v = random_bath(3, 5, seed)
    m = make_model(3, 5, U=2.5, Jh=0.4, Ust=1.7, e_bath=e, v_bath=v, name="kanamori3_ns18")
    return Workload("kanamori_norb3_ns18_n9_9", m, 9, 9, gf_steps=0,
                    description=f"Norb=3 Nbath=5 Ns=18 sector (9,9) D=2363904400 U=2.5 J=0.4 seed={seed}")


def with_exchange(model: ImpurityModel, Jx=None, Jp=None, name=None) -> ImpurityModel:
    """The same model with the spin-exchange and pair-hopping couplings of
    Eq. Ham1 switched on (default J_X = J_P = J: with U' = U - 2J the fully
    rotation-invariant Kanamori interaction)."""
    return ImpurityModel(norb=model.norb, nbath=model.nbath, U=model.U, Ust=model.Ust,
                         Jh=model.Jh, e_imp=model.e_imp, e_bath=model.e_bath,
                         v_bath=model.v_bath, Jx=model.Jh if Jx is None else Jx,
                         Jp=model.Jh if Jp is None else Jp,
                         name=(model.name + "_full") if name is None else name)


def workload_full_norb3_ns15(seed: int = 0) -> Workload:
    """Full Kanamori AIM (spin exchange and pair hopping, J_X = J_P = J,
    U' = U - 2J), three orbitals, Nbath=4 per orbital (Ns=15), sector (8,7),
    D=41,409,225; U=3, J=0.5.  The three-orbital system of the paper's
    density-density vs full Kanamori comparison (Ns = 15)."""
    e, v = random_bath(3, 4, seed)
    m = make_model(3, 4, U=3.0, Jh=0.5, e_bath=e, v_bath=v, name="kanamori3_ns15")
    return Workload("full_kanamori_norb3_ns15_n8_7", with_exchange(m), 8, 7,
                    description=f"Norb=3 Nbath=4 Ns=15 sector (8,7) D=41409225 U=3 J=JX=JP=0.5 seed={seed}")


def workload_full_norb5_ns15(seed: int = 0) -> Workload:
    """Full Kanamori AIM, five orbitals, Nbath=2 per orbital (Ns=15), sector
    (8,7), D=41,409,225; U=3, J=0.5, J_X = J_P = J, U' = U - 2J."""
    e, v = random_bath(5, 2, seed)
    m = make_model(5, 2, U=3.0, Jh=0.5, e_bath=e, v_bath=v, name="kanamori5_ns15")
    return Workload("full_kanamori_norb5_ns15_n8_7", with_exchange(m), 8, 7,
                    description=f"Norb=5 Nbath=2 Ns=15 sector (8,7) D=41409225 U=3 J=JX=JP=0.5 seed={seed}")


def workload_full_ns18(seed: int = 0) -> Workload:
    """The three-orbital Ns=18 half-filled workload with the spin exchange and
    pair hopping switched on (J_X = J_P = J = 0.4)."""
    w = workload_ns18(seed)
    return Workload("full_kanamori_norb3_ns18_n9_9", with_exchange(w.model), 9, 9, gf_steps=0,
                    description=w.description.replace("J=0.4", "J=JX=JP=0.4"))


def workload_eph_ns12(seed: int = 0, nph: int = 10) -> Workload:
    """Electron-phonon (Holstein) AIM of the paper's phonon benchmark: Ns=12
    (one orbital, Nbath=11), half-filled sector (6,6), D_e = 853,776, one
    phonon mode w0 = 0.5 coupled with g = 0.3, cut-off N_ph (D = D_e (N_ph+1));
    U = 2, e_d = -1, seeded random bath."""
    e, v = random_bath(1, 11, seed)
    m = make_model(1, 11, U=2.0, e_d=-1.0, e_bath=e, v_bath=v, name="holstein_ns12")
    return Workload(f"holstein_norb1_ns12_n6_6_nph{nph}", m, 6, 6, gf_steps=200,
                    extra={"w0": 0.5, "g": [0.3], "nph": nph},
                    description=f"Norb=1 Nbath=11 Ns=12 sector (6,6) D_e=853776 w0=0.5 g=0.3 "
                                f"N_ph={nph} U=2 seed={seed}")


# Valid (norb, ns) pairs for the serving stream: ns must be a multiple of
# norb (Ns = Norb (Nbath+1)), ns in {8,...,16}, norb in {1,2,3}.
SERVING_PAIRS = [(no, ns) for no in (1, 2, 3) for ns in (8, 10, 12, 14, 16)
                 if ns % no == 0 and ns // no >= 2]


@dataclass
class ServingRequest:
    rid: int
    arrival_s: float
    workload: Workload


def serving_stream(n_requests: int = 2000, rate_per_s: float = 50.0,
                   seed: int = 0, max_ns: int = 16):
    """Poisson stream of impurity solves with mixed Norb, Ns and sector.

    Each request draws (Norb, Ns) uniformly among the valid pairs, a sector
    within +-2 electrons of half filling per spin, U~U[1,5], J/U~U[0,0.25],
    U'=U-2J, e_d at the particle-hole point, and a random bath."""
    rng = SplitMix64(seed ^ 0x5E4F1CE)
    pairs = [p for p in SERVING_PAIRS if p[1] <= max_ns]
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        norb, ns = pairs[int(rng.uniform() * len(pairs)) % len(pairs)]
        nbath = ns // norb - 1
        half = ns // 2
        nup = half + int(rng.uniform() * 5) % 5 - 2
        ndw = half + int(rng.uniform() * 5) % 5 - 2
        U = rng.uniform(1.0, 5.0)
        J = U * rng.uniform(0.0, 0.25)
        bseed = rng.next_u64()
        m = make_model(norb, nbath, U=U, Jh=J, seed=bseed, name=f"req{rid}")
        wl = Workload(f"req{rid}_norb{norb}_ns{ns}_{nup}_{ndw}", m, nup, ndw)
        out.append(ServingRequest(rid, t, wl))
    return out


WORKLOADS = {
    "ns8": workload_ns8,
    "ns14": workload_ns14,
    "ns16": workload_ns16,
    "ns18": workload_ns18,
    "full3_ns15": workload_full_norb3_ns15,
    "full5_ns15": workload_full_norb5_ns15,
    "full_ns18": workload_full_ns18,
    "eph_ns12": workload_eph_ns12,
}
