"""Writes oracle-only expected values used by the GPU parity tests.

Calls nothing but ``oracle/`` and ``workloads/``.  Each output file records
the workload recipe and the oracle's FP64 results:

* ``oracle_ns8.json``  — Ns=8 single-orbital AIM, sector (4,4): E0 (Lanczos
  and dense eigh) and G_{0,up}(i w_n), 512 Matsubara points, beta=100,
  200-step chains.
* ``oracle_ns14.json`` — Ns=14 single-orbital AIM, sector (7,7), seeded bath
  (seed 0): E0 and G_{0,up}(i w_n) from 200-step chains, plus sampled
  components of psi.
* ``oracle_norb2_ns14.json`` — Ns=14 two-orbital Kanamori AIM, sector (5,6),
  seeded bath (seed 0): the same quantities (orbital 0, spin up).
* ``oracle_ns16.json`` — Ns=16 two-orbital Kanamori AIM, half filling (8,8),
  D=165,636,900, seeded bath (seed 0): the benchmark sector.  E0, 256 psi
  samples and G_{0,up}(i w_n) from 200-step chains, all from the oracle's
  factorised product (Sec. 6.7 without MPI); about two hours on one core.

Usage: python tests/golden/make_golden.py [ns8] [ns14] [norb2_ns14] [ns16]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fock, gf, lanczos  # noqa: E402
from workloads import (workload_ns8, workload_ns14, workload_norb2_ns14,  # noqa: E402
                       workload_ns16)

SEED = 0x5EED


def run(wl, dense=False, nsamp=0):
    t = time.time()
    s = fock.get_sector(wl.model, wl.nup, wl.ndw)
    r = lanczos.ground_state(s.matvec, s.dim, seed=SEED)
    e_rq, res = lanczos.rayleigh_residual(s.matvec, r["psi"])
    out = dict(workload=wl.name, description=wl.description, nup=wl.nup, ndw=wl.ndw,
               seed=SEED, e0=r["e0"], iterations=int(r["k"]), stop=r["reason"],
               e_rayleigh=e_rq, residual=res)
    if dense:
        out["e0_dense"] = float(np.linalg.eigvalsh(s.hamiltonian().toarray())[0])
    G, parts = gf.impurity_gf(wl.model, wl.nup, wl.ndw, r["psi"], r["e0"], 0, 0,
                              nsteps=wl.gf_steps, beta=wl.beta, nmats=wl.nmats,
                              return_parts=True)
    out["G_re"] = G.real.tolist()
    out["G_im"] = G.imag.tolist()
    out["weight_particle"] = parts[1][0]
    out["weight_hole"] = parts[-1][0]
    if nsamp:
        idx = np.unique(np.linspace(0, s.dim - 1, nsamp).astype(np.int64))
        psi = r["psi"] * np.sign(r["psi"][np.argmax(np.abs(r["psi"]))])
        out["psi_index"] = idx.tolist()
        out["psi_value"] = psi[idx].tolist()
    out["oracle_seconds"] = time.time() - t
    return out


def main(which):
    if "ns8" in which:
        with open(os.path.join(HERE, "oracle_ns8.json"), "w") as f:
            json.dump(run(workload_ns8(), dense=True, nsamp=64), f, indent=1)
    if "ns14" in which:
        with open(os.path.join(HERE, "oracle_ns14.json"), "w") as f:
            json.dump(run(workload_ns14(0), nsamp=256), f, indent=1)
    if "norb2_ns14" in which:
        with open(os.path.join(HERE, "oracle_norb2_ns14.json"), "w") as f:
            json.dump(run(workload_norb2_ns14(0), nsamp=256), f, indent=1)
    if "ns16" in which:
        out = run(workload_ns16(0), nsamp=256)
        with open(os.path.join(HERE, "oracle_ns16.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["ns8", "ns14", "norb2_ns14"])
