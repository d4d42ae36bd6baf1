"""Benchmark of the exact-diagonalisation hot path on GB300.

One step = one impurity solve (ed_solve) of the Ns=16 two-orbital Kanamori
workload (Norb=2, Nbath=7, half filling N_up=N_dw=8, D=165,636,900): sector
build (tables), FP32 Lanczos ground state with FP64 scalars, second pass, FP64
polish, and G(i w_n) of both orbitals (spin down follows by symmetry) from
200-step FP32 Lanczos chains on the N+-1 sectors, run concurrently, 512
Matsubara points at beta=100.  All of it runs in libedgb.so; PyTorch supplies
the stream, the events and the ground-state buffer of the e2e leg.

value   = algorithmic H.v bytes of every product in the timed steps (8 D per
          FP32 product, 16 D per FP64 product; read v + write w) / time.
roofline= the product kernel timed alone with CUDA events on its stream
          (ed_matvec_blocked, FP32, 8 D bytes per launch) against the measured
          HBM copy bandwidth.
e2e     = the same solve timed on the host clock, with the FP64 ground state
          copied back to pinned host memory inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload ns16|ns14|ns18] [--serving N]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lanczos H·v GB/s vs HBM peak, iters/s; served solves/s with p50/p99 latency"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, device_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[3]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        loaded = [r for r in rows if r[2] > 10] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "samples_under_load": len(loaded)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _profiled_traffic(workload):
    """DRAM bytes per launch of the product kernel from the committed ncu
    summary, or None when the kernel source changed since that capture."""
    import hashlib
    import re
    f = os.path.join(ROOT, "profiles", f"k_hv_blocked_fp32_{workload}.md")
    src = os.path.join(ROOT, "paper_2105_06806_gb300", "csrc", "matvec.cu")
    if not os.path.exists(f):
        return None
    txt = open(f).read()
    m = re.search(r"sha256 prefix ([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch: (\d+)", txt)
    if not m or not t:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:len(m.group(1))] != m.group(1):
        return None
    return int(t.group(1))


def combine_ranks(dist, nbytes, iters, seconds):
    """Replicas: every rank ran its own copy of the workload.  Whole-job
    throughput = all ranks' bytes (iterations) / the slowest rank's time."""
    t_max = _max_over_ranks(dist, seconds)
    return (_sum_over_ranks(dist, nbytes) / t_max / 1e9, _sum_over_ranks(dist, iters) / t_max, t_max)


def _workload(name):
    import workloads
    return workloads.WORKLOADS[name](0)


def _sector_dim(ns, n1, n2):
    return math.comb(ns, n1) * math.comb(ns, n2)


# ----------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_06806_gb300 as E

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = _workload(args.workload)
    m = wl.model
    ns = m.ns
    D = wl.dim
    stream = torch.cuda.current_stream()
    psi = torch.empty(D, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2
    gf_steps, nmats, beta = (50 if args.quick_gf else 200), 512, 100.0
    do_gf = args.gf and wl.gf_steps > 0

    def one_step(psi_out=None):
        """One impurity solve through ed_solve.  Returns (products,
        algorithmic bytes, Lanczos iterations, result)."""
        r, G = E.solve(m, wl.nup, wl.ndw, stream=stream, psi=psi_out, precision="fp32_polish",
                       gf_precision="fp32", nmats=nmats if do_gf else 0, beta=beta,
                       gf_steps=gf_steps)
        # ground state: the products the library reports as executed, FP32
        # ones at 8 D bytes (read v + write w), FP64 ones (polish steps and
        # residual products) at 16 D
        k = r["iterations"]
        n64 = r["matvecs_fp64"]
        n32 = r["matvecs"] - n64
        nbytes = 8 * D * n32 + 16 * D * n64 + r["gf_product_bytes"]
        nmv = r["matvecs"] + r["gf_steps_total"]
        iters = k + r["polish_iterations"] + r["gf_steps_total"]
        return nmv, nbytes, iters, r

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    l0 = E.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    tot_bytes = tot_mv = tot_it = 0
    last = None
    _barrier(dist)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                                  # L2 flush between steps
        ev[k][0].record(stream)
        nmv, nb, it, last = one_step()
        ev[k][1].record(stream)
        tot_bytes += nb
        tot_mv += nmv
        tot_it += it
    torch.cuda.synchronize()
    _barrier(dist)
    launches = E.kernel_launches() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_s = sum(step_ms) / 1e3
    clk = clocks.stop()

    # dominant kernel alone: the FP32 block-major product (the one inside
    # the Lanczos steps) on the full sector
    mv = time_products(E, wl, stream, dev, reps=20)
    mv_ms = mv["blocked_fp32_ms"]
    hbm, src = _peaks()
    alg = 8.0 * D
    achieved = alg / (mv_ms / 1e3) / 1e9

    # end to end through the public one-call API: host model arrays in; E0,
    # G and the FP64 ground state back in (pinned) host memory
    e2e = None
    if args.e2e:
        host_psi = torch.empty(D, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nmv_e, nb_e, _, r_e = one_step(psi_out=psi)
        host_psi.copy_(psi, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        mm = E.Model(m)
        h2d = mm.e_imp.nbytes + mm.e_bath.nbytes + mm.v_bath.nbytes
        d2h = 8 * D + (16 * 2 * m.norb * nmats if do_gf else 0) + 8 * 16
        e2e = {"value": round(nb_e / (t1 - t0) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "seconds": round(t1 - t0, 4),
               "api": "ed_solve (host model in; E0, G out) + ground state to pinned host"}

    # plain FP64 GPU Lanczos against FP32 + FP64 polish, ground state only,
    # time to solution at the same 1e-10 accuracy target
    cmp = None
    if rank == 0 and args.compare:
        s = E.Sector(m, wl.nup, wl.ndw, stream=stream)
        out = {}
        for prec in ("fp64", "fp32_polish", "fp64", "fp32_polish"):   # second round timed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = E.lanczos_ground(s, prec, want_vector=False, stream=stream, allow_maxit=True)
            torch.cuda.synchronize()
            out[prec] = (time.perf_counter() - t0, r)
        s.free()
        (t64, r64), (t32, r32) = out["fp64"], out["fp32_polish"]
        cmp = {"fp64_seconds": round(t64, 4), "fp64_iterations": r64["iterations"],
               "fp64_iters_per_s": round(r64["iterations"] / t64, 2), "fp64_e0": r64["e0"],
               "fp32_polish_seconds": round(t32, 4),
               "fp32_polish_iterations": r32["iterations"] + r32["polish_iterations"],
               "fp32_polish_e0": r32["e0"], "fp32_raw_e0": r32["e0_raw"],
               "rel_diff_polished": abs(r32["e0"] - r64["e0"]) / abs(r64["e0"]),
               "rel_diff_raw_fp32": abs(r32["e0_raw"] - r64["e0"]) / abs(r64["e0"]),
               "speedup_time_to_solution": round(t64 / t32, 3)}

    cpu = None
    if rank == 0 and args.cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_seconds)

    serving = None
    if rank == 0 and args.serving > 0:
        serving = run_serving(E, args.serving, args.serving_max_ns, args.serving_rate)
        if args.serving_rate <= 0:
            # the same stream with Poisson arrivals at 0.8 x the saturation rate:
            # latency of a loaded but not saturated server
            lam = round(0.8 * serving["solves_per_s"], 1)
            serving["poisson_0p8"] = run_serving(E, args.serving, args.serving_max_ns, lam)
            if args.serving_max_ns < 16:
                # the configured stream draws Ns up to 16 (D up to 1.66e8)
                serving["full_ns16"] = run_serving(E, args.serving, 16, 0.0)

    value, iters_s, t_max = combine_ranks(dist, tot_bytes, tot_it, t_s)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": wl.name, "dim": D, "norb": m.norb, "ns": ns,
                   "sector": [wl.nup, wl.ndw], "precision": "fp32 Lanczos + fp64 polish",
                   "gf": (f"all orbitals, particle and hole chains ({gf_steps} FP32 steps) "
                          f"concurrently, {nmats} Matsubara points, beta={beta}; spin down by "
                          "symmetry") if do_gf else "none",
                   "l2": "256 MB flush between steps; vectors 0.66 GB > L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "iters_per_s": round(iters_s, 2),
        "matvecs_per_step": tot_mv / args.steps,
        "e0": last["e0"], "e0_raw": last["e0_raw"], "residual": last["residual"],
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": _profiled_traffic(args.workload),
                     "kernel": "k_hv<float, HV_PLAIN> block-major (ed_matvec_blocked)",
                     "peak_source": src, "products_ms": mv,
                     "kernel_ms": round(mv_ms, 4), "algorithmic_bytes": int(alg)},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "cpu_baseline": cpu, "serving": serving, "fp64_vs_fp32_polish": cmp,
    }
    print(json.dumps(line))


def time_products(E, wl, stream, dev, reps=20, which=("blocked_fp32", "sector_fp32")):
    """Median CUDA-event time of single H.v launches on the full sector."""
    import torch
    m = wl.model
    s = E.Sector(m, wl.nup, wl.ndw, stream=stream)
    D = s.dim
    out = {}
    for name in which:
        lay, prec = name.split("_")
        dt = torch.float32 if prec == "fp32" else torch.float64
        n = s.blocked_dim if lay == "blocked" else D    # block-major vectors are padded
        v = torch.randn(n, dtype=dt, device=dev)
        w = torch.empty_like(v)
        f = E.matvec_blocked if lay == "blocked" else E.matvec
        for _ in range(3):
            f(s, v, w, prec, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        durs = []
        for _ in range(reps):
            a.record(stream)
            f(s, v, w, prec, stream=stream)
            b.record(stream)
            b.synchronize()
            durs.append(a.elapsed_time(b))
        out[name + "_ms"] = round(statistics.median(durs), 4)
        del v, w
    s.free()
    return out


def run_matvec_only(args):
    """Product kernels alone (used for kernel profiling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_06806_gb300 as E
    torch.cuda.set_device(0)
    wl = _workload(args.workload)
    which = tuple(args.matvec_only.split(","))
    r = time_products(E, wl, torch.cuda.current_stream(), torch.device("cuda", 0),
                      reps=args.steps, which=which)
    hbm, src = _peaks()
    for k, v in list(r.items()):
        elem = 8 if "fp64" in k else 4
        r[k.replace("_ms", "_gbs")] = round(2 * elem * wl.dim / (v / 1e3) / 1e9, 1)
    print(json.dumps({"workload": wl.name, "dim": wl.dim, "peak_gbs": hbm, **r}))


def cpu_baseline(wl, budget_s):
    """The oracle as it stands: its factorised FP64 product inside its plain
    Lanczos, on a bounded number of steps of the same sector."""
    from oracle import fock, lanczos
    t0 = time.perf_counter()
    s = fock.Sector.__new__(fock.Sector)
    m = wl.model
    s.model, s.nup, s.ndw = m, wl.nup, wl.ndw
    s.map_up = fock.build_sector_map(m.ns, wl.nup)
    s.map_dw = s.map_up if wl.ndw == wl.nup else fock.build_sector_map(m.ns, wl.ndw)
    s.dim_up, s.dim_dw = len(s.map_up), len(s.map_dw)
    s.dim = s.dim_up * s.dim_dw
    s.H_up = fock.spin_hopping_matrix(m, 0, wl.nup, s.map_up)
    s.H_dw = fock.spin_hopping_matrix(m, 1, wl.ndw, s.map_dw)
    s.E_up, s.m_up = fock.spin_diagonal(m, 0, wl.nup, s.map_up)
    s.E_dw, s.m_dw = fock.spin_diagonal(m, 1, wl.ndw, s.map_dw)
    s.W = fock.interaction_table(m)
    t_build = time.perf_counter() - t0
    v0 = lanczos.start_vector(0x5EED, s.dim)
    # one timed product decides how many Lanczos steps fit the budget
    t1 = time.perf_counter()
    s.matvec(v0)
    t_mv = time.perf_counter() - t1
    steps = max(1, min(20, int(budget_s / max(t_mv * 1.3, 1e-9))))
    t2 = time.perf_counter()
    r = lanczos.lanczos_ground(s.matvec, v0, maxit=steps, tol=0.0)
    t = time.perf_counter() - t2
    return {"value": round(16.0 * s.dim * r["k"] / t / 1e9, 4), "unit": "GB/s",
            "cores": 1, "kind": "oracle",
            "sample": f"{r['k']} FP64 Lanczos steps of the oracle (factorised scipy product) on "
                      f"the full D={s.dim} sector; table build {t_build:.1f}s not timed",
            "iters_per_s": round(r["k"] / t, 4), "host_cores_available": os.cpu_count()}


def run_serving(E, n_requests, max_ns, rate=0.0):
    """Serving stream: Poisson arrivals, mixed (Norb, Ns, sector); returns
    solves/s and p50/p99 latency of t_done - t_submit."""
    import numpy as np
    import workloads
    reqs = workloads.serving_stream(n_requests, rate_per_s=rate if rate > 0 else 1e9, seed=0,
                                    max_ns=max_ns)
    srv = E.Server(slots=8)
    t0 = time.perf_counter()
    tickets = []
    for q in reqs:
        now = time.perf_counter() - t0
        if q.arrival_s > now:
            time.sleep(q.arrival_s - now)
        tickets.append(srv.submit(q.workload.model, q.workload.nup, q.workload.ndw,
                                  precision="fp32_polish", gf_precision="fp32", nmats=512,
                                  beta=100.0, gf_steps=200))
    lat, ok = [], 0
    for t in tickets:
        srv.wait(t, 600.0)
        r = srv.poll(t)
        if r is None:
            continue
        res, _ = r
        ok += res["status"] == 0
        lat.append(res["t_done_s"] - res["t_submit_s"])
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array(lat)
    return {"requests": n_requests, "completed_ok": int(ok), "solves_per_s": round(ok / wall, 3),
            "p50_s": round(float(np.percentile(lat, 50)), 4),
            "p99_s": round(float(np.percentile(lat, 99)), 4), "max_ns": max_ns,
            "arrival_rate_per_s": rate if rate > 0 else "all at once (saturation)",
            "work": "FP32 ground state + FP64 polish + G(512 Matsubara, 200-step FP32 chains) "
                    "for every orbital and spin"}


# ----------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle (plain CPU FP64 implementation) on the host cores, same
    metric on the same workload: each step is one oracle Lanczos step on the
    full sector, a bounded sample of the solve."""
    dist, rank, ws = _dist()
    if rank != 0:
        return
    from oracle import fock, lanczos
    wl = _workload(args.workload)
    m = wl.model
    s = fock.Sector.__new__(fock.Sector)
    s.model, s.nup, s.ndw = m, wl.nup, wl.ndw
    s.map_up = fock.build_sector_map(m.ns, wl.nup)
    s.map_dw = s.map_up if wl.ndw == wl.nup else fock.build_sector_map(m.ns, wl.ndw)
    s.dim_up, s.dim_dw = len(s.map_up), len(s.map_dw)
    s.dim = s.dim_up * s.dim_dw
    s.H_up = fock.spin_hopping_matrix(m, 0, wl.nup, s.map_up)
    s.H_dw = fock.spin_hopping_matrix(m, 1, wl.ndw, s.map_dw)
    s.E_up, s.m_up = fock.spin_diagonal(m, 0, wl.nup, s.map_up)
    s.E_dw, s.m_dw = fock.spin_diagonal(m, 1, wl.ndw, s.map_dw)
    s.W = fock.interaction_table(m)
    v0 = lanczos.start_vector(0x5EED, s.dim)
    for _ in range(args.warmup):
        s.matvec(v0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lanczos.lanczos_ground(s.matvec, v0, maxit=1, tol=0.0)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = 16.0 * s.dim * args.steps / t / 1e9
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "dim": s.dim, "parallelism": "host CPU"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "one FP64 oracle Lanczos step per bench step on the "
                                       "full sector (scipy factorised product)"},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ns16", choices=["ns14", "ns16", "ns18"])
    ap.add_argument("--no-gf", dest="gf", action="store_false")
    ap.add_argument("--quick-gf", action="store_true", help="50-step chains instead of 200")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--serving-rate", type=float, default=0.0,
                    help="Poisson arrival rate of the serving stream (0: all at once)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serving", type=int, default=96, help="requests of the serving stream (0: off)")
    ap.add_argument("--serving-max-ns", type=int, default=12)
    ap.add_argument("--matvec-only", default="",
                    help="comma list of {blocked,sector}_{fp32,fp64}: time products only")
    args = ap.parse_args()
    if args.matvec_only:
        run_matvec_only(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = max(args.warmup, 0)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
