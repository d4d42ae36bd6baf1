"""Benchmark of the exact-diagonalisation hot path on GB300.

Headline (N=1): one step = one impurity solve through ed_solve of the
largest single-GPU workload, the Ns=18 three-orbital Kanamori sector
(Norb=3, Nbath=5, half filling N_up=N_dw=9, D=2,363,904,400), ground state
only: sector build (tables), FP32 Lanczos with FP64 scalars, the second pass
for psi (the Krylov basis of 9.5 GB vectors does not fit the device budget),
FP64 polish and FP64 residual.  `--workload ns16` makes the Ns=16 two-orbital
sector (D=165,636,900) with G(i w_n) of both orbitals (200-step FP32 chains
on the N+-1 sectors, 512 Matsubara points, beta=100) the timed step instead;
with the default workload that solve is timed as a sub-record.

value   = algorithmic H.v bytes of every product the library reports as
          executed in the timed steps (8 D per FP32 product, 16 D per FP64
          product: read v + write w) / time.
roofline= the FP32 block-major product of the headline sector timed alone
          with CUDA events on its stream (ed_matvec_blocked: at Ns=18 the
          H_up pass and the H_dw pass, two launches; 8 D bytes per product)
          against the measured HBM copy bandwidth.
e2e     = the same solve through ed_solve on the host clock, with the FP64
          ground state copied back to pinned host memory inside the timed
          region.
cpu_baseline = the oracle's factorised FP64 product (Sec. 6.7 without MPI)
          on the same sector, split over dw-row slabs across all host cores
          (spawned worker processes), and one slab on one core.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload ns18|ns16|ns14] [--serving N]
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
    f = os.path.join(ROOT, "profiles", f"product_fp32_{workload}.md")
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

GF = dict(nmats=512, beta=100.0, steps=200)


def _solve_step(E, wl, stream, with_gf, precision="fp32_polish", psi_out=None):
    """One impurity solve through ed_solve.  Returns (products, algorithmic
    product bytes, Lanczos iterations, result)."""
    D = wl.dim
    do_gf = with_gf and wl.gf_steps > 0
    r, G = E.solve(wl.model, wl.nup, wl.ndw, stream=stream, psi=psi_out, precision=precision,
                   gf_precision="fp32" if precision != "fp64" else "fp64",
                   nmats=GF["nmats"] if do_gf else 0, beta=GF["beta"], gf_steps=GF["steps"])
    # the products the library reports as executed: FP32 ones at 8 D bytes
    # (read v + write w), FP64 ones (polish steps, residual products, or the
    # whole run in FP64) at 16 D
    n64 = r["matvecs_fp64"]
    n32 = r["matvecs"] - n64
    nbytes = 8 * D * n32 + 16 * D * n64 + r["gf_product_bytes"]
    nmv = r["matvecs"] + r["gf_steps_total"]
    iters = r["iterations"] + r["polish_iterations"] + r["gf_steps_total"]
    return nmv, nbytes, iters, r


def _time_solves(E, wl, stream, steps, warmup, with_gf, flush=None):
    """Warm-up then `steps` timed solves (CUDA events on `stream`)."""
    import torch
    for _ in range(warmup):
        _solve_step(E, wl, stream, with_gf)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    tot = dict(bytes=0, mv=0, it=0)
    last = None
    for k in range(steps):
        if flush is not None:
            flush.zero_()                                  # L2 flush between steps
        ev[k][0].record(stream)
        nmv, nb, it, last = _solve_step(E, wl, stream, with_gf)
        ev[k][1].record(stream)
        tot["bytes"] += nb
        tot["mv"] += nmv
        tot["it"] += it
    torch.cuda.synchronize()
    t_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    return t_s, tot, last


def run_ours(args):
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
    D = wl.dim
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2
    with_gf = args.gf and wl.gf_steps > 0

    # timed steps of the headline workload
    for _ in range(args.warmup):
        _solve_step(E, wl, stream, with_gf)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    l0 = E.kernel_launches()
    _barrier(dist)
    torch.cuda.synchronize()
    t_s, tot, last = _time_solves(E, wl, stream, args.steps, 0, with_gf, flush)
    _barrier(dist)
    launches = E.kernel_launches() - l0
    clk = clocks.stop()

    # dominant kernel alone: the FP32 block-major product (the one inside the
    # Lanczos steps) on the full sector
    mv = time_products(E, wl, stream, dev, reps=10 if D > 1e9 else 20)
    mv_ms = mv["blocked_fp32_ms"]
    hbm, src = _peaks()
    alg = 8.0 * D
    achieved = alg / (mv_ms / 1e3) / 1e9

    # end to end through the public one-call API: host model arrays in; E0
    # (and G) out, the FP64 ground state copied back to pinned host memory
    e2e = None
    if args.e2e:
        # torch's cached blocks (the product timing's vectors) back to the
        # device, and the page-locked buffer's first copy done untimed: the
        # first transfer into freshly page-locked memory ran at 35 GB/s
        # against 190 GB/s for every later one
        torch.cuda.empty_cache()
        psi = torch.empty(D, dtype=torch.float64, device=dev)
        host_psi = torch.empty(D, dtype=torch.float64, pin_memory=True)
        host_psi.copy_(psi, non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, nb_e, _, r_e = _solve_step(E, wl, stream, with_gf, psi_out=psi)
        host_psi.copy_(psi, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        del psi
        mm = E.Model(m)
        h2d = mm.e_imp.nbytes + mm.e_bath.nbytes + mm.v_bath.nbytes
        d2h = 8 * D + (16 * 2 * m.norb * GF["nmats"] if with_gf else 0) + 8 * 16
        e2e = {"value": round(nb_e / (t1 - t0) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "seconds": round(t1 - t0, 4),
               "api": "ed_solve (host model in; E0" + (", G" if with_gf else "")
                      + " out) + ground state to pinned host"}
        del host_psi

    subs = {}
    if rank == 0 and args.workload != "ns16" and args.sub_ns16:
        # the Ns=16 full solve with G(i w_n) of both orbitals, as a sub-record
        w16 = _workload("ns16")
        t16, tot16, last16 = _time_solves(E, w16, stream, 3, 1, True, flush)
        mv16 = time_products(E, w16, stream, dev, reps=20)
        subs["ns16_full_solve"] = {
            "workload": w16.name, "dim": w16.dim, "steps": 3,
            "ms_per_step": round(1e3 * t16 / 3, 3), "value": round(tot16["bytes"] / t16 / 1e9, 3),
            "unit": "GB/s", "iters_per_s": round(tot16["it"] / t16, 2),
            "matvecs_per_step": tot16["mv"] / 3, "e0": last16["e0"],
            "gf": "all orbitals, particle and hole chains (200 FP32 steps) concurrently, "
                  "512 Matsubara points, beta=100; spin down by symmetry",
            "product": {**mv16, "frac": round(8.0 * w16.dim / (mv16["blocked_fp32_ms"] / 1e3)
                                              / 1e9 / hbm, 4)}}

    if rank == 0 and args.full_kanamori:
        subs["full_kanamori"] = run_full_kanamori(E, stream, dev, hbm)
    if rank == 0 and args.eph:
        subs["electron_phonon_ns12"] = run_eph(E, stream, dev)

    # plain FP64 GPU Lanczos against FP32 + FP64 polish, ground state only,
    # time to solution at the same 1e-10 accuracy target
    cmp = None
    if rank == 0 and args.compare:
        cmp = {}
        for name in ([args.workload] + (["ns16"] if args.workload != "ns16" else [])):
            wc = _workload(name)
            s = E.Sector(wc.model, wc.nup, wc.ndw, stream=stream)
            out = {}
            order = ("fp64", "fp32_polish") if wc.dim > 1e9 else ("fp64", "fp32_polish") * 2
            for prec in order:   # small sectors: the second round is the timed one
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = E.lanczos_ground(s, prec, want_vector=False, stream=stream, allow_maxit=True)
                torch.cuda.synchronize()
                out[prec] = (time.perf_counter() - t0, r)
            s.free()
            (t64, r64), (t32, r32) = out["fp64"], out["fp32_polish"]
            cmp[wc.name] = {
                "fp64_seconds": round(t64, 4), "fp64_iterations": r64["iterations"],
                "fp64_iters_per_s": round(r64["iterations"] / t64, 2), "fp64_e0": r64["e0"],
                "fp32_polish_seconds": round(t32, 4),
                "fp32_polish_iterations": r32["iterations"] + r32["polish_iterations"],
                "fp32_polish_e0": r32["e0"], "fp32_raw_e0": r32["e0_raw"],
                "rel_diff_polished": abs(r32["e0"] - r64["e0"]) / abs(r64["e0"]),
                "rel_diff_raw_fp32": abs(r32["e0_raw"] - r64["e0"]) / abs(r64["e0"]),
                "speedup_time_to_solution": round(t64 / t32, 3)}

    serving = None
    if rank == 0 and args.serving > 0:
        serving = run_serving(E, args.serving, args.serving_max_ns, 0.0, "fp32_polish")
        lam = round(0.8 * serving["solves_per_s"], 1)
        # the same stream with Poisson arrivals at 0.8 x the saturation rate:
        # latency of a loaded but not saturated server
        serving["poisson_0p8"] = run_serving(E, args.serving, args.serving_max_ns, lam,
                                             "fp32_polish")
        # FP64 arm: the same requests in plain FP64 (ground state and chains)
        serving["fp64"] = run_serving(E, args.serving, args.serving_max_ns, 0.0, "fp64")
        if args.serving_max_ns < 16:
            # the configured stream draws Ns up to 16 (D up to 1.66e8)
            serving["full_ns16"] = run_serving(E, 96, 16, 0.0, "fp32_polish")

    cpu = None
    if rank == 0 and args.cpu_baseline and not (m.Jx or m.Jp):
        # (the parallel oracle product covers the factorised part only)
        cpu = cpu_baseline(wl, args.cpu_steps)

    value, iters_s, t_max = combine_ranks(dist, tot["bytes"], tot["it"], t_s)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": wl.name, "dim": D, "norb": m.norb, "ns": m.ns,
                   "sector": [wl.nup, wl.ndw], "precision": "fp32 Lanczos + fp64 polish",
                   "gf": ("all orbitals, particle and hole chains (200 FP32 steps) concurrently, "
                          "512 Matsubara points, beta=100; spin down by symmetry")
                         if with_gf else "none (ground state only)",
                   "l2": "256 MB flush between steps; vectors "
                         f"{4 * D / 1e9:.2f} GB (FP32) > L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "iters_per_s": round(iters_s, 2),
        "matvecs_per_step": tot["mv"] / args.steps,
        "e0": last["e0"], "e0_raw": last["e0_raw"], "residual": last["residual"],
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": _profiled_traffic(args.workload),
                     "kernel": "FP32 block-major product w = H v (ed_matvec_blocked"
                               + (": H_up pass + H_dw pass)" if D > 1e9 else ", k_hv)"),
                     "peak_source": src, "products_ms": mv,
                     "kernel_ms": round(mv_ms, 4), "algorithmic_bytes": int(alg)},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "cpu_baseline": cpu, "serving": serving, "fp64_vs_fp32_polish": cmp, **subs,
    }
    print(json.dumps(line))


def time_products(E, wl, stream, dev, reps=20, which=("blocked_fp32",), kernel=None):
    """Median CUDA-event time of single H.v launches on the full sector
    (`kernel`: pin the block-major product kernel, else the autotuned one)."""
    import torch
    m = wl.model
    s = E.Sector(m, wl.nup, wl.ndw, stream=stream)
    D = s.dim
    out = {}
    for name in which:
        lay, prec = name.split("_")
        if kernel and lay == "blocked":
            s.set_kernel(kernel, prec)
            out[name + "_kernel"] = s.blocked_kernel(prec)
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
    out["kernel_choice"] = s.blocked_kernel("fp32")
    s.free()
    return out


def _nd_alg_bytes(m, nup, ndw, elem):
    """Algorithmic bytes of one H_nd launch: every element with at least one
    spin-exchange or pair-hopping term is read and written once, and every
    term reads one element of v (counted from the impurity masks)."""
    no, ns = m.norb, m.ns

    def per_mask(n):
        return [math.comb(ns - no, n - bin(mu).count("1"))
                if 0 <= n - bin(mu).count("1") <= ns - no else 0 for mu in range(1 << no)]
    cu, cd = per_mask(nup), per_mask(ndw)
    touched = terms = 0
    for mu in range(1 << no):
        for md in range(1 << no):
            t = 0
            for b in range(no):
                for a in range(no):
                    if a == b or not (mu >> b) & 1 or (mu >> a) & 1:
                        continue
                    t += bool(m.Jx) and bool((md >> a) & 1) and not (md >> b) & 1
                    t += bool(m.Jp) and bool((md >> b) & 1) and not (md >> a) & 1
            terms += t * cu[mu] * cd[md]
            touched += (t > 0) * cu[mu] * cd[md]
    return elem * (2 * touched + terms)


def run_full_kanamori(E, stream, dev, hbm):
    """Spin exchange and pair hopping (H_nd of Eq. Ham1): the FP32 product and
    the FP32 + polish ground state of the Ns = 15 three- and five-orbital
    full-Kanamori sectors against the same models without H_nd; the H_nd
    kernel's time is the difference of the two products."""
    import torch
    import workloads
    out = {}
    for name in ("full3_ns15", "full5_ns15"):
        wl = _workload(name)
        m = wl.model
        dd = workloads.Workload(wl.name + "_dd", workloads.ImpurityModel(
            norb=m.norb, nbath=m.nbath, U=m.U, Ust=m.Ust, Jh=m.Jh, e_imp=m.e_imp,
            e_bath=m.e_bath, v_bath=m.v_bath), wl.nup, wl.ndw)
        rec = {"dim": wl.dim, "Jx": m.Jx, "Jp": m.Jp}
        for tag, w in (("full", wl), ("dd", dd)):
            rec[f"product_fp32_ms_{tag}"] = time_products(E, w, stream, dev, reps=20)["blocked_fp32_ms"]
            s = E.Sector(w.model, w.nup, w.ndw, stream=stream)
            best = None
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = E.lanczos_ground(s, "fp32_polish", want_vector=False, stream=stream)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            s.free()
            rec[f"ground_fp32_polish_s_{tag}"] = round(best, 4)
            rec[f"e0_{tag}"] = r["e0"]
            rec[f"iterations_{tag}"] = r["iterations"] + r["polish_iterations"]
        nd_ms = rec["product_fp32_ms_full"] - rec["product_fp32_ms_dd"]
        alg = _nd_alg_bytes(m, wl.nup, wl.ndw, 4)
        rec["nd_kernel_ms"] = round(nd_ms, 4)
        rec["nd_algorithmic_bytes"] = int(alg)
        rec["nd_gbs"] = round(alg / (nd_ms / 1e3) / 1e9, 1) if nd_ms > 0 else None
        rec["nd_frac"] = round(alg / (nd_ms / 1e3) / 1e9 / hbm, 4) if nd_ms > 0 else None
        out[wl.name] = rec
    return out


def run_eph(E, stream, dev, nphs=(0, 2, 5, 10)):
    """The electron-phonon extension (Sec. 4) on the paper's phonon benchmark
    (Ns = 12, half-filled (6,6), one mode): ground state (FP32 + FP64 polish)
    time against the phonon cut-off N_ph, and the FP32 coupled product in
    sector order (CUDA events, median of 10)."""
    import torch
    import workloads
    out = {}
    for nph in nphs:
        wl = workloads.workload_eph_ns12(0, nph)
        x = wl.extra
        ph = E.phonon(x["w0"], x["g"], x["nph"])
        s = E.Sector(wl.model, wl.nup, wl.ndw, stream=stream)
        D = s.dim * (nph + 1)
        best, r = None, None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = E.eph_lanczos_ground(s, ph, "fp32_polish", stream=stream)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        v = torch.randn(D, dtype=torch.float32, device=dev)
        w = torch.empty_like(v)
        for _ in range(2):
            E.eph_matvec(s, ph, v, w, "fp32", stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        durs = []
        for _ in range(10):
            a.record(stream)
            E.eph_matvec(s, ph, v, w, "fp32", stream=stream)
            b.record(stream)
            b.synchronize()
            durs.append(a.elapsed_time(b))
        del v, w
        s.free()
        out[f"nph{nph}"] = {"dim": D, "ground_fp32_polish_s": round(best, 4), "e0": r["e0"],
                            "iterations": r["iterations"] + r["polish_iterations"],
                            "residual": r["residual"],
                            "product_fp32_ms": round(statistics.median(durs), 4)}
    return out


def run_matvec_only(args):
    """Product kernels alone (used for kernel profiling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_06806_gb300 as E
    torch.cuda.set_device(0)
    wl = _workload(args.workload)
    if args.sector:
        import workloads
        nup, ndw = (int(x) for x in args.sector.split(","))
        wl = workloads.Workload(f"{wl.name}_sector_{nup}_{ndw}", wl.model, nup, ndw)
    which = tuple(args.matvec_only.split(","))
    r = time_products(E, wl, torch.cuda.current_stream(), torch.device("cuda", 0),
                      reps=args.steps, which=which, kernel=args.kernel or None)
    hbm, src = _peaks()
    for k, v in list(r.items()):
        if not k.endswith("_ms"):
            continue
        elem = 8 if "fp64" in k else 4
        r[k.replace("_ms", "_gbs")] = round(2 * elem * wl.dim / (v / 1e3) / 1e9, 1)
    print(json.dumps({"workload": wl.name, "dim": wl.dim, "peak_gbs": hbm, **r}))


# ----------------------------------------------------------------- CPU (oracle) legs

def _oracle_tables(wl):
    """The oracle's per-spin pieces of the sector (Sec. 2.4): CSR H_up, H_dw,
    diagonal energies, impurity masks and the interaction table."""
    from oracle import fock
    m = wl.model
    map_up = fock.build_sector_map(m.ns, wl.nup)
    map_dw = map_up if wl.ndw == wl.nup else fock.build_sector_map(m.ns, wl.ndw)
    H_up = fock.spin_hopping_matrix(m, 0, wl.nup, map_up)
    H_dw = fock.spin_hopping_matrix(m, 1, wl.ndw, map_dw)
    E_up, m_up = fock.spin_diagonal(m, 0, wl.nup, map_up)
    E_dw, m_dw = fock.spin_diagonal(m, 1, wl.ndw, map_dw)
    return dict(H_up=H_up, H_dw=H_dw, E_up=E_up, E_dw=E_dw, m_up=m_up, m_dw=m_dw,
                W=fock.interaction_table(m), dim_up=len(map_up), dim_dw=len(map_dw))


_W = {}


def _worker_init(tables, shm_v, shm_w):
    """Worker process of the CPU legs: attaches the shared vectors."""
    import numpy as np
    from multiprocessing import shared_memory
    _W["t"] = tables
    _W["shm"] = [shared_memory.SharedMemory(name=shm_v), shared_memory.SharedMemory(name=shm_w)]
    shape = (tables["dim_dw"], tables["dim_up"])
    _W["V"] = np.ndarray(shape, dtype=np.float64, buffer=_W["shm"][0].buf)
    _W["Wm"] = np.ndarray(shape, dtype=np.float64, buffer=_W["shm"][1].buf)


def _worker_fill(r0, r1):
    """v rows [r0, r1): the Lanczos start-vector values u_i - 1/2 (SplitMix64,
    sector order) of those rows."""
    from workloads import splitmix64_uniform_array
    t = _W["t"]
    n = (r1 - r0) * t["dim_up"]
    _W["V"][r0:r1] = (splitmix64_uniform_array(0x5EED, n, r0 * t["dim_up"]) - 0.5).reshape(
        r1 - r0, t["dim_up"])
    return r1 - r0


def _worker_slab(r0, r1):
    """w rows [r0, r1) of the oracle's factorised product (Sec. 6.7 without
    MPI, the arithmetic of oracle.fock.Sector.matvec restricted to those dw
    rows): diagonal, H_up along each row, H_dw across rows."""
    t, V, Wm = _W["t"], _W["V"], _W["Wm"]
    t0 = time.perf_counter()
    Vs = V[r0:r1]
    D = t["E_up"][None, :] + t["E_dw"][r0:r1, None] + t["W"][t["m_up"][None, :],
                                                             t["m_dw"][r0:r1, None]]
    out = D * Vs
    out += (t["H_up"] @ Vs.T).T
    out += t["H_dw"][r0:r1] @ V
    Wm[r0:r1] = out
    return time.perf_counter() - t0


class OracleProduct:
    """The oracle's FP64 product on a full sector, split over dw-row slabs
    across worker processes (spawned: this process has used the GPU) that
    share v and w through shared memory.  Only the CPU legs of the benchmark
    use it."""

    def __init__(self, wl, workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import numpy as np
        self.t = _oracle_tables(wl)
        self.dim_dw, self.dim_up = self.t["dim_dw"], self.t["dim_up"]
        nbytes = 8 * self.dim_dw * self.dim_up
        self.shm = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(2)]
        ctx = mp.get_context("spawn")
        self.workers = workers
        self.pool = ctx.Pool(workers, initializer=_worker_init,
                             initargs=(self.t, self.shm[0].name, self.shm[1].name))
        nsl = max(workers * 4, 1)
        edges = np.linspace(0, self.dim_dw, nsl + 1).astype(int)
        self.slabs = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
        self.pool.starmap(_worker_fill, self.slabs)

    def product(self, slabs=None):
        """One product over `slabs` (default all rows); returns (seconds, rows)."""
        sl = self.slabs if slabs is None else slabs
        t0 = time.perf_counter()
        self.pool.starmap(_worker_slab, sl)
        return time.perf_counter() - t0, sum(b - a for a, b in sl)

    def one_core(self, slab):
        """One slab on one core (one worker)."""
        return self.pool.apply(_worker_slab, slab), slab[1] - slab[0]

    def close(self):
        self.pool.close()
        self.pool.join()
        for x in self.shm:
            x.close()
            x.unlink()


def cpu_baseline(wl, steps):
    """The oracle's product on the machine's host cores, same sector and metric:
    `steps` full products over all cores, and `steps` products of one dw-row
    slab on one core (bytes scaled to the slab)."""
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    op = OracleProduct(wl, cores)
    t_setup = time.perf_counter() - t0
    D = op.dim_dw * op.dim_up
    op.product()                                  # warm-up
    ts = [op.product()[0] for _ in range(steps)]
    slab = op.slabs[len(op.slabs) // 2]
    t1 = [op.one_core(slab)[0] for _ in range(steps)]
    op.close()
    rows1 = slab[1] - slab[0]
    val_all = 16.0 * D * steps / sum(ts) / 1e9
    val_one = 16.0 * rows1 * op.dim_up * steps / sum(t1) / 1e9
    return {"value": round(val_all, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 products of the oracle's factorised product (scipy CSR, "
                      f"Sec. 6.7) on the full D={D} sector, dw rows split over {cores} "
                      f"processes; setup (tables, start vector) {t_setup:.1f}s not timed",
            "seconds_per_product": round(sum(ts) / steps, 3),
            "one_core": {"value": round(val_one, 4), "unit": "GB/s", "cores": 1,
                         "sample": f"{steps} products of {rows1} of the {op.dim_dw} dw rows "
                                   "on one core",
                         "seconds_per_full_product_est": round(sum(t1) / steps * op.dim_dw
                                                               / rows1, 2)}}


def run_serving(E, n_requests, max_ns, rate=0.0, precision="fp32_polish"):
    """Serving stream: Poisson arrivals, mixed (Norb, Ns, sector); returns
    solves/s and p50/p99 latency of t_done - t_submit."""
    import numpy as np
    import workloads
    reqs = workloads.serving_stream(n_requests, rate_per_s=rate if rate > 0 else 1e9, seed=0,
                                    max_ns=max_ns)
    srv = E.Server(slots=8)
    gprec = "fp64" if precision == "fp64" else "fp32"
    b0 = E.batch_stats()
    t0 = time.perf_counter()
    tickets = []
    for q in reqs:
        now = time.perf_counter() - t0
        if q.arrival_s > now:
            time.sleep(q.arrival_s - now)
        tickets.append(srv.submit(q.workload.model, q.workload.nup, q.workload.ndw,
                                  precision=precision, gf_precision=gprec, nmats=GF["nmats"],
                                  beta=GF["beta"], gf_steps=GF["steps"]))
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
    b1 = E.batch_stats()
    lat = np.array(lat)
    return {"requests": n_requests, "completed_ok": int(ok), "solves_per_s": round(ok / wall, 3),
            "p50_s": round(float(np.percentile(lat, 50)), 4),
            "p99_s": round(float(np.percentile(lat, 99)), 4), "max_ns": max_ns,
            "precision": precision,
            "batched_chain_launches": b1["launches"] - b0["launches"],
            "batched_chains": b1["chains"] - b0["chains"],
            "arrival_rate_per_s": rate if rate > 0 else "all at once (saturation)",
            "work": ("FP32 ground state + FP64 polish + G(512 Matsubara, 200-step FP32 chains)"
                     if precision != "fp64" else
                     "FP64 ground state + G(512 Matsubara, 200-step FP64 chains)")
                    + " for every orbital and spin"}


# ----------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle (plain CPU FP64 implementation) on the host cores, same
    metric on the same workload: each step is one oracle product over a
    fixed quarter of the dw rows (all cores), a bounded sample of the
    solve's products."""
    dist, rank, ws = _dist()
    if rank != 0:
        return
    wl = _workload(args.workload)
    cores = os.cpu_count() or 1
    op = OracleProduct(wl, cores)
    q = max(1, len(op.slabs) // 4)
    sample = op.slabs[:q]
    for _ in range(args.warmup):
        op.product(sample)
    times, rows = [], 0
    for _ in range(args.steps):
        t, rows = op.product(sample)
        times.append(t)
    op.close()
    t = sum(times)
    value = 16.0 * rows * op.dim_up * args.steps / t / 1e9
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "dim": wl.dim, "parallelism": "host CPU"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"per step one FP64 oracle product over {rows} of the "
                                       f"{op.dim_dw} dw rows (scipy factorised product, rows "
                                       f"split over {cores} processes)"},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    import workloads
    ap.add_argument("--workload", default="ns18", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--no-gf", dest="gf", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-sub-ns16", dest="sub_ns16", action="store_false")
    ap.add_argument("--no-full-kanamori", dest="full_kanamori", action="store_false")
    ap.add_argument("--no-eph", dest="eph", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--serving", type=int, default=1000,
                    help="requests of each serving stream (0: off)")
    ap.add_argument("--serving-max-ns", type=int, default=12)
    ap.add_argument("--matvec-only", default="",
                    help="comma list of {blocked,sector}_{fp32,fp64}: time products only")
    ap.add_argument("--sector", default="",
                    help="with --matvec-only: another sector 'NUP,NDW' of the workload's model")
    ap.add_argument("--kernel", default="",
                    help="with --matvec-only: pin the block-major kernel "
                         "(tiled, two_pass, elementwise)")
    args = ap.parse_args()
    if args.matvec_only:
        run_matvec_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
