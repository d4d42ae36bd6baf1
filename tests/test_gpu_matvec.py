"""a3 on the GPU: w = H v through ed_matvec against the oracle's factorised
product, element by element, FP64 and FP32, on sizes that span several CTAs,
ragged last CTAs, the flattened and the row-loop paths, the shared-memory and
the global-memory staging; plus sampled outputs at the full workload sizes.

Tolerances: FP64 |dw| <= 1e-13 * (sum of |terms| bound) ; FP32 relative to the
same bound <= 2e-6 (FP32 row sums of at most ~30 terms)."""
import numpy as np
import pytest
import torch

from oracle import fock
from workloads import (make_model, workload_ns8, workload_ns14, workload_ns16, workload_ns18,
                       ImpurityModel)

pytestmark = pytest.mark.gpu


def _bound(ref_sector, v):
    """Elementwise bound sum_k |H_ik| |v_k| (scale of the rounding error)."""
    s = ref_sector
    V = np.abs(v).reshape(s.dim_dw, s.dim_up)
    B = np.abs(s.diagonal()) * V + (abs(s.H_up) @ V.T).T + abs(s.H_dw) @ V
    return B.reshape(-1)


SMALL = [
    (workload_ns8().model, 4, 4),                              # D_up=70 < CTA: flattened
    (make_model(2, 4, U=3.0, Jh=0.5, seed=6), 5, 4),           # Ns=10, D=252*210
    (make_model(1, 11, U=2.5, e_d=-1.2, seed=7), 6, 5),        # Ns=12, D_up=924 row loop
    (make_model(1, 16, U=2.0, e_d=-1.0, seed=8), 8, 1),        # Ns=17: D_up=24310, FP64 row
                                                               # beyond shared memory
    (make_model(3, 2, U=2.0, Jh=0.3, seed=9), 0, 9),           # empty up string, full down
]


@pytest.mark.parametrize("ci", range(len(SMALL)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matvec_elementwise(ed, ci, prec):
    m, nup, ndw = SMALL[ci]
    ref = fock.Sector(m, nup, ndw)
    s = ed.Sector(m, nup, ndw)
    rng = np.random.default_rng(100 + ci)
    v = rng.uniform(-1, 1, ref.dim)
    want = ref.matvec(v)
    dt = torch.float64 if prec == "fp64" else torch.float32
    vt = torch.tensor(v, dtype=dt, device="cuda")
    wt = torch.full_like(vt, float("nan"))
    ed.matvec(s, vt, wt, prec)
    torch.cuda.synchronize()
    got = wt.double().cpu().numpy()
    if prec == "fp32":
        # the FP32 path sees the input rounded to FP32 and FP32 matrix elements
        v_used, tol = vt.double().cpu().numpy(), 4e-6
    else:
        v_used, tol = v, 1e-13
    want = ref.matvec(v_used)
    bnd = _bound(ref, v_used)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - want) <= tol * bnd)
    s.free()


def test_matvec_hermitian(ed):
    m = make_model(2, 4, U=3.0, Jh=0.5, seed=6)
    s = ed.Sector(m, 5, 5)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.normal(size=s.dim), device="cuda")
    y = torch.tensor(rng.normal(size=s.dim), device="cuda")
    hx, hy = torch.empty_like(x), torch.empty_like(y)
    ed.matvec(s, x, hx)
    ed.matvec(s, y, hy)
    a, b = float(torch.dot(x, hy)), float(torch.dot(hx, y))
    assert abs(a - b) <= 1e-12 * max(1, abs(a))


def _sampled_reference(ref, v_host_fn, rows, cols):
    """Oracle product at sampled (r, c) computed entry by entry from the
    oracle's per-spin tables (Eq. Hbuild): needs only rows k of v."""
    out = []
    for r, c in zip(rows, cols):
        d = ref.E_up[c] + ref.E_dw[r] + ref.W[ref.m_up[c], ref.m_dw[r]]
        acc = d * v_host_fn(r, c)
        hu = ref.H_up
        for k in range(hu.indptr[c], hu.indptr[c + 1]):
            acc += hu.data[k] * v_host_fn(r, hu.indices[k])
        hd = ref.H_dw
        for k in range(hd.indptr[r], hd.indptr[r + 1]):
            acc += hd.data[k] * v_host_fn(hd.indices[k], c)
        out.append(acc)
    return np.array(out)


def _lite_sector(model, nup, ndw):
    """Oracle per-spin pieces only (no explicit sector matrix)."""
    class S:
        pass
    S.map_up = fock.build_sector_map(model.ns, nup)
    S.map_dw = S.map_up if ndw == nup else fock.build_sector_map(model.ns, ndw)
    S.H_up = fock.spin_hopping_matrix(model, 0, nup, S.map_up)
    S.H_dw = fock.spin_hopping_matrix(model, 1, ndw, S.map_dw)
    S.E_up, S.m_up = fock.spin_diagonal(model, 0, nup, S.map_up)
    S.E_dw, S.m_dw = fock.spin_diagonal(model, 1, ndw, S.map_dw)
    S.W = fock.interaction_table(model)
    return S


@pytest.mark.parametrize("maker", [workload_ns14, workload_ns16, workload_ns18])
def test_matvec_full_size_sampled(ed, maker):
    """Full-size product in the launch configuration of the benchmark (FP32,
    the input is a closed-form function of the index so the oracle can
    evaluate any entry), checked on sampled outputs."""
    wl = maker(0)
    m = wl.model
    s = ed.Sector(m, wl.nup, wl.ndw)
    dup, ddw = s.dim_up, s.dim_dw
    n = s.dim
    # v[i] = sin(0.37 i) + cos(0.011 i) computed in FP64 then rounded to FP32
    v = torch.empty(n, device="cuda", dtype=torch.float32)
    step = 1 << 27
    for o in range(0, n, step):
        idx = torch.arange(o, min(n, o + step), device="cuda", dtype=torch.float64)
        v[o:o + len(idx)] = (torch.sin(0.37 * idx) + torch.cos(0.011 * idx)).float()
    del idx
    w = torch.empty_like(v)
    ed.matvec(s, v, w, "fp32")
    torch.cuda.synchronize()
    ref = _lite_sector(m, wl.nup, wl.ndw)

    def vf(r, c):
        i = int(r) * int(dup) + int(c)
        return float(np.float32(np.sin(0.37 * i) + np.cos(0.011 * i)))
    rng = np.random.default_rng(5)
    rows = np.concatenate([[0, ddw - 1, ddw // 2], rng.integers(0, ddw, 40)])
    cols = np.concatenate([[0, dup - 1, dup // 3], rng.integers(0, dup, 40)])
    want = _sampled_reference(ref, vf, rows, cols)
    flat = torch.tensor(rows.astype(np.int64) * dup + cols.astype(np.int64), device="cuda")
    got = w[flat].double().cpu().numpy()
    assert np.abs(got - want).max() <= 2e-5 * max(1.0, np.abs(want).max())
    s.free()


@pytest.mark.parametrize("ci", range(len(SMALL)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_major_layout(ed, ci, prec):
    """Block-major order: the permutation round-trips exactly, is a
    permutation of the entries, and the block-major product equals the
    sector-order product up to rounding (only the summation order of the
    H_up terms differs)."""
    m, nup, ndw = SMALL[ci]
    ref = fock.Sector(m, nup, ndw)
    s = ed.Sector(m, nup, ndw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(ci)
    v = torch.rand(s.dim, device="cuda", dtype=dt, generator=g) * 2 - 1
    assert s.blocked_dim == s.dim_dw * s.blocked_stride and s.blocked_stride % 4 == 0
    vb = torch.full((s.blocked_dim,), float("nan"), device="cuda", dtype=dt)
    back = torch.empty_like(v)
    ed.permute(s, v, vb, True, prec)
    ed.permute(s, vb, back, False, prec)
    assert torch.equal(back, v)
    pad = torch.zeros(s.blocked_dim - s.dim, device="cuda", dtype=dt)
    assert torch.equal(torch.sort(vb).values, torch.sort(torch.cat([v, pad])).values)
    w, w2 = torch.empty_like(v), torch.empty_like(v)
    wb = torch.empty_like(vb)
    ed.matvec(s, v, w, prec)
    ed.matvec_blocked(s, vb, wb, prec)
    ed.permute(s, wb, w2, False, prec)
    bnd = _bound(ref, v.double().cpu().numpy())
    tol = 1e-13 if prec == "fp64" else 4e-6
    assert np.all(np.abs((w2 - w).double().cpu().numpy()) <= tol * bnd)
    s.free()


# Both one-pass block-major product kernels against the oracle element by
# element, each pinned in turn (ed_sector_set_kernel): one, two and three
# orbitals, ragged sectors off half filling, several work items per block
# pair; the two kernels must also agree bit for bit (they take the same
# operations per element in the same order).
KERNEL_CASES = [
    (make_model(2, 4, U=3.0, Jh=0.5, seed=6), 5, 4),      # D = 52,920 (below the tuning range)
    (make_model(1, 11, U=2.5, e_d=-1.2, seed=7), 6, 5),   # D = 731,808
    (make_model(3, 3, U=2.5, Jh=0.4, seed=14), 6, 5),     # D = 731,808
    (make_model(1, 13, U=4.0, e_d=-2.0, seed=11), 7, 6),  # D = 10,306,296
    (make_model(2, 6, U=3.0, Jh=0.5, seed=12), 5, 6),     # D = 6,012,006
    (make_model(3, 4, U=2.5, Jh=0.4, seed=13), 5, 4),     # D = 4,099,095
]


@pytest.mark.parametrize("ci", range(len(KERNEL_CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blocked_kernels_against_oracle(ed, ci, prec):
    m, nup, ndw = KERNEL_CASES[ci]
    s = ed.Sector(m, nup, ndw)
    assert s.blocked_kernel(prec) in ("tiled", "elementwise")
    ref = fock.Sector(m, nup, ndw)
    rng = np.random.default_rng(200 + ci)
    dt = torch.float64 if prec == "fp64" else torch.float32
    v = torch.tensor(rng.uniform(-1, 1, ref.dim), dtype=dt, device="cuda")
    vb = torch.empty(s.blocked_dim, dtype=dt, device="cuda")
    ed.permute(s, v, vb, True, prec)
    v_used = v.double().cpu().numpy()
    want = ref.matvec(v_used)
    bnd = _bound(ref, v_used)
    tol = 1e-13 if prec == "fp64" else 4e-6
    out = {}
    for kernel in ("tiled", "elementwise"):
        s.set_kernel(kernel, prec)
        assert s.blocked_kernel(prec) == kernel
        wb = torch.full_like(vb, float("nan"))
        w = torch.empty_like(v)
        ed.matvec_blocked(s, vb, wb, prec)
        ed.permute(s, wb, w, False, prec)
        torch.cuda.synchronize()
        got = w.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - want) <= tol * bnd), kernel
        # the padding entries of the block-major output are never written
        assert np.count_nonzero(np.isnan(wb.double().cpu().numpy())) == s.blocked_dim - ref.dim
        out[kernel] = wb
    assert torch.equal(out["tiled"].nan_to_num(), out["elementwise"].nan_to_num())
    s.free()


def test_autotuner_picks_the_faster_kernel_per_shape(ed):
    """Sectors above 2^17 padded elements: the first sector of a model
    shape (Norb, Nbath, precision) times both kernels and uses the faster;
    another sector of the same shape (other parameters, other fillings)
    inherits the choice without timing."""
    m1 = make_model(2, 5, U=2.0, Jh=0.3, seed=41)  # Norb=2, Nbath=5 (Ns=12)
    m2 = make_model(2, 5, U=3.5, Jh=0.6, seed=42)
    s1 = ed.Sector(m1, 6, 5)  # D = 731,808
    k1, ms1 = s1.tune_info("fp32")
    s2 = ed.Sector(m2, 5, 7)  # D = 627,264
    k2, ms2 = s2.tune_info("fp32")
    assert k1 == k2 and k1 in ("tiled", "elementwise")
    assert ms2 == {"tiled": -1.0, "elementwise": -1.0}
    if ms1["tiled"] >= 0:  # this process had not tuned the shape before
        assert ms1["elementwise"] > 0 and ms1["tiled"] > 0
        assert k1 == ("elementwise" if ms1["elementwise"] < ms1["tiled"] else "tiled")
    # below the tuning range the element-parallel kernel is used without timing
    s3 = ed.Sector(make_model(1, 7, U=2.0, seed=43), 4, 4)
    assert s3.tune_info("fp32") == ("elementwise", {"tiled": -1.0, "elementwise": -1.0})
    for s in (s1, s2, s3):
        s.free()


@pytest.mark.parametrize("maker,prec,kernel", [
    (workload_ns16, "fp32", "tiled"),
    (workload_ns16, "fp64", "two_pass"), (workload_ns16, "fp64", "elementwise"),
    (workload_ns18, "fp32", "two_pass"), (workload_ns18, "fp32", "elementwise")])
def test_full_size_sampled(ed, maker, prec, kernel):
    """The full-size products of the Lanczos runs, checked on sampled outputs
    against the oracle (input a closed-form function of the sector index):
    the one-pass tiled block-major product at Ns=16 in FP32 (the kernel the
    benchmark times and the FP32 Lanczos runs use there), the two-pass
    block-major product (H_up pass, then H_dw pass over column chunks; taken
    where the block pairs exceed L2) and the element-parallel product with
    several chunks of 256 elements per CTA (10 at Ns=16, 141 at Ns=18), the
    kernels the autotuner chooses between at these sizes."""
    wl = maker(0)
    m = wl.model
    s = ed.Sector(m, wl.nup, wl.ndw)
    s.set_kernel(kernel, prec)
    assert s.blocked_kernel(prec) == kernel
    dup, ddw, n = s.dim_up, s.dim_dw, s.dim
    dt = torch.float64 if prec == "fp64" else torch.float32
    v = torch.empty(n, device="cuda", dtype=dt)
    step = 1 << 27
    for o in range(0, n, step):
        idx = torch.arange(o, min(n, o + step), device="cuda", dtype=torch.float64)
        v[o:o + len(idx)] = (torch.sin(0.37 * idx) + torch.cos(0.011 * idx)).to(dt)
    del idx
    vb = torch.empty(s.blocked_dim, device="cuda", dtype=dt)
    ed.permute(s, v, vb, True, prec)
    wb = torch.empty_like(vb)
    ed.matvec_blocked(s, vb, wb, prec)
    del vb
    w = v  # reuse the memory: v is no longer needed on the device
    ed.permute(s, wb, w, False, prec)
    del wb
    torch.cuda.synchronize()
    ref = _lite_sector(m, wl.nup, wl.ndw)

    def vf(r, c):
        i = int(r) * int(dup) + int(c)
        x = np.sin(0.37 * i) + np.cos(0.011 * i)
        return float(np.float32(x)) if prec == "fp32" else float(x)
    rng = np.random.default_rng(9)
    rows = np.concatenate([[0, ddw - 1, ddw // 2], rng.integers(0, ddw, 40)])
    cols = np.concatenate([[0, dup - 1, dup // 3], rng.integers(0, dup, 40)])
    want = _sampled_reference(ref, vf, rows, cols)
    flat = torch.tensor(rows.astype(np.int64) * dup + cols.astype(np.int64), device="cuda")
    got = w[flat].double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max())
    s.free()


def test_vector_length_checked(ed):
    """Mismatched vector lengths are rejected before any kernel runs."""
    s = ed.Sector(workload_ns8().model, 4, 4)
    assert s.blocked_dim != s.dim          # 70 columns padded to 72
    v = torch.zeros(s.dim, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(v)
    with pytest.raises(ed.EDError) as e:
        ed.matvec_blocked(s, v, w)
    assert e.value.status == ed.ED_ERR_ARG
    vb = torch.zeros(s.blocked_dim, dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError):
        ed.matvec(s, vb, torch.zeros_like(vb))
    with pytest.raises(ed.EDError):
        ed.permute(s, v, torch.zeros_like(v), True)
    # block-major vectors are accessed as 16-byte vectors: an offset view of
    # the right length is rejected on the host
    big = torch.zeros(s.blocked_dim + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError) as e:
        ed.matvec_blocked(s, big[1:], torch.zeros_like(vb))
    assert e.value.status == ed.ED_ERR_ARG
    s.free()


def test_tiled_family_bit_identical_to_elementwise_ns18(ed):
    """Ns=18 (D = 2,363,904,400), FP32: the product the Lanczos runs use here
    (the tiled family: one pass on the block pairs that fit L2, two passes
    on the larger ones) gives the same w bit for bit as the element-parallel
    product (the same order of operations per element), which
    test_full_size_sampled pins against the oracle at this size."""
    wl = workload_ns18(0)
    s = ed.Sector(wl.model, wl.nup, wl.ndw)
    g = torch.Generator(device="cuda").manual_seed(18)
    vs = torch.empty(s.dim, dtype=torch.float32, device="cuda")
    step = 1 << 28
    for o in range(0, s.dim, step):
        n = min(step, s.dim - o)
        vs[o:o + n] = torch.rand(n, dtype=torch.float32, device="cuda", generator=g) - 0.5
    v = torch.empty(s.blocked_dim, dtype=torch.float32, device="cuda")
    ed.permute(s, vs, v, True, "fp32")       # padding columns written as zero
    del vs
    out = {}
    for kernel in ("two_pass", "elementwise"):
        s.set_kernel(kernel, "fp32")
        w = torch.zeros_like(v)              # padding is not written: stays zero
        ed.matvec_blocked(s, v, w, "fp32")
        out[kernel] = w
    torch.cuda.synchronize()
    assert torch.equal(out["two_pass"], out["elementwise"])
    assert bool(torch.isfinite(out["two_pass"]).all())
    s.free()
