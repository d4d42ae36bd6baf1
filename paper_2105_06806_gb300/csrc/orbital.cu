// Per-orbital sectors (Sec. 2.2, N_ud = Norb).  The block-major order of a
// sector is already the concatenation of its finer sectors: a block pair (one
// up block x one dw block, blocks labelled by the per-orbital occupations) is
// one finer sector, and H maps it to itself (Sec. 2.4: H_sigma is a Kronecker
// sum over the orbital groups; the diagonal and the density-density
// interaction are diagonal).  The product kernels address vectors only
// through their work items (absolute rows, padded columns) and the row
// stride, so a finer sector's vectors are the block pair's [rows][padded
// columns] alone: the kernels get the block pair's items, the block's padded
// width as stride and a base pointer shifted by the block pair's first row
// and column (every access stays inside the block pair).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

struct OrbView {
  int bu = -1, bd = -1;
  int64_t R0 = 0, nr = 0;    // rows of the dw block
  int64_t C0 = 0, nc = 0;    // block-major columns of the up block
  int64_t C0p = 0, ncp = 0;  // its padded columns
};

int find_block(const BlockInfo &b, int norb, const int32_t *occ) {
  for (int k = 0; k < b.nblocks; ++k) {
    bool eq = true;
    for (int a = 0; a < norb; ++a)
      if (b.keys[(size_t)k * norb + a] != occ[a]) eq = false;
    if (eq) return k;
  }
  return -1;
}

ed_status make_view(ed_sector s, const int32_t *nu, const int32_t *nd, OrbView *v) {
  if (!s || !nu || !nd) return ED_ERR_ARG;
  const int norb = s->mp.norb;
  v->bu = find_block(s->bi[0], norb, nu);
  v->bd = find_block(s->bi[1], norb, nd);
  if (v->bu < 0 || v->bd < 0) return ED_ERR_ARG;
  v->R0 = s->bi[1].offset[v->bd];
  v->nr = s->bi[1].offset[v->bd + 1] - v->R0;
  v->C0 = s->bi[0].offset[v->bu];
  v->nc = s->bi[0].offset[v->bu + 1] - v->C0;
  v->C0p = s->up_off_pad[v->bu];
  v->ncp = s->up_off_pad[v->bu + 1] - v->C0p;
  return ED_OK;
}

// seeded start vector on the finer sector's [rows][padded columns], padding zero
template <typename T>
__global__ void k_orb_start(T *v, int64_t nr, int64_t ncp, int64_t C0p, const int32_t *padinv,
                            uint64_t seed) {
  const int64_t n = nr * ncp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i % ncp;
    T x = T(0);
    if (padinv[C0p + c] >= 0) {
      const double u = (double)(ed_splitmix64_at(seed, (uint64_t)i) >> 11) *
                       (1.0 / 9007199254740992.0);
      x = (T)(u - 0.5);
    }
    v[i] = x;
  }
}

// the finer sector's vector into a sector-order vector of s (zero elsewhere)
template <typename Ti, typename To>
__global__ void k_orb_scatter(const Ti *in, To *out, int64_t R0, int64_t nr, int64_t ncp,
                              int64_t C0p, const int32_t *pidx_dw, const int32_t *pidx_up,
                              const int32_t *padinv, int64_t dup) {
  const int64_t n = nr * ncp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ncp, c = i - r * ncp;
    const int32_t cb = padinv[C0p + c];
    if (cb < 0) continue;
    out[(int64_t)pidx_dw[R0 + r] * dup + pidx_up[cb]] = (To)in[i];
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

struct Mem {
  void *p = nullptr;
  cudaStream_t cs = nullptr;
  ~Mem() {
    if (p) ed_dfree(p, cs);
  }
  ed_status alloc(size_t bytes, cudaStream_t st, const char *what) {
    cs = st;
    return ed_dmalloc(&p, std::max<size_t>(bytes, 256), st, what);
  }
};

// The block pair's work items of precision T (both passes of the two-pass
// product where the sector uses it), copied to the device.
template <typename T>
ed_status view_tables(ed_sector s, const OrbView &v, Mem &store, HvTables<T> *tb, cudaStream_t cs) {
  const int e = sizeof(T) == 8 ? 1 : 0;
  ED_TRY(ed_build_items(s, 1, (int)sizeof(T)));
  const ItemList &il = s->items[1][e];
  std::vector<HvItem> all(il.nitems), keep;
  std::vector<DwItem> dall(il.nditems), dkeep;
  if (il.nitems)
    ED_TRY_CUDA(cudaMemcpy(all.data(), il.d_items, il.nitems * sizeof(HvItem), cudaMemcpyDeviceToHost));
  if (il.nditems)
    ED_TRY_CUDA(cudaMemcpy(dall.data(), il.d_ditems, il.nditems * sizeof(DwItem), cudaMemcpyDeviceToHost));
  for (const HvItem &it : all)
    if (it.r0 >= v.R0 && it.r0 < v.R0 + v.nr && it.c0 == v.C0) keep.push_back(it);
  for (const DwItem &it : dall)
    if (it.r0 >= v.R0 && it.r0 < v.R0 + v.nr && it.c0p >= v.C0p && it.c0p < v.C0p + v.ncp)
      dkeep.push_back(it);
  const size_t ib = (keep.size() * sizeof(HvItem) + 255) & ~(size_t)255;
  ED_TRY(store.alloc(ib + dkeep.size() * sizeof(DwItem) + 256, cs, "finer-sector items"));
  HvItem *d_items = (HvItem *)store.p;
  DwItem *d_ditems = (DwItem *)((char *)store.p + ib);
  if (!keep.empty())
    ED_TRY_CUDA(cudaMemcpyAsync(d_items, keep.data(), keep.size() * sizeof(HvItem),
                                cudaMemcpyHostToDevice, cs));
  if (!dkeep.empty())
    ED_TRY_CUDA(cudaMemcpyAsync(d_ditems, dkeep.data(), dkeep.size() * sizeof(DwItem),
                                cudaMemcpyHostToDevice, cs));
  *tb = ed_hv_tables<T>(s, 1);
  tb->items = d_items;
  tb->nitems = (int64_t)keep.size();
  tb->ditems = il.d_ditems ? d_ditems : nullptr;
  tb->nditems = il.d_ditems ? (int64_t)dkeep.size() : 0;
  tb->small_cols = nullptr;  // the tiled family: the items carry the block pair
  tb->stride = v.ncp;
  tb->nd_up = nullptr;
  return ED_OK;
}

template <typename T>
LinOp<T> view_op(ed_sector s, const OrbView &v, const HvTables<T> &tb) {
  LinOp<T> op;
  op.n = v.nr * v.ncp;
  const int64_t shift = v.R0 * v.ncp + v.C0p;
  op.apply = [s, tb, shift](const T *x, T *w, cudaStream_t cs) {
    // base pointers moved so that [row * ncp + padded column] of the block
    // pair lands on the finer sector's [row - R0][column - C0p]
    const T *xs = (const T *)((uintptr_t)x - (uintptr_t)shift * sizeof(T));
    T *ws = (T *)((uintptr_t)w - (uintptr_t)shift * sizeof(T));
    return ed_launch_hv<T>(s, tb, HV_PLAIN, xs, ws, nullptr, nullptr, nullptr, nullptr, nullptr, cs);
  };
  return op;
}

}  // namespace

extern "C" ed_status ed_orbital_sector_dims(ed_sector s, const int32_t *nup_orb,
                                            const int32_t *ndw_orb, int64_t *dim_up,
                                            int64_t *dim_dw) {
  OrbView v;
  ED_TRY(make_view(s, nup_orb, ndw_orb, &v));
  if (dim_up) *dim_up = v.nc;
  if (dim_dw) *dim_dw = v.nr;
  return ED_OK;
}

extern "C" ed_status ed_lanczos_ground_orbital(ed_sector s, const int32_t *nup_orb,
                                               const int32_t *ndw_orb, const ed_lanczos_opts *o,
                                               ed_lanczos_result *res, void *d_psi, void *stream) {
  if (!s || !o || !res) return ED_ERR_ARG;
  if (s->mp.Jx != 0.0 || s->mp.Jp != 0.0) {
    ed_set_error_msg("per-orbital sectors need J_X = J_P = 0");
    return ED_ERR_UNSUPPORTED;
  }
  OrbView v;
  ED_TRY(make_view(s, nup_orb, ndw_orb, &v));
  memset(res, 0, sizeof(*res));
  const int maxit = o->max_iter > 0 ? o->max_iter : 512;
  if (maxit > ED_MAX_LANCZOS) return ED_ERR_ARG;
  const ed_precision prec = o->precision;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  const double tol = o->tol > 0 ? o->tol : (prec == ED_FP64 ? 1e-12 : 1e-6);
  cudaStream_t cs = (cudaStream_t)stream;
  const int64_t n = v.nr * v.ncp;
  Mem it64, psi64, start;
  HvTables<double> tb64;
  ED_TRY(view_tables<double>(s, v, it64, &tb64, cs));
  const LinOp<double> op64 = view_op<double>(s, v, tb64);
  ED_TRY(psi64.alloc((size_t)n * 8, cs, "finer-sector ground state"));
  OpRun run;
  int mv = 0, mv32 = 0;
  if (prec == ED_FP64) {
    ED_TRY(start.alloc((size_t)n * 8, cs, "finer-sector start vector"));
    k_orb_start<double><<<grid_of(n), 256, 0, cs>>>((double *)start.p, v.nr, v.ncp, v.C0p,
                                                    s->padinv, o->seed);
    ED_LAUNCHED(1);
    ED_TRY(ed_op_lanczos<double>(op64, (const double *)start.p, maxit, tol, true, &run, nullptr,
                                 (double *)psi64.p, cs));
    mv = run.matvecs;
    res->e0 = res->e0_raw = run.theta;
  } else {
    Mem it32, psi32, s32;
    HvTables<float> tb32;
    ED_TRY(view_tables<float>(s, v, it32, &tb32, cs));
    ED_TRY(psi32.alloc((size_t)n * 4, cs, "finer-sector FP32 ground state"));
    ED_TRY(s32.alloc((size_t)n * 4, cs, "finer-sector start vector"));
    k_orb_start<float><<<grid_of(n), 256, 0, cs>>>((float *)s32.p, v.nr, v.ncp, v.C0p, s->padinv,
                                                   o->seed);
    ED_LAUNCHED(1);
    ED_TRY(ed_op_lanczos<float>(view_op<float>(s, v, tb32), (const float *)s32.p, maxit, tol, true,
                                &run, nullptr, (float *)psi32.p, cs));
    mv = mv32 = run.matvecs;
    res->e0 = res->e0_raw = run.theta;
    ED_TRY((ed_op_normalised_copy<float, double>((const float *)psi32.p, (double *)psi64.p, n, cs)));
    if (prec == ED_FP32_POLISH) {
      const int steps = o->polish_steps > 0 ? o->polish_steps : 4;
      ED_TRY(start.alloc((size_t)n * 8, cs, "polish start"));
      ED_TRY_CUDA(cudaMemcpyAsync(start.p, psi64.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, cs));
      OpRun pol;
      ED_TRY(ed_op_lanczos<double>(op64, (const double *)start.p, steps, 1e-300, true, &pol,
                                   nullptr, (double *)psi64.p, cs));
      mv += pol.matvecs;
      res->e0 = pol.theta;
      res->polish_iterations = pol.k;
    } else if (d_psi) {
      ED_TRY_CUDA(cudaMemsetAsync(d_psi, 0, (size_t)s->dim * 4, cs));
      k_orb_scatter<float, float><<<grid_of(n), 256, 0, cs>>>(
          (const float *)psi32.p, (float *)d_psi, v.R0, v.nr, v.ncp, v.C0p, s->bi[1].pidx,
          s->bi[0].pidx, s->padinv, s->sp[0].dim);
      ED_LAUNCHED(1);
    }
  }
  res->iterations = run.k;
  res->residual_estimate = run.resid_est;
  res->stop_reason = run.stop;
  double e = 0.0, r = 0.0;
  ED_TRY(ed_op_residual(op64, (const double *)psi64.p, &e, &r, cs));
  ++mv;
  res->residual = r;
  if (d_psi && prec != ED_FP32) {
    ED_TRY_CUDA(cudaMemsetAsync(d_psi, 0, (size_t)s->dim * 8, cs));
    k_orb_scatter<double, double><<<grid_of(n), 256, 0, cs>>>(
        (const double *)psi64.p, (double *)d_psi, v.R0, v.nr, v.ncp, v.C0p, s->bi[1].pidx,
        s->bi[0].pidx, s->padinv, s->sp[0].dim);
    ED_LAUNCHED(1);
  }
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  res->matvecs = mv;
  res->matvecs_fp64 = mv - mv32;
  if (run.stop == 2) {
    ed_set_error_msg("max_iter reached before the Lanczos tolerance");
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}
