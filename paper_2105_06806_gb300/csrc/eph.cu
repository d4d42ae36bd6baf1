// Electron-phonon (Holstein) extension (Sec. 4): one local phonon mode,
// H = H_e + w0 b^+ b + sum_{alpha sigma} g_alpha n_{alpha sigma} (b + b^+),
// phonon number cut off at N_ph.  A coupled vector is D_ph = N_ph + 1
// electronic vectors (phonon slices, phonon index slowest, Eq. Vdecomp2);
// the sector matrix is Eq. HephBuild.
//
// Product: the electronic product kernels on every slice (the slices are
// independent for H_e), then one pass k_phonon over the electronic elements
// that walks each element's D_ph slices with a three-value window, adding
// w0 p v[p] + N_g (sqrt(p) v[p-1] + sqrt(p+1) v[p+1]): v is read once and w
// read and written once (the paper's observation that the phonon terms stay
// local to an electronic element, Sec. 4.4).  N_g = sum_alpha g_alpha
// (n_{alpha up} + n_{alpha dw}) comes from the two impurity masks through a
// 2^Norb table.  The Lanczos solves run through the operator-generic driver.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int PH_THREADS = 256;

struct PhParams {
  double w0;
  double gm[1 << ED_MAX_NORB];  // sum_alpha g_alpha over the bits of an impurity mask
  int nph;
};

bool make_params(const ed_sector s, const ed_phonon *ph, PhParams *out) {
  if (!ph || ph->nph < 0 || ph->nph > ED_MAX_NPH || !isfinite(ph->w0)) return false;
  memset(out, 0, sizeof(*out));
  out->w0 = ph->w0;
  out->nph = ph->nph;
  const int norb = s->mp.norb;
  for (int a = 0; a < norb; ++a)
    if (!isfinite(ph->g[a])) return false;
  for (int m = 0; m < (1 << norb); ++m) {
    double t = 0.0;
    for (int a = 0; a < norb; ++a)
      if ((m >> a) & 1) t += ph->g[a];
    out->gm[m] = t;
  }
  return true;
}

// w[p][i] += w0 p v[p][i] + N_g(i) (sqrt(p) v[p-1][i] + sqrt(p+1) v[p+1][i])
// for every electronic element i of a slice (padding columns skipped).
// Layout: element i = r * stride + c; the up mask of column c is
// mup[padinv ? padinv[c] : c] (padinv < 0: padding), the dw mask mdw[r].
template <typename T>
__global__ void __launch_bounds__(PH_THREADS) k_phonon(const T *v, T *w, int64_t slice,
                                                       int64_t stride, const int32_t *padinv,
                                                       const uint8_t *mup, const uint8_t *mdw,
                                                       PhParams ph) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slice;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / stride, c = i - r * stride;
    int64_t cu = c;
    if (padinv) {
      cu = padinv[c];
      if (cu < 0) continue;
    }
    const T ng = (T)(ph.gm[mup[cu]] + ph.gm[mdw[r]]);
    const T w0 = (T)ph.w0;
    T xm = T(0), x0 = v[i];
    for (int p = 0; p <= ph.nph; ++p) {
      const T xp = p < ph.nph ? v[(int64_t)(p + 1) * slice + i] : T(0);
      const T sp = sqrt((T)p), sp1 = sqrt((T)(p + 1));
      const T disp = sp * xm + sp1 * xp;
      T *o = w + (int64_t)p * slice + i;
      *o = *o + (w0 * (T)p * x0 + ng * disp);
      xm = x0;
      x0 = xp;
    }
  }
}

// Seeded start vector over padded block-major slices: element (p, r', pc)
// holds u - 1/2 with u the uniform double of SplitMix64 output
// p * D + pidx_dw[r'] * D_up + pidx_up[padinv[pc]] (the coupled sector index);
// padding holds zero.
template <typename T>
__global__ void k_eph_start(T *v, int64_t slice, int64_t dph, int64_t stride, int64_t dup,
                            int64_t de, const int32_t *pidx_up, const int32_t *pidx_dw,
                            const int32_t *padinv, uint64_t seed) {
  const int64_t n = slice * dph;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / slice, e = i - p * slice;
    const int64_t r = e / stride, pc = e - r * stride;
    const int32_t cb = padinv[pc];
    T x = T(0);
    if (cb >= 0) {
      const uint64_t q = (uint64_t)p * (uint64_t)de + (uint64_t)pidx_dw[r] * (uint64_t)dup +
                         (uint64_t)pidx_up[cb];
      const double u = (double)(ed_splitmix64_at(seed, q) >> 11) * (1.0 / 9007199254740992.0);
      x = (T)(u - 0.5);
    }
    v[i] = x;
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + PH_THREADS - 1) / PH_THREADS,
                                                          152 * 16));
}

// The coupled operator on `layout` (0: sector order, 1: padded block-major)
// (`tables`, nullable: the electronic product's tables instead of the
// sector's, e.g. the shifted diagonal of an FP32 chain)
template <typename T>
ed_status eph_apply(ed_sector s, const PhParams &ph, int layout, const T *v, T *w,
                    cudaStream_t cs, const HvTables<T> *tables = nullptr) {
  const HvTables<T> tb = tables ? *tables : ed_hv_tables<T>(s, layout);
  const int64_t slice = layout == 1 ? s->bdim : s->dim;
  for (int p = 0; p <= ph.nph; ++p)
    ED_TRY(ed_launch_hv<T>(s, tb, HV_PLAIN, v + (int64_t)p * slice, w + (int64_t)p * slice,
                           nullptr, nullptr, nullptr, nullptr, nullptr, cs));
  const SpinTables *t = layout == 1 ? s->bk : s->sp;
  k_phonon<T><<<grid_of(slice), PH_THREADS, 0, cs>>>(v, w, slice, tb.stride,
                                                     layout == 1 ? s->padinv : nullptr, t[0].imask,
                                                     t[1].imask, ph);
  ED_LAUNCHED(1);
  return ED_OK;
}

template <typename T>
LinOp<T> eph_op(ed_sector s, const PhParams &ph) {
  LinOp<T> op;
  op.n = s->bdim * (int64_t)(ph.nph + 1);
  op.apply = [s, ph](const T *v, T *w, cudaStream_t cs) { return eph_apply<T>(s, ph, 1, v, w, cs); };
  return op;
}

// the coupled operator with the electronic product on the given tables
template <typename T>
LinOp<T> eph_op(ed_sector s, const PhParams &ph, const HvTables<T> &tb) {
  LinOp<T> op;
  op.n = s->bdim * (int64_t)(ph.nph + 1);
  op.apply = [s, ph, tb](const T *v, T *w, cudaStream_t cs) {
    return eph_apply<T>(s, ph, 1, v, w, cs, &tb);
  };
  return op;
}

struct Buf {
  void *p = nullptr;
  cudaStream_t cs = nullptr;
  ~Buf() {
    if (p) ed_dfree(p, cs);
  }
  ed_status alloc(size_t bytes, cudaStream_t st, const char *what) {
    cs = st;
    return ed_dmalloc(&p, std::max<size_t>(bytes, 256), st, what);
  }
};

// coupled sector order <-> padded block-major slices
ed_status permute_slices(ed_sector s, ed_precision prec, bool to_blocked, const void *in, void *out,
                         int dph, cudaStream_t cs) {
  const size_t el = prec == ED_FP64 ? 8 : 4;
  const int64_t si = to_blocked ? s->dim : s->bdim, so = to_blocked ? s->bdim : s->dim;
  for (int p = 0; p < dph; ++p)
    ED_TRY(ed_permute_vec(s, prec, to_blocked, (const char *)in + (size_t)p * si * el,
                          (char *)out + (size_t)p * so * el, cs));
  return ED_OK;
}

template <typename T>
ed_status eph_solve(ed_sector s, const PhParams &ph, int maxit, double tol, uint64_t seed,
                    const T *start, T *psi, OpRun *run, cudaStream_t cs) {
  const LinOp<T> op = eph_op<T>(s, ph);
  Buf v0;
  if (!start) {
    ED_TRY(v0.alloc((size_t)op.n * sizeof(T), cs, "coupled start vector"));
    k_eph_start<T><<<grid_of(op.n), PH_THREADS, 0, cs>>>(
        (T *)v0.p, s->bdim, ph.nph + 1, s->bstride, s->sp[0].dim, s->dim, s->bi[0].pidx,
        s->bi[1].pidx, s->padinv, seed);
    ED_LAUNCHED(1);
    start = (const T *)v0.p;
  }
  return ed_op_lanczos<T>(op, start, maxit, tol, true, run, nullptr, psi, cs);
}

}  // namespace

extern "C" ed_status ed_eph_matvec(ed_sector s, const ed_phonon *ph, ed_precision prec,
                                   const void *d_v, void *d_w, int64_t n, void *stream) {
  PhParams pp;
  if (!s || !d_v || !d_w || d_v == d_w || !make_params(s, ph, &pp)) return ED_ERR_ARG;
  if (n != s->dim * (int64_t)(pp.nph + 1)) {
    ed_set_error_msg("vector length does not match the coupled sector");
    return ED_ERR_ARG;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  if (prec == ED_FP64) {
    ED_TRY(ed_build_items(s, 0, 8));
    return eph_apply<double>(s, pp, 0, (const double *)d_v, (double *)d_w, cs);
  }
  if (prec == ED_FP32 || prec == ED_FP32_POLISH) {
    ED_TRY(ed_build_items(s, 0, 4));
    return eph_apply<float>(s, pp, 0, (const float *)d_v, (float *)d_w, cs);
  }
  return ED_ERR_ARG;
}

extern "C" ed_status ed_eph_lanczos_ground(ed_sector s, const ed_phonon *ph,
                                           const ed_lanczos_opts *o, ed_lanczos_result *res,
                                           void *d_psi, void *stream) {
  PhParams pp;
  if (!s || !o || !res || !make_params(s, ph, &pp)) return ED_ERR_ARG;
  memset(res, 0, sizeof(*res));
  const int maxit = o->max_iter > 0 ? o->max_iter : 512;
  if (maxit > ED_MAX_LANCZOS || s->dim <= 0) return ED_ERR_ARG;
  const ed_precision prec = o->precision;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  const double tol = o->tol > 0 ? o->tol : (prec == ED_FP64 ? 1e-12 : 1e-6);
  cudaStream_t cs = (cudaStream_t)stream;
  const int dph = pp.nph + 1;
  const int64_t n = s->bdim * (int64_t)dph;
  ED_TRY(ed_build_items(s, 1, 8));
  Buf psi64;
  ED_TRY(psi64.alloc((size_t)n * 8, cs, "coupled ground state"));
  ED_TRY_CUDA(cudaMemsetAsync(psi64.p, 0, (size_t)n * 8, cs));
  OpRun run;
  int mv = 0, mv32 = 0;
  if (prec == ED_FP64) {
    ED_TRY(eph_solve<double>(s, pp, maxit, tol, o->seed, nullptr, (double *)psi64.p, &run, cs));
    mv = run.matvecs;
    res->e0 = res->e0_raw = run.theta;
  } else {
    ED_TRY(ed_build_items(s, 1, 4));
    Buf psi32;
    ED_TRY(psi32.alloc((size_t)n * 4, cs, "coupled FP32 ground state"));
    ED_TRY(eph_solve<float>(s, pp, maxit, tol, o->seed, nullptr, (float *)psi32.p, &run, cs));
    mv = mv32 = run.matvecs;
    res->e0 = res->e0_raw = run.theta;
    if (prec == ED_FP32) {
      if (d_psi) ED_TRY(permute_slices(s, ED_FP32, false, psi32.p, d_psi, dph, cs));
    }
    ED_TRY((ed_op_normalised_copy<float, double>((const float *)psi32.p, (double *)psi64.p, n, cs)));
    if (prec == ED_FP32_POLISH) {
      // a few FP64 steps from the FP32 ground state (a6)
      const int steps = o->polish_steps > 0 ? o->polish_steps : 4;
      OpRun pol;
      Buf start;
      ED_TRY(start.alloc((size_t)n * 8, cs, "polish start"));
      ED_TRY_CUDA(cudaMemcpyAsync(start.p, psi64.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, cs));
      ED_TRY((eph_solve<double>(s, pp, steps, 1e-300, 0, (const double *)start.p,
                                (double *)psi64.p, &pol, cs)));
      mv += pol.matvecs;
      res->e0 = pol.theta;
      res->polish_iterations = pol.k;
    }
  }
  res->iterations = run.k;
  res->residual_estimate = run.resid_est;
  res->stop_reason = run.stop;
  double e = 0.0, r = 0.0;
  ED_TRY(ed_op_residual(eph_op<double>(s, pp), (const double *)psi64.p, &e, &r, cs));
  ++mv;
  res->residual = r;
  if (d_psi && prec != ED_FP32) ED_TRY(permute_slices(s, ED_FP64, false, psi64.p, d_psi, dph, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  res->matvecs = mv;
  res->matvecs_fp64 = mv - mv32;
  if (run.stop == 2) {
    ed_set_error_msg("max_iter reached before the Lanczos tolerance");
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}

extern "C" ed_status ed_eph_gf_lanczos_z(ed_sector s, const ed_phonon *ph, ed_precision prec,
                                         const void *d_psi, double e0, int32_t orb, int32_t spin,
                                         int32_t nsteps, const double *host_z, int32_t nz,
                                         double *host_G, ed_gf_info *info, void *stream) {
  PhParams pp;
  if (!s || !d_psi || !host_G || !make_params(s, ph, &pp) || nz < 0 || (nz > 0 && !host_z))
    return ED_ERR_ARG;
  if (orb < 0 || orb >= s->mp.norb || spin < 0 || spin > 1) return ED_ERR_ARG;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (nsteps <= 0) nsteps = 200;
  if (nsteps > ED_MAX_LANCZOS) return ED_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  const int dph = pp.nph + 1;
  if (info) memset(info, 0, sizeof(*info));
  Buf zg;
  const size_t zb = (size_t)std::max(nz, 1) * sizeof(double2);
  ED_TRY(zg.alloc(2 * zb + ((sizeof(LanczosState) + 255) & ~(size_t)255), cs, "coupled G"));
  double2 *dz = (double2 *)zg.p, *dG = (double2 *)((char *)zg.p + zb);
  LanczosState *st = (LanczosState *)((char *)zg.p + 2 * zb);
  if (nz > 0) {
    ED_TRY_CUDA(cudaMemcpyAsync(dz, host_z, nz * sizeof(double2), cudaMemcpyHostToDevice, cs));
    ED_TRY_CUDA(cudaMemsetAsync(dG, 0, nz * sizeof(double2), cs));
  }
  for (int create = 1; create >= -1; create -= 2) {
    ed_sector nb = nullptr;
    ED_TRY(ed_neighbor_sector(s, spin, create, cs, &nb));
    if (!nb || nb->dim == 0) continue;
    const int64_t n = nb->bdim * (int64_t)dph;
    OpRun run;
    double sigma = 0.0;  // the chain's operator is H - sigma
    if (prec == ED_FP64) {
      ED_TRY(ed_build_items(nb, 1, 8));
      Buf phi;
      ED_TRY(phi.alloc((size_t)n * 8, cs, "coupled chain start"));
      for (int p = 0; p < dph; ++p)
        ED_TRY((ed_apply_op_launch<double, double>(s, nb, (const double *)d_psi + (int64_t)p * s->dim,
                                                   (double *)phi.p + (int64_t)p * nb->bdim, orb,
                                                   spin, create, cs)));
      ED_TRY(ed_op_lanczos<double>(eph_op<double>(nb, pp), (const double *)phi.p, nsteps, 0.0,
                                   false, &run, st, nullptr, cs));
    } else {
      ED_TRY(ed_build_items(nb, 1, 4));
      Buf phi;
      ED_TRY(phi.alloc((size_t)n * 4, cs, "coupled chain start"));
      for (int p = 0; p < dph; ++p) {
        float *dst = (float *)phi.p + (int64_t)p * nb->bdim;
        if (prec == ED_FP32)
          ED_TRY((ed_apply_op_launch<float, float>(s, nb, (const float *)d_psi + (int64_t)p * s->dim,
                                                   dst, orb, spin, create, cs)));
        else
          ED_TRY((ed_apply_op_launch<double, float>(s, nb,
                                                    (const double *)d_psi + (int64_t)p * s->dim,
                                                    dst, orb, spin, create, cs)));
      }
      // FP32 chains run on H - e0: the electronic diagonal tables shifted in
      // FP64 before their rounding (the phonon terms are unchanged), so that
      // the continued fraction takes e0 - e0 = 0
      HvTables<float> tb = ed_hv_tables<float>(nb, 1);
      Buf shifted;
      ED_TRY(shifted.alloc(ed_shift_diag_bytes(nb), cs, "shifted diagonal"));
      ED_TRY(ed_shift_diag32(nb, e0, shifted.p, &tb, cs));
      ED_TRY(ed_op_lanczos<float>(eph_op<float>(nb, pp, tb), (const float *)phi.p, nsteps, 0.0,
                                  false, &run, st, nullptr, cs));
      sigma = e0;
    }
    if (info) {
      if (create > 0) {
        info->weight_particle = run.weight;
        info->steps_particle = run.k;
      } else {
        info->weight_hole = run.weight;
        info->steps_hole = run.k;
      }
    }
    if (run.weight > 0.0 && run.k > 0)
      ED_TRY(ed_cfrac_z_launch(st, run.weight, e0 - sigma, dz, nz, create, dG, cs));
  }
  if (nz > 0)
    ED_TRY_CUDA(cudaMemcpyAsync(host_G, dG, nz * sizeof(double2), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  return ED_OK;
}
