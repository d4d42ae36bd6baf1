// Impurity Green's function on the Matsubara axis (Sec. 6.8, Eq. KLgf at
// T = 0): start vectors c^+_{a s}|gs> and c_{a s}|gs> built on the device in
// gather form, Lanczos chains on the N+-1 sectors, continued fractions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

constexpr int GF_THREADS = 256;

__device__ __forceinline__ double gf_warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

struct ApplyArgs {
  // target sector (dst) in block-major order, source psi in sector order
  const uint32_t *dst_map;     // strings of the spin that changes, block-major order
  const int32_t *dst_pother;   // sector index of the unchanged spin's block-major index
  const int32_t *dst_padinv;   // padded column -> block-major up column (-1: padding)
  int64_t dst_stride, dst_dim; // padded row length, D_dw * stride
  int64_t src_dup;
  int level;                 // level a of the operator (impurity orbital)
  int create;                // +1: c^+, -1: c
  int spin;
  int nup_src;               // N_up of the source (sign of down operators)
};

// phi[r',c'] = sign * psi[r,c] where the changed spin string of the target
// element, with level a removed (c^+) or added (c), is the source string;
// sign = (-1)^(occupied modes before (a,s)) in the order 1up..Ns up,
// 1dw..Ns dw (Sec. 2.3).  phi is written in the target's block-major order,
// psi is read in sector order (sector index = colex rank of the strings).
// Partial sums of phi^2 per CTA.
template <typename Ti, typename To>
__global__ void __launch_bounds__(GF_THREADS) k_apply_op(ApplyArgs a, const Ti *psi, To *phi,
                                                         double *part) {
  __shared__ double red[GF_THREADS / 32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint32_t bit = 1u << a.level;
  const uint32_t below = bit - 1u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.dst_dim; i += stride) {
    const int64_t r2 = i / a.dst_stride;
    const int32_t c2 = a.dst_padinv[i - r2 * a.dst_stride];
    To out = To(0);
    const uint32_t I2 = c2 < 0 ? 0u : a.dst_map[a.spin == 0 ? (int64_t)c2 : r2];
    const bool occ = (I2 & bit) != 0u;
    if (c2 >= 0 && occ == (a.create > 0)) {
      const uint32_t I = I2 ^ bit;
      const int64_t src_idx = ed_rank(I);
      int parity = __popc(I & below);
      if (a.spin == 1) parity += a.nup_src;
      const int64_t r = a.spin == 0 ? (int64_t)a.dst_pother[r2] : src_idx;
      const int64_t c = a.spin == 0 ? src_idx : (int64_t)a.dst_pother[c2];
      const Ti x = psi[r * a.src_dup + c];
      out = (To)((parity & 1) ? -x : x);
    }
    phi[i] = out;
    acc += (double)out * (double)out;
  }
  acc = gf_warp_sum(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < GF_THREADS / 32; ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

// Continued fraction of one chain: G[n] += sgn * weight / f(z_n) with
// z_n = e0 + sgn * i w_n and f from the backward recurrence
// f = z - a_{k-1};  f = z - a_m - b_{m+1}^2 / f  (m = k-2 .. 0).
__global__ void k_cfrac(const LanczosState *st, double weight, double e0, double beta, int nmats,
                        int sgn, double2 *G) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nmats) return;
  const int k = st->j;
  if (k <= 0 || weight == 0.0) return;
  const double wn = (2.0 * n + 1.0) * M_PI / beta;
  const double zr = e0, zi = sgn * wn;
  double fr = zr - st->alpha[k - 1], fi = zi;
  for (int m = k - 2; m >= 0; --m) {
    const double b2 = st->beta[m + 1] * st->beta[m + 1];
    const double den = fr * fr + fi * fi;
    // b2 / f = b2 * conj(f) / |f|^2
    const double qr = b2 * fr / den, qi = -b2 * fi / den;
    fr = zr - st->alpha[m] - qr;
    fi = zi - qi;
  }
  const double den = fr * fr + fi * fi;
  const double gr = weight * fr / den, gi = -weight * fi / den;
  G[n].x += sgn * gr;
  G[n].y += sgn * gi;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename Ti, typename To>
static ed_status one_chain(ed_sector s, const Ti *psi, int orb, int spin, int create, int nsteps,
                           double e0, double beta, int nmats, double2 *dG, double *weight,
                           int *steps, cudaStream_t cs) {
  *weight = 0.0;
  *steps = 0;
  ed_sector nb = nullptr;
  ED_TRY(ed_neighbor_sector(s, spin, create, cs, &nb));
  if (!nb || nb->dim == 0) return ED_OK;
  const int64_t n = nb->bdim;  // padded block-major vectors
  const int64_t np1 = ed_hv_num_parts(nb, 1, (int)sizeof(To));
  const int64_t g2 = ed_reduce_grid(n);
  const int64_t nparts = std::max<int64_t>(np1, 3 * g2);
  const size_t vb = al256(n * sizeof(To));
  const size_t bytes = 3 * vb + al256(sizeof(LanczosState)) + 2 * al256(nparts * sizeof(double));
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, bytes, cs, "gf chain workspace"));
  cudaError_t e = cudaSuccess;
  char *p = (char *)mem;
  To *bufs[3];
  for (int b = 0; b < 3; ++b) {
    bufs[b] = (To *)p;
    p += vb;
  }
  LanczosState *st = (LanczosState *)p;
  p += al256(sizeof(LanczosState));
  double *part = (double *)p;
  p += al256(nparts * sizeof(double));
  double *part2 = (double *)p;

  ApplyArgs a;
  a.dst_map = nb->bk[spin].map;
  a.dst_pother = nb->bi[1 - spin].pidx;
  a.dst_padinv = nb->padinv;
  a.dst_stride = nb->bstride;
  a.dst_dim = n;
  a.src_dup = s->sp[0].dim;
  a.level = orb;  // impurity orbital alpha is level alpha
  a.create = create;
  a.spin = spin;
  a.nup_src = s->nup;
  ed_status rs = ED_OK;
  // padding entries must stay zero in every chain vector
  if (cudaMemsetAsync(mem, 0, 3 * vb, cs) != cudaSuccess) rs = ED_ERR_CUDA;
  PinnedFlag flag;
  if (rs == ED_OK && !flag.p) rs = ED_ERR_OOM;
  if (rs == ED_OK) {
    k_apply_op<Ti, To><<<(unsigned)g2, GF_THREADS, 0, cs>>>(a, psi, bufs[0], part);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  if (rs == ED_OK) rs = ed_lanczos_chain<To>(nb, bufs, st, part, part2, g2, nsteps, cs, flag.p);
  double hw[2] = {0, 0};
  int32_t hj = 0;
  if (rs == ED_OK) {
    // weight = ||phi||^2 was stored by the state initialisation in acc[0]
    e = cudaMemcpyAsync(hw, &st->acc[0], sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hj, &st->j, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "gf chain read-back", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  if (rs == ED_OK && hw[0] > 0.0 && nmats > 0) {
    k_cfrac<<<(nmats + 127) / 128, 128, 0, cs>>>(st, hw[0], e0, beta, nmats, create, dG);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  *weight = hw[0];
  *steps = hj;
  ed_dfree(mem, cs);
  return rs;
}

ed_status ed_gf_impl(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                     int spin, int nsteps, double beta, int nmats, double *host_G,
                     ed_gf_info *info, cudaStream_t cs) {
  if (!s || !d_psi || orb < 0 || orb >= s->mp.norb || spin < 0 || spin > 1 || nsteps <= 0 ||
      nsteps > ED_MAX_LANCZOS || nmats < 0 || (nmats > 0 && (!host_G || !(beta > 0))))
    return ED_ERR_ARG;
  double2 *dG = nullptr;
  ED_TRY(ed_dmalloc((void **)&dG, std::max(1, nmats) * sizeof(double2), cs, "gf accumulator"));
  ed_status rs = ED_OK;
  if (cudaMemsetAsync(dG, 0, std::max(1, nmats) * sizeof(double2), cs) != cudaSuccess) rs = ED_ERR_CUDA;
  double wp = 0, wh = 0;
  int sp = 0, sh = 0;
  for (int create = 1; create >= -1 && rs == ED_OK; create -= 2) {
    double *w = create > 0 ? &wp : &wh;
    int *k = create > 0 ? &sp : &sh;
    if (prec == ED_FP64)
      rs = one_chain<double, double>(s, (const double *)d_psi, orb, spin, create, nsteps, e0, beta,
                                     nmats, dG, w, k, cs);
    else if (prec == ED_FP32)
      rs = one_chain<float, float>(s, (const float *)d_psi, orb, spin, create, nsteps, e0, beta,
                                   nmats, dG, w, k, cs);
    else
      rs = one_chain<double, float>(s, (const double *)d_psi, orb, spin, create, nsteps, e0, beta,
                                    nmats, dG, w, k, cs);
  }
  if (rs == ED_OK && nmats > 0) {
    cudaError_t e = cudaMemcpyAsync(host_G, dG, nmats * sizeof(double2), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "gf result copy", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  ed_dfree(dG, cs);
  if (info) {
    info->weight_particle = wp;
    info->weight_hole = wh;
    info->steps_particle = sp;
    info->steps_hole = sh;
  }
  return rs;
}

// One chain (particle: create = +1, hole: -1) of G_{orb,spin}, on its own
// stream ordered after `after`; its contribution to G goes to host_G
// (2*nmats doubles, overwritten).  Used by ed_solve to run the chains of a
// solve concurrently; the neighbour sector and its work lists must already
// exist (ed_gf_prepare) so that concurrent jobs share no mutable state.
ed_status ed_gf_chain_job(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                          int spin, int create, int nsteps, double beta, int nmats,
                          double *host_G, double *weight, int *steps, int64_t *dim,
                          cudaEvent_t after) {
  *weight = 0.0;
  *steps = 0;
  *dim = 0;
  cudaStream_t cs = nullptr;
  ED_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  ed_status rs = ED_OK;
  if (after && cudaStreamWaitEvent(cs, after, 0) != cudaSuccess) rs = ED_ERR_CUDA;
  double2 *dG = nullptr;
  if (rs == ED_OK)
    rs = ed_dmalloc((void **)&dG, std::max(1, nmats) * sizeof(double2), cs, "gf accumulator");
  if (rs == ED_OK && cudaMemsetAsync(dG, 0, std::max(1, nmats) * sizeof(double2), cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (rs == ED_OK) {
    if (prec == ED_FP64)
      rs = one_chain<double, double>(s, (const double *)d_psi, orb, spin, create, nsteps, e0,
                                     beta, nmats, dG, weight, steps, cs);
    else if (prec == ED_FP32)
      rs = one_chain<float, float>(s, (const float *)d_psi, orb, spin, create, nsteps, e0, beta,
                                   nmats, dG, weight, steps, cs);
    else
      rs = one_chain<double, float>(s, (const double *)d_psi, orb, spin, create, nsteps, e0,
                                    beta, nmats, dG, weight, steps, cs);
  }
  if (rs == ED_OK && nmats > 0) {
    cudaError_t e = cudaMemcpyAsync(host_G, dG, nmats * sizeof(double2), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) rs = ED_ERR_CUDA;
  }
  ed_dfree(dG, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  cudaStreamDestroy(cs);
  ed_sector nb = s->nb[spin][create > 0 ? 1 : 0];
  *dim = nb ? nb->dim : 0;
  return rs;
}

// Builds the neighbour sector of a chain and its product work lists on the
// calling thread (before concurrent chain jobs start).
ed_status ed_gf_prepare(ed_sector s, int spin, int create, int elem, cudaStream_t cs) {
  ed_sector nb = nullptr;
  ED_TRY(ed_neighbor_sector(s, spin, create, cs, &nb));
  if (nb && nb->dim > 0) ED_TRY(ed_build_items(nb, 1, elem));
  return ED_OK;
}

extern "C" ed_status ed_gf_lanczos(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                                   int32_t orb, int32_t spin, int32_t nsteps, double beta,
                                   int32_t nmats, double *host_G, ed_gf_info *info, void *stream) {
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  return ed_gf_impl(s, prec, d_psi, e0, orb, spin, nsteps, beta, nmats, host_G, info,
                    (cudaStream_t)stream);
}
