// Self-energy and local observables (Sec. 6.8 and App. B: the impurity
// self-energy on the Matsubara axis, functions on the real axis, impurity
// densities and double occupancies).
//
// ed_sigma: the non-interacting impurity function of the normal bath,
// G0_{a s}(z)^-1 = z - e_{a s} - sum_nu V_{nu a s}^2 / (z - eps_{nu a s})
// (Eq. Ham1 with a diagonal H^loc and bath h), and the Dyson equation
// Sigma(z) = G0(z)^-1 - G(z)^-1, one thread per frequency.
//
// ed_observables: every density-density observable of the impurity depends
// on a basis state only through its impurity occupation masks (m_up, m_dw),
// so they all follow from the table P[m_up][m_dw] = sum of |psi_i|^2 over
// the states with those masks.  The spin exchange and pair hopping add
// <psi|H_nd|psi> to the interaction energy (the H_nd kernel's dot mode).  The table is formed in a fixed order (no
// atomics): one warp per dw row sums |psi|^2 over the row's columns per up
// mask (lanes in a fixed stride, a fixed shuffle tree), then one thread per
// mask pair sums the rows in row order.  One thread then forms the
// densities, the correlators <n_{a s} n_{b t}> and the interaction energy of
// Eq. Ham1 (U, U', U' - J terms) from the table.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int OB_WARPS = 8;  // warps (dw rows) per CTA of the row pass

__global__ void k_sigma(const double *e_bath, const double *v_bath, double e_imp, int nbath,
                        const double2 *z, const double2 *G, int nz, double2 *sigma) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nz) return;
  const double zr = z[n].x, zi = z[n].y;
  // G0^-1 = z - e_imp - sum_nu V^2 / (z - eps)
  double gr = zr - e_imp, gi = zi;
  for (int nu = 0; nu < nbath; ++nu) {
    const double dr = zr - e_bath[nu], di = zi;
    const double inv = 1.0 / (dr * dr + di * di);
    const double v2 = v_bath[nu] * v_bath[nu];
    gr -= v2 * dr * inv;
    gi += v2 * di * inv;
  }
  // - 1 / G
  const double inv = 1.0 / (G[n].x * G[n].x + G[n].y * G[n].y);
  sigma[n] = make_double2(gr - G[n].x * inv, gi + G[n].y * inv);
}

// S[r][mu] = sum over the columns c of row r with impurity mask mu of
// |psi[r][c]|^2 (FP64), one warp per row
template <typename T>
__global__ void __launch_bounds__(32 * OB_WARPS) k_mask_rows(const T *psi, int64_t dup, int64_t ddw,
                                                            const uint8_t *m_up, int nm,
                                                            double *S) {
  const int64_t r = (int64_t)blockIdx.x * OB_WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= ddw) return;
  double acc[ED_MAX_NORB > 5 ? 32 : (1 << ED_MAX_NORB)];
  for (int k = 0; k < nm; ++k) acc[k] = 0.0;
  const T *row = psi + r * dup;
  for (int64_t c = lane; c < dup; c += 32) {
    const double x = (double)row[c];
    acc[m_up[c]] += x * x;
  }
  for (int k = 0; k < nm; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) S[r * nm + k] = v;
  }
}

// P[mu][md] = sum over the rows r with dw mask md of S[r][mu], rows in order
__global__ void k_mask_pairs(const double *S, const uint8_t *m_dw, int64_t ddw, int nm,
                             double *P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * nm) return;
  const int mu = t / nm, md = t - mu * nm;
  double acc = 0.0;
  for (int64_t r = 0; r < ddw; ++r)
    if (m_dw[r] == md) acc += S[r * nm + mu];
  P[t] = acc;
}

// out: dens[2][norb], nn[2][2][norb][norb], e_int, norm (normalised by norm);
// nd: nnd partial sums of <psi|H_nd|psi> (spin exchange, pair hopping)
__global__ void k_observables(const double *P, int norb, double U, double Ust, double Jh,
                              const double *nd, int nnd, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nm = 1 << norb;
  double norm = 0.0;
  for (int t = 0; t < nm * nm; ++t) norm += P[t];
  const double inv = norm > 0.0 ? 1.0 / norm : 0.0;
  double *dens = out, *nn = out + 2 * norb;
  for (int k = 0; k < 2 * norb + 4 * norb * norb; ++k) out[k] = 0.0;
  for (int mu = 0; mu < nm; ++mu)
    for (int md = 0; md < nm; ++md) {
      const double p = P[mu * nm + md] * inv;
      if (p == 0.0) continue;
      const int m[2] = {mu, md};
      for (int s = 0; s < 2; ++s)
        for (int a = 0; a < norb; ++a) {
          if (!((m[s] >> a) & 1)) continue;
          dens[s * norb + a] += p;
          for (int t = 0; t < 2; ++t)
            for (int b = 0; b < norb; ++b)
              if ((m[t] >> b) & 1) nn[((s * 2 + t) * norb + a) * norb + b] += p;
        }
    }
  double e_int = 0.0;
  for (int a = 0; a < norb; ++a) {
    e_int += U * nn[((0 * 2 + 1) * norb + a) * norb + a];
    for (int b = 0; b < norb; ++b) {
      if (a != b) e_int += Ust * nn[((0 * 2 + 1) * norb + a) * norb + b];
      if (a < b)
        e_int += (Ust - Jh) * (nn[((0 * 2 + 0) * norb + a) * norb + b] +
                               nn[((1 * 2 + 1) * norb + a) * norb + b]);
    }
  }
  double e_nd = 0.0;
  for (int k = 0; k < nnd; ++k) e_nd += nd[k];
  e_int += e_nd * inv;
  out[2 * norb + 4 * norb * norb] = e_int;
  out[2 * norb + 4 * norb * norb + 1] = norm;
}

}  // namespace

extern "C" ed_status ed_sigma(const ed_model *model, int32_t orb, int32_t spin,
                              const double *host_z, int32_t nz, const double *host_G,
                              double *host_sigma, void *stream) {
  if (!model || !host_z || !host_G || !host_sigma || nz < 0 || spin < 0 || spin > 1 || orb < 0 ||
      orb >= model->norb || model->nbath < 0 || (model->nbath > 0 && (!model->e_bath || !model->v_bath)) ||
      !model->e_imp)
    return ED_ERR_ARG;
  if (nz == 0) return ED_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  const int nb = model->nbath;
  const size_t zb = (size_t)nz * sizeof(double2);
  const size_t bytes = 3 * zb + 2 * (size_t)std::max(nb, 1) * sizeof(double);
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, bytes, cs, "self-energy"));
  char *p = (char *)mem;
  double2 *dz = (double2 *)p, *dG = (double2 *)(p + zb), *dS = (double2 *)(p + 2 * zb);
  double *de = (double *)(p + 3 * zb), *dv = de + std::max(nb, 1);
  const size_t boff = ((size_t)spin * model->norb + orb) * nb;
  ed_status rs = ED_OK;
  auto h2d = [&](void *dst, const void *src, size_t n) {
    if (rs == ED_OK && n && cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, cs) != cudaSuccess)
      rs = ED_ERR_CUDA;
  };
  h2d(dz, host_z, zb);
  h2d(dG, host_G, zb);
  if (nb) {
    h2d(de, model->e_bath + boff, nb * sizeof(double));
    h2d(dv, model->v_bath + boff, nb * sizeof(double));
  }
  if (rs == ED_OK) {
    k_sigma<<<(nz + 127) / 128, 128, 0, cs>>>(de, dv, model->e_imp[spin * model->norb + orb], nb,
                                              dz, dG, nz, dS);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  if (rs == ED_OK && cudaMemcpyAsync(host_sigma, dS, zb, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  ed_dfree(mem, cs);
  return rs;
}

extern "C" ed_status ed_observables(ed_sector s, ed_precision prec, const void *d_psi,
                                    int64_t n, double *host_out, void *stream) {
  if (!s || !d_psi || !host_out) return ED_ERR_ARG;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (n != s->dim) {
    ed_set_error_msg("vector length does not match the sector dimension");
    return ED_ERR_ARG;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  const int norb = s->mp.norb, nm = 1 << norb;
  const int64_t ddw = s->sp[1].dim, dup = s->sp[0].dim;
  const int nout = 2 * norb + 4 * norb * norb + 2;
  const size_t sb = ((size_t)ddw * nm * sizeof(double) + 255) & ~(size_t)255;
  const size_t pb = ((size_t)nm * nm * sizeof(double) + 255) & ~(size_t)255;
  const int nnd = (s->nd[0].up && ddw > 0 && dup > 0) ? (int)ed_nd_grid(ddw, s->nd[0].ncols) : 0;
  const size_t ndb = ((size_t)std::max(nnd, 1) * sizeof(double) + 255) & ~(size_t)255;
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, sb + pb + ndb + nout * sizeof(double), cs, "observables"));
  double *S = (double *)mem, *P = (double *)((char *)mem + sb);
  double *ndp = (double *)((char *)mem + sb + pb), *dout = (double *)((char *)mem + sb + pb + ndb);
  ed_status rs = ED_OK;
  if (nnd > 0) {  // <psi|H_nd|psi>, one partial per CTA
    rs = prec == ED_FP32
             ? ed_launch_nd<float>(ed_hv_tables<float>(s, 0), ND_DOT, (const float *)d_psi,
                                   nullptr, nullptr, nullptr, nullptr, ndp, cs)
             : ed_launch_nd<double>(ed_hv_tables<double>(s, 0), ND_DOT, (const double *)d_psi,
                                    nullptr, nullptr, nullptr, nullptr, ndp, cs);
  }
  const unsigned rows_grid = (unsigned)((ddw + OB_WARPS - 1) / OB_WARPS);
  if (rs != ED_OK) {
  } else if (ddw > 0 && dup > 0) {
    if (prec == ED_FP32)
      k_mask_rows<float><<<rows_grid, 32 * OB_WARPS, 0, cs>>>((const float *)d_psi, dup, ddw,
                                                              s->sp[0].imask, nm, S);
    else
      k_mask_rows<double><<<rows_grid, 32 * OB_WARPS, 0, cs>>>((const double *)d_psi, dup, ddw,
                                                               s->sp[0].imask, nm, S);
    ed_count_launches(1);
    k_mask_pairs<<<(nm * nm + 127) / 128, 128, 0, cs>>>(S, s->sp[1].imask, ddw, nm, P);
    ed_count_launches(1);
  } else if (cudaMemsetAsync(P, 0, nm * nm * sizeof(double), cs) != cudaSuccess) {
    rs = ED_ERR_CUDA;
  }
  if (rs == ED_OK) {
    k_observables<<<1, 32, 0, cs>>>(P, norb, s->U, s->Ust, s->Jh, ndp, nnd, dout);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  if (rs == ED_OK &&
      cudaMemcpyAsync(host_out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  ed_dfree(mem, cs);
  return rs;
}
