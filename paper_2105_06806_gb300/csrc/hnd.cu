// Spin exchange and pair hopping: the part H_nd of Eq. Ham1 that the
// per-spin factorisation of Sec. 2.4 cannot hold (Sec. 3.2: the paper applies
// it as a separate sparse term over the whole sector).
//
//   -J_X sum_{a != b} d+_{a up} d_{a dw} d+_{b dw} d_{b up}
//   +J_P sum_{a != b} d+_{a up} d+_{a dw} d_{b dw} d_{b up}
//
// Both terms keep N_up and N_dw and move one electron of each spin between
// two impurity orbitals, so each factorises into a move on the up string and
// a move on the dw string.  The library tabulates, per spin and layout, the
// index of the moved string (and its sign) for every ordered pair of
// impurity orbitals, and adds H_nd v after the factorised product with one
// gather kernel: a CTA takes a row (dw string), lists the up moves that the
// row's dw string can pair with (at most Norb^2, typically 4 for Norb = 3)
// with the target row and coefficient in shared memory, and its threads run
// along the row's columns, each gathering v at the moved (row, column) pairs.
// The column tables (Norb^2 x D_up entries) stay in L2.
#include <algorithm>

#include "internal.cuh"

BlockView ed_block_view(ed_sector s, int spin);

namespace {

constexpr int ND_THREADS = 256;
constexpr int ND_MOVES = ED_MAX_NORB * ED_MAX_NORB;
constexpr int ND_FLUSH = 16;  // terms summed in T before the FP64 partial

// Entry k = b * norb + a (move of an electron from impurity level b to a) of
// index i of one spin's layout; ORDER 0: sector order (ascending strings),
// 1: block-major (padinv maps a padded column to its column or -1, colpos
// maps a block-major column back to its padded column; both null for rows).
template <int ORDER>
__global__ void k_nd_table(const uint32_t *map, const int32_t *padinv, const int32_t *colpos,
                           int64_t n, int norb, BlockView bv, int32_t *tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t c = i;
  if (padinv) c = padinv[i];
  const bool valid = c >= 0;
  const uint32_t I = valid ? map[c] : 0u;
  for (int b = 0; b < norb; ++b)
    for (int a = 0; a < norb; ++a) {
      int32_t e = -1;
      if (valid && a != b && ((I >> b) & 1u) && !((I >> a) & 1u)) {
        const uint32_t J = I ^ (1u << b) ^ (1u << a);
        const int lo = min(a, b), hi = max(a, b);
        const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
        const int neg = __popc(I & between) & 1;
        int64_t t = ORDER == 0 ? ed_rank(J) : ed_blocked_rank(bv, J);
        if (colpos) t = colpos[t];
        e = (int32_t)((t << 1) | neg);
      }
      tab[(int64_t)(b * norb + a) * n + i] = e;
    }
}

template <typename T>
__device__ __forceinline__ T nd_fma(T a, T b, T c);
template <>
__device__ __forceinline__ float nd_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double nd_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct NdLaunch {
  HvTables<T> tb;
  const T *v;                // HV_PLAIN, ND_DOT
  T *w;                      // HV_PLAIN
  T *b0, *b1, *b2;           // Lanczos modes: v_j = scale[j % 3] * b[j % 3]
  T *const *basis;           // HV_LANCZOS with a kept basis: v_j at basis[j]
  const LanczosState *st;
  double *part;              // HV_LANCZOS, ND_DOT: one partial per CTA
};

// MODE HV_PLAIN: w += H_nd v.  HV_LANCZOS: out += s H_nd g with g, out and
// s = scale[j % 3] of step j (the product kernel wrote s H g there), and the
// partial <s g, s H_nd g> of alpha_j.  HV_SECOND: out += s H_nd g.  ND_DOT:
// the partial <v, H_nd v>.
template <typename T, int MODE>
__global__ void __launch_bounds__(ND_THREADS) k_nd(NdLaunch<T> a) {
  __shared__ int s_n;
  __shared__ int s_kup[ND_MOVES];
  __shared__ int64_t s_roff[ND_MOVES];
  __shared__ T s_cf[ND_MOVES];
  __shared__ double red[ND_THREADS / 32];
  const HvTables<T> &tb = a.tb;
  const T *g = a.v;
  T *out = a.w;
  T s_cur = T(1);
  if (MODE == HV_LANCZOS || MODE == HV_SECOND) {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    const int j = st->j;
    T *bufs[3] = {a.b0, a.b1, a.b2};
    g = bufs[j % 3];
    out = bufs[(j + 1) % 3];
    if (MODE == HV_LANCZOS && a.basis) {
      g = a.basis[j];
      out = a.basis[j + 1];
    }
    s_cur = (T)st->scale[j % 3];
  }
  const int no = tb.nd_norb;
  const int64_t ncols = tb.nd_ncols, stride = tb.stride;
  double dsum = 0.0;
  T dt = T(0);
  int cnt = 0;
  for (int64_t r = blockIdx.x; r < tb.ddw; r += gridDim.x) {
    __syncthreads();  // the previous row's list has been read
    if (threadIdx.x == 0) {
      const int md = tb.m_dw[r];
      int n = 0;
      for (int b = 0; b < no; ++b)
        for (int q = 0; q < no; ++q) {
          if (q == b) continue;
          int kd = -1;
          T cf = T(0);
          if (((md >> q) & 1) && !((md >> b) & 1)) {  // spin exchange: dw q -> b
            kd = q * no + b;
            cf = tb.nd_jx;
          } else if (((md >> b) & 1) && !((md >> q) & 1)) {  // pair hopping: dw b -> q
            kd = b * no + q;
            cf = tb.nd_jp;
          }
          if (kd < 0 || cf == T(0)) continue;
          const int32_t e = tb.nd_dw[(int64_t)kd * tb.ddw + r];
          s_kup[n] = b * no + q;
          s_roff[n] = (int64_t)(e >> 1) * stride;
          s_cf[n] = (e & 1) ? -cf : cf;
          ++n;
        }
      s_n = n;
    }
    __syncthreads();
    const int n = s_n;
    if (n == 0) continue;
    const int64_t rb = r * stride;
    for (int64_t c = threadIdx.x; c < ncols; c += ND_THREADS) {
      T acc = T(0);
      bool any = false;
      for (int q = 0; q < n; ++q) {
        const int32_t e = __ldg(tb.nd_up + (int64_t)s_kup[q] * ncols + c);
        if (e < 0) continue;
        const T x = g[s_roff[q] + (e >> 1)];
        acc = nd_fma<T>((e & 1) ? -s_cf[q] : s_cf[q], x, acc);
        any = true;
      }
      if (!any) continue;
      if (MODE == HV_PLAIN) {
        out[rb + c] += acc;
      } else if (MODE == ND_DOT) {
        dt = nd_fma<T>(g[rb + c], acc, dt);
      } else {
        const T w1 = acc * s_cur;
        out[rb + c] += w1;
        if (MODE == HV_LANCZOS) dt = nd_fma<T>(g[rb + c] * s_cur, w1, dt);
      }
      if (MODE == HV_LANCZOS || MODE == ND_DOT) {
        if (++cnt == ND_FLUSH) {
          dsum += (double)dt;
          dt = T(0);
          cnt = 0;
        }
      }
    }
  }
  if (MODE == HV_LANCZOS || MODE == ND_DOT) {
    dsum += (double)dt;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < ND_THREADS / 32; ++k) t += red[k];
      a.part[blockIdx.x] = t;
    }
  }
}

template <typename P>
ed_status nd_alloc(ed_sector s, cudaStream_t st, P **p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(P);
  ED_TRY(ed_dmalloc((void **)p, bytes, st, "spin-exchange / pair-hopping tables"));
  s->device_bytes += (int64_t)bytes;
  return ED_OK;
}

template <int ORDER>
ed_status nd_table(ed_sector s, const SpinTables &t, const int32_t *padinv, const int32_t *colpos,
                   int64_t n, BlockView bv, int32_t **out, cudaStream_t st) {
  const int no = s->mp.norb;
  ED_TRY(nd_alloc(s, st, out, (size_t)no * no * n));
  if (n > 0) {
    k_nd_table<ORDER><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t.map, padinv, colpos, n, no,
                                                                   bv, *out);
    ED_LAUNCHED(1);
  }
  return ED_OK;
}

}  // namespace

int64_t ed_nd_grid(int64_t ddw) { return std::max<int64_t>(1, std::min<int64_t>(ddw, 152 * 8)); }

ed_status ed_build_nd_tables(ed_sector s, cudaStream_t st) {
  if (s->mp.Jx == 0.0 && s->mp.Jp == 0.0) return ED_OK;
  BlockView none{};
  // sector order
  NdTables &t0 = s->nd[0];
  t0.ncols = s->sp[0].dim;
  ED_TRY(nd_table<0>(s, s->sp[0], nullptr, nullptr, s->sp[0].dim, none, &t0.up, st));
  ED_TRY(nd_table<0>(s, s->sp[1], nullptr, nullptr, s->sp[1].dim, none, &t0.dw, st));
  // block-major order: up columns padded
  NdTables &t1 = s->nd[1];
  t1.ncols = s->bstride;
  ED_TRY(nd_table<1>(s, s->bk[0], s->padinv, s->colpos, s->bstride, ed_block_view(s, 0), &t1.up,
                     st));
  ED_TRY(nd_table<1>(s, s->bk[1], nullptr, nullptr, s->sp[1].dim, ed_block_view(s, 1), &t1.dw,
                     st));
  return ED_OK;
}

void ed_free_nd_tables(ed_sector s, cudaStream_t st) {
  for (int l = 0; l < 2; ++l) {
    ed_dfree(s->nd[l].up, st);
    ed_dfree(s->nd[l].dw, st);
    s->nd[l] = NdTables();
  }
}

template <typename T>
ed_status ed_launch_nd(const HvTables<T> &tb, int mode, const T *v, T *w, T *const *bufs,
                       T *const *basis, const LanczosState *state, double *part, cudaStream_t st) {
  if (!tb.nd_up || tb.ddw == 0 || tb.nd_ncols == 0) return ED_OK;
  NdLaunch<T> a;
  a.tb = tb;
  a.v = v;
  a.w = w;
  a.b0 = bufs ? bufs[0] : nullptr;
  a.b1 = bufs ? bufs[1] : nullptr;
  a.b2 = bufs ? bufs[2] : nullptr;
  a.basis = basis;
  a.st = state;
  a.part = part;
  const unsigned grid = (unsigned)ed_nd_grid(tb.ddw);
  if (mode == HV_PLAIN)
    k_nd<T, HV_PLAIN><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == HV_LANCZOS)
    k_nd<T, HV_LANCZOS><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == HV_SECOND)
    k_nd<T, HV_SECOND><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == ND_DOT)
    k_nd<T, ND_DOT><<<grid, ND_THREADS, 0, st>>>(a);
  else
    return ED_ERR_ARG;
  ED_LAUNCHED(1);
  return ED_OK;
}

template ed_status ed_launch_nd<float>(const HvTables<float> &, int, const float *, float *,
                                       float *const *, float *const *, const LanczosState *,
                                       double *, cudaStream_t);
template ed_status ed_launch_nd<double>(const HvTables<double> &, int, const double *, double *,
                                        double *const *, double *const *, const LanczosState *,
                                        double *, cudaStream_t);
