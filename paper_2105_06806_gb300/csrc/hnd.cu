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
// gather kernel: a warp takes a row (dw string), lists the up moves that the
// row's dw string can pair with (at most Norb (Norb - 1), 4 for Norb = 3)
// with the target row and coefficient, and its lanes run along the row's
// columns, each gathering v at the moved (row, column) pairs.  The column
// tables (Norb^2 x D_up entries) stay in L2.
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

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float *p, float (&x)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  }
  static __device__ __forceinline__ void store(float *p, const float (&x)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double *p, double (&x)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
  static __device__ __forceinline__ void store(double *p, const double (&x)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(x[2], x[3]);
  }
};

constexpr int ND_WARPS = ND_THREADS / 32;
constexpr int ND_CHUNK_LANE = 8;  // iterations of a warp per work unit (row, column chunk)
constexpr int ND_CTAS_PER_SM = 5;  // FP32 (48 registers); FP64 kernels take 4

// MODE HV_PLAIN: w += H_nd v.  HV_LANCZOS: out += s H_nd g with g, out and
// s = scale[j % 3] of step j (the product kernel wrote s H g there), and the
// partial <s g, s H_nd g> of alpha_j.  HV_SECOND: out += s H_nd g.  ND_DOT:
// the partial <v, H_nd v>.
//
// A warp takes work units (row, column chunk) in grid-stride order; for a
// new row its lanes form the row's list of moves in parallel (lane l takes
// the orbital pair (l / Norb, l % Norb), a ballot packs the pairs that the
// row's dw string allows into shared memory), then run along the chunk.  VEC (block-major layout: rows and up blocks padded to
// multiples of 4 columns, 16-byte aligned): a lane takes 4 consecutive
// columns, reads the 4 table entries of a move as one int4 and updates the 4
// outputs with one 16-byte (FP32) access; padding columns have no moves and
// keep their value.  Otherwise one column per lane.
template <typename T, int MODE, bool VEC>
__global__ void __launch_bounds__(ND_THREADS, sizeof(T) == 4 ? ND_CTAS_PER_SM : 4) k_nd(NdLaunch<T> a) {
  __shared__ int s_kup[ND_WARPS][ND_MOVES];
  __shared__ int64_t s_roff[ND_WARPS][ND_MOVES];
  __shared__ T s_cf[ND_WARPS][ND_MOVES];
  __shared__ double red[ND_WARPS];
  const HvTables<T> &tb = a.tb;
  const T *g = a.v;
  T *out = a.w;
  T s_cur = T(1);
  if (MODE == HV_LANCZOS || MODE == HV_SECOND) {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    const int j = st->j, m3 = j % 3;
    g = m3 == 0 ? a.b0 : (m3 == 1 ? a.b1 : a.b2);
    out = m3 == 0 ? a.b1 : (m3 == 1 ? a.b2 : a.b0);
    if (MODE == HV_LANCZOS && a.basis) {
      g = a.basis[j];
      out = a.basis[j + 1];
    }
    s_cur = (T)st->scale[j % 3];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int no = tb.nd_norb;
  const int64_t ncols = tb.nd_ncols, stride = tb.stride;
  double dsum = 0.0;
  T dt = T(0);
  int cnt = 0;
  // work units: (row, chunk of ND_CHUNK columns), grid-stride over the warps
  const int64_t chunk = VEC ? 4 * ND_CHUNK_LANE * 32 : ND_CHUNK_LANE * 32;
  const int64_t nchunk = (ncols + chunk - 1) / chunk;
  const int64_t units = tb.ddw * nchunk;
  int64_t r_prev = -1;
  int n = 0;
  for (int64_t u = (int64_t)blockIdx.x * ND_WARPS + wid; u < units;
       u += (int64_t)gridDim.x * ND_WARPS) {
    const int64_t r = u / nchunk;
    const int64_t c0 = (u - r * nchunk) * chunk;
    if (r != r_prev) {
      // the row's moves: up b -> q paired with dw q -> b (spin exchange) or
      // dw b -> q (pair hopping)
      r_prev = r;
      const int md = tb.m_dw[r];
      const int b = lane / no, q = lane - b * no;
      int kd = -1;
      T cf = T(0);
      if (lane < no * no && b != q) {
        if (((md >> q) & 1) && !((md >> b) & 1)) {
          kd = q * no + b;
          cf = tb.nd_jx;
        } else if (((md >> b) & 1) && !((md >> q) & 1)) {
          kd = b * no + q;
          cf = tb.nd_jp;
        }
      }
      const bool has = kd >= 0 && cf != T(0);
      const unsigned bal = __ballot_sync(0xffffffffu, has);
      __syncwarp();  // the previous row's list has been read
      if (has) {
        const int pos = __popc(bal & ((1u << lane) - 1u));
        const int32_t e = tb.nd_dw[(int64_t)kd * tb.ddw + r];
        s_kup[wid][pos] = b * no + q;
        s_roff[wid][pos] = (int64_t)(e >> 1) * stride;
        s_cf[wid][pos] = (e & 1) ? -cf : cf;
      }
      __syncwarp();
      n = __popc(bal);
    }
    if (n == 0) continue;
    const int64_t rb = r * stride;
    const int64_t c1 = min(ncols, c0 + chunk);
    if (VEC) {
      for (int64_t c = c0 + 4 * lane; c < c1; c += 128) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        int any = 0;
        for (int k = 0; k < n; ++k) {
          const int4 e4 = __ldg(reinterpret_cast<const int4 *>(tb.nd_up + (int64_t)s_kup[wid][k] * ncols + c));
          const int32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
          const T cfk = s_cf[wid][k];
          const T *row = g + s_roff[wid][k];
#pragma unroll
          for (int uu = 0; uu < 4; ++uu) {
            if (e[uu] < 0) continue;
            acc[uu] = nd_fma<T>((e[uu] & 1) ? -cfk : cfk, __ldg(row + (e[uu] >> 1)), acc[uu]);
            any = 1;
          }
        }
        if (!any) continue;
        T o[4], x[4];
        if (MODE == ND_DOT || MODE == HV_LANCZOS) Vec4<T>::load(g + rb + c, x);
        if (MODE == ND_DOT) {
#pragma unroll
          for (int uu = 0; uu < 4; ++uu) dt = nd_fma<T>(x[uu], acc[uu], dt);
        } else {
          Vec4<T>::load(out + rb + c, o);
#pragma unroll
          for (int uu = 0; uu < 4; ++uu) {
            const T w1 = MODE == HV_PLAIN ? acc[uu] : acc[uu] * s_cur;
            o[uu] += w1;
            if (MODE == HV_LANCZOS) dt = nd_fma<T>(x[uu] * s_cur, w1, dt);
          }
          Vec4<T>::store(out + rb + c, o);
        }
        if (MODE == HV_LANCZOS || MODE == ND_DOT) {
          if ((cnt += 4) >= ND_FLUSH) {
            dsum += (double)dt;
            dt = T(0);
            cnt = 0;
          }
        }
      }
    } else {
      for (int64_t c = c0 + lane; c < c1; c += 32) {
        T acc = T(0);
        bool any = false;
        for (int k = 0; k < n; ++k) {
          const int32_t e = __ldg(tb.nd_up + (int64_t)s_kup[wid][k] * ncols + c);
          if (e < 0) continue;
          const T x = __ldg(g + s_roff[wid][k] + (e >> 1));
          acc = nd_fma<T>((e & 1) ? -s_cf[wid][k] : s_cf[wid][k], x, acc);
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
  }
  if (MODE == HV_LANCZOS || MODE == ND_DOT) {
    dsum += (double)dt;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    if (lane == 0) red[wid] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < ND_WARPS; ++k) t += red[k];
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

int64_t ed_nd_grid(int64_t ddw, int64_t ncols) {
  // work units of one warp: (row, chunk of 32 * ND_CHUNK_LANE columns, 4x with
  // 16-byte accesses); at most ND_CTAS_PER_SM resident CTAs per SM
  const int64_t units = ddw * ((ncols + 32 * ND_CHUNK_LANE - 1) / (32 * ND_CHUNK_LANE));
  return std::max<int64_t>(1, std::min<int64_t>((units + ND_WARPS - 1) / ND_WARPS,
                                                 152 * ND_CTAS_PER_SM));
}

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

ed_status ed_move_tables(ed_sector s, int32_t *up, int32_t *dw, cudaStream_t st) {
  const int no = s->mp.norb;
  const int64_t nu = s->bstride, nd = s->sp[1].dim;
  if (nu > 0) {
    k_nd_table<1><<<(unsigned)((nu + 255) / 256), 256, 0, st>>>(
        s->bk[0].map, s->padinv, s->colpos, nu, no, ed_block_view(s, 0), up);
    ED_LAUNCHED(1);
  }
  if (nd > 0) {
    k_nd_table<1><<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(
        s->bk[1].map, nullptr, nullptr, nd, no, ed_block_view(s, 1), dw);
    ED_LAUNCHED(1);
  }
  return ED_OK;
}

void ed_free_nd_tables(ed_sector s, cudaStream_t st) {
  for (int l = 0; l < 2; ++l) {
    ed_dfree(s->nd[l].up, st);
    ed_dfree(s->nd[l].dw, st);
    s->nd[l] = NdTables();
  }
}

template <typename T, bool VEC>
static ed_status launch_nd(const NdLaunch<T> &a, int mode, unsigned grid, cudaStream_t st) {
  if (mode == HV_PLAIN)
    k_nd<T, HV_PLAIN, VEC><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == HV_LANCZOS)
    k_nd<T, HV_LANCZOS, VEC><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == HV_SECOND)
    k_nd<T, HV_SECOND, VEC><<<grid, ND_THREADS, 0, st>>>(a);
  else if (mode == ND_DOT)
    k_nd<T, ND_DOT, VEC><<<grid, ND_THREADS, 0, st>>>(a);
  else
    return ED_ERR_ARG;
  return ED_OK;
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
  const unsigned grid = (unsigned)ed_nd_grid(tb.ddw, tb.nd_ncols);
  // block-major vectors: rows, blocks and tables padded to 4 columns, 16-byte aligned
  // (and the vectors 16-byte aligned: sector-order vectors need not be)
  const uintptr_t al = (uintptr_t)tb.nd_up | (uintptr_t)v | (uintptr_t)w |
                       (bufs ? (uintptr_t)bufs[0] | (uintptr_t)bufs[1] | (uintptr_t)bufs[2] : 0);
  const bool vec = tb.nd_ncols % 4 == 0 && tb.stride == tb.nd_ncols && (al & 15) == 0;
  if (vec) ED_TRY((launch_nd<T, true>(a, mode, grid, st)));
  else ED_TRY((launch_nd<T, false>(a, mode, grid, st)));
  ED_LAUNCHED(1);
  return ED_OK;
}

template ed_status ed_launch_nd<float>(const HvTables<float> &, int, const float *, float *,
                                       float *const *, float *const *, const LanczosState *,
                                       double *, cudaStream_t);
template ed_status ed_launch_nd<double>(const HvTables<double> &, int, const double *, double *,
                                        double *const *, double *const *, const LanczosState *,
                                        double *, cudaStream_t);
