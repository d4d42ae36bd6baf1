// Sector product w = H v (Sec. 6.7 without MPI, Eq. Hbuild) with optional
// Lanczos epilogues (Sec. 6.6).
//
// Layout: v is a row-major [D_dw][stride] array (Eq. Vmatrix); row r is one
// down configuration.  The product is cut into work items, rectangles of rows
// x columns inside one (dw block, up block) pair of the block-major order, so
// that H_up of a column never leaves the item's columns and H_dw of a row
// never leaves the dw block (in sector order there is one block per spin).
//
// Per item a CTA stages its rows in shared memory, transposed so that the RT
// rows a thread owns are contiguous: one 16-byte shared load then feeds the
// same H_up entry to RT rows (a small SpMM along the up axis).  Each thread
// owns a tile of 4 consecutive columns x RT rows.  In block-major order the
// H_up table is an ELL copy per up block interleaved by tiles (the entries
// of a tile's 4 columns are one 16-byte word), and every up block is padded
// to a multiple of 4 columns, so both the table and the H_dw neighbour rows
// are read with aligned, coalesced vector loads; the neighbour lists and
// diagonal pieces of the item's rows sit in shared memory.  No transpose is
// formed: the strided axis of Sec. 3.2 is read directly by row segments,
// which stay in L2 while the block pair is processed.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <type_traits>

#include "internal.cuh"

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <typename T>
__device__ __forceinline__ T mul_t(T a, T b);
template <>
__device__ __forceinline__ float mul_t<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_t<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ __forceinline__ T add_t(T a, T b);
template <>
__device__ __forceinline__ float add_t<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double add_t<double>(double a, double b) { return __dadd_rn(a, b); }

// Register tile: 4 consecutive columns x RT rows; the RT rows of one column
// form one 16-byte vector in shared memory (FP32: RT = 4, or 2 with an
// 8-byte vector when EDGB_RT_F32 = 2).
#ifndef EDGB_RT_F32
#define EDGB_RT_F32 4
#endif
template <typename T>
struct Tile;
template <>
struct Tile<float> {
  static constexpr int CU = 4, RT = EDGB_RT_F32;
  using V = typename std::conditional<EDGB_RT_F32 == 4, float4, float2>::type;
};
template <>
struct Tile<double> {
  static constexpr int CU = 4, RT = 2;
  using V = double2;
};
// register tile of a given height; the H_up pass of the two-pass product
// has two shapes, chosen per sector by its widest up block:
//  - narrow blocks (at most EDGB_PASSA_WIDE padded columns): 2 FP32 rows per
//    thread in 512-thread CTAs, two CTAs per SM;
//  - wide blocks: 4 FP32 rows per thread in 1024-thread CTAs, one CTA per SM,
//    the 4 staged rows of a column read with one 16-byte load.
// Measured per product: three orbitals at Ns=18 (8000-column blocks), FP32,
// 25.0 ms wide against 26.8 ms narrow; one orbital at Ns=16 (6436 columns)
// 1.50 ms either way; two orbitals at Ns=16 (4900 columns), FP64, 5.85 ms
// narrow against 6.47 ms wide.  FP64 keeps 2 rows per thread in both shapes.
template <typename T, int RTX>
struct TileOf;
template <>
struct TileOf<float, 4> {
  using V = float4;
};
template <>
struct TileOf<float, 2> {
  using V = float2;
};
template <>
struct TileOf<double, 2> {
  using V = double2;
};
#ifndef EDGB_PASSA_WIDE
#define EDGB_PASSA_WIDE 6000
#endif
template <typename T, bool WIDE>
constexpr int rt_passa() { return sizeof(T) == 4 && WIDE ? 4 : 2; }
template <bool WIDE>
constexpr int passa_threads() { return WIDE ? 1024 : 512; }

// four consecutive values of a 16-byte aligned row segment
__device__ __forceinline__ void load4(const float *p, float *y) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  y[0] = v.x;
  y[1] = v.y;
  y[2] = v.z;
  y[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double *y) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  y[0] = a.x;
  y[1] = a.y;
  y[2] = b.x;
  y[3] = b.y;
}

__device__ __forceinline__ void store4(float *p, const float *y) {
  *reinterpret_cast<float4 *>(p) = make_float4(y[0], y[1], y[2], y[3]);
}
__device__ __forceinline__ void store4(double *p, const double *y) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(y[0], y[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(y[2], y[3]);
}
__device__ __forceinline__ void vec_get(const float4 &v, float *x) {
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void vec_get(const double2 &v, double *x) {
  x[0] = v.x;
  x[1] = v.y;
}
__device__ __forceinline__ void vec_get(const float2 &v, float *x) {
  x[0] = v.x;
  x[1] = v.y;
}

// Element-parallel product (one thread per element of the padded block-major
// vector, striding for large sectors).  Below EDGB_TUNE_MIN elements the
// tiled kernel has too few work items to fill the GPU and its time is set by
// the serial per-thread tile, so the element-parallel kernel is used; above
// it, which one is faster depends on the block shapes and the precision (the
// tiled kernel reuses staged rows and ELL entries, the element-parallel one
// keeps more loads in flight): the autotuner times both.
constexpr int HVS_THREADS = 256;
#ifndef EDGB_TUNE_MIN
#define EDGB_TUNE_MIN (1 << 17)
#endif
// Elements per thread of the element-parallel product: 1 up to
// EDGB_SMALL_PARTS CTAs, then K, so that the grid (= the Lanczos partials)
// stays within EDGB_SMALL_PARTS.  CTA b takes the K consecutive 256-element
// chunks b*K .. b*K+K-1: CTAs are dispatched in order, so the part of the
// vector in flight stays a compact window of (resident CTAs) x K chunks, and
// the H_dw neighbour rows that nearby rows share are still in L2 when they
// are read again.  (A grid-stride loop over one resident wave measured 1.9x
// slower at 2.4e9 elements: its CTAs drift apart and the window spreads over
// the whole vector.)  One CTA sums the partials every Lanczos step: at
// D = 1.66e8 an FP32 step takes 3.2 ms with 2^16 partials, 3.7 ms with
// 2.2e5 and 5.3 ms with 6.5e5 (one element per thread), while the product
// itself stays within 4% of one element per thread at every size.
#ifndef EDGB_SMALL_PARTS
#define EDGB_SMALL_PARTS (1 << 16)
#endif
static int64_t small_chunk_of(int64_t n) {
  const int64_t nblk = (n + HVS_THREADS - 1) / HVS_THREADS;
  return std::max<int64_t>(1, (nblk + EDGB_SMALL_PARTS - 1) / EDGB_SMALL_PARTS);
}
static int64_t small_grid_of(int64_t n) {
  const int64_t nblk = (n + HVS_THREADS - 1) / HVS_THREADS;
  const int64_t k = small_chunk_of(n);
  return (nblk + k - 1) / k;
}

static bool passa_is_wide(ed_sector s);

template <typename T>
static void fill_tables(HvTables<T> &t, const SpinTables &u, const SpinTables &d, const T *vu,
                        const T *vd, const T *eu, const T *e_d, const T *W, int norb) {
  t.dup = u.dim;
  t.ddw = d.dim;
  t.rp_up = u.rowptr;
  t.col_up = u.col;
  t.val_up = vu;
  t.e_up = eu;
  t.m_up = u.imask;
  t.rp_dw = d.rowptr;
  t.col_dw = d.col;
  t.val_dw = vd;
  t.e_dw = e_d;
  t.m_dw = d.imask;
  t.W = W;
  t.nmask = 1 << norb;
}

template <typename T>
static void set_nd(HvTables<T> &t, ed_sector s, int layout) {
  const NdTables &nd = s->nd[layout];
  t.nd_up = nd.up;
  t.nd_dw = nd.dw;
  t.nd_ncols = nd.ncols;
  t.nd_norb = s->mp.norb;
  t.nd_jx = (T)s->mp.Jx;
  t.nd_jp = (T)s->mp.Jp;
}

template <>
HvTables<double> ed_hv_tables<double>(ed_sector s, int layout) {
  HvTables<double> t;
  const SpinTables *T2 = layout == 0 ? s->sp : s->bk;
  fill_tables<double>(t, T2[0], T2[1], T2[0].val, T2[1].val, T2[0].ediag, T2[1].ediag, s->W,
                      s->mp.norb);
  const ItemList &il = s->items[layout][1];
  t.items = il.d_items;
  t.nitems = il.nitems;
  t.smem = il.smem;
  t.ditems = il.d_ditems;
  t.nditems = il.nditems;
  t.stride = layout == 0 ? s->sp[0].dim : s->bstride;
  t.ell_col = layout == 0 ? nullptr : s->ell_col;
  t.ell_val = layout == 0 ? nullptr : s->ell_v64;
  t.small_cols = (layout == 1 && s->hv_kernel[1] == 1) ? s->small_cols : nullptr;
  t.small_grid = t.small_cols ? small_grid_of(s->bdim) : 0;
  t.small_chunk = (int32_t)small_chunk_of(s->bdim);
  t.passa_wide = layout == 1 && passa_is_wide(s);
  set_nd<double>(t, s, layout);
  return t;
}
template <>
HvTables<float> ed_hv_tables<float>(ed_sector s, int layout) {
  HvTables<float> t;
  const SpinTables *T2 = layout == 0 ? s->sp : s->bk;
  fill_tables<float>(t, T2[0], T2[1], T2[0].val32, T2[1].val32, T2[0].ediag32, T2[1].ediag32,
                     s->W32, s->mp.norb);
  const ItemList &il = s->items[layout][0];
  t.items = il.d_items;
  t.nitems = il.nitems;
  t.smem = il.smem;
  t.ditems = il.d_ditems;
  t.nditems = il.nditems;
  t.stride = layout == 0 ? s->sp[0].dim : s->bstride;
  t.ell_col = layout == 0 ? nullptr : s->ell_col;
  t.ell_val = layout == 0 ? nullptr : s->ell_v32;
  t.small_cols = (layout == 1 && s->hv_kernel[0] == 1) ? s->small_cols : nullptr;
  t.small_grid = t.small_cols ? small_grid_of(s->bdim) : 0;
  t.small_chunk = (int32_t)small_chunk_of(s->bdim);
  t.passa_wide = layout == 1 && passa_is_wide(s);
  set_nd<float>(t, s, layout);
  return t;
}

template <typename T>
struct HvLaunch {
  HvTables<T> tb;
  const T *v;
  T *w;
  T *b0, *b1, *b2;
  T *const *basis;  // Lanczos mode: vector j at basis[j] (else b[j % 3])
  T *psi;
  LanczosState *st;
  double *part;
};

constexpr int HV_THREADS = 512;
// H_dw pass of the two-pass product (k_hv_dw)
constexpr int DW_THREADS = 256;
constexpr int DW_ROWS = 32;    // rows of an item
constexpr int DW_COLS = 512;   // columns of an item (a multiple of 4)
constexpr size_t HV_SMEM_TWO = 88 * 1024;   // two CTAs per SM (with the static tables)
constexpr size_t HV_SMEM_MAX = 190 * 1024;  // one CTA per SM (very wide blocks)
constexpr int HV_MAXROWS = 64;              // rows of an item (G * RT <= 16 * 4)
#ifndef EDGB_MIN_CTAS
#define EDGB_MIN_CTAS 2
#endif

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ELL copy of H_up per up block (block-major order), interleaved by tiles of
// 4 columns: entry e of local column c = 4 t + u sits at
// ell_off + (e * ntile + t) * 4 + u.  Past a column's degree the entry is
// (the column itself, 0), which adds an exact zero.  One grid row per block.
__global__ void k_fill_ell(const int32_t *rowptr, const int32_t *col, const double *val,
                           const int64_t *blk_off, const int32_t *ell_off, const int32_t *ell_deg,
                           const int64_t *pad_off, const int32_t *run_len, int32_t *ell_col,
                           float *v32, double *v64) {
  const int b = blockIdx.y;
  const int64_t C0 = blk_off[b], nc = blk_off[b + 1] - C0;
  const int64_t ncp = pad_off[b + 1] - pad_off[b];
  const int64_t ntile = ncp / 4;
  const int deg = ell_deg[b];
  const int64_t base = ell_off[b];
  const int64_t dF = run_len[b];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncp;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = c >> 2, u = c & 3;
    int32_t k0 = 0, n = 0;
    if (c < nc) {
      k0 = rowptr[C0 + c];
      n = rowptr[C0 + c + 1] - k0;
    }
    // entry order: first the hops that keep the last group's string (they
    // shift the column by whole runs of dF, the same for every column of a
    // run), then the others, each in ascending target order
    int e = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int32_t k = k0; k < k0 + n; ++k) {
        const int64_t tgt = col[k] - C0;
        const bool same_run_pos = (tgt % dF) == (c % dF);
        if (same_run_pos != (pass == 0)) continue;
        const int64_t o = base + ((int64_t)e * ntile + t) * 4 + u;
        ell_col[o] = (int32_t)tgt;
        v64[o] = val[k];
        v32[o] = (float)val[k];
        ++e;
      }
    for (; e < deg; ++e) {
      const int64_t o = base + ((int64_t)e * ntile + t) * 4 + u;
      ell_col[o] = c < nc ? (int32_t)c : 0;
      v64[o] = 0.0;
      v32[o] = 0.0f;
    }
  }
}

ed_status ed_build_ell(ed_sector s, cudaStream_t st) {
  if (s->ell_col) return ED_OK;
  const BlockInfo &b = s->bi[0];
  const int nb = b.nblocks;
  std::vector<int32_t> rp(s->bk[0].dim + 1);
  ED_TRY_CUDA(cudaMemcpyAsync(rp.data(), s->bk[0].rowptr, rp.size() * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  s->ell_deg.assign(nb, 0);
  s->ell_off.assign(nb + 1, 0);
  for (int k = 0; k < nb; ++k) {
    int d = 0;
    for (int64_t c = b.offset[k]; c < b.offset[k + 1]; ++c) d = std::max(d, rp[c + 1] - rp[c]);
    s->ell_deg[k] = d;
    const int64_t ncp = s->up_off_pad[k + 1] - s->up_off_pad[k];
    const int64_t next = (int64_t)s->ell_off[k] + (int64_t)d * ncp;
    if (next >= (int64_t)INT32_MAX) return ED_ERR_UNSUPPORTED;
    s->ell_off[k + 1] = (int32_t)next;
  }
  const int64_t total = std::max<int64_t>(1, s->ell_off[nb]);
  int64_t *d_blk = nullptr, *d_pad = nullptr;
  int32_t *d_off = nullptr, *d_deg = nullptr;
  int32_t *ell_col = nullptr;
  float *ell_v32 = nullptr;
  double *ell_v64 = nullptr;
  ed_status rs = ed_dmalloc((void **)&ell_col, total * sizeof(int32_t), st, "ell");
  if (rs == ED_OK) rs = ed_dmalloc((void **)&ell_v32, total * sizeof(float), st, "ell");
  if (rs == ED_OK) rs = ed_dmalloc((void **)&ell_v64, total * sizeof(double), st, "ell");
  // block bounds for the fill kernel, released (stream-ordered) after it
  if (rs == ED_OK) rs = ed_dmalloc((void **)&d_blk, (nb + 1) * sizeof(int64_t), st, "ell bounds");
  if (rs == ED_OK) rs = ed_dmalloc((void **)&d_pad, (nb + 1) * sizeof(int64_t), st, "ell bounds");
  if (rs == ED_OK) rs = ed_dmalloc((void **)&d_off, (nb + 1) * sizeof(int32_t), st, "ell bounds");
  if (rs == ED_OK) rs = ed_dmalloc((void **)&d_deg, nb * sizeof(int32_t), st, "ell bounds");
  // run length of every up block: the strings of its last orbital group
  // (Norb = 1: the whole block); inside a block the index is (slow, run)
  std::vector<int32_t> run(std::max(nb, 1), 1);
  {
    const int norb = s->mp.norb, g = s->mp.nbath + 1;
    for (int k = 0; k < nb; ++k) {
      int64_t d = b.offset[k + 1] - b.offset[k];
      if (norb >= 2) {
        const int m = b.keys[(size_t)k * norb + norb - 1];
        d = 1;
        for (int i = 1; i <= m; ++i) d = d * (g - m + i) / i;
      }
      run[k] = (int32_t)std::max<int64_t>(d, 1);
    }
  }
  int32_t *d_run = nullptr;
  if (rs == ED_OK) rs = ed_dmalloc((void **)&d_run, run.size() * sizeof(int32_t), st, "ell bounds");
  auto h2d = [&](void *dst, const void *src, size_t bytes) {
    if (rs == ED_OK && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rs = ED_ERR_CUDA;
  };
  h2d(d_blk, b.offset.data(), (nb + 1) * sizeof(int64_t));
  h2d(d_pad, s->up_off_pad.data(), (nb + 1) * sizeof(int64_t));
  h2d(d_off, s->ell_off.data(), (nb + 1) * sizeof(int32_t));
  h2d(d_deg, s->ell_deg.data(), nb * sizeof(int32_t));
  h2d(d_run, run.data(), run.size() * sizeof(int32_t));
  if (rs == ED_OK) {
    int64_t maxw = 1;
    for (int k = 0; k < nb; ++k)
      maxw = std::max<int64_t>(maxw, s->up_off_pad[k + 1] - s->up_off_pad[k]);
    dim3 grid((unsigned)std::min<int64_t>((maxw + 255) / 256, 1024), (unsigned)nb);
    k_fill_ell<<<grid, 256, 0, st>>>(s->bk[0].rowptr, s->bk[0].col, s->bk[0].val, d_blk, d_off,
                                     d_deg, d_pad, d_run, ell_col, ell_v32, ell_v64);
    ed_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "k_fill_ell", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  ed_dfree(d_blk, st);
  ed_dfree(d_pad, st);
  ed_dfree(d_off, st);
  ed_dfree(d_deg, st);
  ed_dfree(d_run, st);
  if (rs == ED_OK && cudaStreamSynchronize(st) != cudaSuccess) rs = ED_ERR_CUDA;
  if (rs != ED_OK) {
    ed_dfree(ell_col, st);
    ed_dfree(ell_v32, st);
    ed_dfree(ell_v64, st);
    return rs;
  }
  // published only once filled
  s->ell_col = ell_col;
  s->ell_v32 = ell_v32;
  s->ell_v64 = ell_v64;
  s->device_bytes += total * 16;
  return ED_OK;
}

// Column table of the element-parallel product (small sectors): built once,
// after the ELL table.  Sectors whose blocks do not fit the packing stay on
// the tiled kernel.
static ed_status build_small_cols(ed_sector s, cudaStream_t cs) {
  if (s->small_cols || s->bdim == 0) return ED_OK;
  const BlockInfo &b = s->bi[0];
  std::vector<int4> cols(s->bstride);
  for (int k = 0; k < b.nblocks; ++k) {
    const int64_t C0 = b.offset[k], nc = b.offset[k + 1] - C0;
    const int64_t p0 = s->up_off_pad[k], ncp = s->up_off_pad[k + 1] - p0;
    if (ncp >= (1 << 23) || s->ell_deg[k] > 255) return ED_OK;
    for (int64_t c = 0; c < ncp; ++c)
      cols[p0 + c] = make_int4(c < nc ? (int)(C0 + c) : -1, s->ell_off[k] + (int)c, (int)p0,
                               (int)(ncp << 8) | s->ell_deg[k]);
  }
  int4 *d = nullptr;
  ED_TRY(ed_dmalloc((void **)&d, cols.size() * sizeof(int4), cs, "small-sector columns"));
  cudaError_t e = cudaMemcpyAsync(d, cols.data(), cols.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "small-sector columns upload", __FILE__, __LINE__);
    ed_dfree(d, cs);
    return ED_ERR_CUDA;
  }
  s->small_cols = d;
  s->device_bytes += (int64_t)(cols.size() * sizeof(int4));
  return ED_OK;
}

// Two-pass product: used when the largest (dw block x up block) slice of a
// vector exceeds EDGB_TWO_PASS_MB, so that the neighbour rows the one-pass
// kernel reads for H_dw no longer stay in L2.  The H_dw pass then walks
// column chunks of DW_COLS through all rows of a dw block.
#ifndef EDGB_TWO_PASS_MB
#define EDGB_TWO_PASS_MB 160
#endif
static bool two_pass_wanted(ed_sector s, int elem) {
  const std::vector<int64_t> &ob_dw = s->bi[1].offset;
  int64_t max_rows = 0, max_cols = 0;
  for (size_t k = 0; k + 1 < ob_dw.size(); ++k) max_rows = std::max(max_rows, ob_dw[k + 1] - ob_dw[k]);
  for (size_t k = 0; k + 1 < s->up_off_pad.size(); ++k)
    max_cols = std::max(max_cols, s->up_off_pad[k + 1] - s->up_off_pad[k]);
  return max_rows * max_cols * elem > ((int64_t)EDGB_TWO_PASS_MB << 20);
}

// the H_up pass shape of this sector (see rt_passa)
static bool passa_is_wide(ed_sector s) {
  int64_t w = 0;
  for (size_t k = 0; k + 1 < s->up_off_pad.size(); ++k)
    w = std::max<int64_t>(w, s->up_off_pad[k + 1] - s->up_off_pad[k]);
  return w > (int64_t)EDGB_PASSA_WIDE;
}

static ed_status build_dw_items(ed_sector s, ItemList &il, int elem, cudaStream_t cs) {
  if (il.d_ditems || !two_pass_wanted(s, elem)) return ED_OK;
  const std::vector<int64_t> &ob_dw = s->bi[1].offset, &ob_up = s->bi[0].offset;
  std::vector<DwItem> items;
  for (size_t bd = 0; bd + 1 < ob_dw.size(); ++bd) {
    const int64_t R0 = ob_dw[bd], R1 = ob_dw[bd + 1];
    for (size_t bu = 0; bu + 1 < ob_up.size(); ++bu) {
      const int64_t nc = ob_up[bu + 1] - ob_up[bu], p0 = s->up_off_pad[bu];
      for (int64_t c = 0; c < nc; c += DW_COLS)
        for (int64_t r = R0; r < R1; r += DW_ROWS)
          items.push_back(DwItem{(int32_t)r, (int32_t)std::min<int64_t>(DW_ROWS, R1 - r),
                                 (int32_t)(p0 + c), (int32_t)std::min<int64_t>(DW_COLS, nc - c)});
    }
  }
  DwItem *d = nullptr;
  ED_TRY(ed_dmalloc((void **)&d, std::max<size_t>(items.size(), 1) * sizeof(DwItem), cs,
                    "H_dw work items"));
  cudaError_t e = cudaSuccess;
  if (!items.empty())
    e = cudaMemcpyAsync(d, items.data(), items.size() * sizeof(DwItem), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "H_dw work items upload", __FILE__, __LINE__);
    ed_dfree(d, cs);
    return ED_ERR_CUDA;
  }
  il.nditems = (int64_t)items.size();
  il.d_ditems = d;
  s->device_bytes += (int64_t)(items.size() * sizeof(DwItem));
  return ED_OK;
}

// ----------------------------------------------------------------- autotuner
//
// For sectors above EDGB_TUNE_MIN padded elements the faster of the tiled
// family (one or two passes) and the element-parallel product depends on the
// block shapes and the precision, so it is measured: both kernels, one
// warm-up and three timed launches each (alternating) on a scratch vector,
// on this thread's private stream.  The choice is kept per model shape
// (Norb, Nbath, precision) for the life of the process, so every sector of a
// shape uses the same kernel and results do not depend on which call came
// first.  The sectors of one shape share the block structure that decides
// between the kernels (block widths set by the orbital count, bath strings
// of one length); where two sectors of a shape were measured (Ns = 14, at
// and next to half filling) both chose the same kernel wherever the two
// kernels differed by more than 5%.  Keying on the sector as well made
// a serving stream whose requests are mostly distinct sectors tune on almost
// every request (15% fewer solves/s at Ns <= 16).  Both kernels give the
// same w = H v bit for bit.
namespace {
struct TuneKey {
  int norb, nbath, elem;
  bool operator<(const TuneKey &o) const {
    return std::tie(norb, nbath, elem) < std::tie(o.norb, o.nbath, o.elem);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
}  // namespace

// Autotuning input: v_i = u_i - 1/2 at every real element (u_i a uniform
// from a hash of the index, the distribution of the Lanczos start vector),
// zero at padding columns; timings on a zero vector run faster than on the
// vectors the solves see.
template <typename T>
__global__ void k_tune_fill(T *v, int64_t n, int64_t stride, const int32_t *padinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pc = i % stride;
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x5EEDull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = padinv[pc] < 0 ? T(0) : (T)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
}

template <typename T>
static ed_status time_hv_kernels(ed_sector s, int e, cudaStream_t cs, double ms[2]) {
  const int64_t n = s->bdim;
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, 2 * n * sizeof(T), cs, "autotune vectors"));
  T *v = (T *)mem, *w = v + n;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ed_status rs = ED_OK;
  if (cudaMemsetAsync(w, 0, n * sizeof(T), cs) != cudaSuccess ||
      cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (rs == ED_OK) {
    k_tune_fill<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, cs>>>(
        v, n, s->bstride, s->padinv);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  // one warm-up launch of each kernel, then three rounds that alternate the
  // two, so that a clock that is still ramping up favours neither
  ms[0] = ms[1] = 0.0;
  for (int r = -1; r < 3 && rs == ED_OK; ++r)
    for (int k = 0; k < 2 && rs == ED_OK; ++k) {
      s->hv_kernel[e] = (int8_t)k;
      const HvTables<T> tb = ed_hv_tables<T>(s, 1);
      if (cudaEventRecord(ev[0], cs) != cudaSuccess) rs = ED_ERR_CUDA;
      if (rs == ED_OK)
        rs = ed_launch_hv<T>(s, tb, HV_PLAIN, v, w, nullptr, nullptr, nullptr, nullptr, nullptr, cs);
      float t = 0.0f;
      if (rs == ED_OK && (cudaEventRecord(ev[1], cs) != cudaSuccess ||
                          cudaEventSynchronize(ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess))
        rs = ED_ERR_CUDA;
      if (r >= 0) ms[k] += t / 3.0;
    }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  ed_dfree(mem, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  return rs;
}

static ed_status decide_kernel(ed_sector s, int elem, cudaStream_t cs) {
  const int e = elem == 8 ? 1 : 0;
  if (s->hv_kernel[e] >= 0) return ED_OK;
  if (!s->small_cols) {
    s->hv_kernel[e] = 0;
    return ED_OK;
  }
  if (s->bdim <= (int64_t)EDGB_TUNE_MIN) {
    s->hv_kernel[e] = 1;
    return ED_OK;
  }
  const TuneKey key{s->mp.norb, s->mp.nbath, elem};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      s->hv_kernel[e] = (int8_t)it->second;
      return ED_OK;
    }
  }
  double ms[2] = {-1.0, -1.0};
  const ed_status rs = elem == 8 ? time_hv_kernels<double>(s, e, cs, ms)
                                 : time_hv_kernels<float>(s, e, cs, ms);
  if (rs != ED_OK) {
    s->hv_kernel[e] = 0;
    return rs;
  }
  int choice = ms[1] < ms[0] ? 1 : 0;
  s->tune_ms[e][0] = ms[0];
  s->tune_ms[e][1] = ms[1];
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);  // another thread may have tuned the shape meanwhile
    if (it != g_tune.end()) choice = it->second;
    else g_tune[key] = choice;
  }
  s->hv_kernel[e] = (int8_t)choice;
  return ED_OK;
}

// Rows of an item and the shared-memory bytes of one row group: the CTA is
// split into G groups of P threads (P = the item's columns rounded up to a
// warp, at most the CTA); group q owns rows q*RT .. q*RT+RT-1.
static void item_shape(int64_t nc, int elem, int RT, int threads, int64_t *rows,
                       size_t *bytes_per_group) {
  const int64_t ntile = (nc + 3) / 4;
  const int64_t P = ntile >= threads ? threads : round_up(ntile, 32);
  const int64_t G = threads / P;
  *rows = G * RT;
  *bytes_per_group = (size_t)round_up(nc, 4) * RT * elem;
}

// Work items, ordered dw block by dw block, up block by up block, rows
// ascending: while one block pair is processed, its |dw block| x |up block|
// slice of v is the L2 working set of the H_dw reads.
ed_status ed_build_items(ed_sector s, int layout, int elem) {
  ItemList &il = s->items[layout][elem == 8 ? 1 : 0];
  if (il.d_items) return ED_OK;
  // built once per sector on this thread's private stream, complete on return
  ed_status ps = ED_OK;
  cudaStream_t cs = ed_private_stream(&ps);
  if (ps != ED_OK) return ps;
  std::vector<int64_t> ob_up, ob_dw, op_up;
  if (layout == 0) {
    ob_up = {0, s->sp[0].dim};
    op_up = ob_up;
    ob_dw = {0, s->sp[1].dim};
  } else {
    ED_TRY(ed_build_ell(s, cs));
    ED_TRY(build_small_cols(s, cs));
    ob_up = s->bi[0].offset;
    op_up = s->up_off_pad;
    ob_dw = s->bi[1].offset;
  }
  // the H_up pass of the two-pass product has its own tile height and CTA size
  const bool passa = layout == 1 && two_pass_wanted(s, elem);
  const bool wide = passa_is_wide(s);
  const int RT = passa ? (elem == 4 ? (wide ? rt_passa<float, true>() : rt_passa<float, false>())
                                    : (wide ? rt_passa<double, true>() : rt_passa<double, false>()))
                       : (elem == 4 ? Tile<float>::RT : Tile<double>::RT);
  const int threads = passa ? (wide ? passa_threads<true>() : passa_threads<false>()) : HV_THREADS;
  std::vector<HvItem> items;
  size_t smem = 0;
  for (size_t bd = 0; bd + 1 < ob_dw.size(); ++bd) {
    const int64_t R0 = ob_dw[bd], R1 = ob_dw[bd + 1];
    if (R1 <= R0) continue;
    for (size_t bu = 0; bu + 1 < ob_up.size(); ++bu) {
      const int64_t C0 = ob_up[bu], C1 = ob_up[bu + 1];
      const int64_t nc = C1 - C0;
      if (nc <= 0) continue;
      int64_t R;
      size_t per_group;
      item_shape(nc, elem, RT, threads, &R, &per_group);
      // shared memory holds ceil(R/RT) row groups; shrink R until it fits
      while (R > RT && (size_t)((R + RT - 1) / RT) * per_group > HV_SMEM_TWO) R -= RT;
      // the per-row lists of an item live in arrays of HV_MAXROWS rows
      R = std::min<int64_t>(std::min<int64_t>(R, HV_MAXROWS), R1 - R0);
      const size_t need = (size_t)((R + RT - 1) / RT) * per_group;
      if (need <= HV_SMEM_MAX) smem = std::max(smem, need);
      const int32_t deg = layout == 0 ? 0 : s->ell_deg[bu];
      const int32_t eoff = layout == 0 ? 0 : s->ell_off[bu];
      const int32_t ncp = (int32_t)(op_up[bu + 1] - op_up[bu]);
      for (int64_t r = R0; r < R1; r += R)
        items.push_back(HvItem{(int32_t)r, (int32_t)std::min<int64_t>(R, R1 - r), (int32_t)C0,
                               (int32_t)nc, (int32_t)op_up[bu], deg, eoff, ncp});
    }
  }
  HvItem *d_items = nullptr;
  ED_TRY(ed_dmalloc((void **)&d_items, std::max<size_t>(items.size(), 1) * sizeof(HvItem), cs,
                    "work items"));
  cudaError_t e = cudaSuccess;
  if (!items.empty())
    e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(HvItem),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "work items upload", __FILE__, __LINE__);
    ed_dfree(d_items, cs);
    return ED_ERR_CUDA;
  }
  // published only once complete
  il.nitems = (int64_t)items.size();
  il.smem = smem;
  il.d_items = d_items;
  s->device_bytes += (int64_t)(items.size() * sizeof(HvItem));
  if (layout == 1) {
    ED_TRY(build_dw_items(s, il, elem, cs));
    ED_TRY(decide_kernel(s, elem, cs));
  }
  return ED_OK;
}

template <typename T>
__device__ __forceinline__ double block_sum(double x, double *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  }
  return s;
}

// Slot of column c in a staged row group of ncp = 4 q4 columns: columns are
// interleaved by c mod 4 (all columns 0 mod 4 first, then 1 mod 4, ...).  The
// lanes of a warp own consecutive 4-column tiles, so when they all read
// member u of their tiles (the diagonal, or hops that shift whole runs of
// columns) they read consecutive 16-byte slots: no bank conflicts.
__device__ __forceinline__ int stage_pos(int c, int q4) { return (c & 3) * q4 + (c >> 2); }

// One tile: 4 consecutive columns cb..cb+3 x RT rows of the thread's row
// group.  FULL: all RT rows exist and all 4 columns are inside the block
// (no predication).  BLK: block-major layout (ELL table, aligned vectors).
// Asynchronous copy of one element from global to shared memory (cp.async,
// cached in L1), so that all the loads of a staging loop are in flight at
// once instead of each waiting in a register for its shared-memory store.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst_smem, const T *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T, bool FULL, bool BLK, bool NODW, int RTX>
__device__ __forceinline__ void hv_tile(const HvTables<T> &tb, const HvItem &it, const T *g,
                                        const T *smq, bool staged, int lr0, int nrt, int cb,
                                        const int32_t *s_dn, const int32_t *s_dcol,
                                        const T *s_dval, const int32_t *s_mdw, const T *s_edw,
                                        T (&acc)[4][RTX]) {
  constexpr int RT = RTX;
  using VT = typename TileOf<T, RTX>::V;
  const int64_t stride = tb.stride;
  const int r0 = it.r0, c0 = it.c0, nc = it.nc;
  const int q4 = (nc + 3) >> 2;
  const int64_t cp0 = it.c0p;
  auto rows_at = [&](int c, T *y) {
    if (staged) {
      vec_get(*reinterpret_cast<const VT *>(smq + (size_t)stage_pos(c, q4) * RT), y);
    } else {
#pragma unroll
      for (int i = 0; i < RT; ++i)
        y[i] = (FULL || i < nrt) ? g[(int64_t)(r0 + lr0 + i) * stride + cp0 + c] : T(0);
    }
  };
  // diagonal
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = cb + u;
#pragma unroll
    for (int i = 0; i < RT; ++i) acc[u][i] = T(0);
    if (FULL || c < nc) {
      T x[RT];
      rows_at(c, x);
      const int64_t cg = (int64_t)c0 + c;
      const T eu = tb.e_up[cg];
      const int mu = (int)tb.m_up[cg] * tb.nmask;
#pragma unroll
      for (int i = 0; i < RT; ++i)
        if (FULL || i < nrt)
          acc[u][i] =
              mul_t<T>(add_t<T>(add_t<T>(eu, s_edw[lr0 + i]), tb.W[mu + s_mdw[lr0 + i]]), x[i]);
    }
  }
  // H_up
  if (BLK) {
    const int64_t ntile4 = (int64_t)it.ncp;  // entries of one ELL row (4 per tile)
    const int4 *ec = reinterpret_cast<const int4 *>(tb.ell_col + it.ell_off + cb);
    const T *ev = tb.ell_val + it.ell_off + cb;
    for (int e = 0; e < it.deg; ++e) {
      const int4 kc = __ldg(ec + (e * ntile4) / 4);
      T h[4];
      load4(ev + e * ntile4, h);
      const int kk[4] = {kc.x, kc.y, kc.z, kc.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (FULL || cb + u < nc) {
          T y[RT];
          rows_at(kk[u], y);
#pragma unroll
          for (int i = 0; i < RT; ++i) acc[u][i] = fma_t<T>(h[u], y[i], acc[u][i]);
        }
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = cb + u;
      if (FULL || c < nc) {
        const int64_t cg = (int64_t)c0 + c;
        const int32_t k0 = __ldg(tb.rp_up + cg), k1 = __ldg(tb.rp_up + cg + 1);
        for (int32_t k = k0; k < k1; ++k) {
          const int kc = __ldg(tb.col_up + k) - c0;
          const T h = __ldg(tb.val_up + k);
          T y[RT];
          rows_at(kc, y);
#pragma unroll
          for (int i = 0; i < RT; ++i) acc[u][i] = fma_t<T>(h, y[i], acc[u][i]);
        }
      }
    }
  }
  // H_dw: neighbour rows at the same 4 columns (the second pass does it when NODW)
#pragma unroll
  for (int i = 0; i < (NODW ? 0 : RT); ++i) {
    if (!FULL && i >= nrt) continue;
    const int n = s_dn[lr0 + i];
    const int32_t *dc = s_dcol + (lr0 + i) * ED_MAX_NS;
    const T *dv = s_dval + (lr0 + i) * ED_MAX_NS;
    int t = 0;
    if (BLK) {
      // two neighbour rows in flight (four measured 5% slower: spills at the
      // 64-register cap)
      for (; t + 2 <= n; t += 2) {
        T y[2][4];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
          load4(g + (int64_t)dc[t + q2] * stride + cp0 + cb, y[q2]);
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const T h = dv[t + q2];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][i] = fma_t<T>(h, y[q2][u], acc[u][i]);
        }
      }
    }
    for (; t < n; ++t) {
      const T h = dv[t];
      const T *nb = g + (int64_t)dc[t] * stride + cp0 + cb;
      T y[4];
      if (BLK) {
        load4(nb, y);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = (FULL || cb + u < nc) ? __ldg(nb + u) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][i] = fma_t<T>(h, y[u], acc[u][i]);
    }
  }
}

// PASSA: first pass of the two-pass product (block pairs larger than L2): the
// diagonal and H_up only, written unscaled to the output vector; k_hv_dw adds
// H_dw and applies the epilogue.
template <typename T, int MODE, bool BLK, bool PASSA = false, int RTX = Tile<T>::RT,
          int NT = HV_THREADS>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : EDGB_MIN_CTAS) k_hv(HvLaunch<T> a) {
  constexpr int RT = RTX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  __shared__ int32_t s_dcol[HV_MAXROWS * ED_MAX_NS];
  __shared__ T s_dval[HV_MAXROWS * ED_MAX_NS];
  __shared__ int32_t s_dn[HV_MAXROWS], s_mdw[HV_MAXROWS];
  __shared__ T s_edw[HV_MAXROWS];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const HvTables<T> &tb = a.tb;

  // Epilogue state of the Lanczos modes, kept in shared memory and read in
  // the epilogue only: held in registers across the tile it made the
  // Lanczos-mode kernel spill at the 64-register cap (152 bytes; the FP32
  // Lanczos step at D = 1.66e8 went from 2.60 to 2.46 ms without them).
  struct EpState {
    T *out;
    const T *prev;
    T s_cur, s_prev, beta_j, alpha_j, y_j;
    int j;
  };
  __shared__ EpState ep_s;
  const T *g;
  T *out_plain = nullptr;
  if (MODE == HV_PLAIN) {
    g = a.v;
    out_plain = a.w;
  } else {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    const int j = st->j;
    T *bufs[3] = {a.b0, a.b1, a.b2};
    g = bufs[j % 3];
    if (MODE == HV_LANCZOS && a.basis) g = a.basis[j];
    if (threadIdx.x == 0) {
      EpState e;
      e.j = j;
      e.prev = bufs[(j + 2) % 3];
      e.out = bufs[(j + 1) % 3];
      if (MODE == HV_LANCZOS && a.basis) {
        e.prev = a.basis[j > 0 ? j - 1 : 0];
        e.out = a.basis[j + 1];
      }
      e.s_cur = (T)st->scale[j % 3];
      e.s_prev = (T)st->scale[(j + 2) % 3];
      e.beta_j = (T)st->beta[j];
      e.alpha_j = MODE == HV_SECOND ? (T)st->alpha[j] : T(0);
      e.y_j = MODE == HV_SECOND ? (T)st->y[j] : T(0);
      ep_s = e;
    }
  }

  const HvItem it = tb.items[blockIdx.x];
  const int64_t stride = tb.stride;
  const int r0 = it.r0, nr = it.nr, nc = it.nc;
  const int64_t cp0 = it.c0p;  // first column of the item in the vector layout
  const int ncp = (nc + 3) & ~3;
  const int ngroups = (nr + RT - 1) / RT;
  const bool staged = (size_t)ngroups * ncp * RT * sizeof(T) <= tb.smem;
  // staging, transposed: sm[(q * ncp + stage_pos(c)) * RT + i] = v[r0 + q*RT + i][c],
  // by asynchronous copies that complete before the barrier below (issued all
  // at once: with the copies waited for one by one through registers the
  // FP32 product at D = 1.66e8 took 1.50 ms, with cp.async 1.17 ms)
  if (staged) {
    for (int lr = 0; lr < ngroups * RT; ++lr) {
      const int q = lr / RT, i = lr - q * RT;
      T *dst = sm + (size_t)q * ncp * RT + i;
      if (lr < nr) {
        const T *src = g + (int64_t)(r0 + lr) * stride + cp0;
        for (int c = threadIdx.x; c < ncp; c += blockDim.x) {
          T *d = dst + stage_pos(c, ncp >> 2) * RT;
          if (c < nc)
            cp_async_elem<T>(d, src + c);
          else
            *d = T(0);
        }
      } else {
        for (int c = threadIdx.x; c < ncp; c += blockDim.x) dst[stage_pos(c, ncp >> 2) * RT] = T(0);
      }
    }
  }
  // per-row data of the item: diagonal pieces and the H_dw neighbour lists
  for (int lr = threadIdx.x; lr < nr; lr += blockDim.x) {
    const int64_t r = r0 + lr;
    const int32_t d0 = __ldg(tb.rp_dw + r), d1 = __ldg(tb.rp_dw + r + 1);
    s_dn[lr] = d1 - d0;
    s_mdw[lr] = tb.m_dw[r];
    s_edw[lr] = tb.e_dw[r];
    if (!PASSA)
      for (int32_t k = d0; k < d1; ++k) {
      s_dcol[lr * ED_MAX_NS + (k - d0)] = __ldg(tb.col_dw + k);
      s_dval[lr * ED_MAX_NS + (k - d0)] = __ldg(tb.val_dw + k);
    }
  }
  if (staged) cp_async_wait_all();  // the staged rows, loaded while the lists above were read
  __syncthreads();

  const int ntile = ncp / 4;
  const int P = ntile >= (int)blockDim.x ? (int)blockDim.x : ((ntile + 31) & ~31);
  const int q = threadIdx.x / P, p = threadIdx.x - q * P;
  const int lr0 = q * RT;
  const int nrt = min(RT, nr - lr0);  // rows of this thread (may be <= 0)
  const T *smq = sm + (size_t)q * ncp * RT;

  // Lanczos mode: <v_j, w1> summed in T over this thread's tiles of the item
  // (at most ceil(1225 / 512) = 3 tiles of 16 products at Ns=16), then in
  // FP64 across threads and CTAs.  An FP64 accumulator per thread (or a
  // shared-memory FP64 slot per tile) doubled the register spills of this
  // kernel at its 64-register cap and slowed the FP32 Lanczos step.
  T dot = T(0);
  if (nrt > 0) {
    for (int tl = p; tl < ntile; tl += P) {
      const int cb = tl * 4;
      T acc[4][RT];
      const bool full = nrt == RT && cb + 4 <= nc;
      if (full)
        hv_tile<T, true, BLK, PASSA, RT>(tb, it, g, smq, staged, lr0, nrt, cb, s_dn, s_dcol,
                                         s_dval, s_mdw, s_edw, acc);
      else
        hv_tile<T, false, BLK, PASSA, RT>(tb, it, g, smq, staged, lr0, nrt, cb, s_dn, s_dcol,
                                          s_dval, s_mdw, s_edw, acc);
      // epilogue: one 16-byte store (and, in the Lanczos modes, one 16-byte
      // load of v_{j-1}) per row of a full tile in the block-major layout,
      // whose rows and blocks are padded to multiples of 4 elements (the
      // sector-order layout is not aligned: element accesses there)
      const bool vec = BLK && full;
      const volatile EpState &ep = ep_s;
      T *const out = MODE == HV_PLAIN ? out_plain : ep.out;
      if (MODE == HV_PLAIN || PASSA) {
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          if (i >= nrt) continue;
          T *o = out + (int64_t)(r0 + lr0 + i) * stride + cp0 + cb;
          if (vec) {
            const T res[4] = {acc[0][i], acc[1][i], acc[2][i], acc[3][i]};
            store4(o, res);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (cb + u < nc) o[u] = acc[u][i];
          }
        }
      } else {
        if (MODE == HV_LANCZOS) {
          // w1 = H v_j (the update kernel subtracts beta_j v_{j-1} and
          // alpha_j v_j); each column's RT staged rows of v_j in one 16-byte
          // shared load for <v_j, w1>
          const T s_cur = ep.s_cur;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = cb + u;
            T xr[RT];
            if (staged) {
              vec_get(*reinterpret_cast<const typename TileOf<T, RTX>::V *>(
                          smq + (size_t)stage_pos(c, ncp >> 2) * RT),
                      xr);
            } else {
#pragma unroll
              for (int i = 0; i < RT; ++i)
                xr[i] = (i < nrt && (full || c < nc))
                            ? g[(int64_t)(r0 + lr0 + i) * stride + cp0 + c]
                            : T(0);
            }
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              if (i >= nrt || (!full && c >= nc)) continue;
              const T w1 = mul_t<T>(acc[u][i], s_cur);
              acc[u][i] = w1;
              dot = fma_t<T>(mul_t<T>(xr[i], s_cur), w1, dot);
            }
          }
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            if (i >= nrt) continue;
            T *o = out + (int64_t)(r0 + lr0 + i) * stride + cp0 + cb;
            if (vec) {
              const T res[4] = {acc[0][i], acc[1][i], acc[2][i], acc[3][i]};
              store4(o, res);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (cb + u < nc) o[u] = acc[u][i];
            }
          }
          continue;
        }
        // second pass: the step's scalars, read from shared memory once per tile
        const T s_cur = ep.s_cur, s_prev = ep.s_prev, beta_j = ep.beta_j;
        const T alpha_j = ep.alpha_j, y_j = ep.y_j;
        const T *const prev = ep.prev;
        const bool has_prev = ep.j > 0;
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          if (i >= nrt) continue;
          const int64_t rb = (int64_t)(r0 + lr0 + i) * stride + cp0 + cb;
          T pv[4] = {T(0), T(0), T(0), T(0)};
          if (has_prev) {
            if (vec) {
              load4(prev + rb, pv);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (cb + u < nc) pv[u] = prev[rb + u];
            }
          }
          T res[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = cb + u;
            res[u] = T(0);
            if (!full && c >= nc) continue;
            const T xv = staged ? smq[(size_t)stage_pos(c, ncp >> 2) * RT + i] : g[rb + u];
            const T v = mul_t<T>(xv, s_cur);
            T w1 = mul_t<T>(acc[u][i], s_cur);
            if (has_prev) w1 = fma_t<T>(-beta_j, mul_t<T>(pv[u], s_prev), w1);
            if (MODE == HV_LANCZOS) {
              res[u] = w1;
              dot = fma_t<T>(v, w1, dot);
            } else {
              res[u] = fma_t<T>(-alpha_j, v, w1);
              a.psi[rb + u] = fma_t<T>(y_j, v, a.psi[rb + u]);
            }
          }
          if (vec) {
            store4(out + rb, res);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (cb + u < nc) out[rb + u] = res[u];
          }
        }
      }
    }
  }
  if (MODE == HV_LANCZOS && !PASSA) {
    double smv = block_sum<T>((double)dot, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = smv;
  }
}

// Second pass of the two-pass product: out += H_dw v over DwItems (rows of
// one dw block x a column chunk of one up block), then the epilogue of k_hv.
// Items run column chunk by column chunk through all rows of a dw block, so
// the chunk's strip of v (rows of the dw block x chunk columns) is the L2
// working set of the neighbour-row reads.  Each accumulator continues from
// the first pass's value and adds the H_dw terms in the same order as k_hv,
// so the product equals the one-pass product bit for bit.

template <typename T, int MODE>
__global__ void __launch_bounds__(DW_THREADS) k_hv_dw(HvLaunch<T> a) {
  constexpr int RT = Tile<T>::RT;
  __shared__ double red[DW_THREADS / 32];
  __shared__ int32_t s_dcol[DW_ROWS * ED_MAX_NS];
  __shared__ T s_dval[DW_ROWS * ED_MAX_NS];
  __shared__ int32_t s_dn[DW_ROWS];
  const HvTables<T> &tb = a.tb;
  int j = 0;
  T s_cur = T(1), s_prev = T(0), beta_j = T(0), alpha_j = T(0), y_j = T(0);
  const T *g;
  const T *prev = nullptr;
  T *out;
  if (MODE == HV_PLAIN) {
    g = a.v;
    out = a.w;
  } else {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    j = st->j;
    const int m3 = j % 3;
    g = m3 == 0 ? a.b0 : (m3 == 1 ? a.b1 : a.b2);
    out = m3 == 0 ? a.b1 : (m3 == 1 ? a.b2 : a.b0);
    prev = m3 == 0 ? a.b2 : (m3 == 1 ? a.b0 : a.b1);
    if (MODE == HV_LANCZOS && a.basis) {
      g = a.basis[j];
      prev = a.basis[j > 0 ? j - 1 : 0];
      out = a.basis[j + 1];
    }
    s_cur = (T)st->scale[m3];
    s_prev = (T)st->scale[(j + 2) % 3];
    beta_j = (T)st->beta[j];
    if (MODE == HV_SECOND) {
      alpha_j = (T)st->alpha[j];
      y_j = (T)st->y[j];
    }
  }
  const DwItem it = tb.ditems[blockIdx.x];
  const int64_t stride = tb.stride;
  for (int lr = threadIdx.x; lr < it.nr; lr += blockDim.x) {
    const int64_t r = it.r0 + lr;
    const int32_t d0 = __ldg(tb.rp_dw + r), d1 = __ldg(tb.rp_dw + r + 1);
    s_dn[lr] = d1 - d0;
    for (int32_t k = d0; k < d1; ++k) {
      s_dcol[lr * ED_MAX_NS + (k - d0)] = __ldg(tb.col_dw + k);
      s_dval[lr * ED_MAX_NS + (k - d0)] = __ldg(tb.val_dw + k);
    }
  }
  __syncthreads();
  const int ntile = (it.nc + 3) >> 2, ngrp = (it.nr + RT - 1) / RT;
  T dot = T(0);       // one tile's products (at most 16)
  double dotd = 0.0;  // the thread's tiles
  for (int idx = threadIdx.x; idx < ngrp * ntile; idx += blockDim.x) {
    dotd += (double)dot;
    dot = T(0);
    const int q = idx / ntile, cb = (idx - q * ntile) * 4;
    const int lr0 = q * RT, nrt = min(RT, it.nr - lr0);
    const int64_t col0 = (int64_t)it.c0p + cb;
    T acc[RT][4];
#pragma unroll
    for (int i = 0; i < RT; ++i)
      if (i < nrt) load4(out + (int64_t)(it.r0 + lr0 + i) * stride + col0, acc[i]);
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      if (i >= nrt) continue;
      const int n = s_dn[lr0 + i];
      const int32_t *dc = s_dcol + (lr0 + i) * ED_MAX_NS;
      const T *dv = s_dval + (lr0 + i) * ED_MAX_NS;
      int t = 0;
      for (; t + 2 <= n; t += 2) {
        T y[2][4];
        load4(g + (int64_t)dc[t] * stride + col0, y[0]);
        load4(g + (int64_t)dc[t + 1] * stride + col0, y[1]);
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const T h = dv[t + q2];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[i][u] = fma_t<T>(h, y[q2][u], acc[i][u]);
        }
      }
      for (; t < n; ++t) {
        T y[4];
        load4(g + (int64_t)dc[t] * stride + col0, y);
        const T h = dv[t];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[i][u] = fma_t<T>(h, y[u], acc[i][u]);
      }
    }
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      if (i >= nrt) continue;
      const int64_t rowbase = (int64_t)(it.r0 + lr0 + i) * stride + col0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (cb + u >= it.nc) continue;  // padding is not written
        const int64_t gi = rowbase + u;
        if (MODE == HV_PLAIN) {
          out[gi] = acc[i][u];
        } else {
          const T v = mul_t<T>(g[gi], s_cur);
          T w1 = mul_t<T>(acc[i][u], s_cur);
          if (MODE == HV_SECOND && j > 0)  // the Lanczos step does this in its update
            w1 = fma_t<T>(-beta_j, mul_t<T>(prev[gi], s_prev), w1);
          if (MODE == HV_LANCZOS) {
            out[gi] = w1;
            dot = fma_t<T>(v, w1, dot);
          } else {
            out[gi] = fma_t<T>(-alpha_j, v, w1);
            a.psi[gi] = fma_t<T>(y_j, v, a.psi[gi]);
          }
        }
      }
    }
  }
  if (MODE == HV_LANCZOS) {
    double smv = block_sum<T>(dotd + (double)dot, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = smv;
  }
}

// The same product, one thread per element of the padded block-major vector
// (small sectors).  Every element takes the same operations in the same
// order as in k_hv: the diagonal, the H_up entries in ELL order, the H_dw
// entries in CSR order, then the same epilogue; the Lanczos mode leaves one
// partial of <v_j, w1> per CTA.
template <typename T, int MODE, bool CHUNKED>
__global__ void __launch_bounds__(HVS_THREADS) k_hv_small(HvLaunch<T> a) {
  __shared__ double red[HVS_THREADS / 32];
  const HvTables<T> &tb = a.tb;
  int j = 0;
  T s_cur = T(1), s_prev = T(0), beta_j = T(0), alpha_j = T(0), y_j = T(0);
  const T *g;
  const T *prev = nullptr;
  T *out;
  if (MODE == HV_PLAIN) {
    g = a.v;
    out = a.w;
  } else {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    j = st->j;
    const int m3 = j % 3;  // buffers selected without a local array
    g = m3 == 0 ? a.b0 : (m3 == 1 ? a.b1 : a.b2);
    out = m3 == 0 ? a.b1 : (m3 == 1 ? a.b2 : a.b0);
    prev = m3 == 0 ? a.b2 : (m3 == 1 ? a.b0 : a.b1);
    if (MODE == HV_LANCZOS && a.basis) {
      g = a.basis[j];
      prev = a.basis[j > 0 ? j - 1 : 0];
      out = a.basis[j + 1];
    }
    s_cur = (T)st->scale[j % 3];
    s_prev = (T)st->scale[(j + 2) % 3];
    beta_j = (T)st->beta[j];
    if (MODE == HV_SECOND) {
      alpha_j = (T)st->alpha[j];
      y_j = (T)st->y[j];
    }
  }
  const int64_t stride = tb.stride;
  T dot = T(0);
  double dot_sum = 0.0;  // the per-thread sum, flushed from T every 16 elements
  const int64_t n = tb.ddw * stride;
  // one element per thread unless CHUNKED (separate instances: the chunk loop
  // costs registers, and the small sectors run at full occupancy without it)
  const int K = CHUNKED ? tb.small_chunk : 1;
  for (int k = 0; k < K; ++k) {
    const int64_t gi = ((int64_t)blockIdx.x * K + k) * HVS_THREADS + threadIdx.x;
    if (gi >= n) break;
    if (CHUNKED && MODE == HV_LANCZOS && (k & 15) == 15) {
      dot_sum += (double)dot;
      dot = T(0);
    }
    const int64_t r = gi / stride;
    const int pc = (int)(gi - r * stride);
    const int4 ci = __ldg(tb.small_cols + pc);
    if (ci.x >= 0) {
      const T x = g[gi];
      const T *row = g + r * stride + ci.z;
      const int deg = ci.w & 255, ncp = ci.w >> 8;
      const int mu = (int)tb.m_up[ci.x] * tb.nmask;
      T acc = mul_t<T>(add_t<T>(add_t<T>(tb.e_up[ci.x], tb.e_dw[r]), tb.W[mu + tb.m_dw[r]]), x);
      for (int e = 0; e < deg; ++e) {
        const int o = ci.y + e * ncp;
        acc = fma_t<T>(__ldg(tb.ell_val + o), row[__ldg(tb.ell_col + o)], acc);
      }
      const int32_t d0 = __ldg(tb.rp_dw + r), d1 = __ldg(tb.rp_dw + r + 1);
      for (int32_t k = d0; k < d1; ++k)
        acc = fma_t<T>(__ldg(tb.val_dw + k), g[(int64_t)__ldg(tb.col_dw + k) * stride + pc], acc);
      if (MODE == HV_PLAIN) {
        out[gi] = acc;
      } else {
        const T v = mul_t<T>(x, s_cur);
        T w1 = mul_t<T>(acc, s_cur);
        if (MODE == HV_SECOND && j > 0)  // the Lanczos step does this in its update
          w1 = fma_t<T>(-beta_j, mul_t<T>(prev[gi], s_prev), w1);
        if (MODE == HV_LANCZOS) {
          out[gi] = w1;
          dot = fma_t<T>(v, w1, dot);
        } else {
          out[gi] = fma_t<T>(-alpha_j, v, w1);
          a.psi[gi] = fma_t<T>(y_j, v, a.psi[gi]);
        }
      }
    }
  }
  if (MODE == HV_LANCZOS) {
    double smv = block_sum<T>(dot_sum + (double)dot, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = smv;
  }
}

int64_t ed_hv_num_parts(ed_sector s, int layout, int elem_size) {
  if (ed_build_items(s, layout, elem_size) != ED_OK) return 0;
  // the H_nd kernel's partials follow the product's
  const int64_t nd = s->nd[layout].up ? ed_nd_grid(s->sp[1].dim, s->nd[layout].ncols) : 0;
  if (layout == 1 && s->hv_kernel[elem_size == 8 ? 1 : 0] == 1) return small_grid_of(s->bdim) + nd;
  const ItemList &il = s->items[layout][elem_size == 8 ? 1 : 0];
  return (il.d_ditems ? il.nditems : il.nitems) + nd;
}

// Opt the product kernels into large dynamic shared memory, once per device
// (outside any stream capture).
template <typename T, bool WIDE>
static ed_status prepare_passa() {
  constexpr int RT = rt_passa<T, WIDE>(), NT = passa_threads<WIDE>();
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_PLAIN, true, true, RT, NT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_LANCZOS, true, true, RT, NT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_SECOND, true, true, RT, NT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  return ED_OK;
}

template <typename T, bool BLK>
static ed_status prepare_layout() {
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_PLAIN, BLK>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_LANCZOS, BLK>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_SECOND, BLK>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  if (BLK) {
    ED_TRY((prepare_passa<T, true>()));
    ED_TRY((prepare_passa<T, false>()));
  }
  return ED_OK;
}

template <typename T>
ed_status ed_hv_prepare() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return ED_OK;
  ED_TRY((prepare_layout<T, false>()));
  ED_TRY((prepare_layout<T, true>()));
  if (dev < 64) done[dev] = true;
  return ED_OK;
}
template ed_status ed_hv_prepare<float>();
template ed_status ed_hv_prepare<double>();

template <typename T, int MODE>
static ed_status launch_mode(const HvLaunch<T> &a, cudaStream_t st) {
  if (a.tb.small_cols) {
    if (a.tb.small_chunk > 1)
      k_hv_small<T, MODE, true><<<(unsigned)a.tb.small_grid, HVS_THREADS, 0, st>>>(a);
    else
      k_hv_small<T, MODE, false><<<(unsigned)a.tb.small_grid, HVS_THREADS, 0, st>>>(a);
  } else if (a.tb.ditems) {
    if (a.tb.passa_wide)
      k_hv<T, MODE, true, true, rt_passa<T, true>(), passa_threads<true>()>
          <<<(unsigned)a.tb.nitems, passa_threads<true>(), a.tb.smem, st>>>(a);
    else
      k_hv<T, MODE, true, true, rt_passa<T, false>(), passa_threads<false>()>
          <<<(unsigned)a.tb.nitems, passa_threads<false>(), a.tb.smem, st>>>(a);
    ED_LAUNCHED(1);
    k_hv_dw<T, MODE><<<(unsigned)a.tb.nditems, DW_THREADS, 0, st>>>(a);
  } else if (a.tb.ell_col) {
    k_hv<T, MODE, true><<<(unsigned)a.tb.nitems, HV_THREADS, a.tb.smem, st>>>(a);
  } else {
    k_hv<T, MODE, false><<<(unsigned)a.tb.nitems, HV_THREADS, a.tb.smem, st>>>(a);
  }
  ED_LAUNCHED(1);
  return ED_OK;
}

template <typename T>
ed_status ed_launch_hv(ed_sector s, const HvTables<T> &tb, int mode, const T *v, T *w,
                       T *const *bufs, T *psi, LanczosState *state, double *part,
                       int64_t *nparts, cudaStream_t st, T *const *basis) {
  ED_TRY(ed_hv_prepare<T>());
  HvLaunch<T> a;
  a.tb = tb;
  if (nparts) *nparts = tb.small_cols ? tb.small_grid : (tb.ditems ? tb.nditems : tb.nitems);
  if (tb.nitems == 0 || tb.dup == 0) return ED_OK;
  if (!tb.items) return ED_ERR_ARG;
  a.v = v;
  a.w = w;
  a.b0 = bufs ? bufs[0] : nullptr;
  a.b1 = bufs ? bufs[1] : nullptr;
  a.b2 = bufs ? bufs[2] : nullptr;
  a.basis = basis;
  a.psi = psi;
  a.st = state;
  a.part = part;
  if (mode == HV_PLAIN) ED_TRY((launch_mode<T, HV_PLAIN>(a, st)));
  else if (mode == HV_LANCZOS) ED_TRY((launch_mode<T, HV_LANCZOS>(a, st)));
  else ED_TRY((launch_mode<T, HV_SECOND>(a, st)));
  if (!tb.nd_up) return ED_OK;
  // spin exchange and pair hopping, added to the product (partials after the product's)
  const int64_t np = tb.small_cols ? tb.small_grid : (tb.ditems ? tb.nditems : tb.nitems);
  if (nparts) *nparts = np + ed_nd_grid(tb.ddw, tb.nd_ncols);
  return ed_launch_nd<T>(tb, mode, v, w, bufs, basis, state, part ? part + np : nullptr, st);
}

template ed_status ed_launch_hv<float>(ed_sector, const HvTables<float> &, int, const float *,
                                       float *, float *const *, float *, LanczosState *, double *,
                                       int64_t *, cudaStream_t, float *const *);
template ed_status ed_launch_hv<double>(ed_sector, const HvTables<double> &, int, const double *,
                                        double *, double *const *, double *, LanczosState *,
                                        double *, int64_t *, cudaStream_t, double *const *);

static ed_status matvec_layout(ed_sector s, ed_precision prec, const void *d_v, void *d_w,
                               int64_t n, void *stream, int layout) {
  if (!s || !d_v || !d_w || d_v == d_w) return ED_ERR_ARG;
  if (n != (layout == 0 ? s->dim : s->bdim)) {
    ed_set_error_msg("vector length does not match the sector layout");
    return ED_ERR_ARG;
  }
  // block-major rows are read and written as 16-byte vectors; sector-order
  // elements need their natural alignment
  const uintptr_t amask = layout == 1 ? 15 : (prec == ED_FP64 ? 7 : 3);
  if (((uintptr_t)d_v | (uintptr_t)d_w) & amask) {
    ed_set_error_msg(layout == 1 ? "block-major vectors must be 16-byte aligned"
                                 : "vectors must be aligned to their element size");
    return ED_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == ED_FP64) {
    ED_TRY(ed_build_items(s, layout, 8));
    return ed_launch_hv<double>(s, ed_hv_tables<double>(s, layout), HV_PLAIN,
                                (const double *)d_v, (double *)d_w, nullptr, nullptr, nullptr,
                                nullptr, nullptr, st);
  }
  if (prec == ED_FP32 || prec == ED_FP32_POLISH) {
    ED_TRY(ed_build_items(s, layout, 4));
    return ed_launch_hv<float>(s, ed_hv_tables<float>(s, layout), HV_PLAIN, (const float *)d_v,
                               (float *)d_w, nullptr, nullptr, nullptr, nullptr, nullptr, st);
  }
  return ED_ERR_ARG;
}

extern "C" ed_status ed_matvec(ed_sector s, ed_precision prec, const void *d_v, void *d_w,
                               int64_t n, void *stream) {
  return matvec_layout(s, prec, d_v, d_w, n, stream, 0);
}

extern "C" ed_status ed_matvec_blocked(ed_sector s, ed_precision prec, const void *d_v, void *d_w,
                                       int64_t n, void *stream) {
  return matvec_layout(s, prec, d_v, d_w, n, stream, 1);
}

static ed_status kernel_of(ed_sector s, ed_precision prec, int *e, int32_t *kernel) {
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  const int elem = prec == ED_FP64 ? 8 : 4;
  *e = elem == 8 ? 1 : 0;
  ED_TRY(ed_build_items(s, 1, elem));
  *kernel = s->hv_kernel[*e] == 1
                ? ED_KERNEL_ELEMENTWISE
                : (s->items[1][*e].d_ditems ? ED_KERNEL_TWO_PASS : ED_KERNEL_TILED);
  return ED_OK;
}

extern "C" ed_status ed_sector_blocked_kernel(ed_sector s, ed_precision prec, int32_t *kernel) {
  if (!s || !kernel) return ED_ERR_ARG;
  int e = 0;
  return kernel_of(s, prec, &e, kernel);
}

extern "C" ed_status ed_sector_tune_info(ed_sector s, ed_precision prec, int32_t *kernel,
                                         double *host_ms) {
  if (!s || !kernel || !host_ms) return ED_ERR_ARG;
  int e = 0;
  ED_TRY(kernel_of(s, prec, &e, kernel));
  host_ms[0] = s->tune_ms[e][0];
  host_ms[1] = s->tune_ms[e][1];
  return ED_OK;
}

extern "C" ed_status ed_sector_set_kernel(ed_sector s, ed_precision prec, int32_t kernel) {
  if (!s) return ED_ERR_ARG;
  int e = 0;
  int32_t cur = 0;
  ED_TRY(kernel_of(s, prec, &e, &cur));
  if (kernel == ED_KERNEL_ELEMENTWISE) {
    if (!s->small_cols) {
      ed_set_error_msg("this sector's blocks do not fit the element-parallel column table");
      return ED_ERR_UNSUPPORTED;
    }
    s->hv_kernel[e] = 1;
  } else if (kernel == ED_KERNEL_TILED || kernel == ED_KERNEL_TWO_PASS) {
    // the tiled family: one or two passes as the sector's size decides
    if ((kernel == ED_KERNEL_TWO_PASS) != (s->items[1][e].d_ditems != nullptr)) {
      ed_set_error_msg("one or two passes is fixed by the sector's block sizes");
      return ED_ERR_UNSUPPORTED;
    }
    s->hv_kernel[e] = 0;
  } else {
    return ED_ERR_ARG;
  }
  return ED_OK;
}
