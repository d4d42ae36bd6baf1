// Device and pinned-host memory of the library, and the per-thread private
// stream.
//
// Every device buffer (sector tables, work lists, Lanczos and chain
// workspaces, psi) comes from one stream-ordered pool per device, owned by
// the library.  Allocation and release are ordered on a stream and never
// synchronise the device, so concurrent solves on other streams (the serving
// loop, the concurrent Green's function chains) do not wait for one another
// when one of them sets up or tears down a sector.  Freed blocks stay mapped
// in the pool for the next allocation: the first use of fresh device memory
// through a pool costs about 5.6 ms per GB on GB300 (about 0.04 ms once
// mapped), and a solve allocates its Krylov vectors one by one while the
// device waits on the host (56 GB per Ns=16 ground state, about 0.12 s of its
// 0.33 s).  ed_memory_trim returns the cached blocks to the device, as a
// caching allocator's release call does; the budgets that look at free memory
// (the kept Krylov basis, the server's admission) count the pool's cached
// blocks as available.
//
// The 4-byte host words that the Lanczos drivers poll for the device stop
// flag are page-locked (so that the copy of the flag is a true async copy);
// they are recycled through a free list instead of being allocated and freed
// per call, because releasing page-locked memory synchronises the device.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {nullptr};

std::mutex g_flag_mu;
std::vector<int32_t *> g_free_flags;
constexpr int kFlagStride = 16;   // one 64-byte line per flag
constexpr int kFlagsPerChunk = 64;

ed_status device_pool(cudaMemPool_t *out) {
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    ed_set_error_msg("device ordinal out of range");
    return ED_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    ED_TRY_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = ~0ull;  // freed blocks stay cached (see the file comment)
    cudaError_t e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    // a block freed on another stream is reused only once its free has
    // completed, never by making the new stream wait on the old one:
    // concurrent requests (the server's slots, the concurrent chains) would
    // otherwise wait on each other through the memory they exchange
    int no = 0;
    if (e == cudaSuccess)
      e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      ed_set_cuda_error(e, "cudaMemPoolSetAttribute", __FILE__, __LINE__);
      return ED_ERR_CUDA;
    }
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return ED_OK;
}

// Private streams of a host thread, one per device; destroyed when the
// thread exits.
struct ThreadStreams {
  cudaStream_t s[kMaxDevices] = {nullptr};
  ~ThreadStreams() {
    for (int d = 0; d < kMaxDevices; ++d)
      if (s[d]) {
        cudaSetDevice(d);
        cudaStreamDestroy(s[d]);
      }
  }
};

}  // namespace

ed_status ed_dmalloc(void **p, size_t bytes, cudaStream_t st, const char *what) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  ED_TRY(device_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, st);
  if (e == cudaErrorMemoryAllocation) {
    // the device is full of this pool's cached blocks that this stream
    // cannot use (split into other sizes, or freed on streams it does not
    // follow): return the free ones to the device and try once more
    cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, st);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    ed_set_cuda_error(e, what ? what : "cudaMallocFromPoolAsync", __FILE__, __LINE__);
    return e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;
  }
  return ED_OK;
}

void ed_dfree(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

ed_status ed_device_available(size_t *bytes) {
  *bytes = 0;
  size_t fr = 0, tot = 0;
  ED_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
  cudaMemPool_t pool = nullptr;
  ED_TRY(device_pool(&pool));
  uint64_t reserved = 0, used = 0;
  ED_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  ED_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = fr + (size_t)(reserved > used ? reserved - used : 0);
  return ED_OK;
}

extern "C" ed_status ed_memory_trim(int64_t keep_bytes) {
  if (keep_bytes < 0) return ED_ERR_ARG;
  cudaMemPool_t pool = nullptr;
  ED_TRY(device_pool(&pool));
  ED_TRY_CUDA(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
  return ED_OK;
}

extern "C" ed_status ed_memory_cached(int64_t *reserved, int64_t *used) {
  if (!reserved || !used) return ED_ERR_ARG;
  cudaMemPool_t pool = nullptr;
  ED_TRY(device_pool(&pool));
  uint64_t r = 0, u = 0;
  ED_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
  ED_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
  *reserved = (int64_t)r;
  *used = (int64_t)u;
  return ED_OK;
}

cudaStream_t ed_private_stream(ed_status *st) {
  static thread_local ThreadStreams ts;
  int dev = 0;
  *st = ED_OK;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = ED_ERR_CUDA;
    return nullptr;
  }
  if (!ts.s[dev]) {
    cudaError_t e = cudaStreamCreateWithFlags(&ts.s[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
      ts.s[dev] = nullptr;
      *st = ED_ERR_CUDA;
      return nullptr;
    }
  }
  return ts.s[dev];
}

int32_t *ed_pinned_flag_acquire() {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (g_free_flags.empty()) {
    int32_t *chunk = nullptr;
    // chunks stay allocated for the life of the process
    if (cudaMallocHost((void **)&chunk, sizeof(int32_t) * kFlagStride * kFlagsPerChunk) !=
        cudaSuccess)
      return nullptr;
    for (int i = kFlagsPerChunk - 1; i >= 0; --i) g_free_flags.push_back(chunk + i * kFlagStride);
  }
  int32_t *f = g_free_flags.back();
  g_free_flags.pop_back();
  *f = 0;
  return f;
}

void ed_pinned_flag_release(int32_t *f) {
  if (!f) return;
  std::lock_guard<std::mutex> lk(g_flag_mu);
  g_free_flags.push_back(f);
}
