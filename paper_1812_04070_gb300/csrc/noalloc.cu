// noalloc.cu -- BFS for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// runtime's memory pool or a tightly budgeted process (the allocator belongs
// to someone else), code that must not allocate while a CUDA graph is being
// captured elsewhere on the device, and plugins whose host application forbids
// allocations after start-up.  simdx_bfs_noalloc serves them: the caller
// passes a device CSR and the output array, and every byte of scratch the BFS
// kernel needs (task lists, online-filter bins, bitmaps, barrier words,
// statistics) lives in one file-scope __device__ array of fixed size.  Every
// GPU that loads the library holds that array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and that address is what
// the kernels receive.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "simdx_internal.h"

namespace simdx {

const void* bfs_kernel_ptr(int off_bits);
int bfs_launch_raw(int off_bits, int n, long long e, const void* off, const int32_t* idx, int src,
                   int32_t* levels, const Work& w, const Knobs& k, int grid, cudaStream_t st);

namespace noalloc {

constexpr long long kMaxN = 1ll << 18;       // vertices
constexpr int kMaxGrid = 1024;               // CTAs of the persistent launch
constexpr int kBinCap = kThreads;            // online-filter bin: 1 entry per thread per class
constexpr int kTraceCap = 1024;
constexpr long long kWords = kMaxN / 32 + 1;
constexpr long long kListCap = (kMaxN > (long long)kMaxGrid * kBinCap ? kMaxN : (long long)kMaxGrid * kBinCap) + 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffSync = 0;
constexpr size_t kOffStats = align256(kOffSync + sizeof(Sync));
constexpr size_t kOffBad = align256(kOffStats + sizeof(DevStats));
constexpr size_t kOffTrace = align256(kOffBad + sizeof(int));
constexpr size_t kOffBitmaps = align256(kOffTrace + sizeof(long long) * kTraceWords * kTraceCap);
constexpr size_t kOffBins = align256(kOffBitmaps + sizeof(uint32_t) * 4 * kWords);
constexpr size_t kOffLists = align256(kOffBins + sizeof(int32_t) * kClasses * (size_t)kMaxGrid * kBinCap);
constexpr size_t kOffAux3 = align256(kOffLists + sizeof(int32_t) * 2 * kClasses * (size_t)kListCap);
constexpr size_t kBytes = align256(kOffAux3 + sizeof(uint32_t) * 2 * (size_t)kListCap);  // ~14.7 MB

}  // namespace noalloc

// The scratch itself (one copy per device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[noalloc::kBytes];

namespace {

std::mutex g_mu;
unsigned char* g_addr[256] = {};  // device address of the scratch, per device

// Look up (once per device, with that device current) the device address of
// the scratch array.
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return SIMDX_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return SIMDX_OK;
}

template <class OffT>
__global__ void noalloc_prepare_kernel(long long n, long long e, const OffT* off, const int32_t* idx,
                                       uint32_t* bm_nz, int* bad) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long wd = tid; wd < (n + 31) / 32; wd += stride) {
    uint32_t m = 0;
    for (int b = 0; b < 32; ++b) {
      long long v = wd * 32 + b;
      if (v < n) {
        if (off[v + 1] < off[v]) atomicOr(bad, 1);
        if (off[v + 1] > off[v]) m |= 1u << b;
      }
    }
    bm_nz[wd] = m;
  }
  if (tid == 0 && (off[0] != 0 || (long long)off[n] != e)) atomicOr(bad, 2);
  for (long long p = tid; p < e; p += stride) {
    int32_t u = idx[p];
    if (u < 0 || (long long)u >= n) atomicOr(bad, 4);
  }
}

}  // namespace
}  // namespace simdx

using namespace simdx;

extern "C" int simdx_bfs_noalloc(const simdx_csr* csr, int32_t src, int32_t* levels, void* stream) {
  using namespace simdx::noalloc;
  if (!csr || !levels || csr->n <= 0 || csr->n > kMaxN || csr->e < 0 || !csr->offsets ||
      (csr->e > 0 && !csr->indices) || (csr->offset_bits != 32 && csr->offset_bits != 64) || src < 0 ||
      src >= csr->n)
    return SIMDX_EINVAL;
  if (csr->offset_bits == 32 && csr->e >= (1ll << 31)) return SIMDX_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != SIMDX_OK) return rc;
  const int n = (int)csr->n;

  Work w{};
  w.sync = reinterpret_cast<Sync*>(base + kOffSync);
  w.stats = reinterpret_cast<DevStats*>(base + kOffStats);
  int* bad = reinterpret_cast<int*>(base + kOffBad);
  w.trace = reinterpret_cast<long long*>(base + kOffTrace);
  w.trace_cap = kTraceCap;
  uint32_t* bm = reinterpret_cast<uint32_t*>(base + kOffBitmaps);
  const long long words = ((long long)n + 31) / 32 + 1;
  w.bm_nz = bm;
  w.bm_vis = bm + words;
  w.bm_f[0] = bm + 2 * words;
  w.bm_f[1] = bm + 3 * words;
  w.bins = reinterpret_cast<int32_t*>(base + kOffBins);
  w.list_cap = kListCap;
  int32_t* lists = reinterpret_cast<int32_t*>(base + kOffLists);
  uint32_t* aux3 = reinterpret_cast<uint32_t*>(base + kOffAux3);
  for (int b = 0; b < 2; ++b) {
    for (int c = 0; c < kClasses; ++c) w.list[b][c] = lists + ((size_t)b * kClasses + c) * (size_t)kListCap;
    w.aux3[b] = aux3 + (size_t)b * (size_t)kListCap;
  }
  w.chunk_cnt = nullptr;
  w.state = nullptr;

  simdx_config cfg;
  simdx_config_default(&cfg);
  Knobs k{};
  k.small_max = cfg.small_max;
  k.med_max = cfg.med_max;
  k.huge_min = cfg.huge_min;
  k.bin_cap = kBinCap;
  // push only: a push level reads out-edges alone, so a directed CSR gives
  // the same levels as a symmetric one (no in-edge array is passed here)
  k.direction = 1;
  k.filter = 0;
  k.alpha = cfg.alpha;
  k.beta = cfg.beta;
  k.kalpha = cfg.kcore_alpha;
  k.delta = cfg.delta;
  k.timeout_ns = (unsigned long long)cfg.barrier_timeout_ms * 1000000ull;
  k.skip_cta = -1;
  k.skip_phase = -1;

  // grid: co-resident CTAs (the occupancy form of Eq. 1), capped by the scratch
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, csr->offset_bits == 32 ? bfs_kernel_ptr(32) : bfs_kernel_ptr(64), kThreads, 0);
  if (e != cudaSuccess) return cuda_status(e, "occupancy");
  const int grid = std::min(per_sm * sms, kMaxGrid);
  if (grid <= 0) return SIMDX_EUNSUPPORTED;

  // reset what must start at zero, check the CSR, build the in-edge bitmap
  if ((e = cudaMemsetAsync(base, 0, kOffTrace, st)) != cudaSuccess) return cuda_status(e, "cudaMemsetAsync");
  const int blocks = std::max(1, std::min(4 * sms, (int)((csr->e + csr->n) / 256 + 1)));
  if (csr->offset_bits == 32)
    noalloc_prepare_kernel<int32_t><<<blocks, 256, 0, st>>>(n, csr->e, (const int32_t*)csr->offsets,
                                                             csr->indices, w.bm_nz, bad);
  else
    noalloc_prepare_kernel<long long><<<blocks, 256, 0, st>>>(n, csr->e, (const long long*)csr->offsets,
                                                               csr->indices, w.bm_nz, bad);
  int h_bad = 0;
  if ((e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_status(e, "noalloc check");
  if (h_bad) return SIMDX_EINVAL;
  return bfs_launch_raw(csr->offset_bits, n, csr->e, csr->offsets, csr->indices, src, levels, w, k, grid, st);
}
