// graph.cu -- graph residency (Sec. 6, "Storage Format"), workspace, knobs,
// launch helpers and the small host-only entry points of the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "simdx_internal.h"

namespace simdx {

// Kernel handles of the algorithm translation units (for occupancy sizing).
const void* bfs_kernel_ptr(int off_bits);
const void* sssp_kernel_ptr(int off_bits);
const void* kcore_kernel_ptr(int off_bits);
const void* pagerank_kernel_ptr(int off_bits);

static thread_local char g_last_cuda[256] = "";

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaMemPool_t pool_of(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pl = nullptr;
    if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) return nullptr;
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pl;
  }
  return g_pool[dev];
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pl = pool_of(dev);
  if (!pl) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), pl, st);
}

void dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

static std::mutex g_stage_mu;
static std::vector<HostStage*> g_stage_free;

HostStage* host_stage_get() {
  std::lock_guard<std::mutex> lk(g_stage_mu);
  if (g_stage_free.empty()) {
    constexpr int kChunk = 64;
    void* blk = nullptr;
    if (cudaHostAlloc(&blk, sizeof(HostStage) * kChunk, cudaHostAllocDefault) != cudaSuccess) return nullptr;
    for (int i = 0; i < kChunk; ++i) g_stage_free.push_back(static_cast<HostStage*>(blk) + i);
  }
  HostStage* h = g_stage_free.back();
  g_stage_free.pop_back();
  std::memset(h, 0, sizeof(HostStage));
  return h;
}

void host_stage_put(HostStage* h) {
  if (!h) return;
  std::lock_guard<std::mutex> lk(g_stage_mu);
  g_stage_free.push_back(h);
}

int cuda_status(cudaError_t e, const char* what) {
  snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return SIMDX_ENOMEM;
  return SIMDX_ECUDA;
}

// small_frontier = 2 turns the cluster levels on for graphs whose largest
// out-degree is at most this.
constexpr long long kSmallAutoMaxDeg = 64;

Knobs make_knobs(const simdx_graph* g) {
  const simdx_config& c = g->cfg;
  Knobs k{};
  k.small_max = c.small_max;
  k.med_max = c.med_max;
  k.huge_min = c.huge_min;
  k.bin_cap = g->bin_cap;
  k.direction = c.direction;
  k.filter = c.filter;
  k.alpha = c.alpha;
  k.beta = c.beta;
  k.kalpha = c.kcore_alpha;
  k.delta = c.delta;
  k.timeout_ns = (unsigned long long)(c.barrier_timeout_ms > 0 ? c.barrier_timeout_ms : 2000) * 1000000ull;
  k.skip_cta = c.debug_skip_cta;
  k.skip_phase = c.debug_skip_phase;
  k.fusion = c.fusion;
  k.stage = c.stage_edges;
  // small frontiers on one cluster: on, or (2) on for graphs without hubs,
  // whose BFS levels are many and small (meshes, grids, road networks); a
  // graph with hubs has few levels, and the launch in clusters costs its
  // large levels a few CTAs
  k.small = c.small_frontier == 1 || (c.small_frontier == 2 && g->max_deg <= kSmallAutoMaxDeg);
  return k;
}

Work make_work(const simdx_graph* g) {
  Work w{};
  w.bins = g->bins;
  w.list_cap = g->list_cap;
  for (int b = 0; b < 2; ++b) {
    for (int c = 0; c < kClasses; ++c)
      w.list[b][c] = g->lists + ((size_t)b * kClasses + c) * (size_t)g->list_cap;
    w.aux3[b] = g->aux3 + (size_t)b * (size_t)g->list_cap;
  }
  w.chunk_cnt = g->chunk_cnt;
  w.chunk_part = g->chunk_part;
  w.chunk_done = g->chunk_done;
  w.warp_start = g->warp_start;
  long long words = (g->n + 31) / 32 + 1;
  w.bm_nz = g->bitmaps;
  w.bm_vis = g->bitmaps + words;
  w.bm_f[0] = g->bitmaps + 2 * words;
  w.bm_f[1] = g->bitmaps + 3 * words;
  w.state = g->state;
  w.sync = g->sync;
  w.stats = g->dstats;
  w.trace = g->trace;
  w.trace_cap = g->trace_cap;
  return w;
}

static std::mutex g_occ_mu;
static std::unordered_map<const void*, int> g_occ;

static int occupancy(const void* kernel) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto it = g_occ.find(kernel);
  if (it != g_occ.end()) return it->second;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kThreads, 0) != cudaSuccess) blocks = 0;
  g_occ[kernel] = blocks;
  return blocks;
}

int grid_for(const simdx_graph* g, const void* kernel) {
  int per_sm = occupancy(kernel);
  if (g->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, g->cfg.ctas_per_sm);
  int grid = per_sm * g->num_sms;
  return std::min(grid, g->grid_max);
}

int prepare_launch(simdx_graph* g, cudaStream_t st) {
  SIMDX_CUDA(cudaMemsetAsync(g->sync, 0, sizeof(Sync), st));
  SIMDX_CUDA(cudaMemsetAsync(g->chunk_done, 0, sizeof(int) * (size_t)(g->n + 16), st));
  SIMDX_CUDA(cudaMemsetAsync(g->dstats, 0, sizeof(DevStats), st));
  return SIMDX_OK;
}

int prepare_next_launch(simdx_graph* g, cudaStream_t st) {
  char* sy = reinterpret_cast<char*>(g->sync);
  SIMDX_CUDA(cudaMemsetAsync(sy + offsetof(Sync, arrive), 0, sizeof(unsigned long long), st));
  SIMDX_CUDA(cudaMemsetAsync(sy + offsetof(Sync, slot), 0, sizeof(PhaseSlot) * 3 + sizeof(Resume), st));
  SIMDX_CUDA(cudaMemsetAsync(g->chunk_done, 0, sizeof(int) * (size_t)(g->n + 16), st));
  return SIMDX_OK;
}

int prepare_resume(simdx_graph* g, cudaStream_t st) {
  char* sy = reinterpret_cast<char*>(g->sync);
  SIMDX_CUDA(cudaMemsetAsync(sy + offsetof(Sync, arrive), 0, sizeof(unsigned long long), st));
  SIMDX_CUDA(cudaMemsetAsync(sy + offsetof(Sync, slot), 0, sizeof(PhaseSlot) * 3, st));
  return SIMDX_OK;
}

int read_resume(simdx_graph* g, cudaStream_t st, int* done, int* want_dir) {
  SIMDX_CUDA(cudaMemcpyAsync(&g->h_stats->rs_done, &g->sync->rs.done, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                             st));
  SIMDX_CUDA(cudaMemcpyAsync(&g->h_stats->err, &g->sync->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SIMDX_CUDA(cudaStreamSynchronize(st));
  *done = g->h_stats->rs_done || g->h_stats->err;
  *want_dir = g->h_stats->rs_want;
  return SIMDX_OK;
}

// A cooperative launch through the extensible launch API, which stream
// capture records as a cooperative kernel node.
int launch_coop(const void* kernel, int grid, void** args, cudaStream_t st, int cluster) {
  if (grid <= 0 || (cluster > 1 && grid % cluster)) return SIMDX_EUNSUPPORTED;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cluster > 1) {
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = (unsigned)cluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.numAttrs = 2;
  }
  SIMDX_CUDA(cudaLaunchKernelExC(&cfg, kernel, args));
  return SIMDX_OK;
}

// Co-resident grid in clusters of `cluster` CTAs: the occupancy grid, at
// most the clusters that fit at once, a multiple of the cluster size (0 if
// none fits).
int grid_for_cluster(const simdx_graph* g, const void* kernel, int cluster) {
  // per device: the non-portable cluster size is allowed on each device the
  // kernel runs on
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> max_clusters;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const auto key = std::make_pair(dev, kernel);
  int mc = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = max_clusters.find(key);
    if (it != max_clusters.end()) {
      mc = it->second;
    } else {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(cluster * 64);
      cfg.blockDim = dim3(kThreads);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)cluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cluster > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        mc = 0;
      else if (cudaOccupancyMaxActiveClusters(&mc, kernel, &cfg) != cudaSuccess)
        mc = 0;
      max_clusters[key] = mc;
    }
  }
  int grid = std::min(grid_for(g, kernel), mc * cluster);
  return grid - grid % cluster;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

struct PendingStats {
  simdx_graph* g;
  simdx_stats* user;
  int launches;
};

static void CUDART_CB stats_cb(void* p) {
  PendingStats* ps = static_cast<PendingStats*>(p);
  const DevStats& d = ps->g->h_stats->ds;
  simdx_stats* u = ps->user;
  std::memset(u, 0, sizeof(*u));
  u->status = ps->g->h_stats->status();
  u->iterations = d.iterations;
  u->push_iters = d.push_iters;
  u->pull_iters = d.pull_iters;
  u->ballot_iters = d.ballot_iters;
  u->online_iters = d.online_iters;
  u->phases = d.phases;
  u->grid_ctas = d.grid;
  u->edges_visited = d.edges_visited;
  u->frontier_sum = d.frontier_sum;
  u->last_l1 = d.last_l1;
  u->launches = ps->launches;
  delete ps;
}

int finish_launch(simdx_graph* g, simdx_stats* user, cudaStream_t st, int launches) {
  SIMDX_CUDA(cudaMemcpyAsync(&g->h_stats->ds, g->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  SIMDX_CUDA(cudaMemcpyAsync(&g->h_stats->err, &g->sync->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (user) {
    // the host callback owns a one-shot record: a captured graph would replay it
    if (capturing(st)) return SIMDX_EUNSUPPORTED;
    PendingStats* ps = new (std::nothrow) PendingStats{g, user, launches};
    if (!ps) return SIMDX_ENOMEM;
    cudaError_t e = cudaLaunchHostFunc(st, stats_cb, ps);
    if (e != cudaSuccess) {
      delete ps;
      return cuda_status(e, "cudaLaunchHostFunc");
    }
  }
  return SIMDX_OK;
}

// ------------------------------------------------------------ validation
// Checks a CSR on the device: offsets[0] = 0, non-decreasing, offsets[n] = e,
// indices in [0, n).  Also builds the "has an in-edge" bitmap.
template <class OffT>
__global__ void validate_kernel(long long n, long long e, const OffT* off, const int32_t* idx,
                                int* bad) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) atomicOr(bad, 1);
  if (tid == 0 && (off[0] != 0 || (long long)off[n] != e)) atomicOr(bad, 2);
  for (long long p = tid; p < e; p += stride) {
    int32_t u = idx[p];
    if (u < 0 || (long long)u >= n) atomicOr(bad, 4);
  }
}

// Largest edge weight (for the default SSSP bucket width).
__global__ void weight_max_kernel(long long e, const uint32_t* w, unsigned* out) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  unsigned m = 0;
  for (long long p = tid; p < e; p += stride) m = max(m, w[p]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// A vertex of largest degree, smallest id among them: (degree << 32 |
// ~id) maximised.
template <class OffT>
__global__ void hub_kernel(long long n, const OffT* off, unsigned long long* out) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long m = 0;
  for (long long v = tid; v < n; v += stride) {
    const unsigned long long key = ((unsigned long long)(off[v + 1] - off[v]) << 32) | (0xffffffffull - (unsigned long long)v);
    m = key > m ? key : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

template <class OffT>
__global__ void nonzero_bitmap_kernel(long long n, const OffT* off, uint32_t* bm) {
  long long words = (n + 31) / 32;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long wd = tid; wd < words; wd += stride) {
    uint32_t m = 0;
    for (int b = 0; b < 32; ++b) {
      long long v = wd * 32 + b;
      if (v < n && off[v + 1] > off[v]) m |= 1u << b;
    }
    bm[wd] = m;
  }
}

}  // namespace simdx

using namespace simdx;

extern "C" {

const char* simdx_strerror(int s) {
  switch (s) {
    case SIMDX_OK: return "ok";
    case SIMDX_EINVAL: return "invalid argument";
    case SIMDX_ENOMEM: return "out of memory";
    case SIMDX_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case SIMDX_EBARRIER_TIMEOUT: return "grid barrier wait timed out";
    case SIMDX_EUNSUPPORTED: return "unsupported";
    case SIMDX_EBUSY: return "busy";
    case SIMDX_ENOTREADY: return "not ready";
    default: return "unknown status";
  }
}

int simdx_version(void) { return 10000; }

void simdx_config_default(simdx_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->small_max = 32;
  c->med_max = 512;
  c->huge_min = 4096;
  c->bin_per_thread = 64;
  c->direction = 0;
  c->filter = 0;
  c->alpha = 14.f;
  c->beta = 24.f;
  c->kcore_alpha = 8.f;
  c->delta = 32;
  c->ctas_per_sm = 0;
  c->barrier_timeout_ms = 2000;
  c->debug_skip_cta = -1;
  c->debug_skip_phase = -1;
  c->pr_alpha = 8.f;
  c->pr_theta = 2.f;
  c->pr_rho = 0.6f;
  c->small_frontier = 2;
}

int64_t simdx_eq1_ctas(int64_t regs_per_sm, int64_t regs_per_thread, int64_t threads_per_cta,
                       int64_t n_sm) {
  if (regs_per_sm <= 0 || regs_per_thread <= 0 || threads_per_cta <= 0 || n_sm <= 0) return -1;
  return (regs_per_sm / (regs_per_thread * threads_per_cta)) * n_sm;
}

static void free_workspace(simdx_graph* g, cudaStream_t st) {
  dev_free(g->bins, st);
  dev_free(g->lists, st);
  dev_free(g->aux3, st);
  dev_free(g->chunk_part, st);
  dev_free(g->chunk_done, st);
  dev_free(g->warp_start, st);
  g->warp_start = nullptr;
  g->bins = nullptr;
  g->lists = nullptr;
  g->aux3 = nullptr;
  g->chunk_part = nullptr;
  g->chunk_done = nullptr;
}

static int alloc_workspace(simdx_graph* g, cudaStream_t st) {
  free_workspace(g, st);
  int per_sm = 0;
  const void* ks[4] = {bfs_kernel_ptr(g->off_bits), sssp_kernel_ptr(g->off_bits),
                       kcore_kernel_ptr(g->off_bits), pagerank_kernel_ptr(g->off_bits)};
  for (const void* k : ks) per_sm = std::max(per_sm, occupancy(k));
  if (per_sm <= 0) return SIMDX_ECUDA;
  if (g->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, g->cfg.ctas_per_sm);
  g->grid_max = per_sm * g->num_sms;
  int bpt = std::max(0, g->cfg.bin_per_thread);
  g->bin_cap = bpt * kThreads;
  long long online_total = (long long)g->grid_max * g->bin_cap;
  g->list_cap = std::max<long long>(g->n, online_total) + 64;
  size_t bins_bytes = sizeof(int32_t) * (size_t)kClasses * g->grid_max * std::max(1, g->bin_cap);
  size_t list_bytes = sizeof(int32_t) * (size_t)2 * kClasses * g->list_cap;
  SIMDX_CUDA(dev_alloc((void**)&g->bins, bins_bytes, st));
  SIMDX_CUDA(dev_alloc((void**)&g->lists, list_bytes, st));
  SIMDX_CUDA(dev_alloc((void**)&g->aux3, sizeof(uint32_t) * 2 * (size_t)g->list_cap, st));
  // chunked class-3 tasks: at most e / huge_min + (tasks) chunks per phase
  const long long hm = std::max(1, g->cfg.huge_min);
  const size_t parts = (size_t)(g->e / hm + g->n + 16);
  SIMDX_CUDA(dev_alloc((void**)&g->chunk_part, sizeof(unsigned long long) * parts, st));
  SIMDX_CUDA(dev_alloc((void**)&g->chunk_done, sizeof(int) * (size_t)(g->n + 16), st));
  SIMDX_CUDA(cudaMemsetAsync(g->chunk_done, 0, sizeof(int) * (size_t)(g->n + 16), st));
  SIMDX_CUDA(dev_alloc((void**)&g->warp_start, sizeof(int) * ((size_t)g->grid_max * kWarps + 1), st));
  return SIMDX_OK;
}

int simdx_graph_create(const simdx_csr* csr, const simdx_csr* csc, const uint32_t* weights,
                       uint32_t flags, void* stream, simdx_graph** out) {
  if (!out) return SIMDX_EINVAL;
  *out = nullptr;
  if (!csr || csr->n < 0 || csr->n >= (1ll << 31) - 1 || csr->e < 0 ||
      (csr->offset_bits != 32 && csr->offset_bits != 64) || !csr->offsets ||
      (csr->e > 0 && !csr->indices))
    return SIMDX_EINVAL;
  if ((flags & SIMDX_INPUT_HOST) && (flags & SIMDX_BORROW)) return SIMDX_EINVAL;
  if (csr->offset_bits == 32 && csr->e >= (1ll << 31)) return SIMDX_EINVAL;
  if (csc && (csc->n != csr->n || csc->e != csr->e || csc->offset_bits != csr->offset_bits ||
              !csc->offsets || (csc->e > 0 && !csc->indices)))
    return SIMDX_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  simdx_graph* g = new (std::nothrow) simdx_graph();
  if (!g) return SIMDX_ENOMEM;
  simdx_config_default(&g->cfg);
  g->gen = next_graph_gen();
  g->n = csr->n;
  g->e = csr->e;
  g->off_bits = csr->offset_bits;
  g->symmetric = (csc == nullptr);
  g->borrowed = (flags & SIMDX_BORROW) != 0;
  const bool host = (flags & SIMDX_INPUT_HOST) != 0;
  size_t osz = (size_t)(g->off_bits / 8) * (size_t)(g->n + 1);
  size_t isz = sizeof(int32_t) * (size_t)std::max<int64_t>(g->e, 1);
  int rc = SIMDX_OK;
  auto fail = [&](int r) {
    simdx_graph_destroy(g);
    return r;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&g->device)) != cudaSuccess) return fail(cuda_status(e, "cudaGetDevice"));
  if ((e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess)
    return fail(cuda_status(e, "cudaDeviceGetAttribute"));
  auto place = [&](const void* src, size_t bytes, void** dst) -> int {
    if (g->borrowed) {
      *dst = const_cast<void*>(src);
      return SIMDX_OK;
    }
    cudaError_t ee = dev_alloc(dst, bytes, st);
    if (ee != cudaSuccess) return cuda_status(ee, "dev_alloc(graph)");
    if (src && bytes) {
      ee = cudaMemcpyAsync(*dst, src, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
      if (ee != cudaSuccess) return cuda_status(ee, "cudaMemcpyAsync(graph)");
    }
    return SIMDX_OK;
  };
  if ((rc = place(csr->offsets, osz, &g->off)) != SIMDX_OK) return fail(rc);
  if ((rc = place(csr->indices, g->e ? isz : 0, (void**)&g->idx)) != SIMDX_OK) return fail(rc);
  if (csc) {
    if ((rc = place(csc->offsets, osz, &g->in_off)) != SIMDX_OK) return fail(rc);
    if ((rc = place(csc->indices, g->e ? isz : 0, (void**)&g->in_idx)) != SIMDX_OK) return fail(rc);
  } else {
    g->in_off = g->off;
    g->in_idx = g->idx;
  }
  if (weights) {
    if ((rc = place(weights, sizeof(uint32_t) * (size_t)std::max<int64_t>(g->e, 1), (void**)&g->w)) != SIMDX_OK)
      return fail(rc);
  }
  // validate on the device (also catches bad host input after the copy)
  int* d_bad = nullptr;  // [0] validation flags, [1] largest weight, [2..3] hub key
  if ((e = dev_alloc((void**)&d_bad, 4 * sizeof(int), st)) != cudaSuccess) return fail(cuda_status(e, "dev_alloc"));
  cudaMemsetAsync(d_bad, 0, 4 * sizeof(int), st);
  int vblocks = std::max(1, std::min(4 * g->num_sms, (int)((g->e + g->n) / 256 + 1)));
  const simdx_csr* parts[2] = {csr, csc};
  for (int pi = 0; pi < 2; ++pi) {
    if (!parts[pi]) continue;
    void* o = pi == 0 ? g->off : g->in_off;
    int32_t* ix = pi == 0 ? g->idx : g->in_idx;
    if (g->off_bits == 32)
      validate_kernel<int32_t><<<vblocks, 256, 0, st>>>(g->n, g->e, (const int32_t*)o, ix, d_bad);
    else
      validate_kernel<long long><<<vblocks, 256, 0, st>>>(g->n, g->e, (const long long*)o, ix, d_bad);
  }
  if (g->w && g->e > 0)
    weight_max_kernel<<<vblocks, 256, 0, st>>>(g->e, g->w, reinterpret_cast<unsigned*>(d_bad + 1));
  if (g->off_bits == 32)
    hub_kernel<int32_t><<<vblocks, 256, 0, st>>>(g->n, (const int32_t*)g->off,
                                                 reinterpret_cast<unsigned long long*>(d_bad + 2));
  else
    hub_kernel<long long><<<vblocks, 256, 0, st>>>(g->n, (const long long*)g->off,
                                                   reinterpret_cast<unsigned long long*>(d_bad + 2));
  int h_bad[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(h_bad, d_bad, 4 * sizeof(int), cudaMemcpyDeviceToHost, st);
  dev_free(d_bad, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "graph validation"));
  if (h_bad[0]) return fail(SIMDX_EINVAL);
  // default bucket width: 16 x the largest weight (a few buckets cover the
  // distances of a low-diameter graph; a long path gets wide buckets)
  {
    unsigned long long key = 0;
    std::memcpy(&key, h_bad + 2, sizeof(key));
    g->hub = key ? (int32_t)(0xffffffffull - (key & 0xffffffffull)) : 0;
    g->max_deg = (long long)(key >> 32);
  }
  const unsigned wmax = static_cast<unsigned>(h_bad[1]);
  if (wmax) g->cfg.delta = wmax >= (1u << 26) ? (1u << 30) : 16u * wmax;
  // workspace
  long long words = (g->n + 31) / 32 + 1;
  if ((e = dev_alloc((void**)&g->bitmaps, sizeof(uint32_t) * 4 * (size_t)words, st)) != cudaSuccess)
    return fail(cuda_status(e, "dev_alloc(bitmaps)"));
  cudaMemsetAsync(g->bitmaps, 0, sizeof(uint32_t) * 4 * (size_t)words, st);
  if ((e = dev_alloc(&g->state, 20 * (size_t)std::max<int64_t>(g->n, 1) + 64, st)) != cudaSuccess)
    return fail(cuda_status(e, "dev_alloc(state)"));
  if ((e = dev_alloc((void**)&g->sync, sizeof(Sync), st)) != cudaSuccess) return fail(cuda_status(e, "dev_alloc(sync)"));
  {
    long long chunks = (g->n + kBallotChunk - 1) / kBallotChunk + 1;
    if ((e = dev_alloc((void**)&g->chunk_cnt, sizeof(int32_t) * kClasses * (size_t)chunks, st)) != cudaSuccess)
      return fail(cuda_status(e, "dev_alloc(chunk_cnt)"));
  }
  if ((e = dev_alloc((void**)&g->dstats, sizeof(DevStats), st)) != cudaSuccess)
    return fail(cuda_status(e, "dev_alloc(stats)"));
  cudaMemsetAsync(g->dstats, 0, sizeof(DevStats), st);
  g->trace_cap = 1 << 16;
  if ((e = dev_alloc((void**)&g->trace, sizeof(long long) * kTraceWords * (size_t)g->trace_cap, st)) != cudaSuccess)
    return fail(cuda_status(e, "dev_alloc(trace)"));
  if (!(g->h_stats = host_stage_get())) return fail(SIMDX_ENOMEM);
  cudaMemsetAsync(g->sync, 0, sizeof(Sync), st);
  if ((rc = alloc_workspace(g, st)) != SIMDX_OK) return fail(rc);
  int nb = std::max(1, std::min(4 * g->num_sms, (int)(words / 256 + 1)));
  if (g->off_bits == 32)
    nonzero_bitmap_kernel<int32_t><<<nb, 256, 0, st>>>(g->n, (const int32_t*)g->in_off, g->bitmaps);
  else
    nonzero_bitmap_kernel<long long><<<nb, 256, 0, st>>>(g->n, (const long long*)g->in_off, g->bitmaps);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_status(e, "graph create"));
  *out = g;
  return SIMDX_OK;
}

int simdx_graph_destroy(simdx_graph* g) {
  if (!g) return SIMDX_EINVAL;
  cudaDeviceSynchronize();  // no call on this graph is in flight past here
  cudaStream_t st = 0;
  mg_pack_free(g, st);
  if (!g->borrowed) {
    dev_free(g->off, st);
    dev_free(g->idx, st);
    if (!g->symmetric) {
      dev_free(g->in_off, st);
      dev_free(g->in_idx, st);
    }
    dev_free(g->w, st);
  }
  free_workspace(g, st);
  dev_free(g->bitmaps, st);
  dev_free(g->state, st);
  dev_free(g->sync, st);
  dev_free(g->ms_state, st);
  dev_free(g->d_roots, st);
  if (g->h_roots) cudaFreeHost(g->h_roots);
  dev_free(g->sb_state, st);
  dev_free(g->mss_state, st);
  dev_free(g->pr_ws, st);
  dev_free(g->chunk_cnt, st);
  dev_free(g->dstats, st);
  dev_free(g->trace, st);
  host_stage_put(g->h_stats);
  delete g;
  return SIMDX_OK;
}

int simdx_graph_info(const simdx_graph* g, int64_t* n, int64_t* e, int32_t* grid_ctas,
                     int32_t* threads_per_cta) {
  if (!g) return SIMDX_EINVAL;
  if (n) *n = g->n;
  if (e) *e = g->e;
  if (grid_ctas) *grid_ctas = g->grid_max;
  if (threads_per_cta) *threads_per_cta = kThreads;
  return SIMDX_OK;
}

int simdx_graph_get_config(const simdx_graph* g, simdx_config* cfg) {
  if (!g || !cfg) return SIMDX_EINVAL;
  *cfg = g->cfg;
  return SIMDX_OK;
}

int simdx_graph_set_config(simdx_graph* g, const simdx_config* cfg) {
  if (!g || !cfg) return SIMDX_EINVAL;
  if (cfg->small_max < 1 || cfg->med_max < cfg->small_max || cfg->huge_min < cfg->med_max ||
      cfg->bin_per_thread < 0 || cfg->bin_per_thread > 4096 || cfg->direction < 0 ||
      cfg->direction > 2 || (cfg->filter != 0 && cfg->filter != 2) || !(cfg->alpha > 0.f) ||
      !(cfg->beta > 0.f) || !(cfg->kcore_alpha > 0.f) || cfg->ctas_per_sm < 0 || cfg->batch_group < 0 ||
      cfg->fusion < 0 || cfg->fusion > 2 || !(cfg->pr_alpha >= 0.f) || !(cfg->pr_theta >= 0.f) ||
      !(cfg->pr_rho >= 0.f) || cfg->sssp_combine < 0 || cfg->sssp_combine > 1 ||
      (cfg->sssp_batch_width != 0 && cfg->sssp_batch_width != 8 && cfg->sssp_batch_width != 16 &&
       cfg->sssp_batch_width != 32 && cfg->sssp_batch_width != 64) || cfg->pr_row_cost < 0 ||
      cfg->pr_row_cost > 4096 || cfg->stage_edges < 0 || cfg->stage_edges > 1 || cfg->pr_recut < 0 ||
      cfg->small_frontier < 0 || cfg->small_frontier > 2)
    return SIMDX_EINVAL;
  bool realloc_ws = cfg->bin_per_thread != g->cfg.bin_per_thread || cfg->ctas_per_sm != g->cfg.ctas_per_sm ||
                    cfg->huge_min != g->cfg.huge_min;
  cudaDeviceSynchronize();
  g->cfg = *cfg;
  if (realloc_ws) {
    int rc = alloc_workspace(g, 0);
    cudaError_t e = cudaStreamSynchronize(0);
    if (rc == SIMDX_OK && e != cudaSuccess) rc = cuda_status(e, "set_config");
    return rc;
  }
  return SIMDX_OK;
}

int simdx_graph_last_status(simdx_graph* g, void* stream) {
  if (!g) return SIMDX_EINVAL;
  SIMDX_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return g->h_stats->status();
}

int simdx_graph_trace(simdx_graph* g, void* stream, int64_t* rec, int64_t cap, int64_t* count) {
  if (!g || (cap > 0 && !rec)) return SIMDX_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SIMDX_CUDA(cudaStreamSynchronize(st));
  int64_t it = g->h_stats->ds.iterations;
  if (count) *count = it;
  int64_t m = std::min<int64_t>(std::min<int64_t>(it, cap), g->trace_cap);
  if (m > 0)
    SIMDX_CUDA(cudaMemcpy(rec, g->trace, sizeof(long long) * kTraceWords * (size_t)m, cudaMemcpyDeviceToHost));
  return SIMDX_OK;
}

const char* simdx_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
