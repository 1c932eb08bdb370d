// multigraph.cu -- BFS over many separate graphs in one persistent launch
// (growth direction (a): many graphs of uneven size in one launch).
//
// The graphs stay separate objects; the library packs them on the device
// into one block-diagonal CSR (graph i's vertex ids offset by the vertices
// of the graphs before it), runs the multi-root BFS of bfs.cu on the pack
// with one root per block, and scatters each block's levels back into the
// caller's per-graph arrays.  No edge joins two blocks, so each block's
// levels are exactly that graph's BFS.  The pack (and a graph object over
// it) is cached on the first graph of the list and rebuilt only when the
// list changes (graphs are told apart by a creation number, so a graph
// destroyed and re-created at the same address is not mistaken for the old
// one).
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <vector>

#include "simdx_internal.h"

namespace simdx {

namespace {

struct MgDesc {
  const void* off;
  const int32_t* idx;
  const void* ioff;
  const int32_t* iidx;
  long long n, e, vbase, ebase;
  int bits;
  int pad;
};

}  // namespace

struct MgPack {
  std::vector<const simdx_graph*> graphs;
  std::vector<unsigned long long> gens;
  std::vector<long long> vbase;  // [k + 1]
  bool directed = false;
  simdx_graph* packed = nullptr;  // borrows the arrays below
  void* off = nullptr;
  int32_t* idx = nullptr;
  void* ioff = nullptr;
  int32_t* iidx = nullptr;
  int32_t* lev = nullptr;       // levels of the pack
  MgDesc* d_desc = nullptr;     // [k] graph descriptors (device)
  int32_t** d_out = nullptr;    // [k] the caller's output arrays (device copy of the table)
};

void mg_pack_free(simdx_graph* g, cudaStream_t st) {
  MgPack* p = static_cast<MgPack*>(g->mg_pack);
  if (!p) return;
  if (p->packed) simdx_graph_destroy(p->packed);
  dev_free(p->off, st);
  dev_free(p->idx, st);
  if (p->directed) {
    dev_free(p->ioff, st);
    dev_free(p->iidx, st);
  }
  dev_free(p->lev, st);
  dev_free(p->d_desc, st);
  dev_free(p->d_out, st);
  delete p;
  g->mg_pack = nullptr;
}

namespace {

// Block y copies graph y into the pack: offsets shifted by the edges before
// it, neighbour ids by the vertices before it (out-edges, and in-edges when
// some graph of the list is directed).
template <class POff>
__global__ void mg_pack_kernel(const MgDesc* desc, POff* poff, int32_t* pidx, POff* pioff, int32_t* piidx) {
  const MgDesc d = desc[blockIdx.y];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int side = 0; side < (pioff ? 2 : 1); ++side) {
    const void* so = side ? d.ioff : d.off;
    const int32_t* si = side ? d.iidx : d.idx;
    POff* to = side ? pioff : poff;
    int32_t* ti = side ? piidx : pidx;
    for (long long v = tid; v < d.n; v += stride) {
      const long long o = d.bits == 32 ? (long long)static_cast<const int32_t*>(so)[v]
                                       : static_cast<const long long*>(so)[v];
      to[d.vbase + v] = (POff)(d.ebase + o);
    }
    for (long long q = tid; q < d.e; q += stride) ti[d.ebase + q] = (int32_t)(d.vbase + si[q]);
  }
}

template <class POff>
__global__ void mg_last_offset(POff* poff, POff* pioff, long long n, long long e) {
  poff[n] = (POff)e;
  if (pioff) pioff[n] = (POff)e;
}

// Block y copies block y's levels into the caller's array for graph y.
__global__ void mg_scatter_kernel(const MgDesc* desc, int32_t* const* out, const int32_t* lev) {
  const MgDesc d = desc[blockIdx.y];
  int32_t* o = out[blockIdx.y];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < d.n; v += stride) o[v] = lev[d.vbase + v];
}

std::atomic<unsigned long long> g_gen{1};

bool same_list(const MgPack* p, simdx_graph* const* gs, int k) {
  if (!p || (int)p->graphs.size() != k) return false;
  for (int i = 0; i < k; ++i)
    if (p->graphs[i] != gs[i] || p->gens[i] != gs[i]->gen) return false;
  return true;
}

int build_pack(simdx_graph* owner, simdx_graph* const* gs, int k, cudaStream_t st) {
  mg_pack_free(owner, st);
  MgPack* p = new (std::nothrow) MgPack();
  if (!p) return SIMDX_ENOMEM;
  owner->mg_pack = p;
  p->vbase.assign(k + 1, 0);
  std::vector<MgDesc> desc(k);
  long long n = 0, e = 0;
  for (int i = 0; i < k; ++i) {
    const simdx_graph* g = gs[i];
    p->graphs.push_back(g);
    p->gens.push_back(g->gen);
    p->directed |= !g->symmetric;
    desc[i] = MgDesc{g->off, g->idx, g->in_off, g->in_idx, g->n, g->e, n, e, g->off_bits, 0};
    p->vbase[i] = n;
    n += g->n;
    e += g->e;
  }
  p->vbase[k] = n;
  if (n >= (1ll << 31) - 1) return SIMDX_EINVAL;
  const int bits = e < (1ll << 31) ? 32 : 64;
  const size_t osz = (size_t)(bits / 8) * (size_t)(n + 1), isz = sizeof(int32_t) * (size_t)std::max(e, 1ll);
  SIMDX_CUDA(dev_alloc(&p->off, osz, st));
  SIMDX_CUDA(dev_alloc((void**)&p->idx, isz, st));
  if (p->directed) {
    SIMDX_CUDA(dev_alloc(&p->ioff, osz, st));
    SIMDX_CUDA(dev_alloc((void**)&p->iidx, isz, st));
  }
  SIMDX_CUDA(dev_alloc((void**)&p->lev, sizeof(int32_t) * (size_t)std::max(n, 1ll), st));
  SIMDX_CUDA(dev_alloc((void**)&p->d_desc, sizeof(MgDesc) * (size_t)k, st));
  SIMDX_CUDA(dev_alloc((void**)&p->d_out, sizeof(int32_t*) * (size_t)k, st));
  SIMDX_CUDA(cudaMemcpyAsync(p->d_desc, desc.data(), sizeof(MgDesc) * (size_t)k, cudaMemcpyHostToDevice, st));
  long long maxw = 1;
  for (const MgDesc& d : desc) maxw = std::max(maxw, std::max(d.n, d.e));
  const dim3 grid((unsigned)std::min<long long>(64, (maxw + 255) / 256), (unsigned)k);
  if (bits == 32) {
    mg_pack_kernel<int32_t><<<grid, 256, 0, st>>>(p->d_desc, (int32_t*)p->off, p->idx, (int32_t*)p->ioff, p->iidx);
    mg_last_offset<int32_t><<<1, 1, 0, st>>>((int32_t*)p->off, (int32_t*)p->ioff, n, e);
  } else {
    mg_pack_kernel<long long><<<grid, 256, 0, st>>>(p->d_desc, (long long*)p->off, p->idx, (long long*)p->ioff,
                                                   p->iidx);
    mg_last_offset<long long><<<1, 1, 0, st>>>((long long*)p->off, (long long*)p->ioff, n, e);
  }
  SIMDX_CUDA(cudaGetLastError());
  simdx_csr csr{n, e, bits, p->off, p->idx};
  simdx_csr csc{n, e, bits, p->ioff, p->iidx};
  return simdx_graph_create(&csr, p->directed ? &csc : nullptr, nullptr, SIMDX_BORROW, st, &p->packed);
}

}  // namespace

unsigned long long next_graph_gen() { return g_gen.fetch_add(1); }

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_bfs_multigraph(simdx_graph* const* gs, const int32_t* srcs, int32_t k, int32_t* const* levels,
                                    void* stream) {
  if (!gs || !srcs || !levels || k <= 0 || k > 65535) return SIMDX_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SIMDX_ECUDA;
  for (int i = 0; i < k; ++i)
    if (!gs[i] || !levels[i] || gs[i]->device != dev || srcs[i] < 0 || srcs[i] >= gs[i]->n) return SIMDX_EINVAL;
  simdx_graph* owner = gs[0];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (capturing(st)) return SIMDX_EUNSUPPORTED;  // the output table travels from pageable memory
  int rc = SIMDX_OK;
  {
    std::lock_guard<std::mutex> lk(owner->mu);
    if (!same_list(static_cast<MgPack*>(owner->mg_pack), gs, k) && (rc = build_pack(owner, gs, k, st)) != SIMDX_OK) {
      mg_pack_free(owner, st);
      return rc;
    }
  }
  MgPack* p = static_cast<MgPack*>(owner->mg_pack);
  std::vector<int32_t> roots(k);
  for (int i = 0; i < k; ++i) roots[i] = (int32_t)(p->vbase[i] + srcs[i]);
  if ((rc = simdx_bfs_multi(p->packed, roots.data(), k, p->lev, nullptr, stream)) != SIMDX_OK) return rc;
  // the caller's arrays: a pageable copy, staged before the call returns
  SIMDX_CUDA(cudaMemcpyAsync(p->d_out, levels, sizeof(int32_t*) * (size_t)k, cudaMemcpyHostToDevice, st));
  long long maxn = 1;
  for (int i = 0; i < k; ++i) maxn = std::max(maxn, (long long)gs[i]->n);
  const dim3 grid((unsigned)std::min<long long>(64, (maxn + 255) / 256), (unsigned)k);
  mg_scatter_kernel<<<grid, 256, 0, st>>>(p->d_desc, p->d_out, p->lev);
  SIMDX_CUDA(cudaGetLastError());
  return SIMDX_OK;
}
