// msbfs.cu -- batched BFS: up to 64 sources in one persistent ACC kernel.
//
// Growth direction (a) of the hot path: many BFS queries on one graph in one
// launch with per-source frontiers.  Each vertex carries two 64-bit masks:
// visit (bit i = reached by source i) and the frontier of the current level
// (bit i = reached by source i at this level).  In ACC terms (Sec. 3.2) the
// per-vertex state is the mask, Compute offers a neighbour's frontier mask,
// and Combine is bitwise OR -- commutative, associative, and a vote: every
// source that reaches a vertex at a level offers the same level.
//   level 0 -> 1 : push from the sources (atomicOr of the source bit into the
//                  neighbours' next masks; the first offer records the vertex)
//                  and an apply pass over the recorded vertices;
//   level L -> L+1 (L >= 1): pull over every vertex that some source has not
//                  reached yet: OR the in-neighbours' frontier masks (the
//                  owner computes, no atomics), new = OR & ~visit.
// levels[i * ld + v] = level of v from srcs[i] (-1 unreached).
#include "simdx_internal.h"

namespace simdx {

template <class OffT>
struct MsArgs {
  int n, k;
  int32_t srcs[64];     // the sources (a kernel parameter: no copy to stage, so a launch can be captured)
  const OffT* off;
  const int32_t* idx;
  const OffT* ioff;
  const int32_t* iidx;
  int32_t* levels;
  long long ld;
  unsigned long long* visit;
  unsigned long long* fr0;
  unsigned long long* fr1;
  Work w;
  Knobs kn;
};

template <class OffT>
struct MsPush {
  struct Src {
    unsigned long long m;
  };
  const unsigned long long* frc;
  unsigned long long* frn;
  const unsigned long long* visit;
  const OffT* off;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ MsPush(const unsigned long long* c, unsigned long long* nx, const unsigned long long* vi, const OffT* o,
                    CtaShared& s, const Work& ww, const Knobs& kk, unsigned g)
      : frc(c), frn(nx), visit(vi), off(o), sh(s), w(ww), k(kk), grid(g) {}
  __device__ __forceinline__ bool src(int v, Src& s, int, unsigned) {
    s.m = frc[v];
    return s.m != 0ull;
  }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src& s, int l) {
    Src r;
    r.m = __shfl_sync(kFull, s.m, l);
    return r;
  }
  __device__ __forceinline__ void edges(const Src (&s)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&)[kPushBatch], unsigned ok) {
    unsigned long long bits[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) bits[q] = ((ok >> q) & 1u) ? (s[q].m & ~visit[u[q]]) : 0ull;
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      if (bits[q] && atomicOr(&frn[u[q]], bits[q]) == 0ull) {
        long long d = (long long)gload(off + u[q] + 1) - (long long)gload(off + u[q]);
        ++nrec;
        mrec += (unsigned long long)d;
        online_record(u[q], degree_class(d, k), sh, w, k, grid);
      }
    }
  }
};

template <class OffT>
struct MsPull {
  using Acc = unsigned long long;
  const unsigned long long* frc;
  unsigned long long* frn;
  unsigned long long* visit;
  int32_t* levels;
  long long ld;
  int next;
  unsigned long long nrec = 0;
  __device__ __forceinline__ Acc zero() const { return 0ull; }
  __device__ __forceinline__ void combine(Acc& a, Acc b) const { a |= b; }
  __device__ __forceinline__ void edge(Acc& a, int, int v, long long) { a |= frc[v]; }
  __device__ __forceinline__ void finish(int u, Acc m) {
    const unsigned long long vis = visit[u];
    unsigned long long nb = m & ~vis;
    frn[u] = nb;  // owner: every candidate's next mask is written
    if (nb) {
      visit[u] = vis | nb;
      ++nrec;
      while (nb) {
        const int i = __ffsll((long long)nb) - 1;
        nb &= nb - 1;
        levels[(long long)i * ld + u] = next;
      }
    }
  }
};

template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) msbfs_kernel(const __grid_constant__ MsArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ unsigned long long red_m[kWarps];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.kn;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  const unsigned long long all = a.k >= 64 ? ~0ull : ((1ull << a.k) - 1ull);
  unsigned long long* fr[2] = {a.fr0, a.fr1};
  const OffT* off = a.off;
  const OffT* ioff = a.ioff;
  auto odeg = [off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
  auto ideg = [ioff](int v) { return (long long)gload(ioff + v + 1) - (long long)gload(ioff + v); };
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // ---- phase 0: reset masks and levels
  clear_next_slot(s, sh);
  for (long long v = gtid; v < n; v += gthreads) {
    a.visit[v] = 0ull;
    fr[0][v] = 0ull;
    fr[1][v] = 0ull;
  }
  for (long long x = gtid; x < (long long)a.k * n; x += gthreads) {
    const long long i = x / n, v = x - i * n;
    a.levels[i * a.ld + v] = -1;
  }
  if (!grid_sync(s, grid, sh, k)) return;
  // ---- phase 1: seed the sources (level 0) and their task list
  clear_next_slot(s, sh);
  if (blockIdx.x == 0) {
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    for (int i = threadIdx.x; i < a.k; i += kThreads) {
      const int v = a.srcs[i];
      atomicOr(&a.visit[v], 1ull << i);
      a.levels[(long long)i * a.ld + v] = 0;
      if (atomicOr(&fr[0][v], 1ull << i) == 0ull) {
        const int c = degree_class(odeg(v), k);
        const unsigned pos = atomicAdd(&slot.list_cnt[c], 1u);
        a.w.list[0][c][pos] = v;
        if (c == 3) a.w.aux3[0][pos] = 0xffffffffu;
      }
    }
  }
  if (!grid_sync(s, grid, sh, k)) return;
  unsigned cnt[kClasses];
  {
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
  }
  long long evisit = 0;
  int it = 0;
  bool more = true;
  // ---- level 0 -> 1: push from the sources
  {
    const unsigned long long t_it = globaltimer();
    clear_next_slot(s, sh);
    online_reset(sh);
    __syncthreads();
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    MsPush<OffT> f(fr[0], fr[1], a.visit, off, sh, a.w, k, grid);
    const int32_t* lists[kClasses] = {a.w.list[0][0], a.w.list[0][1], a.w.list[0][2], a.w.list[0][3]};
    push_classes<OffT>(f, off, a.idx, lists, cnt, grid, k.huge_min, sh, evisit);
    online_flush(sh, a.w, k, grid, 1, slot);
    unsigned long long tn = cta_sum_u64(f.nrec, sh);
    if (threadIdx.x == 0 && tn) atomicAdd(&slot.nact, tn);
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    const bool ovf = p.overflow != 0;
    const unsigned long long n1 = p.nact;
    unsigned c1[kClasses];
    for (int c = 0; c < kClasses; ++c) c1[c] = p.list_cnt[c];
    // apply level 1: visit |= offered bits, write the levels
    clear_next_slot(s, sh);
    if (!ovf) {
      for (int c = 0; c < kClasses; ++c)
        for (unsigned i = (unsigned)gtid; i < c1[c]; i += (unsigned)gthreads) {
          const int u = a.w.list[1][c][i];
          unsigned long long nb = fr[1][u];
          a.visit[u] |= nb;
          while (nb) {
            const int b = __ffsll((long long)nb) - 1;
            nb &= nb - 1;
            a.levels[(long long)b * a.ld + u] = 1;
          }
        }
    } else {
      for (long long u = gtid; u < n; u += gthreads) {
        unsigned long long nb = fr[1][u];
        if (!nb) continue;
        a.visit[u] |= nb;
        while (nb) {
          const int b = __ffsll((long long)nb) - 1;
          nb &= nb - 1;
          a.levels[(long long)b * a.ld + u] = 1;
        }
      }
    }
    trace_put(a.w, it, 1 | (1 << 8), a.k, (long long)n1, 0, t_it);
    ++it;
    if (!grid_sync(s, grid, sh, k)) return;
    more = n1 != 0;
  }
  // ---- levels L -> L+1 by pull over the vertices not reached by every source
  for (int L = 1; more; ++L) {
    const unsigned long long t_it = globaltimer();
    const int cur = L & 1, nxt = cur ^ 1;
    unsigned long long* frc = fr[cur];
    unsigned long long* frn = fr[nxt];
    // candidates (ballot filter); every other vertex gets an empty next mask
    clear_next_slot(s, sh);
    {
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      unsigned long long* visit = a.visit;
      auto pred = [=](int u) {
        if (visit[u] == all || ideg(u) == 0) {
          frn[u] = 0ull;
          return false;
        }
        return true;
      };
      auto none = [](int) {};
      ballot_filter(n, pred, ideg, none, sh, a.w, k, grid, 0, slot);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    {
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    }
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    MsPull<OffT> f;
    f.frc = frc;
    f.frn = frn;
    f.visit = a.visit;
    f.levels = a.levels;
    f.ld = a.ld;
    f.next = L + 1;
    const int32_t* lists[kClasses] = {a.w.list[0][0], a.w.list[0][1], a.w.list[0][2], a.w.list[0][3]};
    pull_classes<OffT>(f, ioff, a.iidx, lists, cnt, grid, red_m, k.huge_min, sh, a.w, evisit);
    unsigned long long tn = cta_sum_u64(f.nrec, sh);
    if (threadIdx.x == 0 && tn) atomicAdd(&slot.nact, tn);
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    const unsigned long long nn = p.nact;
    trace_put(a.w, it, 2 | (2 << 8), (long long)(cnt[0] + cnt[1] + cnt[2] + cnt[3]), (long long)nn, L, t_it);
    trace_classes(a.w, it, p);
    ++it;
    if (nn == 0) break;
  }
  {
    unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
    if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  }
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = it;
    st.push_iters = 1;
    st.pull_iters = it - 1;
    st.ballot_iters = it - 1;
    st.online_iters = 1;
    st.phases = (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = 0;
    st.last_l1 = 0.0;
  }
}

const void* msbfs_kernel_ptr(int off_bits) {
  return off_bits == 32 ? (const void*)msbfs_kernel<int32_t> : (const void*)msbfs_kernel<long long>;
}

// Batch state: visit + two frontier masks per vertex, and the device copy of
// the sources.  Allocated on the first batched call, kept with the graph.
int ensure_msbfs_state(simdx_graph* g, cudaStream_t st) {
  if (g->ms_state) return SIMDX_OK;
  SIMDX_CUDA(dev_alloc((void**)&g->ms_state, sizeof(unsigned long long) * 3 * (size_t)(g->n + 1) + 64 * sizeof(int32_t),
                       st));
  return SIMDX_OK;
}

template <class OffT>
static int run_msbfs(simdx_graph* g, const int32_t* srcs, int k, int32_t* levels, long long ld, simdx_stats* stats,
                     cudaStream_t st) {
  MsArgs<OffT> a{};
  a.n = (int)g->n;
  a.k = k;
  for (int i = 0; i < k; ++i) a.srcs[i] = srcs[i];
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.ioff = (const OffT*)g->in_off;
  a.iidx = g->in_idx;
  a.levels = levels;
  a.ld = ld;
  a.visit = g->ms_state;
  a.fr0 = g->ms_state + (g->n + 1);
  a.fr1 = g->ms_state + 2 * (g->n + 1);
  a.w = make_work(g);
  a.kn = make_knobs(g);
  const void* kern = (const void*)msbfs_kernel<OffT>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st);
}

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_bfs_batch(simdx_graph* g, const int32_t* srcs, int32_t k, int32_t* levels, simdx_stats* stats,
                               void* stream) {
  if (!g || !srcs || !levels || k <= 0 || g->n <= 0) return SIMDX_EINVAL;
  for (int i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_msbfs_state(g, st);
  if (rc) return rc;
  for (int b = 0; b < k; b += 64) {
    const int kb = k - b < 64 ? k - b : 64;
    int32_t* lv = levels + (size_t)b * (size_t)g->n;
    rc = g->off_bits == 32 ? run_msbfs<int32_t>(g, srcs + b, kb, lv, g->n, b + kb >= k ? stats : nullptr, st)
                           : run_msbfs<long long>(g, srcs + b, kb, lv, g->n, b + kb >= k ? stats : nullptr, st);
    if (rc) return rc;
  }
  return SIMDX_OK;
}
