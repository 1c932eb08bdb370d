// msssp.cu -- batched SSSP: up to 64 sources in one persistent launch, the
// sources of a group sharing each edge read (growth direction (a); Sec. 2.1
// / Sec. 3.3 per source, aggregation combine = min).
//
// The sources run in groups of G (8, 16, 32 or 64; the sssp_batch_width
// knob, 32 by default), one group after another inside the launch.  A
// group's distances are kept vertex-major, dvm[v * G + i] for its source i,
// so the relaxations of one edge for all the group's sources touch one
// contiguous row of G words (G = 8: one 32-byte sector).  Measured at R-MAT
// scale 22 with 64 sources: G = 8 / 16 / 32 / 64 run 75 / 61 / 55 / 57 ms
// (narrow groups keep the state in L2 but repeat every iteration's fixed
// cost once per group; wide rows stream from DRAM).  A vertex is active
// for the sources in the mask chg[v] (their distance at v changed since v
// last relaxed them); one task per active vertex, whatever the number of
// sources.  Tasks are walked by the degree-class driver of the single query
// (lanes over edges, 32 small tasks per warp, chunked hubs); a lane reads
// an edge's index and weight once and relaxes it for every claimed source
// of its task from 32-byte pieces of the two rows, with an atomicMin for
// each source that improves (Combine = min).  The improving sources of an
// edge are added to chg[u] with one atomicOr; the add that makes chg[u] non-zero
// records u in the next task lists (online filter, degree-class bins;
// ballot filter over chg != 0 on overflow), so lists hold no duplicates.
// Each iteration claims the masks of its tasks first (chg -> cm, a phase of
// its own), then relaxes; a group ends when no distance changed and writes
// its source-major rows of the result through a shared-memory transpose.
#include "simdx_internal.h"

namespace simdx {

constexpr int kMsMaxInst = 64;     // sources per launch
constexpr int kMsDefaultWidth = 32;  // sources per group (row width of the state)

template <class OffT>
struct MsspArgs {
  int n, k, K;                 // vertices, sources, row stride of dvm (the group width)
  int32_t srcs[kMsMaxInst];    // the batch's sources (kernel parameter)
  const OffT* off;
  const int32_t* idx;
  const uint32_t* wt;
  uint32_t* dvm;               // [n][K] distances, vertex-major
  unsigned long long* chg;     // [n] sources whose distance at v changed since v relaxed them
  unsigned long long* cm;      // [n] sources a task relaxes in the current iteration
  uint32_t* out;               // [k][n] the caller's distances, source-major
  Work w;
  Knobs kn;
};

// Push functor for the degree-class driver (push_classes): a lane relaxes
// one edge (v -> u, weight w) for every source in v's claimed mask, eight
// sources at a time from 32-byte pieces of the two rows (two 16-byte loads
// each; the pieces of one row share a sector, so the rest hit L1).
template <class OffT, int G>
struct MsPush {
  struct Src {
    unsigned long long m;  // sources claimed by the task
  };
  const MsspArgs<OffT>& a;
  CtaShared& sh;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;

  __device__ MsPush(const MsspArgs<OffT>& aa, CtaShared& s, unsigned g) : a(aa), sh(s), grid(g) {}
  __device__ __forceinline__ bool src(int v, Src& s, int, unsigned) {
    s.m = a.cm[v];
    return s.m != 0ull;
  }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src& s, int l) {
    Src r;
    r.m = __shfl_sync(kFull, s.m, l);
    return r;
  }
  // The improved sources `bits` of target u: add them to chg[u]; the add
  // that makes it non-zero records u for the next iteration.
  __device__ __forceinline__ void mark(int u, unsigned long long bits) {
    if (atomicOr(a.chg + u, bits) == 0ull) {
      const long long d = (long long)gload(a.off + u + 1) - (long long)gload(a.off + u);
      ++nrec;
      mrec += (unsigned long long)d;
      online_record(u, degree_class(d, a.kn), sh, a.w, a.kn, grid);
    }
  }
  __device__ __forceinline__ void edges(const Src (&s)[kPushBatch], const int (&v)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&p)[kPushBatch],
                                        unsigned ok) {
    uint32_t w[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) w[q] = ((ok >> q) & 1u) ? gload(a.wt + p[q]) : 0u;
#pragma unroll 1
    for (int q = 0; q < kPushBatch; ++q) {
      if (!((ok >> q) & 1u)) continue;
      unsigned long long imp = 0;
#pragma unroll 1
      for (int c = 0; c < G / 8; ++c) {
        const unsigned m8 = (unsigned)(s[q].m >> (8 * c)) & 0xffu;
        if (!m8) continue;
        const uint4* dv = reinterpret_cast<const uint4*>(a.dvm + (size_t)v[q] * G + 8 * c);
        uint4* duv = reinterpret_cast<uint4*>(a.dvm + (size_t)u[q] * G + 8 * c);
        const uint4 s0 = dv[0], s1 = dv[1], t0 = duv[0], t1 = duv[1];
        const uint32_t dsv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        const uint32_t dtv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
        uint32_t* du = a.dvm + (size_t)u[q] * G + 8 * c;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (!((m8 >> i) & 1u)) continue;
          const unsigned long long nd = (unsigned long long)dsv[i] + w[q];
          if (nd < dtv[i] && nd < atomicMin(du + i, (uint32_t)nd)) imp |= 1ull << (8 * c + i);
        }
      }
      if (imp) mark(u[q], imp);
    }
  }
};

// One launch answers up to 64 sources, G at a time: each group of G sources
// runs its own iterations on the [n][G] state, writes its rows of the result
// and leaves the state to the next group.
template <class OffT, int G>
__global__ void __launch_bounds__(kThreads, 4) msssp_kernel(const __grid_constant__ MsspArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ uint32_t tile[32][G + 1];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.kn;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();
  int it = 0, ballot_it = 0;
  long long evisit = 0, fsum = 0;

  for (int g0 = 0; g0 < a.k; g0 += G) {
    const int gk = a.k - g0 < G ? a.k - g0 : G;
    // ---- every distance of the group infinite, no source active
    for (long long x = gtid; x < (long long)n * G; x += gthreads) a.dvm[x] = 0xffffffffu;
    for (long long v = gtid; v < n; v += gthreads) a.chg[v] = 0ull;
    clear_next_slot(s, sh);
    if (!grid_sync(s, grid, sh, k)) return;
    // ---- the group's sources (a vertex may be the source of several)
    clear_next_slot(s, sh);
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < gk; i += kThreads) {
        const int v = a.srcs[g0 + i];
        a.dvm[(size_t)v * G + i] = 0u;
        if (atomicOr(a.chg + v, 1ull << i) == 0ull) {
          const long long d = (long long)gload(a.off + v + 1) - (long long)gload(a.off + v);
          const int c = degree_class(d, k);
          const unsigned pos = atomicAdd(&s->slot[slot_of(sh.phase)].list_cnt[c], 1u);
          a.w.list[0][c][pos] = v;
        }
      }
    if (!grid_sync(s, grid, sh, k)) return;

    unsigned cnt[kClasses];
    {
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    }
    int lbuf = 0;
    bool lists_ok = true;
    while (true) {
      const unsigned long long t_it = globaltimer();
      int filt = 1;
      if (!lists_ok || k.filter == 2) {
        // ballot filter: every vertex with a changed source
        clear_next_slot(s, sh);
        PhaseSlot& slot = s->slot[slot_of(sh.phase)];
        const unsigned long long* chg = a.chg;
        auto pred = [chg](int v) { return chg[v] != 0ull; };
        auto deg = [off = a.off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
        auto none = [](int) {};
        ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
        if (!grid_sync(s, grid, sh, k)) return;
        const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
        for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
        filt = 2;
        ++ballot_it;
      }
      const unsigned total = cnt[0] + cnt[1] + cnt[2] + cnt[3];
      if (total == 0) break;
      // ---- claim: the sources each task relaxes in this iteration
      clear_next_slot(s, sh);
      for (int c = 0; c < kClasses; ++c) {
        const int32_t* list = a.w.list[lbuf][c];
        for (long long i = gtid; i < cnt[c]; i += gthreads) {
          const int v = list[i];
          a.cm[v] = atomicExch(a.chg + v, 0ull);
        }
      }
      if (!grid_sync(s, grid, sh, k)) return;
      // ---- relax, the sources of a task on the lanes of a warp
      clear_next_slot(s, sh);
      online_reset(sh);
      __syncthreads();
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      MsPush<OffT, G> f(a, sh, grid);
      {
        const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                          a.w.list[lbuf][3]};
        push_classes<OffT>(f, a.off, a.idx, lists, cnt, grid, k.huge_min, sh, evisit);
      }
      online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
      const unsigned long long tn = cta_sum_u64(f.nrec, sh);
      const unsigned long long tmm = cta_sum_u64(f.mrec, sh);
      if (threadIdx.x == 0 && tn) {
        atomicAdd(&slot.nact, tn);
        atomicAdd(&slot.mact, tmm);
      }
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      trace_put(a.w, it, 1 | (filt << 8), (long long)total, (long long)p.mact, g0, t_it);
      trace_classes(a.w, it, p);
      fsum += total;
      ++it;
      for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
      lists_ok = p.overflow == 0;
      if (p.nact == 0) break;  // no distance changed
      lbuf ^= 1;
    }
    // ---- the group's source-major rows, through a shared-memory transpose
    for (long long t = blockIdx.x; t * 32 < n; t += grid) {
      const long long v0 = t * 32;
      for (int j = threadIdx.x; j < 32 * G; j += kThreads) {
        const int vv = j / G, ii = j - vv * G;
        tile[vv][ii] = v0 + vv < n ? a.dvm[(size_t)(v0 + vv) * G + ii] : 0u;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < 32 * gk; j += kThreads) {
        const int ii = j >> 5, vv = j & 31;
        if (v0 + vv < n) a.out[(size_t)(g0 + ii) * n + v0 + vv] = tile[vv][ii];
      }
      __syncthreads();
    }
    // the next group rewrites the state: every CTA must be done reading it
    if (!grid_sync(s, grid, sh, k)) return;
  }
  const unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the launches of a batch of more than 64 sources add up
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations += it;
    st.push_iters += it;
    st.ballot_iters += ballot_it;
    st.online_iters += it - ballot_it;
    st.phases += (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum += fsum;
    st.last_l1 = 0.0;
  }
}

// Vertex-major state of one group: the distances (G words per vertex) and
// two 64-bit masks per vertex.  Allocated on the first call (or a wider
// group), kept with the graph.
static int ensure_ms_state(simdx_graph* g, int G, cudaStream_t st) {
  const size_t n = (size_t)std::max<int64_t>(g->n, 1);
  const size_t bytes = ((sizeof(uint32_t) * (size_t)G * n + 255) & ~(size_t)255) + 2 * sizeof(unsigned long long) * n;
  if (g->mss_state && g->mss_bytes >= bytes) return SIMDX_OK;
  if (capturing(st)) return SIMDX_EUNSUPPORTED;
  dev_free(g->mss_state, st);
  g->mss_state = nullptr;
  g->mss_bytes = 0;
  SIMDX_CUDA(dev_alloc(&g->mss_state, bytes, st));
  g->mss_bytes = bytes;
  return SIMDX_OK;
}

template <class OffT, int G>
static int run_msssp(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                     cudaStream_t st) {
  int rc = ensure_ms_state(g, G, st);
  if (rc) return rc;
  const size_t n = (size_t)std::max<int64_t>(g->n, 1);
  char* base = static_cast<char*>(g->mss_state);
  MsspArgs<OffT> a{};
  a.n = (int)g->n;
  a.K = G;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.wt = g->w;
  a.dvm = reinterpret_cast<uint32_t*>(base);
  a.chg = reinterpret_cast<unsigned long long*>(base + ((sizeof(uint32_t) * G * n + 255) & ~(size_t)255));
  a.cm = a.chg + n;
  a.w = make_work(g);
  a.kn = make_knobs(g);
  const void* kern = (const void*)msssp_kernel<OffT, G>;
  const int grid = grid_for(g, kern);
  if ((rc = prepare_launch(g, st)) != SIMDX_OK) return rc;
  int launches = 0;
  for (int g0 = 0; g0 < k; g0 += kMsMaxInst, ++launches) {
    const int gk = std::min(kMsMaxInst, k - g0);
    if (g0 > 0 && (rc = prepare_next_launch(g, st)) != SIMDX_OK) return rc;
    a.k = gk;
    for (int i = 0; i < gk; ++i) a.srcs[i] = srcs[g0 + i];
    a.out = dist + (size_t)g0 * n;
    void* args[] = {&a};
    if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  }
  return finish_launch(g, stats, st, launches);
}

template <class OffT>
static int run_msssp_width(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                           cudaStream_t st) {
  int G = g->cfg.sssp_batch_width;
  if (G == 0) G = kMsDefaultWidth;
  // no wider rows than the batch needs
  while (G > 8 && G / 2 >= k) G /= 2;
  switch (G) {
    case 8: return run_msssp<OffT, 8>(g, srcs, k, dist, stats, st);
    case 16: return run_msssp<OffT, 16>(g, srcs, k, dist, stats, st);
    case 32: return run_msssp<OffT, 32>(g, srcs, k, dist, stats, st);
    default: return run_msssp<OffT, 64>(g, srcs, k, dist, stats, st);
  }
}

int sssp_batch_shared(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                      cudaStream_t st) {
  return g->off_bits == 32 ? run_msssp_width<int32_t>(g, srcs, k, dist, stats, st)
                           : run_msssp_width<long long>(g, srcs, k, dist, stats, st);
}

}  // namespace simdx
