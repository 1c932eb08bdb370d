// msssp.cu -- batched SSSP: up to 64 sources in one persistent launch, the
// sources sharing each edge read (growth direction (a); Sec. 2.1 / Sec. 3.3
// per source, aggregation combine = min).
//
// Distances are kept vertex-major, dvm[v * K + i] for source i (K = 32 or
// 64), so the relaxations of one edge for all sources touch one contiguous
// row of K words.  A vertex is active for the sources in the mask chg[v]
// (their distance at v changed since v last relaxed them); one task per
// active vertex, whatever the number of sources.  A task's edges are walked
// by a warp whose lane l holds sources l and l + 32: per edge one index and
// one weight load (the same address in every lane), one coalesced load of
// the target's row, and an atomicMin for each source that improves (Combine
// = min).  The improving sources of an edge are gathered by a ballot and
// added to chg[u] with one atomicOr; the add that makes chg[u] non-zero
// records u in the next task lists (online filter, degree-class bins;
// ballot filter over chg != 0 on overflow), so lists hold no duplicates.
// Each iteration claims the masks of its tasks first (chg -> cm, a phase of
// its own), then relaxes; the run ends when no distance changed.  A last
// phase writes the source-major result through a shared-memory transpose.
#include "simdx_internal.h"

namespace simdx {

constexpr int kMsMaxInst = 64;

template <class OffT>
struct MsspArgs {
  int n, k, K;                 // vertices, sources, row stride of dvm (32 or 64)
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

// Relaxations of a warp: edges [b, e) of task v for the sources in m.
template <class OffT>
struct MsRelax {
  const MsspArgs<OffT>& a;
  CtaShared& sh;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;

  __device__ MsRelax(const MsspArgs<OffT>& aa, CtaShared& s, unsigned g) : a(aa), sh(s), grid(g) {}

  __device__ __forceinline__ void run(int v, unsigned long long m, long long b, long long e) {
    if (b >= e || m == 0) return;
    const int lane = lane_id();
    const int K = a.K;
    const bool hi = (m >> 32) != 0;  // same in every lane
    const bool a0 = (m >> lane) & 1ull;
    const bool a1 = hi && ((m >> (lane + 32)) & 1ull);
    const uint32_t* dv = a.dvm + (size_t)v * K;
    const uint32_t d0 = a0 ? dv[lane] : 0u;
    const uint32_t d1 = a1 ? dv[lane + 32] : 0u;
    constexpr int kU = 4;
    for (long long p = b; p < e; p += kU) {
      int u[kU];
      uint32_t w[kU], c0[kU], c1[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        u[q] = -1;
        w[q] = 0u;
        if (p + q < e) {
          u[q] = gload(a.idx + p + q);
          w[q] = gload(a.wt + p + q);
        }
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        c0[q] = 0u;
        c1[q] = 0u;
        if (u[q] >= 0) {
          const uint32_t* du = a.dvm + (size_t)u[q] * K;
          if (a0) c0[q] = du[lane];
          if (a1) c1[q] = du[lane + 32];
        }
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        if (u[q] < 0) continue;  // the same in every lane
        uint32_t* du = a.dvm + (size_t)u[q] * K;
        const unsigned long long n0 = (unsigned long long)d0 + w[q];
        const unsigned long long n1 = (unsigned long long)d1 + w[q];
        bool g0 = false, g1 = false;
        if (a0 && n0 < c0[q]) g0 = n0 < atomicMin(du + lane, (uint32_t)n0);
        if (a1 && n1 < c1[q]) g1 = n1 < atomicMin(du + lane + 32, (uint32_t)n1);
        const unsigned b0 = __ballot_sync(kFull, g0);
        const unsigned b1 = hi ? __ballot_sync(kFull, g1) : 0u;
        if ((b0 | b1) && lane == 0) {
          const unsigned long long bits = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
          if (atomicOr(a.chg + u[q], bits) == 0ull) {
            const long long d = (long long)gload(a.off + u[q] + 1) - (long long)gload(a.off + u[q]);
            ++nrec;
            mrec += (unsigned long long)d;
            online_record(u[q], degree_class(d, a.kn), sh, a.w, a.kn, grid);
          }
        }
      }
    }
  }
};

template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) msssp_kernel(const __grid_constant__ MsspArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ uint32_t tile[32][65];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.kn;
  const int n = a.n, K = a.K;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kWarps + warp, nw = (long long)grid * kWarps;
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // ---- phase 0: every distance infinite, no source active
  for (long long x = gtid; x < (long long)n * K; x += gthreads) a.dvm[x] = 0xffffffffu;
  for (long long v = gtid; v < n; v += gthreads) a.chg[v] = 0ull;
  clear_next_slot(s, sh);
  if (!grid_sync(s, grid, sh, k)) return;
  // ---- phase 1: the sources (a vertex may be the source of several)
  clear_next_slot(s, sh);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < a.k; i += kThreads) {
      const int v = a.srcs[i];
      a.dvm[(size_t)v * K + i] = 0u;
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
  int lbuf = 0, it = 0, ballot_it = 0;
  bool lists_ok = true;
  long long evisit = 0, fsum = 0;
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
    MsRelax<OffT> f(a, sh, grid);
    {
      ClassTimer tm(&slot);
      // class 3: each task's edges split over every warp of the grid
      for (unsigned i = 0; i < cnt[3]; ++i) {
        const int v = a.w.list[lbuf][3][i];
        const long long vb = gload(a.off + v), ve = gload(a.off + v + 1);
        const long long ch = ((ve - vb + nw - 1) / nw + 31) & ~31ll;
        const long long b = vb + gw * ch;
        f.run(v, a.cm[v], b, b + ch < ve ? b + ch : ve);
        if (lane == 0 && b < ve) evisit += (b + ch < ve ? b + ch : ve) - b;
      }
      tm.lap(3);
      // class 2: one CTA per task, its warps splitting the edges
      for (unsigned i = blockIdx.x; i < cnt[2]; i += grid) {
        const int v = a.w.list[lbuf][2][i];
        const long long vb = gload(a.off + v), ve = gload(a.off + v + 1);
        const long long ch = ((ve - vb + kWarps - 1) / kWarps + 31) & ~31ll;
        const long long b = vb + (long long)warp * ch;
        f.run(v, a.cm[v], b, b + ch < ve ? b + ch : ve);
        if (lane == 0 && b < ve) evisit += (b + ch < ve ? b + ch : ve) - b;
      }
      tm.lap(2);
      // classes 1 and 0: one warp per task
      for (int c = 1; c >= 0; --c) {
        const int32_t* list = a.w.list[lbuf][c];
        for (long long i = gw; i < cnt[c]; i += nw) {
          const int v = list[i];
          const long long vb = gload(a.off + v), ve = gload(a.off + v + 1);
          f.run(v, a.cm[v], vb, ve);
          if (lane == 0) evisit += ve - vb;
        }
        tm.lap(c);
      }
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
    trace_put(a.w, it, 1 | (filt << 8), (long long)total, (long long)p.mact, -1, t_it);
    trace_classes(a.w, it, p);
    fsum += total;
    ++it;
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    lists_ok = p.overflow == 0;
    if (p.nact == 0) break;  // no distance changed
    lbuf ^= 1;
  }
  // ---- the caller's source-major rows, through a shared-memory transpose
  for (long long t = blockIdx.x; t * 32 < n; t += grid) {
    const long long v0 = t * 32;
    for (int j = threadIdx.x; j < 32 * K; j += kThreads) {
      const int vv = j / K, ii = j - vv * K;
      tile[vv][ii] = v0 + vv < n ? a.dvm[(size_t)(v0 + vv) * K + ii] : 0u;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 32 * a.k; j += kThreads) {
      const int ii = j >> 5, vv = j & 31;
      if (v0 + vv < n) a.out[(size_t)ii * n + v0 + vv] = tile[vv][ii];
    }
    __syncthreads();
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

// Vertex-major state for one launch of up to 64 sources: the distances
// (K words per vertex) and two 64-bit masks per vertex.  Allocated on the
// first call (or a larger K), kept with the graph.
static int ensure_ms_state(simdx_graph* g, int K, cudaStream_t st) {
  const size_t n = (size_t)std::max<int64_t>(g->n, 1);
  const size_t bytes = sizeof(uint32_t) * (size_t)K * n + 2 * sizeof(unsigned long long) * n + 512;
  if (g->mss_state && g->mss_bytes >= bytes) return SIMDX_OK;
  if (capturing(st)) return SIMDX_EUNSUPPORTED;
  dev_free(g->mss_state, st);
  g->mss_state = nullptr;
  g->mss_bytes = 0;
  SIMDX_CUDA(dev_alloc(&g->mss_state, bytes, st));
  g->mss_bytes = bytes;
  return SIMDX_OK;
}

template <class OffT>
static int run_msssp(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                     cudaStream_t st) {
  const int K = k > 32 ? 64 : 32;
  int rc = ensure_ms_state(g, K, st);
  if (rc) return rc;
  const size_t n = (size_t)std::max<int64_t>(g->n, 1);
  char* base = static_cast<char*>(g->mss_state);
  MsspArgs<OffT> a{};
  a.n = (int)g->n;
  a.K = K;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.wt = g->w;
  a.dvm = reinterpret_cast<uint32_t*>(base);
  a.chg = reinterpret_cast<unsigned long long*>(base + ((sizeof(uint32_t) * K * n + 255) & ~(size_t)255));
  a.cm = a.chg + n;
  a.w = make_work(g);
  a.kn = make_knobs(g);
  const void* kern = (const void*)msssp_kernel<OffT>;
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

int sssp_batch_shared(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                      cudaStream_t st) {
  return g->off_bits == 32 ? run_msssp<int32_t>(g, srcs, k, dist, stats, st)
                           : run_msssp<long long>(g, srcs, k, dist, stats, st);
}

}  // namespace simdx
