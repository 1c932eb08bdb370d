// kcore.cu -- k-core as one persistent ACC kernel (Sec. 6 "k-Core";
// aggregation combine, Sec. 3.2).
//
// Iteration 0 deletes every vertex of degree < k (a ballot-filter scan of the
// offsets: the degree is offsets[v+1] - offsets[v], no edges are read).
// Iteration i then propagates the deletions of iteration i-1 (the frontier
// R_{i-1}, removed_at == i-1):
//   push : every frontier vertex decrements the degree of each still-alive
//          neighbour; the decrement that takes a degree from k to k-1 deletes
//          that neighbour (removed_at = i) and records it -- exactly one
//          thread sees that transition, so lists carry no duplicates.  A
//          deleted destination is no longer decremented (Sec. 7.1, k-Core).
//   pull : every alive vertex recounts its neighbours alive at the start of
//          the iteration (removed_at >= i) and is deleted if the count is < k;
//          the owner writes, no atomics.
// Pull runs while the deleted vertices carry many edges (the start), push
// once they become few, the order Sec. 5 gives for k-core; the switch
// compares the frontier's edges with the alive vertices' edges.
#include <climits>

#include "simdx_internal.h"

namespace simdx {

template <class OffT>
struct KcoreArgs {
  int n;
  unsigned kk;
  const OffT* off;
  const int32_t* idx;
  uint8_t* in_core;
  uint32_t* resid;
  Work w;
  Knobs k;
};

template <class OffT>
struct KcorePush {
  struct Src {};
  int32_t* removed_at;
  uint32_t* cnt;
  const OffT* off;
  unsigned kk;
  int it;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ KcorePush(int32_t* r, uint32_t* c, const OffT* o, unsigned kv, int i, CtaShared& s,
                       const Work& ww, const Knobs& kn, unsigned g)
      : removed_at(r), cnt(c), off(o), kk(kv), it(i), sh(s), w(ww), k(kn), grid(g) {}
  __device__ __forceinline__ bool src(int, Src&, int, unsigned) { return true; }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src&, int) { return Src{}; }
  // State of all the lane's targets is loaded first.  Then, per slot, lanes
  // of the warp that decrement the same vertex (hubs neighbour most deleted
  // vertices) combine into one atomicSub of their count; the one subtraction
  // that takes the degree from >= k to < k deletes the vertex.
  __device__ __forceinline__ void edges(const Src (&)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&)[kPushBatch],
                                        unsigned ok) {
    bool want[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      want[q] = false;
      if ((ok >> q) & 1u) want[q] = removed_at[u[q]] == INT_MAX;
    }
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q)
      if (want[q]) want[q] = cnt[u[q]] >= kk;  // stop once below k
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      const unsigned mask = __activemask();
      const int key = want[q] ? u[q] : (int)(0x80000000u | lane_id());
      const unsigned peers = __match_any_sync(mask, key);
      if (!want[q] || (int)lane_id() != __ffs(peers) - 1) continue;
      const unsigned c = (unsigned)__popc(peers);
      const unsigned old = atomicSub(&cnt[u[q]], c);
      if (old >= kk && old - c < kk) {
        removed_at[u[q]] = it;
        long long d = (long long)gload(off + u[q] + 1) - (long long)gload(off + u[q]);
        ++nrec;
        mrec += (unsigned long long)d;
        online_record(u[q], degree_class(d, k), sh, w, k, grid);
      }
    }
  }
};

template <class OffT>
struct KcorePull {
  using Acc = unsigned;
  const int32_t* removed_at;
  int32_t* removed_w;
  uint32_t* cnt;
  const OffT* off;
  unsigned kk;
  int it;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ KcorePull(int32_t* r, uint32_t* c, const OffT* o, unsigned kv, int i, CtaShared& s,
                       const Work& ww, const Knobs& kn, unsigned g)
      : removed_at(r), removed_w(r), cnt(c), off(o), kk(kv), it(i), sh(s), w(ww), k(kn), grid(g) {}
  __device__ __forceinline__ Acc zero() const { return 0u; }
  __device__ __forceinline__ void combine(Acc& a, Acc b) const { a += b; }
  __device__ __forceinline__ void edge(Acc& a, int, int v, long long) { a += removed_at[v] >= it ? 1u : 0u; }
  __device__ __forceinline__ void finish(int u, Acc c) {
    cnt[u] = c;
    if (c < kk) {
      removed_w[u] = it;
      long long d = (long long)gload(off + u + 1) - (long long)gload(off + u);
      ++nrec;
      mrec += (unsigned long long)d;
      online_record(u, degree_class(d, k), sh, w, k, grid);
    }
  }
};

template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) kcore_kernel(KcoreArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ unsigned red_u32[kWarps];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const unsigned kk = a.kk;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  int32_t* removed_at = reinterpret_cast<int32_t*>(a.w.state);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(removed_at + n);
  const OffT* off = a.off;
  auto deg = [off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // ---- phase 0: degrees, first deletions (ballot filter over the offsets)
  int lbuf = 0;
  {
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[0];
    unsigned long long m_rm = 0, m_alive = 0, n_rm = 0;
    auto pred = [&](int v) {
      const long long d = deg(v);
      cnt[v] = (uint32_t)d;
      const bool rm = d < (long long)kk;
      removed_at[v] = rm ? 0 : INT_MAX;
      if (rm) { m_rm += d; ++n_rm; } else m_alive += d;
      return rm;
    };
    auto none = [](int) {};
    ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
    unsigned long long t0 = cta_sum_u64(n_rm, sh), t1 = cta_sum_u64(m_rm, sh), t2 = cta_sum_u64(m_alive, sh);
    if (threadIdx.x == 0) {
      atomicAdd(&slot.nact, t0);
      atomicAdd(&slot.mact, t1);
      atomicAdd(&slot.aux0, t2);
    }
  }
  if (!grid_sync(s, grid, sh, k)) return;
  unsigned cnt_l[kClasses];
  unsigned long long n_f, m_f, m_alive;
  {
    const PhaseSlot& p = s->slot[0];
    for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
    n_f = p.nact;
    m_f = p.mact;
    m_alive = p.aux0;
  }
  bool lists_ok = true;
  int it = 1, push_it = 0, pull_it = 0, ballot_it = 0, online_it = 0;
  long long evisit = 0, fsum = (long long)n_f;
  trace_put(a.w, 0, 2 | (2 << 8), (long long)n_f, (long long)m_f, 0);

  while (n_f > 0) {
    const unsigned long long t_it = globaltimer();
    int dir;
    if (k.direction == 1) dir = 1;
    else if (k.direction == 2) dir = 2;
    else dir = exceeds_share(m_f, (long long)m_alive, k.kalpha) ? 2 : 1;
    int filt = 1;
    if (dir == 1 && (!lists_ok || k.filter == 2)) {
      // rebuild the frontier lists from the metadata
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      const int prev = it - 1;
      auto pred = [=](int v) { return removed_at[v] == prev; };
      auto none = [](int) {};
      ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
      filt = 2;
    }
    if (dir == 2) {
      // task lists of the alive vertices (ballot filter)
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      auto pred = [=](int v) { return removed_at[v] == INT_MAX; };
      auto none = [](int) {};
      ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
      filt = 2;
    }
    clear_next_slot(s, sh);
    online_reset(sh);
    __syncthreads();
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                      a.w.list[lbuf][3]};
    unsigned long long nrec = 0, mrec = 0;
    if (dir == 1) {
      KcorePush<OffT> f(removed_at, cnt, a.off, kk, it, sh, a.w, k, grid);
      push_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, k.huge_min, sh, evisit, &slot);
      nrec = f.nrec;
      mrec = f.mrec;
      ++push_it;
    } else {
      KcorePull<OffT> f(removed_at, cnt, a.off, kk, it, sh, a.w, k, grid);
      pull_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, red_u32, k.huge_min, sh, a.w, evisit, &slot);
      nrec = f.nrec;
      mrec = f.mrec;
      ++pull_it;
    }
    if (filt == 2) ++ballot_it; else ++online_it;
    online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
    unsigned long long tn = cta_sum_u64(nrec, sh), tm = cta_sum_u64(mrec, sh);
    if (threadIdx.x == 0 && tn) {
      atomicAdd(&slot.nact, tn);
      atomicAdd(&slot.mact, tm);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    trace_put(a.w, it, dir | (filt << 8), (long long)n_f, (long long)m_f, it, t_it);
    trace_classes(a.w, it, p);
    for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
    lists_ok = p.overflow == 0;
    m_alive -= p.mact;
    n_f = p.nact;
    m_f = p.mact;
    fsum += (long long)n_f;
    lbuf ^= 1;
    ++it;
  }
  // ---- outputs
  for (long long v = gtid; v < n; v += gthreads) {
    const bool in = removed_at[v] == INT_MAX;
    a.in_core[v] = in ? 1 : 0;
    if (a.resid) a.resid[v] = in ? cnt[v] : 0u;
  }
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = it;
    st.push_iters = push_it;
    st.pull_iters = pull_it;
    st.ballot_iters = ballot_it + 1;
    st.online_iters = online_it;
    st.phases = (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = fsum;
    st.last_l1 = 0.0;
  }
}

// ---------------------------------------------------------------------------
// k-core decomposition: the coreness of every vertex, i.e. the largest k
// whose k-core holds it.  Sec. 6 defines the k-core by repeatedly deleting
// the vertices of degree < k; running that deletion for k = 1, 2, ... on the
// shrinking graph deletes at level K exactly the vertices of coreness K.  At
// level K every alive vertex of residual degree <= K is deleted (core = K);
// its push decrements its alive neighbours (warp-combined atomicSub, as in
// the fixed-k push), and the one decrement that takes a neighbour from > K
// to <= K deletes and records it, so lists carry no duplicates.  When a
// level's lists run dry, one scan of the alive vertices (ballot filter)
// opens level K + 1, or, if no alive vertex has degree K + 1, a second scan
// jumps to the smallest alive degree.  All levels run in one persistent
// launch.
template <class OffT>
struct CoreArgs {
  int n;
  const OffT* off;
  const int32_t* idx;
  uint32_t* core;
  Work w;
  Knobs k;
};

template <class OffT>
struct CorePush {
  struct Src {};
  int32_t* removed_at;
  uint32_t* cnt;
  uint32_t* core;
  const OffT* off;
  unsigned K;
  int it;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ CorePush(int32_t* r, uint32_t* c, uint32_t* co, const OffT* o, unsigned kv, int i, CtaShared& s,
                      const Work& ww, const Knobs& kn, unsigned g)
      : removed_at(r), cnt(c), core(co), off(o), K(kv), it(i), sh(s), w(ww), k(kn), grid(g) {}
  __device__ __forceinline__ bool src(int, Src&, int, unsigned) { return true; }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src&, int) { return Src{}; }
  __device__ __forceinline__ void edges(const Src (&)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&)[kPushBatch],
                                        unsigned ok) {
    bool want[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      want[q] = false;
      if ((ok >> q) & 1u) want[q] = removed_at[u[q]] == INT_MAX;
    }
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q)
      if (want[q]) want[q] = cnt[u[q]] > K;  // already at or below the level: deleted at it
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      const unsigned mask = __activemask();
      const int key = want[q] ? u[q] : (int)(0x80000000u | lane_id());
      const unsigned peers = __match_any_sync(mask, key);
      if (!want[q] || (int)lane_id() != __ffs(peers) - 1) continue;
      const unsigned c = (unsigned)__popc(peers);
      const unsigned old = atomicSub(&cnt[u[q]], c);
      if (old > K && old - c <= K) {
        removed_at[u[q]] = it;
        core[u[q]] = K;
        long long d = (long long)gload(off + u[q] + 1) - (long long)gload(off + u[q]);
        ++nrec;
        mrec += (unsigned long long)d;
        online_record(u[q], degree_class(d, k), sh, w, k, grid);
      }
    }
  }
};

// One level scan.  Walks `count` entries of the domain (vertex i, or dom[i]
// once the remaining vertices are listed) and sorts each into: gone (deleted
// before), deleted now (residual degree <= kt: core = kt, removed_at = prev;
// listed by degree class unless it has no edges to push), or kept (appended
// to `keep`, the next scan's domain).  Counts the remaining vertices,
// the deleted ones (slot.nact) and the smallest remaining degree.  Each CTA
// reserves its chunk's entries with one atomic per category, as the ballot
// filter does.
constexpr int kCoreCats = kClasses + 1;  // the degree classes, then "kept"

template <class OffT>
__device__ void core_scan(long long count, const int32_t* dom, int32_t* keep, unsigned kt, int prev,
                          int32_t* removed_at, const uint32_t* cnt, uint32_t* core, const OffT* off,
                          const Work& w, const Knobs& k, unsigned grid, int nbuf, PhaseSlot& slot,
                          int (&cw)[kCoreCats][kWarps], int (&cb)[kCoreCats], unsigned long long& nalive,
                          unsigned long long& ndel, unsigned long long& mymin) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int J = ballot_steps(count, grid);
  const long long csz = (long long)kThreads * J;
  for (long long chunk = blockIdx.x; chunk * csz < count; chunk += grid) {
    const long long wbase = chunk * csz + (long long)warp * 32 * J;
    unsigned my[kCoreCats] = {0u, 0u, 0u, 0u, 0u};
    for (int j = 0; j < J; ++j) {
      const long long i = wbase + j * 32 + lane;
      int cat = -1;
      if (i < count) {
        const int v = dom ? dom[i] : (int)i;
        if (removed_at[v] == INT_MAX) {
          const unsigned c = cnt[v];
          ++nalive;
          if (c < mymin) mymin = c;
          if (c > kt) {
            cat = kClasses;
          } else {
            removed_at[v] = prev;
            core[v] = kt;
            ++ndel;
            const long long d = (long long)gload(off + v + 1) - (long long)gload(off + v);
            if (d > 0) cat = degree_class(d, k);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < kCoreCats; ++c) {
        const unsigned m = __ballot_sync(kFull, cat == c);
        if (lane == j) my[c] = m;
      }
    }
    int pre[kCoreCats];
#pragma unroll
    for (int c = 0; c < kCoreCats; ++c) {
      const int x = __popc(my[c]);
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      pre[c] = incl - x;
      if (lane == 31) cw[c][warp] = incl;
    }
    __syncthreads();
    if (threadIdx.x < kCoreCats) {
      const int c = threadIdx.x;
      int run = 0;
      for (int q = 0; q < kWarps; ++q) {
        const int t = cw[c][q];
        cw[c][q] = run;
        run += t;
      }
      int b = 0;
      if (run > 0)
        b = c < kClasses ? (int)atomicAdd(&slot.list_cnt[c], (unsigned)run)
                         : (int)atomicAdd(&slot.aux0, (unsigned long long)run);
      cb[c] = b;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kCoreCats; ++c) {
      unsigned m = my[c];
      int pos = cb[c] + cw[c][warp] + pre[c];
      int32_t* dst = c < kClasses ? w.list[nbuf][c] : keep;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const long long idx = wbase + lane * 32 + b;
        dst[pos++] = dom ? dom[idx] : (int)idx;
      }
    }
    __syncthreads();
  }
}

template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) coreness_kernel(CoreArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ int cw[kCoreCats][kWarps];
  __shared__ int cb[kCoreCats];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  int32_t* removed_at = reinterpret_cast<int32_t*>(a.w.state);  // push iteration of the deletion
  uint32_t* cnt = reinterpret_cast<uint32_t*>(removed_at + n);   // residual degree
  int32_t* doms[2] = {reinterpret_cast<int32_t*>(cnt + n), reinterpret_cast<int32_t*>(cnt + n) + n};
  const OffT* off = a.off;
  auto deg = [off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();
  for (long long v = gtid; v < n; v += gthreads) {
    cnt[v] = (uint32_t)deg((int)v);
    removed_at[v] = INT_MAX;
  }
  clear_next_slot(s, sh);
  if (!grid_sync(s, grid, sh, k)) return;

  int lbuf = 0;
  unsigned cnt_l[kClasses] = {0u, 0u, 0u, 0u};
  bool lists_ok = true;
  unsigned long long pending = 0;  // vertices deleted by the last push, still to push
  long long K = -1;                // current level
  const int32_t* dom = nullptr;    // the scans' domain: all vertices, then the remaining ones
  long long dcount = n;
  int dsel = 0;
  int it = 0, ballot_it = 0, online_it = 0;
  long long evisit = 0, fsum = 0;
  while (true) {
    const unsigned long long t_it = globaltimer();
    int filt = 1;
    if (pending == 0) {
      // level advance: scan the alive vertices, delete those at the guessed
      // level, count the alive ones and find their smallest degree
      bool done = false;
      unsigned long long Kt = (unsigned long long)(K + 1);
      for (int attempt = 0; attempt < 2; ++attempt) {
        clear_next_slot(s, sh);
        PhaseSlot& slot = s->slot[slot_of(sh.phase)];
        unsigned long long nalive = 0, ndel = 0, mymin = ~0ull;
        int32_t* keep = doms[dsel];
        // deleted as if by the push before the next one
        core_scan<OffT>(dcount, dom, keep, (unsigned)Kt, it - 1, removed_at, cnt, a.core, off, a.w, k, grid,
                        lbuf, slot, cw, cb, nalive, ndel, mymin);
        const unsigned long long td = cta_sum_u64(ndel, sh);
        if (threadIdx.x == 0 && td) atomicAdd(&slot.nact, td);
        const unsigned long long ta = cta_sum_u64(nalive, sh);
        {
          unsigned long long m = mymin;
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(kFull, m, o);
            m = y < m ? y : m;
          }
          __syncthreads();
          if (lane_id() == 0) sh.red64[threadIdx.x >> 5] = m;
          __syncthreads();
          if (threadIdx.x == 0 && ta) {
            unsigned long long t = ~0ull;
            for (int q = 0; q < kWarps; ++q) t = sh.red64[q] < t ? sh.red64[q] : t;
            atomicAdd(&slot.aux1, ta);
            atomicMax(&slot.aux2, ~t);  // slots start at 0: keep the min inverted
          }
        }
        if (!grid_sync(s, grid, sh, k)) return;
        const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
        dom = doms[dsel];
        dcount = (long long)p.aux0;
        dsel ^= 1;
        for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
        if (p.aux1 == 0) {
          done = true;
          break;
        }
        if (p.nact > 0) {
          K = (long long)Kt;
          pending = cnt_l[0] + cnt_l[1] + cnt_l[2] + cnt_l[3];
          break;
        }
        Kt = ~p.aux2;  // no alive vertex has degree K + 1: jump to the smallest
      }
      if (done) break;
      ++ballot_it;
      if (pending == 0) continue;  // the level deleted isolated vertices only
      filt = 2;
      lists_ok = true;
    } else if (!lists_ok || k.filter == 2) {
      // the online bins overflowed: list the last push's deletions again
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      const int prev = it - 1;
      auto pred = [=](int v) { return removed_at[v] == prev; };
      auto none = [](int) {};
      ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
      ++ballot_it;
      filt = 2;
    } else {
      ++online_it;
    }
    clear_next_slot(s, sh);
    online_reset(sh);
    __syncthreads();
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                      a.w.list[lbuf][3]};
    CorePush<OffT> f(removed_at, cnt, a.core, a.off, (unsigned)K, it, sh, a.w, k, grid);
    push_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, k.huge_min, sh, evisit, &slot);
    online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
    const unsigned long long tn = cta_sum_u64(f.nrec, sh), tm = cta_sum_u64(f.mrec, sh);
    if (threadIdx.x == 0 && tn) {
      atomicAdd(&slot.nact, tn);
      atomicAdd(&slot.mact, tm);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    trace_put(a.w, it, 1 | (filt << 8), (long long)(cnt_l[0] + cnt_l[1] + cnt_l[2] + cnt_l[3]),
              (long long)p.mact, K, t_it);
    trace_classes(a.w, it, p);
    fsum += (long long)(cnt_l[0] + cnt_l[1] + cnt_l[2] + cnt_l[3]);
    for (int c = 0; c < kClasses; ++c) cnt_l[c] = p.list_cnt[c];
    lists_ok = p.overflow == 0;
    pending = p.nact;
    lbuf ^= 1;
    ++it;
  }
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = it;
    st.push_iters = it;
    st.pull_iters = 0;
    st.ballot_iters = ballot_it;
    st.online_iters = online_it;
    st.phases = (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = fsum;
    st.last_l1 = 0.0;
  }
}

template <class OffT>
static int run_coreness(simdx_graph* g, uint32_t* core, simdx_stats* stats, cudaStream_t st) {
  CoreArgs<OffT> a{};
  a.n = (int)g->n;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.core = core;
  a.w = make_work(g);
  a.k = make_knobs(g);
  const void* kern = (const void*)coreness_kernel<OffT>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st);
}

const void* kcore_kernel_ptr(int off_bits) {
  return off_bits == 32 ? (const void*)kcore_kernel<int32_t> : (const void*)kcore_kernel<long long>;
}

template <class OffT>
static int run_kcore(simdx_graph* g, uint32_t kk, uint8_t* in_core, uint32_t* resid, simdx_stats* stats,
                     cudaStream_t st) {
  KcoreArgs<OffT> a{};
  a.n = (int)g->n;
  a.kk = kk;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.in_core = in_core;
  a.resid = resid;
  a.w = make_work(g);
  a.k = make_knobs(g);
  const void* kern = (const void*)kcore_kernel<OffT>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st);
}

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_kcore(simdx_graph* g, uint32_t k, uint8_t* in_core, uint32_t* residual_deg,
                           simdx_stats* stats, void* stream) {
  if (!g || !in_core || !g->symmetric) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    int rc = prepare_launch(g, st);
    return rc ? rc : finish_launch(g, stats, st);
  }
  return g->off_bits == 32 ? run_kcore<int32_t>(g, k, in_core, residual_deg, stats, st)
                           : run_kcore<long long>(g, k, in_core, residual_deg, stats, st);
}

extern "C" int simdx_kcore_decompose(simdx_graph* g, uint32_t* coreness, simdx_stats* stats, void* stream) {
  if (!g || !coreness || !g->symmetric) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    int rc = prepare_launch(g, st);
    return rc ? rc : finish_launch(g, stats, st);
  }
  return g->off_bits == 32 ? run_coreness<int32_t>(g, coreness, stats, st)
                           : run_coreness<long long>(g, coreness, stats, st);
}
