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
#include <mutex>
#include <set>
#include <utility>
#include <type_traits>

#include "acc_cluster.cuh"
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
      push_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, k.huge_min, sh, evisit);
      nrec = f.nrec;
      mrec = f.mrec;
      ++push_it;
    } else {
      KcorePull<OffT> f(removed_at, cnt, a.off, kk, it, sh, a.w, k, grid);
      pull_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, red_u32, k.huge_min, sh, a.w, evisit);
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
  int split;     // 1: stop at the first level whose domain fits the cluster; 2: stop before a large
                 // push (at least kCoreBigM edges) that deletes most of what remains (the densest
                 // core's level); the loop state goes to the resume record
  int resume;    // continue the run a launch stopped with this split value (nothing to do if it
                 // finished or stopped otherwise)
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
                          unsigned long long& ndel, unsigned long long& mymin, unsigned long long& mdel) {
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
            mdel += (unsigned long long)d;
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

// ------------------------------------------------ small frontiers
// Most peeling steps of a power-law graph delete a handful of vertices, and
// most levels scan a small remaining domain; each would cost a grid barrier
// and a chain of global round trips.  While a push frontier is small, or the
// domain holds at most kCoreLocDom vertices, the steps run on the first
// thread-block cluster (acc_cluster.cuh).  A push step decrements each
// neighbour's residual degree (atomicSub, the target's offsets loaded
// alongside; the decrement that takes it from K + 1 to K deletes it, the
// same unique transition as the grid's push).  A scan step splits the domain
// into one segment per CTA; each CTA compacts its kept vertices into its own
// segment of the other domain buffer, so no CTA waits on another's order.
// The episode hands back when the frontier grows (lists rebuilt by the
// ballot filter from removed_at), compacting the segments into one domain,
// or when a level ends with a domain too large to scan here.
constexpr long long kCoreLocDom = 65536;  // scan the domain here when it holds at most this many
constexpr int kScanPer = 4;              // domain vertices per thread in flight

enum { kCcK, kCcPending, kCcMpend, kCcDomSel, kCcDcount, kCcDsel, kCcIt, kCcBallotIt, kCcOnlineIt, kCcFsum,
       kCcDone, kCcBeat = 15 };

template <class OffT>
__device__ bool core_local(const CoreArgs<OffT>& a, LocalShared& ls, CtaShared& sh, int32_t* removed_at,
                           uint32_t* cnt, int32_t* const (&doms)[2], const unsigned* cnt_l, int lbuf, long long& K,
                           unsigned long long& pending, unsigned long long& m_pend, const int32_t*& dom,
                           long long& dcount, int& dsel, int& it, int& ballot_it, int& online_it, long long& fsum,
                           long long& evisit, unsigned long long& episodes, bool& done) {
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const OffT* off = a.off;
  if (blockIdx.x < kCluster) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned r = cl.block_rank();
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x < 3) loc_clear(ls, threadIdx.x);
    if (threadIdx.x == 0) ls.stop = 0;
    __syncthreads();
    // the entry frontier: the class lists' entries j with j % kCluster == r
    if (pending > 0) {
      unsigned base = 0;
      for (int c = 0; c < kClasses; ++c) {
        const int32_t* list = a.w.list[lbuf][c];
        for (unsigned i = threadIdx.x; i < cnt_l[c]; i += kThreads)
          if ((base + i) % kCluster == r) {
            const int v = list[i];
            const long long b0 = (long long)gload(off + v);
            loc_put(ls, 0, 0, b0, (long long)gload(off + v + 1) - b0);
          }
        base += cnt_l[c];
      }
    }
    loc_publish(cl, ls, 0, r);
    cl.sync();
    unsigned cc, cp, zc, zp;
    const LocTotals T0 = loc_counts(ls, 0, cc, cp, zc, zp);
    unsigned N = T0.n;
    // the domain: this CTA's segment [seg_lo, seg_lo + seg_n) of src (the
    // identity when src is null), compacted into the other buffer
    const long long seg_lo = dcount * (long long)r / kCluster;
    long long seg_n = dcount * (long long)(r + 1) / kCluster - seg_lo;
    const int32_t* src = dom;
    int wsel = dsel;         // the buffer the next scan writes
    bool segmented = false;  // the domain lives in per-CTA segments
    long long seg_pre = 0;   // this CTA's segment's place in a compacted domain
    long long dtotal = dcount;
    unsigned long long m_cur = m_pend;
    bool first_push = false;  // the push right after a scan lists by ballot in the grid's count
    int cur = 0, fc = 0;
    unsigned long long Kt = (unsigned long long)(K + 1);
    int attempt = 0;  // scans of this level that deleted nothing (jumps)
    long long steps = 0;
    long long c_scans = 0;  // SM clock cycles of scans since the last push
    // the entry lists' pieces may overflow a CTA's buffer (a few vertices of
    // many edges in one CTA's share): then nothing is walked here, and the
    // grid lists and pushes the pending vertices itself
    bool handback = T0.ovf != 0;
    unsigned long long t_it = trace_clock();
    while (!handback) {
      const int nx = cur == 2 ? 0 : cur + 1, nn = nx == 2 ? 0 : nx + 1;
      unsigned ab = 0;
      if (threadIdx.x == 0) {
        loc_clear(ls, nn);
        if (r == 0) {
          ab = (unsigned)ld_volatile_i32(&s->abort);
          if (blockIdx.x == 0) *(volatile long long*)&s->loc[kCcBeat] = ++steps;  // progress for the waiting CTAs
        }
      }
      const bool scan = N == 0;
      const long long c0 = clock64();
      unsigned long long mrec = 0;
      if (scan) {
        // ---- scan the segment at level Kt: gone, deleted now (core = Kt,
        // removed_at = it - 1, listed if it has edges), or kept
        int32_t* dst = doms[wsel];
        unsigned long long nalive = 0, ndel = 0, mymin = ~0ull;
        for (long long i0 = 0; i0 < seg_n; i0 += (long long)kThreads * kScanPer) {
          int v[kScanPer], ra[kScanPer];
          unsigned c[kScanPer];
          long long b0[kScanPer], e0[kScanPer];
#pragma unroll
          for (int q = 0; q < kScanPer; ++q) {
            const long long i = i0 + (long long)q * kThreads + threadIdx.x;
            v[q] = -1;
            if (i < seg_n) v[q] = src ? src[seg_lo + i] : (int)(seg_lo + i);
          }
#pragma unroll
          for (int q = 0; q < kScanPer; ++q) {
            ra[q] = 0;
            c[q] = 0u;
            b0[q] = e0[q] = 0;
            if (v[q] >= 0) {
              // read at L2: other CTAs' pushes wrote these since this SM may
              // have cached them (a cluster barrier does not refresh L1)
              ra[q] = __ldcg(removed_at + v[q]);
              c[q] = __ldcg(cnt + v[q]);
              b0[q] = (long long)gload(off + v[q]);
              e0[q] = (long long)gload(off + v[q] + 1);
            }
          }
#pragma unroll
          for (int q = 0; q < kScanPer; ++q) {
            const bool alive = v[q] >= 0 && ra[q] == INT_MAX;
            const bool del = alive && c[q] <= (unsigned)Kt;
            if (alive) {
              ++nalive;
              if (c[q] < mymin) mymin = c[q];
            }
            if (del) {
              removed_at[v[q]] = it - 1;
              a.core[v[q]] = (uint32_t)Kt;
              ++ndel;
              mrec += (unsigned long long)(e0[q] - b0[q]);
            }
            loc_append(ls, fc ^ 1, nx, del, b0[q], e0[q] - b0[q]);
            const bool kept = alive && !del;
            const unsigned mk = __ballot_sync(kFull, kept);
            if (mk) {
              const int leader = __ffs(mk) - 1;
              unsigned bq = 0;
              if (lane == leader) bq = atomicAdd(&ls.z[nx], (unsigned)__popc(mk));
              bq = __shfl_sync(kFull, bq, leader);
              if (kept) dst[seg_lo + bq + (unsigned)__popc(mk & lanemask_lt())] = v[q];
            }
          }
        }
        nalive = warp_sum_u64(nalive | (ndel << 32));
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const unsigned long long y = __shfl_xor_sync(kFull, mymin, d);
          mymin = y < mymin ? y : mymin;
        }
        if (lane == 0) {
          if (nalive) atomicAdd(&ls.x[nx], nalive);
          if (mymin != ~0ull) atomicMin(&ls.y[nx], mymin);
        }
      } else {
        // ---- push: this CTA's slice of the frontier
        const unsigned lo = (unsigned)(((unsigned long long)N * r) / kCluster);
        const unsigned myc = (unsigned)(((unsigned long long)N * (r + 1)) / kCluster) - lo;
        const unsigned Kv = (unsigned)K;
        unsigned gs = (myc + kWarps - 1) / kWarps;
        gs = gs < 1 ? 1 : (gs > 64 ? 64 : gs);
        for (unsigned b = (unsigned)warp * gs; b < myc; b += (unsigned)kWarps * gs) {
          const unsigned lim = b + gs < myc ? b + gs : myc;
          const unsigned i0 = b + lane, i1 = b + 32 + lane;
          const unsigned g0 = lo + (i0 < lim ? i0 : 0), g1 = lo + (i1 < lim ? i1 : 0);
          const int t0 = loc_owner(cp, g0), t1 = loc_owner(cp, g1);
          const unsigned p0 = __shfl_sync(kFull, cp, t0), p1 = __shfl_sync(kFull, cp, t1);
          unsigned long long e0 = 0, e1 = 0;
          if (i0 < lim) e0 = cl.map_shared_rank(&ls, (unsigned)t0)->f[fc][g0 - p0];
          if (i1 < lim) e1 = cl.map_shared_rank(&ls, (unsigned)t1)->f[fc][g1 - p1];
          const long long b0 = (long long)(e0 >> 24), b1 = (long long)(e1 >> 24);
          const int d0 = (int)(e0 & kLocDegMask), d1 = (int)(e1 & kLocDegMask);
          int ia = d0, ib = d1;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(kFull, ia, o), yb = __shfl_up_sync(kFull, ib, o);
            if (lane >= o) {
              ia += ya;
              ib += yb;
            }
          }
          const int ta = __shfl_sync(kFull, ia, 31);
          ib += ta;
          const int total = __shfl_sync(kFull, ib, 31);
          for (int q0 = 0; q0 < total; q0 += 32 * kLocBatch) {
            int u[kLocBatch];
#pragma unroll
            for (int q = 0; q < kLocBatch; ++q) {
              const int j = q0 + 32 * q + lane;
              bool hi;
              const int t = loc_find(ia, ib, ta, j < total ? j : total - 1, hi);
              const long long s0 = __shfl_sync(kFull, b0, t), s1 = __shfl_sync(kFull, b1, t);
              const int x0 = __shfl_sync(kFull, ia - d0, t), x1 = __shfl_sync(kFull, ib - d1, t);
              const long long bj = hi ? s1 : s0;
              const int ej = hi ? x1 : x0;
              u[q] = j < total ? gload(a.idx + bj + (j - ej)) : -1;
            }
            // decrement the neighbours still above the level: a residual
            // degree <= K means deleted (earlier, by this level's scan, or by
            // the decrement that crossed K + 1 -> K), and degrees only fall,
            // so the L2 value of the last barrier can skip them; the atomic
            // decides the one crossing
            unsigned c[kLocBatch];
            long long ob[kLocBatch], oe[kLocBatch];
#pragma unroll
            for (int q = 0; q < kLocBatch; ++q) {
              c[q] = 0;
              ob[q] = oe[q] = 0;
              if (u[q] >= 0) {
                c[q] = __ldcg(cnt + u[q]);
                ob[q] = (long long)gload(off + u[q]);
                oe[q] = (long long)gload(off + u[q] + 1);
              }
            }
            bool got[kLocBatch];
#pragma unroll
            for (int q = 0; q < kLocBatch; ++q) {
              got[q] = false;
              if (c[q] > Kv) {
                const unsigned old = atomicSub(&cnt[u[q]], 1u);
                if (old == Kv + 1) {
                  removed_at[u[q]] = it;
                  a.core[u[q]] = Kv;
                  mrec += (unsigned long long)(oe[q] - ob[q]);
                  got[q] = true;
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kLocBatch; ++q) loc_append(ls, fc ^ 1, nx, got[q], ob[q], oe[q] - ob[q]);
          }
          evisit += d0 + d1;
        }
      }
      mrec = warp_sum_u64(mrec);
      if (lane == 0 && mrec) atomicAdd(&ls.medges[nx], mrec);
      if (threadIdx.x == 0 && r == 0) ls.stop = ab;
      const long long c1 = clock64();
      loc_publish(cl, ls, nx, r, (unsigned)(c1 - c0));
      cl.sync();
      const LocTotals T = loc_counts(ls, nx, cc, cp, zc, zp);
      const long long c2 = clock64();
      if (scan) c_scans += c2 - c0;
      if (T.stop) {
        handback = true;  // aborted: the waiting CTAs see the flag
        break;
      }
      if (scan) {
        const unsigned long long nalive = T.x & 0xffffffffull, ndel = T.x >> 32;
        src = doms[wsel];
        wsel ^= 1;
        segmented = true;
        seg_n = (long long)ls.z[nx];
        seg_pre = (long long)__shfl_sync(kFull, zp, (int)r);
        dtotal = (long long)T.z;
        if (nalive == 0) {
          done = true;
          break;
        }
        if (ndel == 0) {
          Kt = T.y;  // no alive vertex has degree Kt: jump to the smallest
          ++attempt;
        } else {
          K = (long long)Kt;
          Kt = (unsigned long long)(K + 1);
          attempt = 0;
          ++ballot_it;
          first_push = true;
        }
        N = T.n;
        m_cur = T.m;
        if (T.ovf || N > kLocExitN || T.m > kLocEnterM) {
          handback = true;  // a large frontier: the grid lists and pushes it
          cur = nx;
          break;
        }
      } else {
        const unsigned long long t_end = trace_clock();
        trace_put(a.w, it, 1 | ((first_push ? 2 : 1) << 8) | (1 << 19), (long long)N, (long long)T.m, K, t_it,
                  t_end);
        if (blockIdx.x == 0 && threadIdx.x == 0 && it < a.w.trace_cap) {
          a.w.trace[(long long)kTraceWords * it + 6] = c_scans;  // CTA 0's cycles in scans since the last push
          a.w.trace[(long long)kTraceWords * it + 7] = (long long)T.walk;  // ... the slowest CTA's push walk
        }
        c_scans = 0;
        t_it = t_end;
        fsum += (long long)N;
        if (!first_push) ++online_it;
        first_push = false;
        ++it;
        N = T.n;
        m_cur = T.m;
        if (T.ovf || N > kLocExitN || T.m > kLocEnterM) {
          handback = true;
          cur = nx;
          break;
        }
        if (N == 0 && !segmented && dcount > kCoreLocDom) break;  // the level ends; the grid scans
      }
      cur = nx;
      fc ^= 1;
    }
    // a frontier handed back is pending (its vertices have removed_at ==
    // it - 1); a segmented domain is compacted into the buffer not holding it
    if (handback && segmented && !done) {
      int32_t* dst = doms[wsel];
      for (long long i = threadIdx.x; i < seg_n; i += kThreads) dst[seg_pre + i] = src[seg_lo + i];
    }
    __threadfence();
    cl.sync();  // no CTA leaves while another still reads its shared memory
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      long long* w = s->loc;
      w[kCcK] = K;
      w[kCcPending] = done ? 0 : (long long)N;
      w[kCcMpend] = (long long)m_cur;
      w[kCcDomSel] = segmented ? (handback ? wsel : -2) : -1;
      w[kCcDcount] = dtotal;
      w[kCcDsel] = segmented ? (wsel ^ 1) : dsel;
      w[kCcIt] = it; w[kCcBallotIt] = ballot_it; w[kCcOnlineIt] = online_it; w[kCcFsum] = fsum;
      w[kCcDone] = done;
      red_release_add_u64(&s->loc_epoch, 1ull);
    }
  }
  if (!loc_wait_handback(s, k, sh, &s->loc_epoch, &s->loc[kCcBeat], episodes)) return false;
  ++episodes;
  const volatile long long* w = s->loc;
  K = w[kCcK];
  pending = (unsigned long long)w[kCcPending];
  m_pend = (unsigned long long)w[kCcMpend];
  const long long ds = w[kCcDomSel];
  if (ds >= 0) dom = doms[ds];
  dcount = w[kCcDcount];
  dsel = (int)w[kCcDsel];
  it = (int)w[kCcIt]; ballot_it = (int)w[kCcBallotIt]; online_it = (int)w[kCcOnlineIt]; fsum = w[kCcFsum];
  done = w[kCcDone] != 0;
  return true;
}

// Loop state words of the resume record when a run is split between a grid
// launch (the large levels) and a cluster launch (the rest).
enum { kCrK, kCrDom, kCrDcount, kCrDsel, kCrIt, kCrBallotIt, kCrOnlineIt, kCrFsum, kCrPhases, kCrPending, kCrMpend };
constexpr unsigned long long kCoreBigM = 1ull << 20;  // a push this large goes back to the plain grid
constexpr long long kCoreAutoMaxN = 1ll << 22;        // small_frontier = 2: clusters up to this many vertices

// CLU: small frontiers and small domains run on the first thread-block
// cluster (the small_frontier knob; launched in clusters of kCluster).
template <class OffT, bool CLU = false>
__global__ void __launch_bounds__(kThreads, CLU ? 3 : 4) coreness_kernel(CoreArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ typename std::conditional<CLU, LocalShared, char>::type loc_sm;
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
  // a resumed run skips the set-up; a run the first launch finished ends here
  const bool resumed = a.resume && ld_volatile_i32(&s->rs.active) == a.resume;
  if (a.resume && !resumed) return;
  if (!resumed) {
    for (long long v = gtid; v < n; v += gthreads) {
      cnt[v] = (uint32_t)deg((int)v);
      removed_at[v] = INT_MAX;
    }
    clear_next_slot(s, sh);
    if (!grid_sync(s, grid, sh, k)) return;
  }

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
  unsigned long long m_pend = 0;    // out-edges of the pending vertices
  unsigned long long episodes = 0;  // small-frontier episodes so far
  long long phases0 = 0;            // barrier phases of the first launch
  if (resumed) {
    const volatile long long* r = s->rs.v;
    K = r[kCrK];
    const long long ds = r[kCrDom];
    dom = ds < 0 ? nullptr : doms[ds];
    dcount = r[kCrDcount];
    dsel = (int)r[kCrDsel];
    it = (int)r[kCrIt];
    ballot_it = (int)r[kCrBallotIt];
    online_it = (int)r[kCrOnlineIt];
    fsum = r[kCrFsum];
    phases0 = r[kCrPhases];
    pending = (unsigned long long)r[kCrPending];
    m_pend = (unsigned long long)r[kCrMpend];
    lists_ok = pending == 0;  // a pending frontier is listed again from removed_at
  }
  while (true) {
    if ((a.split == 1 && pending == 0 && dcount <= kCoreLocDom) ||
        (a.split == 2 && pending > 0 && m_pend >= kCoreBigM && 2 * pending >= (unsigned long long)dcount)) {
      // the rest of the run is the cluster launch's: hand the loop state over
      const unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
      if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long* r = s->rs.v;
        r[kCrK] = K;
        r[kCrDom] = dom == nullptr ? -1 : (dom == doms[0] ? 0 : 1);
        r[kCrDcount] = dcount;
        r[kCrDsel] = dsel;
        r[kCrIt] = it;
        r[kCrBallotIt] = ballot_it;
        r[kCrOnlineIt] = online_it;
        r[kCrFsum] = fsum;
        r[kCrPhases] = phases0 + (long long)sh.phase;
        r[kCrPending] = (long long)pending;
        r[kCrMpend] = (long long)m_pend;
        s->rs.active = a.split;
      }
      return;
    }
    if constexpr (CLU) {
      const bool scan_here = pending == 0 && dcount <= kCoreLocDom;
      const bool push_here = pending > 0 && lists_ok && pending <= kLocEnterN && m_pend <= kLocEnterM;
      if (k.small && (scan_here || push_here)) {
        bool done = false;
        if (!core_local(a, loc_sm, sh, removed_at, cnt, doms, cnt_l, lbuf, K, pending, m_pend, dom, dcount, dsel,
                        it, ballot_it, online_it, fsum, evisit, episodes, done))
          return;
        if (done) break;
        lists_ok = false;  // a pending frontier is listed again from removed_at
        continue;
      }
    }
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
        unsigned long long nalive = 0, ndel = 0, mymin = ~0ull, mdel = 0;
        int32_t* keep = doms[dsel];
        // deleted as if by the push before the next one
        core_scan<OffT>(dcount, dom, keep, (unsigned)Kt, it - 1, removed_at, cnt, a.core, off, a.w, k, grid,
                        lbuf, slot, cw, cb, nalive, ndel, mymin, mdel);
        const unsigned long long td = cta_sum_u64(ndel, sh);
        const unsigned long long tmd = cta_sum_u64(mdel, sh);
        if (threadIdx.x == 0 && td) {
          atomicAdd(&slot.nact, td);
          atomicAdd(&slot.mact, tmd);
        }
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
          m_pend = p.mact;
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
    push_classes<OffT>(f, a.off, a.idx, lists, cnt_l, grid, k.huge_min, sh, evisit);
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
    m_pend = p.mact;
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
    st.phases = (int)(phases0 + (long long)sh.phase);
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = fsum;
    st.last_l1 = 0.0;
  }
}

// The decomposition's launches on `st` (no statistics read-back); returns
// their count in *launches.
template <class OffT>
static int launch_coreness(simdx_graph* g, uint32_t* core, cudaStream_t st, int* launches) {
  CoreArgs<OffT> a{};
  a.n = (int)g->n;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.core = core;
  a.w = make_work(g);
  a.k = make_knobs(g);
  // the peeling's tail is small steps whatever the degrees; the automatic
  // setting turns the cluster on up to kCoreAutoMaxN vertices (measured on
  // R-MAT: 34 % faster at 2^18, 24 % at 2^20, 6 % at 2^22, 5 % slower at
  // 2^24, where the tail's larger pushes dominate and run on fewer CTAs)
  a.k.small = g->cfg.small_frontier == 1 || (g->cfg.small_frontier == 2 && g->n <= kCoreAutoMaxN);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  const void* kern = (const void*)coreness_kernel<OffT>;
  const void* kclu = (const void*)coreness_kernel<OffT, true>;
  const int gclu = a.k.small ? grid_for_cluster(g, kclu, kCluster) : 0;
  if (gclu >= kCluster) {
    // the large levels on the plain grid (every CTA it fits), the tail --
    // levels whose remaining vertices fit the cluster's scans -- in
    // clusters; the second launch finds the first one's state in the
    // resume record (or nothing to do)
    a.split = 1;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    if ((rc = prepare_resume(g, st)) != SIMDX_OK) return rc;
    a.split = 2;
    a.resume = 1;
    if ((rc = launch_coop(kclu, gclu, args, st, kCluster)) != SIMDX_OK) return rc;
    // a large push of the tail (the densest core's level) back on the plain grid
    if ((rc = prepare_resume(g, st)) != SIMDX_OK) return rc;
    a.split = 0;
    a.resume = 2;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    *launches = 3;
    return SIMDX_OK;
  }
  a.k.small = 0;  // off, or no cluster fits: the grid runs every step
  if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
  *launches = 1;
  return SIMDX_OK;
}

template <class OffT>
static int run_coreness(simdx_graph* g, uint32_t* core, simdx_stats* stats, cudaStream_t st) {
  int launches = 0;
  const int rc = launch_coreness<OffT>(g, core, st, &launches);
  return rc ? rc : finish_launch(g, stats, st, launches);
}

// ---------------------------------------------------------------- k-core batch
// The k-core of every k in one list from one decomposition: v is in the
// k-core exactly when coreness(v) >= k, and its degree inside the k-core
// counts the neighbours u with min(coreness(u), coreness(v)) >= k.  A warp
// takes 32 consecutive vertices one after another, streams each one's
// edges, and for every edge finds how many of the (sorted) k values
// min(coreness(u), coreness(v)) reaches; one ballot per k value counts them
// for all 32 edges of a round.  The counts go to shared memory and leave as
// coalesced rows, one per k.
constexpr int kKcoreBatchMax = 64;
constexpr long long kKcoreRowsHeavy = 128;  // vertices of more edges are counted by a whole CTA

struct KcoreRows {
  uint32_t ks[kKcoreBatchMax];   // ascending
  int32_t row[kKcoreBatchMax];   // the caller's row of ks[i]
  int nk;
};

template <class OffT>
__global__ void __launch_bounds__(kThreads) kcore_rows_kernel(int n, const OffT* off, const int32_t* idx,
                                                             const uint32_t* core, const KcoreRows q,
                                                             uint8_t* in_core, uint32_t* resid) {
  extern __shared__ uint32_t s_cnt[];  // [warp][k][32 vertices]
  __shared__ uint32_t ks[kKcoreBatchMax];
  const int nk = q.nk;
  for (int i = threadIdx.x; i < nk; i += kThreads) ks[i] = q.ks[i];
  __syncthreads();
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* cntw = s_cnt + (size_t)warp * nk * 32;
  const long long tiles = ((long long)n + 31) / 32;
  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < tiles; tile += (long long)gridDim.x * kWarps) {
    const long long base = tile * 32;
    const int nv = (int)((long long)n - base < 32 ? (long long)n - base : 32);
    for (int vi = 0; vi < nv; ++vi) {
      const long long v = base + vi;
      const uint32_t cv = __ldg(core + v);
      uint32_t c0 = 0, c1 = 0;  // counts of k values lane and lane + 32
      const long long b = (long long)__ldg(off + v), e = (long long)__ldg(off + v + 1);
      if (cv >= ks[0] && resid && e - b <= kKcoreRowsHeavy) {  // in some core: count its neighbours in each
        int nkv = 0;  // the k values this vertex's core reaches (the others count nothing)
        while (nkv < nk && ks[nkv] <= cv) ++nkv;
        for (long long p0 = b; p0 < e; p0 += 32) {
          const long long p = p0 + lane;
          int j = 0;  // k values reached by this edge
          if (p < e) {
            const uint32_t cu = __ldg(core + __ldg(idx + p));
            const uint32_t m = cu < cv ? cu : cv;
            int lo = 0, hi = nk;  // first i with ks[i] > m
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (ks[mid] <= m) lo = mid + 1;
              else hi = mid;
            }
            j = lo;
          }
          for (int i = 0; i < nkv; ++i) {
            const unsigned c = (unsigned)__popc(__ballot_sync(kFull, j > i));
            if (lane == (i & 31)) {
              if (i < 32) c0 += c;
              else c1 += c;
            }
          }
        }
      }
      if (lane < nk) cntw[lane * 32 + vi] = c0;
      if (lane + 32 < nk) cntw[(lane + 32) * 32 + vi] = c1;
    }
    __syncwarp();
    const long long vl = base + lane;
    const bool heavy = lane < nv && resid &&
                       (long long)__ldg(off + vl + 1) - (long long)__ldg(off + vl) > kKcoreRowsHeavy;
    if (lane < nv && !heavy) {  // a heavy vertex's rows come from kcore_rows_heavy_kernel
      const long long v = vl;
      const uint32_t cv = __ldg(core + v);
      for (int i = 0; i < nk; ++i) {
        const bool inc = cv >= ks[i];
        const size_t at = (size_t)q.row[i] * (size_t)n + (size_t)v;
        in_core[at] = inc ? 1 : 0;
        if (resid) resid[at] = inc ? cntw[i * 32 + lane] : 0u;
      }
    }
    __syncwarp();
  }
}

// The vertices of more than kKcoreRowsHeavy edges, one CTA each: every
// thread takes edges, finds how many k values min(coreness(u),
// coreness(v)) reaches, and adds one to that bin of a shared histogram
// (one atomic per distinct bin of a warp); the counts of k value i are the
// bins above i.
template <class OffT>
__global__ void __launch_bounds__(kThreads) kcore_rows_heavy_kernel(int n, const OffT* off, const int32_t* idx,
                                                                   const uint32_t* core, const KcoreRows q,
                                                                   uint8_t* in_core, uint32_t* resid) {
  __shared__ uint32_t ks[kKcoreBatchMax];
  __shared__ unsigned hist[kKcoreBatchMax + 1];
  __shared__ int heavy[kThreads];
  __shared__ int nheavy;
  const int nk = q.nk;
  for (int i = threadIdx.x; i < nk; i += kThreads) ks[i] = q.ks[i];
  const int lane = lane_id();
  // vertex v goes to CTA v % grid: the hubs, low ids in a power-law graph
  // without relabelling, spread over the CTAs
  const long long per = ((long long)n + gridDim.x - 1) / gridDim.x;
  for (long long c0 = 0; c0 < per; c0 += kThreads) {
    if (threadIdx.x == 0) nheavy = 0;
    __syncthreads();
    const long long v = (c0 + threadIdx.x) * (long long)gridDim.x + blockIdx.x;
    if (c0 + threadIdx.x < per && v < n && (long long)__ldg(off + v + 1) - (long long)__ldg(off + v) > kKcoreRowsHeavy)
      heavy[atomicAdd(&nheavy, 1)] = (int)v;
    __syncthreads();
    const int nh = nheavy;
    for (int h = 0; h < nh; ++h) {
      const int hv = heavy[h];
      const uint32_t cv = __ldg(core + hv);
      for (int i = threadIdx.x; i <= nk; i += kThreads) hist[i] = 0;
      __syncthreads();
      if (cv >= ks[0]) {
        const long long b = (long long)__ldg(off + hv), e = (long long)__ldg(off + hv + 1);
        constexpr int kPer = 4;  // edges per thread in flight
        for (long long p0 = b; p0 < e; p0 += (long long)kThreads * kPer) {
          uint32_t cu[kPer];
#pragma unroll
          for (int q = 0; q < kPer; ++q) {
            const long long p = p0 + (long long)q * kThreads + threadIdx.x;
            cu[q] = p < e ? __ldg(core + __ldg(idx + p)) : 0u;
          }
#pragma unroll
          for (int q = 0; q < kPer; ++q) {
            const long long p = p0 + (long long)q * kThreads + threadIdx.x;
            int j = -1;
            if (p < e) {
              const uint32_t m = cu[q] < cv ? cu[q] : cv;
              int lo = 0, hi = nk;
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ks[mid] <= m) lo = mid + 1;
                else hi = mid;
              }
              j = lo;
            }
            const unsigned peers = __match_any_sync(kFull, j);
            if (j >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[j], (unsigned)__popc(peers));
          }
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nk; i += kThreads) {
        const bool inc = cv >= ks[i];
        unsigned c = 0;
        for (int t = i + 1; t <= nk; ++t) c += hist[t];
        const size_t at = (size_t)q.row[i] * (size_t)n + (size_t)hv;
        in_core[at] = inc ? 1 : 0;
        resid[at] = inc ? c : 0u;
      }
      __syncthreads();
    }
  }
}

template <class OffT>
static int run_kcore_batch(simdx_graph* g, const uint32_t* ks, int nk, uint8_t* in_core, uint32_t* resid,
                           simdx_stats* stats, cudaStream_t st) {
  // the decomposition's output lives in the spare fifth of the algorithm
  // state (the peeling uses four n-word arrays)
  uint32_t* core = reinterpret_cast<uint32_t*>(g->state) + 4 * (size_t)g->n;
  int launches = 0;
  int rc = launch_coreness<OffT>(g, core, st, &launches);
  if (rc) return rc;
  KcoreRows q{};
  q.nk = nk;
  for (int i = 0; i < nk; ++i) {
    q.ks[i] = ks[i];
    q.row[i] = i;
  }
  for (int i = 1; i < nk; ++i)  // insertion sort of (k, row) by k
    for (int j = i; j > 0 && q.ks[j - 1] > q.ks[j]; --j) {
      std::swap(q.ks[j - 1], q.ks[j]);
      std::swap(q.row[j - 1], q.row[j]);
    }
  const void* kern = (const void*)kcore_rows_kernel<OffT>;
  const size_t smem = sizeof(uint32_t) * (size_t)kWarps * (size_t)nk * 32;
  // the largest row buffer, allowed once per device (not a stream
  // operation, so a call inside a stream capture does not repeat it)
  {
    static std::mutex mu;
    static std::set<int> allowed;
    int dev = 0;
    SIMDX_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!allowed.count(dev)) {
      SIMDX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(uint32_t) * kWarps * kKcoreBatchMax * 32)));
      allowed.insert(dev);
    }
  }
  const long long tiles = ((long long)g->n + 31) / 32;
  const long long blocks = (tiles + kWarps - 1) / kWarps;
  const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
  kcore_rows_kernel<OffT><<<grid, kThreads, smem, st>>>((int)g->n, (const OffT*)g->off, g->idx, core, q, in_core,
                                                       resid);
  SIMDX_CUDA(cudaGetLastError());
  if (!resid) return finish_launch(g, stats, st, launches + 1);
  const long long hb = ((long long)g->n + kThreads - 1) / kThreads;
  kcore_rows_heavy_kernel<OffT><<<(unsigned)(hb < 1216 ? hb : 1216), kThreads, 0, st>>>(
      (int)g->n, (const OffT*)g->off, g->idx, core, q, in_core, resid);
  SIMDX_CUDA(cudaGetLastError());
  return finish_launch(g, stats, st, launches + 2);
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

extern "C" int simdx_kcore_batch(simdx_graph* g, const uint32_t* ks, int32_t nk, uint8_t* in_core,
                                 uint32_t* residual_deg, simdx_stats* stats, void* stream) {
  if (!g || !ks || !in_core || !g->symmetric || nk < 1 || nk > kKcoreBatchMax) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    int rc = prepare_launch(g, st);
    return rc ? rc : finish_launch(g, stats, st);
  }
  return g->off_bits == 32 ? run_kcore_batch<int32_t>(g, ks, nk, in_core, residual_deg, stats, st)
                           : run_kcore_batch<long long>(g, ks, nk, in_core, residual_deg, stats, st);
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
