// sssp.cu -- SSSP as one persistent ACC kernel (Sec. 2.1; Sec. 3.3 uses
// SSSP as its running example; aggregation combine = min, Sec. 3.2).
//
// Active(v)  : v's distance changed since its out-edges were last relaxed
//              (Sec. 3.2, "Active": metadata differs from the prior
//              iteration).  pdist[v] holds the distance v's edges were last
//              relaxed with, so "active" is dist[v] < pdist[v].
// Delta-step : only active vertices below the bucket bound T are processed
//              (Sec. 3.3, delta-step); when none is left, T advances by delta
//              (or jumps to the bucket of the smallest pending distance).
// Compute    : push: offer dist[v] + w(v,u) to every out-neighbour u.
// Combine    : min.  In push the min lands with one atomicMin per improving
//              edge (the one atomic of the path; Sec. 3.2 gives no
//              atomic-free scheme for scattered aggregation).  Improved
//              vertices below T go to the online-filter bins; every improved
//              vertex gets its pending flag set (a plain byte store).  A
//              dense iteration (task lists holding over 1/16 of the edges)
//              lands its improvements only, with no flags or records.
// Task lists : online filter; on overflow the ballot filter rebuilds sorted
//              lists from {pending and dist < pdist and dist < T}; after a
//              dense iteration it scans dist < pdist over every vertex and
//              flags the ones it leaves for a later bucket.
// Grid class : a very-high-degree task is relaxed by all CTAs; they agree on
//              one source distance through a per-entry "first reader wins"
//              word, so pdist records a distance every slice really used.
#include <type_traits>

#include "acc_cluster.cuh"
#include "simdx_internal.h"

namespace simdx {

// With V (a batch of k SSSP queries) the kernel runs on k virtual copies of
// the graph: task / state id x = inst * nreal + v, inst = x / nreal; every
// copy walks the one CSR, and copy inst starts at srcs[inst].
template <class OffT>
struct SsspArgs {
  int n, src;           // n: state ids (nreal, or k * nreal for a batch)
  int nreal, ninst;
  const int32_t* srcs;  // device [ninst] (batch of more than 64 only)
  int32_t src_list[64]; // the sources of a batch of up to 64, as a kernel parameter (no copy to stage)
  const OffT* off;
  const int32_t* idx;
  const uint32_t* wt;
  uint32_t* dist;
  Work w;
  Knobs k;
};

// With W (connected components) the relaxed value is the neighbour's label
// itself: no weight is read.
template <class OffT, bool V, bool W = false>
struct SsspPush {
  struct Src {
    uint32_t d;
    int base;  // inst * nreal: state id of the task's graph copy
  };
  int nreal;
  uint32_t* dist;
  uint32_t* pdist;
  uint8_t* pend;
  const OffT* off;
  const uint32_t* wt;
  uint32_t* aux3;
  unsigned long long T;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  bool dense = false;  // land improvements only: no pending flags, no records
  bool plain = false;  // combine by plain stores (no atomics); sweeps verify the result
  unsigned long long nrec = 0, mrec = 0;
  __device__ SsspPush(const SsspArgs<OffT>& a, uint32_t* pd, uint8_t* pe, uint32_t* ax, unsigned long long t,
                      CtaShared& s, unsigned g)
      : nreal(a.nreal), dist(a.dist), pdist(pd), pend(pe), off(a.off), wt(a.wt), aux3(ax), T(t), sh(s), w(a.w),
        k(a.k), grid(g) {}
  __device__ __forceinline__ int base_of(int x) const { return V ? (int)(((unsigned)x / (unsigned)nreal) * nreal) : 0; }
  __device__ __forceinline__ int rv(int x) const { return V ? x - base_of(x) : x; }

  // Decide once per task whether v still needs relaxing and with what d.
  __device__ __forceinline__ bool claim(int v, uint32_t& d) {
    d = dist[v];
    if (d >= pdist[v]) return false;  // already relaxed with this or a better distance
    pdist[v] = d;
    return true;
  }
  __device__ __forceinline__ bool src(int v, Src& s, int cls, unsigned item) {
    s.base = base_of(v);
    if (cls == 0) return claim(v, s.d);
    if (cls == 1) {
      uint32_t d = 0;
      int go = 0;
      if (lane_id() == 0) go = claim(v, d);
      go = __shfl_sync(kFull, go, 0);
      s.d = __shfl_sync(kFull, d, 0);
      return go != 0;
    }
    if (cls == 2) {
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t d = 0;
        sh.bcast_i[0] = claim(v, d);
        sh.bcast_i[1] = (int)d;
      }
      __syncthreads();
      s.d = (uint32_t)sh.bcast_i[1];
      return sh.bcast_i[0] != 0;
    }
    // cls 3: all CTAs relax slices of v; the first CTA to look fixes d.
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t mine = dist[v];
      uint32_t old = atomicCAS(&aux3[item], 0xffffffffu, mine);
      uint32_t d = (old == 0xffffffffu) ? mine : old;
      if (d < pdist[v]) pdist[v] = d;  // benign: every CTA stores the agreed d
      sh.bcast_i[1] = (int)d;
    }
    __syncthreads();
    s.d = (uint32_t)sh.bcast_i[1];
    return true;
  }
  static __device__ __forceinline__ Src shfl(const Src& s, int l) {
    Src r;
    r.d = __shfl_sync(kFull, s.d, l);
    r.base = V ? __shfl_sync(kFull, s.base, l) : 0;
    return r;
  }
  // Weights and current distances of all the lane's edges are loaded first,
  // then the improving ones land with atomicMin (issued back to back), then
  // the improved vertices are flagged and recorded.
  __device__ __forceinline__ void edges(const Src (&s)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&p)[kPushBatch],
                                        unsigned ok) {
    unsigned long long nd[kPushBatch];
    uint32_t cur[kPushBatch];
    int x[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      nd[q] = ~0ull;
      cur[q] = 0;
      x[q] = s[q].base + u[q];
      if ((ok >> q) & 1u) {
        nd[q] = (unsigned long long)s[q].d + (W ? 0u : gload(wt + p[q]));
        cur[q] = dist[x[q]];
      }
    }
    if (dense) {
      // fire-and-forget min; the next filter finds the improved vertices by
      // scanning dist < pdist
#pragma unroll
      for (int q = 0; q < kPushBatch; ++q)
        if (nd[q] < cur[q]) {
          if (plain) dist[x[q]] = (uint32_t)nd[q];
          else atomicMin(&dist[x[q]], (uint32_t)nd[q]);
        }
      return;
    }
    uint32_t old[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      old[q] = 0;
      if (nd[q] < cur[q]) {
        if (plain) {
          // a racing smaller store may be overwritten: the sweeps at the end
          // find every distance left too large
          dist[x[q]] = (uint32_t)nd[q];
          old[q] = cur[q];
        } else {
          old[q] = atomicMin(&dist[x[q]], (uint32_t)nd[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      if (nd[q] < cur[q] && nd[q] < old[q]) {
        pend[x[q]] = 1;
        if (nd[q] < T) {
          long long d = (long long)gload(off + u[q] + 1) - (long long)gload(off + u[q]);
          ++nrec;
          mrec += (unsigned long long)d;
          online_record(x[q], degree_class(d, k), sh, w, k, grid);
        }
      }
    }
  }
};

// Pull (Sec. 5: SSSP pushes in the first and last iterations and pulls in
// between): every vertex with an in-edge takes the min of pdist[v] + w over
// its in-neighbours v on the frontier (bitmap `fbm`, pdist = the distance v
// was claimed with) and, the owner, lowers its own distance -- min combine,
// no atomics.  Symmetric graphs only (the in-edge weight is the CSR weight).
template <class OffT>
struct SsspPull {
  using Acc = unsigned;
  const uint32_t* fbm;
  const uint32_t* pdist;
  const uint32_t* wt;
  uint32_t* dist;
  uint8_t* pend;
  const OffT* off;
  unsigned long long T;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ SsspPull(const uint32_t* fb, const uint32_t* pd, const uint32_t* wts, uint32_t* d, uint8_t* pe,
                      const OffT* o, unsigned long long t, CtaShared& s, const Work& ww, const Knobs& kk, unsigned g)
      : fbm(fb), pdist(pd), wt(wts), dist(d), pend(pe), off(o), T(t), sh(s), w(ww), k(kk), grid(g) {}
  __device__ __forceinline__ Acc zero() const { return 0xffffffffu; }
  __device__ __forceinline__ void combine(Acc& a, Acc b) const { a = b < a ? b : a; }
  __device__ __forceinline__ void edge(Acc& a, int, int v, long long p) {
    if ((fbm[v >> 5] >> (v & 31)) & 1u) {
      const unsigned long long c = (unsigned long long)pdist[v] + gload(wt + p);
      if (c < a) a = (unsigned)c;
    }
  }
  __device__ __forceinline__ void finish(int u, Acc best) {
    if (best < dist[u]) {
      dist[u] = best;
      pend[u] = 1;
      if ((unsigned long long)best < T) {
        const long long d = (long long)gload(off + u + 1) - (long long)gload(off + u);
        ++nrec;
        mrec += (unsigned long long)d;
        online_record(u, degree_class(d, k), sh, w, k, grid);
      }
    }
  }
};

// Verification sweep of the atomic-free combine (scope reading: plain-store
// min in push, then pull sweeps until no distance drops): every vertex with
// an in-edge takes the min of dist[v] + w over all its in-neighbours and, the
// owner, lowers its own distance (owner writes, no atomics).  A vertex it
// lowers becomes pending, so its out-edges are pushed again.  When a sweep
// lowers nothing, dist[u] <= dist[v] + w holds on every edge: the distances
// are the shortest.  Symmetric graphs (in-edge weight = CSR weight).
template <class OffT>
struct SsspVerify {
  using Acc = unsigned;
  const uint32_t* wt;
  uint32_t* dist;
  uint8_t* pend;
  unsigned long long changed = 0;
  __device__ __forceinline__ Acc zero() const { return 0xffffffffu; }
  __device__ __forceinline__ void combine(Acc& a, Acc b) const { a = b < a ? b : a; }
  __device__ __forceinline__ void edge(Acc& a, int, int v, long long p) {
    const uint32_t dv = dist[v];
    if (dv != 0xffffffffu) {
      const unsigned long long c = (unsigned long long)dv + gload(wt + p);
      if (c < a) a = (unsigned)c;
    }
  }
  __device__ __forceinline__ void finish(int u, Acc best) {
    if (best < dist[u]) {
      dist[u] = best;
      pend[u] = 1;
      ++changed;
    }
  }
};

// A push iteration whose task lists hold more than 1/kDenseDiv of all edges
// is dense: most of its improvements would be recorded, and one scan of
// dist < pdist over all vertices costs less than recording them.
constexpr unsigned long long kDenseDiv = 16;

// With W the kernel computes weakly connected components (Sec. 3.2 lists
// WCC with the voting algorithms).  A BFS from a highest-degree vertex,
// launched just before, left its levels in `dist`: the vertices it reached
// form one component and take its smallest id as their final label (every
// vote for them is the same).  The other vertices start with their own id
// and propagate the minimum (relaxations add no weight, no buckets), so the
// fixed point labels each component with its smallest id.
// Loop state words of the resume record (Resume::v) for a run with one
// launch per iteration.
enum { kRsT, kRsLbuf, kRsCnt0, kRsListsOk = kRsCnt0 + kClasses, kRsMf, kRsScanAll, kRsIt, kRsBallotIt,
       kRsOnlineIt, kRsPullIt, kRsFsum, kRsPhases };
static_assert(kRsPhases < kResumeWords, "resume record too small");

// SPLIT: the no-fusion instantiation, which stops after one iteration and
// leaves its loop state in the resume record for the next launch.
// VERIFY: the atomic-free combine (plain-store min in push, then pull
// sweeps until no distance drops).
// STAGE: CTA-class push ranges staged in shared memory by bulk copy.
// ------------------------------------------------ small frontiers
// While the frontier below the bucket bound is small (at most kLocEnterN
// vertices and kLocEnterM edges), the push iterations of a single-source
// run go to the first thread-block cluster (acc_cluster.cuh).  An entry
// carries the vertex, the distance it was improved to and its edge range.
// A walk claims the entry (atomicMin on pdist: relaxed with this distance
// or a better one already, skip) while the edge targets and weights load,
// then lands each offer with atomicMin, the target's offsets loaded
// alongside; an improved target gets its pending flag, and joins the next
// frontier when it is below the bound.  The cluster hands back when the
// frontier below the bound is exhausted (the grid advances the bucket) or
// grows (the grid lists the pending vertices by the ballot filter).
struct SsspLocalShared : LocalShared {
  unsigned long long g[2][kLocCap];  // (vertex << 32) | the distance it was appended with
};

enum { kScIt, kScOnlineIt, kScFsum, kScN, kScM, kScBeat = 15 };

// Appends each lane's claimed entry (kLocClaim set on the range word) with
// its vertex word: one shared atomic per warp.
__device__ __forceinline__ void loc_append2(SsspLocalShared& ls, int buf, int sl, unsigned long long ent,
                                            unsigned long long vw) {
  const bool mine = (ent & kLocClaim) != 0;
  const unsigned mk = __ballot_sync(kFull, mine);
  if (mk == 0) return;
  const int leader = __ffs(mk) - 1;
  unsigned base = 0;
  if (lane_id() == leader) base = atomicAdd(&ls.cnt[sl], (unsigned)__popc(mk));
  base = __shfl_sync(kFull, base, leader);
  if (mine) {
    const unsigned pos = base + (unsigned)__popc(mk & lanemask_lt());
    if (pos < (unsigned)kLocCap) {
      ls.f[buf][pos] = ent & ~kLocClaim;
      ls.g[buf][pos] = vw;
    } else {
      ls.ovf[sl] = 1;
    }
  }
}

template <class OffT>
__device__ bool sssp_local(const SsspArgs<OffT>& a, SsspLocalShared& ls, CtaShared& sh, uint32_t* pdist,
                           uint8_t* pend, const unsigned* cnt, int lbuf, unsigned long long T, int& it, int& online_it,
                           long long& fsum, long long& evisit, unsigned long long& episodes, unsigned long long& n_out,
                           unsigned long long& m_out) {
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  if (blockIdx.x < kCluster) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned r = cl.block_rank();
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x < 3) loc_clear(ls, threadIdx.x);
    if (threadIdx.x == 0) ls.stop = 0;
    __syncthreads();
    // the current frontier: the class lists' entries j with j % kCluster == r
    unsigned base = 0;
    for (int c = 0; c < kClasses; ++c) {
      const int32_t* list = a.w.list[lbuf][c];
      for (unsigned i = threadIdx.x; i < cnt[c]; i += kThreads)
        if ((base + i) % kCluster == r) {
          const int v = list[i];
          const long long b0 = (long long)gload(a.off + v);
          const unsigned pos = atomicAdd(&ls.cnt[0], 1u);
          ls.f[0][pos] = loc_pack(b0, (long long)gload(a.off + v + 1) - b0);
          ls.g[0][pos] = ((unsigned long long)(unsigned)v << 32) | __ldcg(a.dist + v);
        }
      base += cnt[c];
    }
    loc_publish(cl, ls, 0, r);
    cl.sync();
    unsigned cc, cp, zc, zp;
    unsigned N = loc_counts(ls, 0, cc, cp, zc, zp).n;
    unsigned long long M = 0;
    int cur = 0, fc = 0;
    unsigned long long t_it = trace_clock();
    while (true) {
      const int nx = cur == 2 ? 0 : cur + 1, nn = nx == 2 ? 0 : nx + 1;
      const long long c_it = clock64();
      unsigned ab = 0;
      if (threadIdx.x == 0) {
        loc_clear(ls, nn);
        if (r == 0) {
          ab = (unsigned)ld_volatile_i32(&s->abort);
          if (blockIdx.x == 0) *(volatile long long*)&s->loc[kScBeat] = it;  // progress for the waiting CTAs
        }
      }
      const unsigned lo = (unsigned)(((unsigned long long)N * r) / kCluster);
      const unsigned myc = (unsigned)(((unsigned long long)N * (r + 1)) / kCluster) - lo;
      unsigned long long mrec = 0;
      unsigned gs = (myc + kWarps - 1) / kWarps;
      gs = gs < 1 ? 1 : (gs > 64 ? 64 : gs);
      for (unsigned b = (unsigned)warp * gs; b < myc; b += (unsigned)kWarps * gs) {
        const unsigned lim = b + gs < myc ? b + gs : myc;
        const unsigned i0 = b + lane, i1 = b + 32 + lane;
        const unsigned g0 = lo + (i0 < lim ? i0 : 0), g1 = lo + (i1 < lim ? i1 : 0);
        const int t0 = loc_owner(cp, g0), t1 = loc_owner(cp, g1);
        const unsigned p0 = __shfl_sync(kFull, cp, t0), p1 = __shfl_sync(kFull, cp, t1);
        unsigned long long e0 = 0, e1 = 0, y0 = 0, y1 = 0;
        if (i0 < lim) {
          const SsspLocalShared* o = cl.map_shared_rank(&ls, (unsigned)t0);
          e0 = o->f[fc][g0 - p0];
          y0 = o->g[fc][g0 - p0];
        }
        if (i1 < lim) {
          const SsspLocalShared* o = cl.map_shared_rank(&ls, (unsigned)t1);
          e1 = o->f[fc][g1 - p1];
          y1 = o->g[fc][g1 - p1];
        }
        // claim: relaxed with this distance or a better one already, skip
        // (the result is used only when the offers land)
        const unsigned nd0 = (unsigned)y0, nd1 = (unsigned)y1;
        unsigned old0 = 0, old1 = 0;
        if (i0 < lim) old0 = atomicMin(pdist + (int)(y0 >> 32), nd0);
        if (i1 < lim) old1 = atomicMin(pdist + (int)(y1 >> 32), nd1);
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
          unsigned long long nd[kLocBatch];
#pragma unroll
          for (int q = 0; q < kLocBatch; ++q) {
            const int j = q0 + 32 * q + lane;
            bool hi;
            const int t = loc_find(ia, ib, ta, j < total ? j : total - 1, hi);
            const long long s0 = __shfl_sync(kFull, b0, t), s1 = __shfl_sync(kFull, b1, t);
            const int x0 = __shfl_sync(kFull, ia - d0, t), x1 = __shfl_sync(kFull, ib - d1, t);
            const unsigned n0 = __shfl_sync(kFull, nd0, t), n1 = __shfl_sync(kFull, nd1, t);
            const unsigned o0 = __shfl_sync(kFull, old0, t), o1 = __shfl_sync(kFull, old1, t);
            const long long bj = hi ? s1 : s0;
            const int ej = hi ? x1 : x0;
            const unsigned dj = hi ? n1 : n0;
            const bool ok = (hi ? o1 : o0) > dj;  // this entry's claim held
            u[q] = -1;
            nd[q] = ~0ull;
            if (j < total && ok) {
              u[q] = gload(a.idx + bj + (j - ej));
              nd[q] = (unsigned long long)dj + gload(a.wt + bj + (j - ej));
            }
          }
          unsigned long long ent[kLocBatch], vw[kLocBatch];
#pragma unroll
          for (int q = 0; q < kLocBatch; ++q) {
            ent[q] = 0;
            vw[q] = 0;
            if (u[q] >= 0 && nd[q] < 0xffffffffull) {
              const unsigned old = atomicMin(a.dist + u[q], (unsigned)nd[q]);
              const long long ob = (long long)gload(a.off + u[q]);
              const long long oe = (long long)gload(a.off + u[q] + 1);
              if (nd[q] < old) {
                pend[u[q]] = 1;
                if (nd[q] < T) {
                  mrec += (unsigned long long)(oe - ob);
                  ent[q] = loc_pack(ob, oe - ob) | kLocClaim;
                  vw[q] = ((unsigned long long)(unsigned)u[q] << 32) | nd[q];
                }
              }
            }
          }
#pragma unroll
          for (int q = 0; q < kLocBatch; ++q) loc_append2(ls, fc ^ 1, nx, ent[q], vw[q]);
        }
        evisit += d0 + d1;
      }
      mrec = warp_sum_u64(mrec);
      if (lane == 0 && mrec) atomicAdd(&ls.medges[nx], mrec);
      if (threadIdx.x == 0 && r == 0) ls.stop = ab;
      const long long c_walk = clock64();
      loc_publish(cl, ls, nx, r, (unsigned)(c_walk - c_it));
      cl.sync();
      const long long c_bar = clock64();
      const LocTotals Tt = loc_counts(ls, nx, cc, cp, zc, zp);
      const unsigned long long t_end = trace_clock();
      trace_put(a.w, it, 1 | (1 << 8) | (1 << 19), (long long)N, (long long)Tt.m,
                (long long)(T == ~0ull ? -1 : (long long)T), t_it, t_end);
      if (blockIdx.x == 0 && threadIdx.x == 0 && it < a.w.trace_cap) {
        a.w.trace[(long long)kTraceWords * it + 6] = (long long)Tt.walk;  // the slowest CTA's walk (SM cycles)
        a.w.trace[(long long)kTraceWords * it + 7] = c_bar - c_walk;     // CTA 0's publication and barrier
      }
      t_it = t_end;
      fsum += (long long)N;
      ++it;
      ++online_it;
      N = Tt.n;
      M = Tt.m;
      if (N == 0 || Tt.ovf || Tt.stop || N > kLocExitN || M > kLocEnterM) break;
      cur = nx;
      fc ^= 1;
    }
    cl.sync();  // no CTA leaves while another still reads its shared memory
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      long long* w = s->loc;
      w[kScIt] = it; w[kScOnlineIt] = online_it; w[kScFsum] = fsum; w[kScN] = N; w[kScM] = (long long)M;
      red_release_add_u64(&s->loc_epoch, 1ull);
    }
  }
  if (!loc_wait_handback(s, k, sh, &s->loc_epoch, &s->loc[kScBeat], episodes)) return false;
  ++episodes;
  const volatile long long* w = s->loc;
  it = (int)w[kScIt]; online_it = (int)w[kScOnlineIt]; fsum = w[kScFsum];
  n_out = (unsigned long long)w[kScN];
  m_out = (unsigned long long)w[kScM];
  return true;
}

// CLU: small push frontiers of a single-source run go to the first
// thread-block cluster (the small_frontier knob; launched in clusters).
template <class OffT, bool V, bool PULL, bool W = false, bool SPLIT = false, bool VERIFY = false, bool STAGE = false,
          bool CLU = false>
__global__ void __launch_bounds__(kThreads, 4) sssp_kernel(const __grid_constant__ SsspArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ typename std::conditional<CLU, SsspLocalShared, char>::type loc_sm;
  __shared__ unsigned red_u[kWarps];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  uint32_t* pdist = reinterpret_cast<uint32_t*>(a.w.state);
  uint8_t* pend = reinterpret_cast<uint8_t*>(pdist + n);
  const unsigned long long delta = (W || !k.delta) ? 0ull : k.delta;
  const unsigned long long kInfT = ~0ull;
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();
  const bool resumed = SPLIT && ld_volatile_i32(&s->rs.active) != 0;
  Stager stg{nullptr, s, (long long)(gload(a.off + a.nreal) - gload(a.off))};
  if constexpr (STAGE) {
    __shared__ StageShared stage_sm;
    stage_init(stage_sm);
    if ((reinterpret_cast<uintptr_t>(a.idx) & 15) == 0) stg.sm = &stage_sm;
  }

  const unsigned nreal = (unsigned)a.nreal;
  // state id -> vertex of the one CSR
  auto realv = [nreal](long long x) { return V ? (int)((unsigned long long)x % nreal) : (int)x; };
  // ---- phase 0: reset state, seed the source(s)
  if (W) {
    unsigned long long mn = ~0ull;  // smallest id the BFS reached (this thread's first)
    for (long long x = gtid; x < n; x += gthreads)
      if ((int)a.dist[x] >= 0) {
        mn = (unsigned long long)x;
        break;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(kFull, mn, o);
      mn = y < mn ? y : mn;
    }
    if (lane_id() == 0) sh.red64[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = ~0ull;
      for (int q = 0; q < kWarps; ++q) t = sh.red64[q] < t ? sh.red64[q] : t;
      if (t != ~0ull) atomicMax(&s->slot[slot_of(sh.phase)].aux2, ~t);  // slots start at 0
    }
    clear_next_slot(s, sh);
    if (!grid_sync(s, grid, sh, k)) return;
    const uint32_t lab0 = (uint32_t)~s->slot[slot_of(sh.phase - 1)].aux2;
    for (long long x = gtid; x < n; x += gthreads) {
      const bool reached = (int)a.dist[x] >= 0;
      const uint32_t l = reached ? lab0 : (uint32_t)x;
      const bool edges = gload(a.off + x + 1) != gload(a.off + x);
      a.dist[x] = l;
      pdist[x] = (reached || !edges) ? l : 0xffffffffu;  // final unless it still has to push
      pend[x] = (!reached && edges) ? 1 : 0;
    }
  }
  for (long long x = gtid; !W && !resumed && x < n; x += gthreads) {
    bool is_src;
    if (V) {
      const long long inst = x / nreal;
      is_src = (x - inst * nreal) == (a.ninst <= 64 ? a.src_list[inst] : a.srcs[inst]);
    } else {
      is_src = x == a.src;
    }
    a.dist[x] = is_src ? 0u : 0xffffffffu;
    pdist[x] = 0xffffffffu;
    pend[x] = is_src ? 1 : 0;  // the source is the first pending vertex
  }
  if (PULL && !resumed)  // pull frontiers (BFS leaves these bitmaps as it likes)
    for (long long q = gtid; q < (((long long)n + 31) >> 5); q += gthreads) {
      a.w.bm_f[0][q] = 0u;
      a.w.bm_f[1][q] = 0u;
    }
  if (!W && !resumed && blockIdx.x == 0) {
    const int nsrc = V ? a.ninst : 1;
    for (int i = threadIdx.x; i < nsrc; i += kThreads) {
      const int v = V ? (a.ninst <= 64 ? a.src_list[i] : a.srcs[i]) : a.src;
      long long d = (long long)a.off[v + 1] - (long long)a.off[v];
      int c = degree_class(d, k);
      const unsigned pos = atomicAdd(&s->slot[0].list_cnt[c], 1u);
      a.w.list[0][c][pos] = V ? i * (int)nreal + v : v;
      if (c == 3) a.w.aux3[0][pos] = 0xffffffffu;
    }
  }
  if (!resumed) {
    clear_next_slot(s, sh);
    if (!grid_sync(s, grid, sh, k)) return;
  }

  unsigned long long T = delta ? delta : kInfT;  // bucket bound: process dist < T
  int lbuf = 0;
  unsigned cnt[kClasses];
  bool lists_ok = !W;  // W: the first filter lists the pending vertices
  {
    const PhaseSlot& p = s->slot[0];
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
  }
  int it = 0, ballot_it = 0, online_it = 0, pull_it = 0;
  long long evisit = 0, fsum = 0;
  int filt = 1;
  // Dense push iterations (frontier edges above 1/kDenseDiv of all edges)
  // only land their improvements; the filter after one scans every vertex.
  const unsigned long long m_all =
      (unsigned long long)(gload(a.off + nreal) - gload(a.off)) * (unsigned long long)(V ? a.ninst : 1);
  unsigned long long mf = 0;  // out-edges of the current task lists
  bool scan_all = false;
  long long phases0 = 0;
  if (resumed) {
    const volatile long long* r = s->rs.v;
    T = (unsigned long long)r[kRsT]; lbuf = (int)r[kRsLbuf];
    for (int c = 0; c < kClasses; ++c) cnt[c] = (unsigned)r[kRsCnt0 + c];
    lists_ok = r[kRsListsOk] != 0; mf = (unsigned long long)r[kRsMf]; scan_all = r[kRsScanAll] != 0;
    it = (int)r[kRsIt]; ballot_it = (int)r[kRsBallotIt]; online_it = (int)r[kRsOnlineIt];
    pull_it = (int)r[kRsPullIt]; fsum = r[kRsFsum]; phases0 = r[kRsPhases];
  }
  const int it_launch = it;
  unsigned long long episodes = 0;  // small-frontier episodes so far

  while (true) {
    if (SPLIT && it > it_launch) {
      // no fusion: the next iteration runs in the next launch
      const unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
      if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long* r = s->rs.v;
        r[kRsT] = (long long)T; r[kRsLbuf] = lbuf;
        for (int c = 0; c < kClasses; ++c) r[kRsCnt0 + c] = cnt[c];
        r[kRsListsOk] = lists_ok; r[kRsMf] = (long long)mf; r[kRsScanAll] = scan_all;
        r[kRsIt] = it; r[kRsBallotIt] = ballot_it; r[kRsOnlineIt] = online_it; r[kRsPullIt] = pull_it;
        r[kRsFsum] = fsum; r[kRsPhases] = phases0 + (long long)sh.phase;
        s->rs.want_dir = PULL ? 2 : 1;
        s->rs.active = 1;
      }
      return;
    }
    const unsigned long long t_it = globaltimer();
    unsigned total = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    filt = 1;
    if (!lists_ok || k.filter == 2 || scan_all) {
      // ballot filter: near active vertices from the metadata (pending
      // flags; after a dense iteration, every vertex)
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      const unsigned long long TT = T;
      uint32_t* dist = a.dist;
      const bool sa = scan_all;
      auto pred = [=](int v) {
        if (!sa && !pend[v]) return false;
        const uint32_t d = dist[v];
        if (d >= pdist[v]) return false;
        if ((unsigned long long)d < TT) return true;
        if (sa) pend[v] = 1;  // improved by the dense iteration, left for a later bucket
        return false;
      };
      unsigned long long msum = 0;
      auto deg = [off = a.off, realv, &msum](int x) {
        const int v = realv(x);
        const long long d = (long long)gload(off + v + 1) - (long long)gload(off + v);
        msum += (unsigned long long)d;
        return d;
      };
      auto visit = [=](int v) { pend[v] = 0; };
      ballot_filter(n, pred, deg, visit, sh, a.w, k, grid, lbuf, slot);
      const unsigned long long tms = cta_sum_u64(msum, sh);
      if (threadIdx.x == 0 && tms) atomicAdd(&slot.mact, tms);
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
      total = cnt[0] + cnt[1] + cnt[2] + cnt[3];
      mf = p.mact;
      lists_ok = true;
      scan_all = false;
      filt = 2;
    }
    if (total == 0) {
      // bucket advance: one scan gives the min pending distance, the pending
      // count and (guessing the next bucket) its task lists
      bool done = false;
      unsigned long long Tn = (T == kInfT) ? kInfT : T + delta;
      for (int attempt = 0; attempt < 2; ++attempt) {
        clear_next_slot(s, sh);
        PhaseSlot& slot = s->slot[slot_of(sh.phase)];
        unsigned long long mymin = ~0ull, mycnt = 0;
        const unsigned long long TT = Tn;
        uint32_t* dist = a.dist;
        auto pred = [&](int v) {
          if (!pend[v]) return false;
          const uint32_t d = dist[v];
          if (d >= pdist[v]) {
            pend[v] = 0;  // stale flag
            return false;
          }
          ++mycnt;
          if (d < mymin) mymin = d;
          return (unsigned long long)d < TT;
        };
        unsigned long long msum = 0;
        auto deg = [off = a.off, realv, &msum](int x) {
          const int v = realv(x);
          const long long d = (long long)gload(off + v + 1) - (long long)gload(off + v);
          msum += (unsigned long long)d;
          return d;
        };
        auto visit = [=](int v) { pend[v] = 0; };
        ballot_filter(n, pred, deg, visit, sh, a.w, k, grid, lbuf, slot);
        const unsigned long long tms = cta_sum_u64(msum, sh);
        if (threadIdx.x == 0 && tms) atomicAdd(&slot.mact, tms);
        unsigned long long c_cnt = cta_sum_u64(mycnt, sh);
        // CTA min
        {
          unsigned long long m = mymin;
          for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = __shfl_xor_sync(kFull, m, o);
            m = y < m ? y : m;
          }
          __syncthreads();
          if (lane_id() == 0) sh.red64[threadIdx.x >> 5] = m;
          __syncthreads();
          if (threadIdx.x == 0) {
            unsigned long long t = ~0ull;
            for (int q = 0; q < kWarps; ++q) t = sh.red64[q] < t ? sh.red64[q] : t;
            if (c_cnt) {
              atomicAdd(&slot.aux1, c_cnt);
              atomicMax(&slot.aux2, ~t);  // slots start at 0: keep the min inverted
            }
          }
        }
        if (!grid_sync(s, grid, sh, k)) return;
        const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
        for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
        total = cnt[0] + cnt[1] + cnt[2] + cnt[3];
        mf = p.mact;
        const unsigned long long pending = p.aux1;
        if (pending == 0) {
          done = true;
          break;
        }
        T = Tn;
        if (total > 0 || delta == 0) break;
        // the guessed bucket was empty: jump to the bucket of the min distance
        const unsigned long long mn = ~p.aux2;
        Tn = delta ? (mn / delta + 1) * delta : kInfT;  // (delta > 0 here)
      }
      if (done) {
        if (!VERIFY) break;
        // atomic-free combine: a pull sweep over every vertex with an
        // in-edge; done when it lowers no distance
        clear_next_slot(s, sh);
        {
          PhaseSlot& slot_c = s->slot[slot_of(sh.phase)];
          auto deg = [off = a.off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
          auto none = [](int) {};
          bitmap_filter(n, a.w.bm_nz, deg, none, sh, a.w, k, grid, lbuf, slot_c);
        }
        if (!grid_sync(s, grid, sh, k)) return;
        unsigned cc[kClasses];
        {
          const PhaseSlot& pc = s->slot[slot_of(sh.phase - 1)];
          for (int c = 0; c < kClasses; ++c) cc[c] = pc.list_cnt[c];
        }
        clear_next_slot(s, sh);
        PhaseSlot& slot_v = s->slot[slot_of(sh.phase)];
        SsspVerify<OffT> fv{a.wt, a.dist, pend};
        const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                          a.w.list[lbuf][3]};
        pull_classes<OffT>(fv, a.off, a.idx, lists, cc, grid, red_u, k.huge_min, sh, a.w, evisit);
        const unsigned long long ch = cta_sum_u64(fv.changed, sh);
        if (threadIdx.x == 0 && ch) atomicAdd(&slot_v.aux0, ch);
        if (!grid_sync(s, grid, sh, k)) return;
        const unsigned long long lowered = s->slot[slot_of(sh.phase - 1)].aux0;
        trace_put(a.w, it, 2 | (2 << 8) | (1 << 18), (long long)(cc[0] + cc[1] + cc[2] + cc[3]),
                  (long long)lowered, (long long)(T == kInfT ? -1 : (long long)T), t_it);
        ++it;
        ++pull_it;
        ++ballot_it;
        if (lowered == 0) break;
        lists_ok = false;  // the lowered vertices are pending: the ballot filter lists them
        continue;
      }
      filt = 2;
      if (total == 0) continue;  // (cannot happen: the jump bucket holds the min)
    }

    // -------- direction: push unless the direction knob forces pull.  A pull
    // iteration sweeps every in-edge (plus two phases to claim the frontier
    // and list the pull tasks); on GB300 that costs more than pushing even
    // the densest frontier of these graphs (R-MAT 20 / 22 / 24, pull in every
    // iteration with more than n / beta frontier vertices for beta 8..64:
    // 1.5-1.8x slower), so the automatic choice is push.
    const bool pull = PULL;  // the pull instantiation runs only when direction forces it
    unsigned long long tn = 0, tm = 0;
    if (pull) {
      uint32_t* fbm = a.w.bm_f[pull_it & 1];
      uint32_t* other = a.w.bm_f[(pull_it & 1) ^ 1];
      // claim the frontier into the bitmap (pdist = the distance relaxed
      // with); clear the other bitmap for the next pull iteration
      clear_next_slot(s, sh);
      for (int c = 0; c < kClasses; ++c) {
        const int32_t* list = a.w.list[lbuf][c];
        for (long long i = gtid; i < cnt[c]; i += gthreads) {
          const int v = list[i];
          const uint32_t d = a.dist[v];
          if (d < pdist[v] && (unsigned long long)d < T) {
            pdist[v] = d;
            atomicOr(&fbm[v >> 5], 1u << (v & 31));
          }
        }
      }
      for (long long q = gtid; q < (((long long)n + 31) >> 5); q += gthreads) other[q] = 0u;
      if (!grid_sync(s, grid, sh, k)) return;
      // the pull tasks: every vertex with an in-edge
      clear_next_slot(s, sh);
      {
        PhaseSlot& slot_c = s->slot[slot_of(sh.phase)];
        auto deg = [off = a.off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
        auto none = [](int) {};
        bitmap_filter(n, a.w.bm_nz, deg, none, sh, a.w, k, grid, lbuf, slot_c);
      }
      if (!grid_sync(s, grid, sh, k)) return;
      unsigned cc[kClasses];
      {
        const PhaseSlot& pc = s->slot[slot_of(sh.phase - 1)];
        for (int c = 0; c < kClasses; ++c) cc[c] = pc.list_cnt[c];
      }
      clear_next_slot(s, sh);
      online_reset(sh);
      __syncthreads();
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      SsspPull<OffT> f(fbm, pdist, a.wt, a.dist, pend, a.off, T, sh, a.w, k, grid);
      const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                        a.w.list[lbuf][3]};
      pull_classes<OffT>(f, a.off, a.idx, lists, cc, grid, red_u, k.huge_min, sh, a.w, evisit);
      online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
      tn = cta_sum_u64(f.nrec, sh);
      tm = cta_sum_u64(f.mrec, sh);
      if (threadIdx.x == 0 && tn) {
        atomicAdd(&slot.nact, tn);
        atomicAdd(&slot.mact, tm);
      }
      ++pull_it;
      ++ballot_it;
    } else {
      if constexpr (CLU) {
        if (k.small && total <= kLocEnterN && mf <= kLocEnterM && mf * kDenseDiv <= m_all) {
          unsigned long long n_out = 0, m_out = 0;
          if (!sssp_local(a, loc_sm, sh, pdist, pend, cnt, lbuf, T, it, online_it, fsum, evisit, episodes, n_out,
                          m_out))
            return;
          // an exhausted bucket hands back empty lists (the grid advances
          // it); a grown frontier is listed again from the pending flags
          lists_ok = n_out == 0;
          for (int c = 0; c < kClasses; ++c) cnt[c] = 0;
          mf = m_out;
          continue;
        }
      }
      // -------- compute: push relaxations from the current task lists
      clear_next_slot(s, sh);
      online_reset(sh);
      __syncthreads();
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      SsspPush<OffT, V, W> f(a, pdist, pend, a.w.aux3[lbuf], T, sh, grid);
      f.plain = VERIFY;
      f.dense = mf * kDenseDiv > m_all;
      scan_all = f.dense;
      const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                        a.w.list[lbuf][3]};
      push_classes<OffT>(f, a.off, a.idx, lists, cnt, grid, k.huge_min, sh, evisit, nullptr, &stg);
      online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
      tn = cta_sum_u64(f.nrec, sh);
      tm = cta_sum_u64(f.mrec, sh);
      if (threadIdx.x == 0 && tn) {
        atomicAdd(&slot.nact, tn);
        atomicAdd(&slot.mact, tm);
      }
      if (filt == 2) ++ballot_it; else ++online_it;
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // a batch's later group launches (and WCC after its BFS) number their
      // records on from the iterations the launches before them recorded
      const int ti = it + ((V || W) ? a.w.stats->iterations : 0);
      trace_put(a.w, ti, (pull ? 2 : 1) | (filt << 8) | (scan_all ? 1 << 16 : 0) | ((VERIFY && !pull) ? 1 << 17 : 0),
                (long long)total, 0,
                (long long)(T == kInfT ? -1 : (long long)T), t_it);
      trace_classes(a.w, ti, p);
    }
    fsum += total;
    ++it;
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    mf = p.mact;
    lists_ok = p.overflow == 0;
    lbuf ^= 1;
  }
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the launches of a batch's groups add up (the host zeroes the record
    // before the first; s->evisit is kept across them)
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations += it;
    st.push_iters += it - pull_it;
    st.pull_iters += pull_it;
    st.ballot_iters += ballot_it;
    st.online_iters += online_it;
    st.phases += (int)(phases0 + (long long)sh.phase);
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum += fsum;
    st.last_l1 = 0.0;
    s->rs.done = 1;
  }
}

const void* sssp_kernel_ptr(int off_bits) {
  return off_bits == 32 ? (const void*)sssp_kernel<int32_t, false, false>
                         : (const void*)sssp_kernel<long long, false, false>;
}

template <class OffT>
static int run_sssp(simdx_graph* g, int32_t src, uint32_t* dist, simdx_stats* stats, cudaStream_t st) {
  SsspArgs<OffT> a{};
  a.n = (int)g->n;
  a.src = src;
  a.nreal = (int)g->n;
  a.ninst = 1;
  a.srcs = nullptr;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.wt = g->w;
  a.dist = dist;
  a.w = make_work(g);
  a.k = make_knobs(g);
  // pull iterations are compiled into their own instantiation, so that the
  // push kernel carries none of their registers
  const bool pull = g->symmetric && g->cfg.direction == 2;
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  // all and selective fusion are one launch (an SSSP run computes in one
  // direction); no fusion runs one launch per iteration until the kernel
  // reports the run finished
  if (g->cfg.sssp_combine == 1) {
    // the atomic-free combine (measured against atomicMin); its sweeps pull
    // with the CSR weights, so the graph must be symmetric
    if (!g->symmetric || pull || a.k.fusion == 2) return SIMDX_EUNSUPPORTED;
    const void* kern = (const void*)sssp_kernel<OffT, false, false, false, false, true>;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    return finish_launch(g, stats, st);
  }
  // small frontiers on the first cluster only when asked for (1): on the
  // 4096^2 grid with the default bucket width, 46 % of the iterations fit
  // the cluster and run 1.6-2.2 us faster, but the larger ones run 0.7 us
  // slower in the launch in clusters (fewer CTAs): 88.0 against 86.3 ms
  a.k.small = g->cfg.small_frontier == 1;
  if (a.k.fusion == 0 && a.k.small && !pull && !a.k.stage) {
    // a cooperative launch in clusters
    const void* kern = (const void*)sssp_kernel<OffT, false, false, false, false, false, false, true>;
    const int grid = grid_for_cluster(g, kern, kCluster);
    if (grid >= kCluster) {
      if ((rc = launch_coop(kern, grid, args, st, kCluster)) != SIMDX_OK) return rc;
      return finish_launch(g, stats, st);
    }
    a.k.small = 0;  // no cluster fits: the grid runs every iteration
  }
  if (a.k.fusion != 2) {
    const void* kern = pull ? (const void*)sssp_kernel<OffT, false, true>
                       : a.k.stage ? (const void*)sssp_kernel<OffT, false, false, false, false, false, true>
                                   : (const void*)sssp_kernel<OffT, false, false>;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    return finish_launch(g, stats, st);
  }
  if (capturing(st)) return SIMDX_EUNSUPPORTED;
  const void* kern = pull ? (const void*)sssp_kernel<OffT, false, true, false, true>
                          : (const void*)sssp_kernel<OffT, false, false, false, true>;
  const int grid = grid_for(g, kern);
  for (int launch = 0;; ++launch) {
    if (launch > 0 && (rc = prepare_resume(g, st)) != SIMDX_OK) return rc;
    if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
    int done = 0, want = 0;
    if ((rc = read_resume(g, st, &done, &want)) != SIMDX_OK) return rc;
    if (done) return finish_launch(g, stats, st, launch + 1);
  }
}

template <class OffT>
static int run_wcc(simdx_graph* g, uint32_t* label, simdx_stats* stats, cudaStream_t st) {
  SsspArgs<OffT> a{};
  a.n = (int)g->n;
  a.src = 0;
  a.nreal = (int)g->n;
  a.ninst = 1;
  a.srcs = nullptr;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.wt = nullptr;  // never read
  a.dist = label;
  a.w = make_work(g);
  a.k = make_knobs(g);
  a.k.fusion = 0;
  const void* kern = (const void*)sssp_kernel<OffT, false, false, true>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  // the hub's component by BFS (levels in `label`), then the rest
  if ((rc = bfs_launch_only(g, g->hub, reinterpret_cast<int32_t*>(label), st)) != SIMDX_OK) return rc;
  if ((rc = prepare_next_launch(g, st)) != SIMDX_OK) return rc;
  a.src = g->hub;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st, 2);
}

// The copies of a batch run in groups of equal size whose distances take at
// most kSsspGroupBytes (or of at most the batch_group knob), one persistent
// launch per group on the stream: a
// group's relaxations stay within a cache-sized window of the distance
// array instead of spreading over all k copies (R-MAT scale 22, 64 sources:
// groups of 8 run 1.17 ms per query, all 64 together 1.44 ms).
constexpr size_t kSsspGroupBytes = size_t(128) << 20;

static int sssp_group(const simdx_graph* g, int k) {
  const size_t per = sizeof(uint32_t) * (size_t)std::max<int64_t>(g->n, 1);
  const size_t want = g->cfg.batch_group > 0 ? (size_t)g->cfg.batch_group : kSsspGroupBytes / per;
  const int fit = (int)std::min<size_t>((size_t)k, std::max<size_t>(1, want));
  const int ngroups = (k + fit - 1) / fit;
  return (k + ngroups - 1) / ngroups;
}

// Batch state for one group of copies: task lists sized for group * n state
// ids, the class-3 words, the processed distances and pending flags; then
// the k sources.
static int ensure_sssp_batch_state(simdx_graph* g, int group, int k, cudaStream_t st) {
  const size_t ids = (size_t)group * (size_t)g->n;
  const size_t cap = std::max<size_t>(ids, (size_t)g->grid_max * (size_t)g->bin_cap) + 64;
  const size_t bytes = sizeof(int32_t) * 2 * kClasses * cap + sizeof(uint32_t) * 2 * cap +
                       sizeof(uint32_t) * ids + ids + sizeof(int32_t) * (size_t)k + 256;
  g->sb_cap = cap;  // the layout follows the current group; any large enough buffer is reused
  if (g->sb_state && g->sb_bytes >= bytes) return SIMDX_OK;
  dev_free(g->sb_state, st);
  g->sb_state = nullptr;
  g->sb_bytes = 0;
  SIMDX_CUDA(dev_alloc(&g->sb_state, bytes, st));
  g->sb_bytes = bytes;
  g->sb_k = group;
  g->sb_cap = cap;
  return SIMDX_OK;
}

template <class OffT>
static int run_sssp_batch(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                          cudaStream_t st) {
  const int group = sssp_group(g, k);
  const size_t ids = (size_t)group * (size_t)g->n;
  const size_t cap = g->sb_cap;
  char* base = static_cast<char*>(g->sb_state);
  int32_t* lists = reinterpret_cast<int32_t*>(base);
  uint32_t* aux3 = reinterpret_cast<uint32_t*>(lists + 2 * kClasses * cap);
  uint32_t* pdist = aux3 + 2 * cap;
  uint8_t* pend = reinterpret_cast<uint8_t*>(pdist + ids);
  int32_t* d_srcs = reinterpret_cast<int32_t*>(((uintptr_t)(pend + ids) + 15) & ~(uintptr_t)15);
  if (group > 64) SIMDX_CUDA(cudaMemcpyAsync(d_srcs, srcs, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st));
  SsspArgs<OffT> a{};
  a.nreal = (int)g->n;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.wt = g->w;
  a.w = make_work(g);
  a.w.list_cap = (long long)cap;
  for (int b = 0; b < 2; ++b) {
    for (int c = 0; c < kClasses; ++c) a.w.list[b][c] = lists + ((size_t)b * kClasses + c) * cap;
    a.w.aux3[b] = aux3 + (size_t)b * cap;
  }
  a.w.state = pdist;  // the kernel finds pend right after the ids processed distances
  a.k = make_knobs(g);
  a.k.fusion = 0;
  const void* kern = (const void*)sssp_kernel<OffT, true, false>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  for (int g0 = 0; g0 < k; g0 += group) {
    const int gk = std::min(group, k - g0);
    if (g0 > 0 && (rc = prepare_next_launch(g, st)) != SIMDX_OK) return rc;
    a.n = gk * (int)g->n;
    a.src = srcs[g0];
    a.ninst = gk;
    a.srcs = gk > 64 ? d_srcs + g0 : nullptr;
    for (int i = 0; i < gk && i < 64; ++i) a.src_list[i] = srcs[g0 + i];
    a.dist = dist + (size_t)g0 * (size_t)g->n;
    void* args[] = {&a};
    if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  }
  return finish_launch(g, stats, st, (k + group - 1) / group);
}

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_sssp(simdx_graph* g, int32_t src, uint32_t* dist, simdx_stats* stats, void* stream) {
  if (!g || !dist || !g->w || src < 0 || src >= g->n) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return g->off_bits == 32 ? run_sssp<int32_t>(g, src, dist, stats, st)
                           : run_sssp<long long>(g, src, dist, stats, st);
}

extern "C" int simdx_sssp_batch(simdx_graph* g, const int32_t* srcs, int32_t k, uint32_t* dist, simdx_stats* stats,
                                void* stream) {
  if (!g || !srcs || !dist || !g->w || k <= 0 || g->n <= 0) return SIMDX_EINVAL;
  if ((long long)k * g->n >= (1ll << 31) - 64) return SIMDX_EINVAL;
  for (int i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // default: every source of a launch shares the edge reads (msssp.cu); the
  // batch_group knob selects virtual graph copies in groups instead
  if (g->cfg.batch_group == 0) return sssp_batch_shared(g, srcs, k, dist, stats, st);
  int rc = ensure_sssp_batch_state(g, sssp_group(g, k), k, st);
  if (rc) return rc;
  return g->off_bits == 32 ? run_sssp_batch<int32_t>(g, srcs, k, dist, stats, st)
                           : run_sssp_batch<long long>(g, srcs, k, dist, stats, st);
}

extern "C" int simdx_wcc(simdx_graph* g, uint32_t* label, simdx_stats* stats, void* stream) {
  if (!g || !label || !g->symmetric) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    int rc = prepare_launch(g, st);
    return rc ? rc : finish_launch(g, stats, st);
  }
  return g->off_bits == 32 ? run_wcc<int32_t>(g, label, stats, st) : run_wcc<long long>(g, label, stats, st);
}
