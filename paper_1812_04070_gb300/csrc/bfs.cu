// bfs.cu -- BFS as one persistent ACC kernel (Sec. 6 "BFS"; voting combine,
// Sec. 3.2).
//
// Active(v)   : level(v) == current level.
// Compute     : push -- every frontier vertex offers level+1 to its
//               out-neighbours; pull -- every unvisited vertex looks for one
//               in-neighbour on the frontier and stops at the first hit
//               (collaborative early termination, Sec. 3.3 "Comparison").
// Combine     : vote.  All updates to a vertex carry the same value; the owner
//               writes in pull.  In push the first writer claims the vertex
//               with one compare-and-swap (only writers that read it
//               unvisited try), so the next frontier holds each vertex once
//               and the vertex / edge counts that drive the direction switch
//               are exact.
// Direction   : push in the first and last levels, pull in between (Sec. 5).
//               The switch uses frontier edge / vertex counts folded into the
//               grid barrier: pull when frontier edges exceed unexplored
//               edges / alpha, back to push when the frontier holds fewer
//               than n / beta vertices and shrinks.
// Task lists  : online filter into degree-class bins during push and pull;
//               on overflow (or when forced) the ballot filter rebuilds
//               sorted, unique lists from the level array or the frontier
//               bitmap (Sec. 4, JIT control).

#include <cstring>
#include <type_traits>

#include "acc_cluster.cuh"
#include "simdx_internal.h"


namespace simdx {

enum { kPush = 1, kPull = 2 };
constexpr int kPullFirst = 8;  // in-edges every pull candidate checks on its own lane
constexpr int kPullPer = 2;    // pull candidates per lane per round (their loads overlap)
enum { kOnline = 1, kBallot = 2 };

template <class OffT>
struct BfsArgs {
  int n, src;
  const int32_t* roots;  // device [nroots]; when nroots > 0 these replace src
  int nroots;
  const OffT* off;
  const int32_t* idx;
  const OffT* ioff;
  const int32_t* iidx;
  int32_t* level;
  long long m_total;
  Work w;
  Knobs k;
};

// The frontier bitmap is rewritten by other CTAs during the kernel, so it is
// read with plain (coherent) loads, never through the non-coherent path.
__device__ __forceinline__ bool bm_test(const uint32_t* bm, int v) {
  return (bm[v >> 5] >> (v & 31)) & 1u;
}

// r-th (0-based) set bit of x.
__device__ __forceinline__ int nth_set_bit(unsigned x, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s; s >>= 1) {
    unsigned lo = x & ((1u << s) - 1u);
    int c = __popc(lo);
    if (r >= c) {
      r -= c;
      x >>= s;
      pos += s;
    } else {
      x = lo;
    }
  }
  return pos;
}

template <class OffT>
struct BfsPush {
  struct Src {};
  int32_t* level;
  const OffT* off;
  int next;
  CtaShared& sh;
  const Work& w;
  const Knobs& k;
  unsigned grid;
  unsigned long long nrec = 0, mrec = 0;
  __device__ BfsPush(int32_t* l, const OffT* o, int nx, CtaShared& s, const Work& ww, const Knobs& kk,
                     unsigned g)
      : level(l), off(o), next(nx), sh(s), w(ww), k(kk), grid(g) {}
  __device__ __forceinline__ bool src(int, Src&, int, unsigned) { return true; }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src&, int) { return Src{}; }
  __device__ __forceinline__ void edges(const Src (&)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&)[kPushBatch],
                                        unsigned ok) {
    int lv[kPushBatch];
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) lv[q] = ((ok >> q) & 1u) ? level[u[q]] : 0;
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      if (((ok >> q) & 1u) && lv[q] == -1 && atomicCAS(&level[u[q]], -1, next) == -1) {
        long long d = (long long)gload(off + u[q] + 1) - (long long)gload(off + u[q]);
        ++nrec;
        mrec += (unsigned long long)d;
        online_record(u[q], degree_class(d, k), sh, w, k, grid);
      }
    }
  }
};

struct PullShared {
  unsigned newbits[kWarps][32];
  int defer_v[kWarps][32 * kPullPer];
  int defer_j[kWarps][32 * kPullPer];
};

// One pull iteration over all unvisited vertices with an in-edge.  Each warp
// takes 32 bitmap words, compacts their candidates and gives kPullPer of them
// to each lane per round; all loads that do not depend on one another are
// issued together (both candidates' in-edge offsets and out-degrees, then
// their first four in-edges, then the frontier bits of those), so a lane has
// several chains in flight.  A candidate checks its first kPullFirst
// in-neighbours on its own lane (sorted adjacency: low ids, the hubs, come
// first, so this resolves almost every candidate); the rest of a higher
// in-degree candidate is scanned by the whole warp, 32 edges at a time,
// stopping at the first frontier hit.  Found vertices go to the next
// frontier bitmap only: a pull level is nearly always followed by another
// pull level, and a push level after it lists the frontier from the bitmap.
template <class OffT>
__device__ void bfs_pull(const BfsArgs<OffT>& a, int cur, const uint32_t* fbm,
                         uint32_t* fbm_next, CtaShared& sh, PullShared& ps, unsigned grid,
                         PhaseSlot& slot, int32_t* big, uint32_t* found_big,
                         unsigned long long& nrec, unsigned long long& mrec, long long& evisit) {
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const long long nwords = ((long long)a.n + 31) >> 5;
  const int next = cur + 1;
  // Tasks of 32 bitmap words: each warp's first is fixed, the rest are taken
  // from a counter in the phase slot in increasing order, one task ahead, so
  // that warps whose candidates resolve fast take more tasks.
  const long long g0 = (long long)grid * kWarps;
  long long g = (long long)blockIdx.x * kWarps + warp;
  while (g * 32 < nwords) {
    unsigned long long gnext = 0;
    if (lane == 0) gnext = g0 + atomicAdd(&slot.aux0, 1ull);
    const long long wid = g * 32 + lane;
    unsigned vis = wid < nwords ? a.w.bm_vis[wid] : ~0u;
    unsigned cand = wid < nwords ? (~vis & a.w.bm_nz[wid]) : 0u;
    int c = __popc(cand);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    ps.newbits[warp][lane] = 0u;
    __syncwarp();
    for (int r = 0; r < total; r += 32 * kPullPer) {
      int u[kPullPer], jb[kPullPer];
      long long beg[kPullPer], end[kPullPer], od[kPullPer];
#pragma unroll
      for (int q = 0; q < kPullPer; ++q) {
        const int kk = r + 32 * q + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          int t = __shfl_sync(kFull, incl, j + step - 1);
          if (t <= kk) j += step;
        }
        const int excl_j = __shfl_sync(kFull, incl - c, j);
        const unsigned cand_j = __shfl_sync(kFull, cand, j);
        u[q] = -1;
        jb[q] = 0;
        beg[q] = end[q] = od[q] = 0;
        if (kk < total) {
          const int bit = nth_set_bit(cand_j, kk - excl_j);
          u[q] = (int)((g * 32 + j) * 32 + bit);
          jb[q] = (j << 5) | bit;
        }
      }
      // the candidates' in-edge ranges and out-degrees
#pragma unroll
      for (int q = 0; q < kPullPer; ++q)
        if (u[q] >= 0) {
          beg[q] = gload(a.ioff + u[q]);
          end[q] = gload(a.ioff + u[q] + 1);
          od[q] = (long long)gload(a.off + u[q] + 1) - (long long)gload(a.off + u[q]);
        }
      // their first four in-neighbours, then the frontier bits of those
      int v[kPullPer][4];
#pragma unroll
      for (int q = 0; q < kPullPer; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) v[q][e] = (u[q] >= 0 && beg[q] + e < end[q]) ? gload(a.iidx + beg[q] + e) : -1;
      bool found[kPullPer];
#pragma unroll
      for (int q = 0; q < kPullPer; ++q) {
        bool f = false;
#pragma unroll
        for (int e = 0; e < 4; ++e) f |= v[q][e] >= 0 && bm_test(fbm, v[q][e]);
        found[q] = f;
      }
      bool deferred[kPullPer];
#pragma unroll
      for (int q = 0; q < kPullPer; ++q) {
        deferred[q] = false;
        if (u[q] < 0) continue;
        // the rest of the first kPullFirst in-neighbours, on this lane
        const long long lim = end[q] - beg[q] < kPullFirst ? end[q] : beg[q] + kPullFirst;
        long long p = beg[q] + 4;
        for (; p < lim && !found[q]; ++p) found[q] = bm_test(fbm, gload(a.iidx + p));
        const long long upto = found[q] ? (p < beg[q] + 4 ? beg[q] + 4 : p) : lim;
        evisit += (upto < end[q] ? upto : end[q]) - beg[q];
        if (found[q]) {
          a.level[u[q]] = next;
          atomicOr(&ps.newbits[warp][jb[q] >> 5], 1u << (jb[q] & 31));
          ++nrec;
          mrec += (unsigned long long)od[q];
        } else if (end[q] - lim >= a.k.huge_min) {
          // scanned later by the whole grid (bfs_pull_big)
          const unsigned pos = (unsigned)atomicAdd(&slot.aux2, 1ull);
          big[pos] = u[q];
          found_big[pos] = 0u;
        } else if (end[q] > lim) {
          deferred[q] = true;  // the warp scans the remaining in-edges
        }
      }
      // warp-cooperative scan of the deferred (higher in-degree) candidates
      int nd = 0;
#pragma unroll
      for (int q = 0; q < kPullPer; ++q) {
        const unsigned dm = __ballot_sync(kFull, deferred[q]);
        if (deferred[q]) {
          const int sl = nd + __popc(dm & lanemask_lt());
          ps.defer_v[warp][sl] = u[q];
          ps.defer_j[warp][sl] = jb[q];
        }
        nd += __popc(dm);
      }
      __syncwarp();
      for (int q = 0; q < nd; ++q) {
        const int vq = ps.defer_v[warp][q];
        const long long b = gload(a.ioff + vq) + kPullFirst, e = gload(a.ioff + vq + 1);
        bool hit_any = false;
        long long seen = 0;
        for (long long base = b; base < e; base += 128) {
          bool hit = false;
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) {
            const long long p = base + lane + 32 * s4;
            if (p < e) hit |= bm_test(fbm, gload(a.iidx + p));
          }
          seen += 128;
          if (__any_sync(kFull, hit)) {
            hit_any = true;
            break;
          }
        }
        if (lane == 0) evisit += seen < e - b ? seen : e - b;
        if (hit_any && lane == 0) {
          a.level[vq] = next;
          const int jj = ps.defer_j[warp][q];
          atomicOr(&ps.newbits[warp][jj >> 5], 1u << (jj & 31));
          const long long odq = (long long)gload(a.off + vq + 1) - (long long)gload(a.off + vq);
          ++nrec;
          mrec += (unsigned long long)odq;
        }
        __syncwarp();
      }
      __syncwarp();
    }
    __syncwarp();
    if (wid < nwords) {
      unsigned nb = ps.newbits[warp][lane];
      fbm_next[wid] = nb;
      if (nb) a.w.bm_vis[wid] = vis | nb;  // owner of the word
    }
    __syncwarp();
    g = (long long)__shfl_sync(kFull, gnext, 0);
  }
}

// Pull for the candidates of in-degree >= huge_min queued by bfs_pull: their
// edges are cut into chunks (huge_min edges, fewer when the batch is small)
// dealt round-robin over all CTAs; a
// chunk is skipped once another chunk found a frontier in-neighbour.  The
// words of the bitmaps were finished by their owners in the previous phase,
// so the few bits set here use atomicOr.
template <class OffT>
__device__ void bfs_pull_big(const BfsArgs<OffT>& a, int cur, const uint32_t* fbm, uint32_t* fbm_next,
                             const int32_t* big, uint32_t* found, unsigned nbig, CtaShared& sh,
                             unsigned grid, unsigned long long& nrec, unsigned long long& mrec,
                             long long& evisit) {
  const long long ch = a.k.huge_min;
  for (unsigned b0 = 0; b0 < nbig; b0 += kChunkBatch) {
    const int nb = (int)min((unsigned)kChunkBatch, nbig - b0);
    const long long cb = chunk_prefix(big + b0, nb, a.ioff, ch, sh, IdentityVertex{}, grid);
    const int total = sh.pref[nb - 1];
    for (int kc = blockIdx.x; kc < total; kc += grid) {
      const int item = chunk_item(sh.pref, nb, kc);
      const int first = item ? sh.pref[item - 1] : 0;
      const int v = big[b0 + item];
      if (threadIdx.x == 0) sh.bcast_i[0] = (int)*reinterpret_cast<volatile uint32_t*>(found + b0 + item);
      __syncthreads();
      const bool skip = sh.bcast_i[0] != 0;
      __syncthreads();
      if (skip) continue;
      const long long vb = gload(a.ioff + v), ve = gload(a.ioff + v + 1);
      const long long beg = vb + (long long)(kc - first) * cb;
      const long long end = beg + cb < ve ? beg + cb : ve;
      bool hit = false;
#pragma unroll 4
      for (long long p = beg + threadIdx.x; p < end; p += kThreads) hit |= bm_test(fbm, gload(a.iidx + p));
      const bool any = __syncthreads_or(hit) != 0;
      if (threadIdx.x == 0) {
        evisit += end - beg;
        if (any && atomicExch(found + b0 + item, 1u) == 0u) {
          a.level[v] = cur + 1;
          atomicOr(fbm_next + (v >> 5), 1u << (v & 31));
          atomicOr(a.w.bm_vis + (v >> 5), 1u << (v & 31));
          ++nrec;
          mrec += (unsigned long long)(gload(a.off + v + 1) - gload(a.off + v));
        }
      }
    }
  }
}

// ------------------------------------------------ small frontiers
// While a push frontier is small (at most kLocEnterN vertices and kLocEnterM
// edges), the levels run on the first thread-block cluster (acc_cluster.cuh):
// a level is two dependent global round trips (edge targets; the claim's
// compare-and-swap with the target's offsets loaded alongside) plus the
// cluster barrier, where the grid pays a grid barrier and its filter.  The
// episode hands the loop state back through the barrier block; levels are
// in the level array, so the grid rebuilds its lists by the ballot filter.

// The pull levels' and the cluster levels' shared memory never live at once
// (a grid barrier or the episode's closing cluster barrier lies between).
union PullLocalShared {
  PullShared ps;
  LocalShared loc;
};
__device__ __forceinline__ PullShared& pull_part(PullShared& x) { return x; }
__device__ __forceinline__ PullShared& pull_part(PullLocalShared& x) { return x.ps; }

enum { kLcL, kLcNf, kLcMf, kLcPrevNf, kLcMu, kLcIt, kLcPushIt, kLcOnlineIt, kLcFsum, kLcDone, kLcBeat = 15 };

// One episode of small-frontier levels (every CTA calls it; cluster 0 works,
// the rest wait).  The current frontier is the class lists (at most
// kLocEnterN entries).  Returns false if the run aborted.
template <class OffT>
__device__ bool bfs_local(const BfsArgs<OffT>& a, LocalShared& ls, CtaShared& sh, const unsigned* cnt, int lbuf,
                          int& L, unsigned long long& n_f, unsigned long long& prev_n_f, unsigned long long& m_f,
                          long long& m_u, int& it, int& push_it, int& online_it, long long& fsum, long long& evisit,
                          unsigned long long& episodes, bool& done) {
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  if (blockIdx.x < kCluster) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned r = cl.block_rank();
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x < 3) loc_clear(ls, threadIdx.x);
    if (threadIdx.x == 0) ls.stop = 0;
    __syncthreads();
    // the current frontier: the entries j of the class lists (in class
    // order) with j % kCluster == r, as if this CTA had claimed them
    unsigned base = 0;
    for (int c = 0; c < kClasses; ++c) {
      const int32_t* list = a.w.list[lbuf][c];
      for (unsigned i = threadIdx.x; i < cnt[c]; i += kThreads)
        if ((base + i) % kCluster == r) {
          const int v = list[i];
          const long long b0 = (long long)gload(a.off + v);
          ls.f[0][atomicAdd(&ls.cnt[0], 1u)] = loc_pack(b0, (long long)gload(a.off + v + 1) - b0);
        }
      base += cnt[c];
    }
    loc_publish(cl, ls, 0, r);
    cl.sync();
    unsigned cc, cp, zc, zp;  // this lane's CTA count and prefix
    unsigned N = loc_counts(ls, 0, cc, cp, zc, zp).n;
    // counter slots rotate over three (the one after next is cleared during
    // a level), entry buffers over two
    int cur = 0, fc = 0;
    unsigned long long t_it = trace_clock();  // a level's start: the previous level's end
    while (true) {
      const int nx = cur == 2 ? 0 : cur + 1, nn = nx == 2 ? 0 : nx + 1;
      const long long c_it = clock64();
      unsigned ab = 0;
      if (threadIdx.x == 0) {
        loc_clear(ls, nn);  // slot nn was last read before the previous barrier
        if (r == 0) {
          ab = (unsigned)ld_volatile_i32(&s->abort);  // stored at the end of the level
          if (blockIdx.x == 0) *(volatile long long*)&s->loc[kLcBeat] = L;  // progress for the waiting CTAs
        }
      }
      // this CTA's slice of the frontier
      const unsigned lo = (unsigned)(((unsigned long long)N * r) / kCluster);
      const unsigned myc = (unsigned)(((unsigned long long)N * (r + 1)) / kCluster) - lo;
      const int next = L + 1;
      unsigned long long mrec = 0;
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
          // claim: compare-and-swap on the level with the target's offsets
          // loaded alongside
          unsigned long long ent[kLocBatch];
#pragma unroll
          for (int q = 0; q < kLocBatch; ++q) {
            ent[q] = 0;
            if (u[q] >= 0) {
              const int old = atomicCAS(&a.level[u[q]], -1, next);
              const long long ob = (long long)gload(a.off + u[q]);
              const long long oe = (long long)gload(a.off + u[q] + 1);
              if (old == -1) {
                mrec += (unsigned long long)(oe - ob);
                ent[q] = loc_pack(ob, oe - ob) | kLocClaim;
              }
            }
          }
#pragma unroll
          for (int q = 0; q < kLocBatch; ++q) loc_append1(ls, fc ^ 1, nx, ent[q]);
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
      // the same values, so the same decisions, in every CTA of the cluster
      const LocTotals T = loc_counts(ls, nx, cc, cp, zc, zp);
      const unsigned long long t_end = trace_clock();
      trace_put(a.w, it, kPush | (kOnline << 8) | (1 << 19), (long long)n_f, (long long)m_f, L, t_it, t_end);
      if (blockIdx.x == 0 && threadIdx.x == 0 && it < a.w.trace_cap) {
        a.w.trace[(long long)kTraceWords * it + 6] = (long long)T.walk;  // the slowest CTA's walk (SM cycles)
        a.w.trace[(long long)kTraceWords * it + 7] = c_bar - c_walk;  // ... its counters and the barrier
      }
      t_it = t_end;
      N = T.n;
      fsum += (long long)n_f;
      ++it;
      ++push_it;
      ++online_it;
      prev_n_f = n_f;
      n_f = N;  // one entry per vertex
      m_f = T.m;
      m_u -= (long long)T.m;
      ++L;
      if (N == 0) {
        done = true;
        break;
      }
      const bool to_pull = k.direction != 1 && exceeds_share(T.m, m_u, k.alpha);
      if (T.ovf || T.stop || N > kLocExitN || T.m > kLocEnterM || to_pull) break;
      cur = nx;
      fc ^= 1;
    }
    cl.sync();  // no CTA leaves while another still reads its shared memory
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      long long* w = s->loc;
      w[kLcL] = L; w[kLcNf] = (long long)n_f; w[kLcMf] = (long long)m_f; w[kLcPrevNf] = (long long)prev_n_f;
      w[kLcMu] = m_u; w[kLcIt] = it; w[kLcPushIt] = push_it; w[kLcOnlineIt] = online_it; w[kLcFsum] = fsum;
      w[kLcDone] = done;
      red_release_add_u64(&s->loc_epoch, 1ull);
    }
  }
  // every CTA: wait for the episode's hand-back, then take its state
  if (!loc_wait_handback(s, k, sh, &s->loc_epoch, &s->loc[kLcBeat], episodes)) return false;
  ++episodes;
  const volatile long long* w = s->loc;
  L = (int)w[kLcL]; n_f = (unsigned long long)w[kLcNf]; m_f = (unsigned long long)w[kLcMf];
  prev_n_f = (unsigned long long)w[kLcPrevNf]; m_u = w[kLcMu]; it = (int)w[kLcIt]; push_it = (int)w[kLcPushIt];
  online_it = (int)w[kLcOnlineIt]; fsum = w[kLcFsum]; done = w[kLcDone] != 0;
  return true;
}

// Loop state words of the resume record (Resume::v) for a run split over
// several launches.
enum { kRsL, kRsLbuf, kRsFb, kRsListsOk, kRsBmOk, kRsPrevDir, kRsCnt0, kRsNf = kRsCnt0 + kClasses, kRsPrevNf,
       kRsMf, kRsMu, kRsIt, kRsPushIt, kRsPullIt, kRsBallotIt, kRsOnlineIt, kRsFsum, kRsPhases };
static_assert(kRsPhases < kResumeWords, "resume record too small");

// DIRS: the directions this instantiation computes (kPush | kPull for the
// all-fusion kernel; kPush or kPull alone for the kernels of selective and
// no fusion, which stop when the next iteration needs the other direction).
// STAGE: CTA-class push ranges staged in shared memory by bulk copy (the
// `stage` knob; a separate instantiation, so the default kernel keeps its
// shared-memory footprint and L1 share).
// CLU: small frontiers run on the first thread-block cluster (the
// small_frontier knob; launched with a cluster dimension of kCluster).
template <class OffT, int DIRS = kPush | kPull, bool STAGE = false, bool CLU = false>
__global__ void __launch_bounds__(kThreads, 4) bfs_kernel(BfsArgs<OffT> a) {
  constexpr bool kHasPush = (DIRS & kPush) != 0;
  constexpr bool kHasPull = (DIRS & kPull) != 0;
  constexpr bool kSplit = DIRS != (kPush | kPull);  // runs may span several launches
  __shared__ CtaShared sh;
  __shared__ typename std::conditional<CLU, PullLocalShared, PullShared>::type pl_sm;
  PullShared& ps = pull_part(pl_sm);
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const long long nwords = ((long long)n + 31) >> 5;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();
  Stager stg{nullptr, s, a.m_total};
  if constexpr (STAGE) {
    __shared__ StageShared stage_sm;
    stage_init(stage_sm);
    if ((reinterpret_cast<uintptr_t>(a.idx) & 15) == 0) stg.sm = &stage_sm;
  }
  // a launch that continues a run split over several launches skips the set-up
  const bool resumed = kSplit && ld_volatile_i32(&s->rs.active) != 0;

  // ---- phase 0: reset levels and bitmaps; seed the first task list
  const int src1 = a.nroots > 0 ? -1 : a.src;
  if (!resumed) {
    for (long long v = gtid; v < n; v += gthreads) a.level[v] = (v == src1) ? 0 : -1;
    for (long long wd = gtid; wd < nwords; wd += gthreads) {
      unsigned m = (src1 >= 0 && wd == (src1 >> 5)) ? (1u << (src1 & 31)) : 0u;
      a.w.bm_vis[wd] = m;
      a.w.bm_f[0][wd] = m;
    }
    if (src1 >= 0 && blockIdx.x == 0 && threadIdx.x == 0) {
      long long d = (long long)a.off[src1 + 1] - (long long)a.off[src1];
      int c = degree_class(d, k);
      a.w.list[0][c][0] = src1;
      if (c == 3) a.w.aux3[0][0] = 0xffffffffu;
      s->slot[0].list_cnt[c] = 1;
      s->slot[0].nact = 1;
      s->slot[0].mact = (unsigned long long)d;
    }
    clear_next_slot(s, sh);
    if (!grid_sync(s, grid, sh, k)) return;
    if (a.nroots > 0) {
      // several roots at level 0 (e.g. one per graph of a block-diagonal batch)
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < a.nroots; i += kThreads) {
          const int r = a.roots[i];
          if (atomicExch(&a.level[r], 0) == 0) continue;  // duplicate root
          atomicOr(&a.w.bm_vis[r >> 5], 1u << (r & 31));
          atomicOr(&a.w.bm_f[0][r >> 5], 1u << (r & 31));
          const long long d = (long long)a.off[r + 1] - (long long)a.off[r];
          const int c = degree_class(d, k);
          const unsigned pos = atomicAdd(&slot.list_cnt[c], 1u);
          a.w.list[0][c][pos] = r;
          if (c == 3) a.w.aux3[0][pos] = 0xffffffffu;
          atomicAdd(&slot.nact, 1ull);
          atomicAdd(&slot.mact, (unsigned long long)d);
        }
      if (!grid_sync(s, grid, sh, k)) return;
    }
  }

  // uniform loop state (identical in every CTA)
  int L = 0;                 // level of the current frontier
  int lbuf = 0, fb = 0;      // current list buffer / frontier bitmap
  bool lists_ok = true;      // current task lists are valid
  bool bm_ok = true;         // fbm[fb] and bm_vis are valid for level L
  int prev_dir = kPush;
  unsigned cnt[kClasses];
  unsigned long long n_f, prev_n_f = 0, m_f;
  {
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    n_f = p.nact;
    m_f = p.mact;
  }
  long long m_u = a.m_total - (long long)m_f;
  int it = 0, push_it = 0, pull_it = 0, ballot_it = 0, online_it = 0;
  long long evisit = 0, fsum = 0, phases0 = 0;
  if (resumed) {
    const volatile long long* r = s->rs.v;
    L = (int)r[kRsL]; lbuf = (int)r[kRsLbuf]; fb = (int)r[kRsFb];
    lists_ok = r[kRsListsOk] != 0; bm_ok = r[kRsBmOk] != 0; prev_dir = (int)r[kRsPrevDir];
    for (int c = 0; c < kClasses; ++c) cnt[c] = (unsigned)r[kRsCnt0 + c];
    n_f = (unsigned long long)r[kRsNf]; prev_n_f = (unsigned long long)r[kRsPrevNf];
    m_f = (unsigned long long)r[kRsMf]; m_u = r[kRsMu];
    it = (int)r[kRsIt]; push_it = (int)r[kRsPushIt]; pull_it = (int)r[kRsPullIt];
    ballot_it = (int)r[kRsBallotIt]; online_it = (int)r[kRsOnlineIt]; fsum = r[kRsFsum];
    phases0 = r[kRsPhases];
  }
  const int it_launch = it;  // first iteration of this launch
  unsigned long long episodes = 0;  // small-frontier episodes so far

  while (true) {
    const unsigned long long t_it = globaltimer();
    // -------- direction for this iteration
    int dir;
    if (k.direction == 1) dir = kPush;
    else if (k.direction == 2) dir = kPull;
    else if (prev_dir == kPush) dir = exceeds_share(m_f, m_u, k.alpha) ? kPull : kPush;
    else dir = ((float)n_f * k.beta < (float)n && n_f <= prev_n_f) ? kPush : kPull;  // n_f < n / beta
    int filt = kOnline;

    // -------- selective / no fusion: leave the loop state to the next launch
    // when this kernel does not compute `dir`, or after one iteration
    if (kSplit && ((dir == kPush && !kHasPush) || (dir == kPull && !kHasPull) || (k.fusion == 2 && it > it_launch))) {
      const unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
      if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long* r = s->rs.v;
        r[kRsL] = L; r[kRsLbuf] = lbuf; r[kRsFb] = fb; r[kRsListsOk] = lists_ok; r[kRsBmOk] = bm_ok;
        r[kRsPrevDir] = prev_dir;
        for (int c = 0; c < kClasses; ++c) r[kRsCnt0 + c] = cnt[c];
        r[kRsNf] = (long long)n_f; r[kRsPrevNf] = (long long)prev_n_f; r[kRsMf] = (long long)m_f;
        r[kRsMu] = m_u; r[kRsIt] = it; r[kRsPushIt] = push_it; r[kRsPullIt] = pull_it;
        r[kRsBallotIt] = ballot_it; r[kRsOnlineIt] = online_it; r[kRsFsum] = fsum;
        r[kRsPhases] = phases0 + (long long)sh.phase;
        s->rs.want_dir = dir;
        s->rs.active = 1;
      }
      return;
    }

    // -------- make the frontier representation match the direction
    if (kHasPull && dir == kPull && !bm_ok) {
      // ballot scan of the level array: visited and frontier bitmaps
      clear_next_slot(s, sh);
      const int lane = lane_id();
      const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
      for (long long wd = gw; wd < nwords; wd += (long long)grid * kWarps) {
        long long v = wd * 32 + lane;
        int lv = v < n ? a.level[v] : -1;
        unsigned vis = __ballot_sync(kFull, lv != -1);
        unsigned fr = __ballot_sync(kFull, lv == L);
        if (lane == 0) {
          a.w.bm_vis[wd] = vis;
          a.w.bm_f[fb][wd] = fr;
        }
      }
      if (!grid_sync(s, grid, sh, k)) return;
      bm_ok = true;
      filt = kBallot;
    }
    if (kHasPush && dir == kPush && (!lists_ok || k.filter == 2)) {
      clear_next_slot(s, sh);
      PhaseSlot& slot = s->slot[slot_of(sh.phase)];
      const OffT* off = a.off;
      auto deg = [off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
      auto none = [](int) {};
      if (bm_ok) {
        bitmap_filter(n, a.w.bm_f[fb], deg, none, sh, a.w, k, grid, lbuf, slot);
      } else {
        const int32_t* lev = a.level;
        const int LL = L;
        auto pred = [lev, LL](int v) { return lev[v] == LL; };
        ballot_filter(n, pred, deg, none, sh, a.w, k, grid, lbuf, slot);
      }
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
      for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
      lists_ok = true;
      filt = kBallot;
    }

    // -------- a small push frontier: levels on one cluster until it grows
    if constexpr (CLU) {
      if (k.small && dir == kPush && k.direction != 2 && cnt[0] + cnt[1] + cnt[2] + cnt[3] <= kLocEnterN &&
          m_f <= kLocEnterM) {
        bool done = false;
        if (!bfs_local(a, pl_sm.loc, sh, cnt, lbuf, L, n_f, prev_n_f, m_f, m_u, it, push_it, online_it, fsum, evisit,
                       episodes, done))
          return;
        lists_ok = false;  // levels are in the level array: the ballot filter lists the frontier
        bm_ok = false;
        prev_dir = kPush;
        if (done) break;
        continue;
      }
    }

    // -------- compute (push or pull) with the online filter recording
    clear_next_slot(s, sh);
    online_reset(sh);
    __syncthreads();
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    unsigned long long nrec = 0, mrec = 0;
    if (kHasPush && (!kHasPull || dir == kPush)) {
      BfsPush<OffT> f(a.level, a.off, L + 1, sh, a.w, k, grid);
      const int32_t* lists[kClasses] = {a.w.list[lbuf][0], a.w.list[lbuf][1], a.w.list[lbuf][2],
                                        a.w.list[lbuf][3]};
      push_classes<OffT>(f, a.off, a.idx, lists, cnt, grid, k.huge_min, sh, evisit, nullptr, &stg);
      nrec = f.nrec;
      mrec = f.mrec;
      ++push_it;
    } else if (kHasPull) {
      bfs_pull<OffT>(a, L, a.w.bm_f[fb], a.w.bm_f[fb ^ 1], sh, ps, grid, slot, a.w.list[lbuf][3],
                     a.w.aux3[lbuf], nrec, mrec, evisit);
      ++pull_it;
    }
    if (filt == kBallot || dir == kPull) ++ballot_it; else ++online_it;
    online_flush(sh, a.w, k, grid, lbuf ^ 1, slot);
    unsigned long long tn = cta_sum_u64(nrec, sh);
    unsigned long long tm = cta_sum_u64(mrec, sh);
    if (threadIdx.x == 0 && tn) {
      atomicAdd(&slot.nact, tn);
      atomicAdd(&slot.mact, tm);
    }
    if (!grid_sync(s, grid, sh, k)) return;

    // -------- read the reductions of the compute phase
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    unsigned long long nn = p.nact, mm = p.mact;
    bool ovf = p.overflow != 0;
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    const unsigned nbig = (kHasPull && dir == kPull) ? (unsigned)p.aux2 : 0u;
    const unsigned long long t_main = globaltimer();
    if (kHasPull && nbig > 0) {
      // grid-wide pull of the high in-degree candidates
      clear_next_slot(s, sh);
      PhaseSlot& slot2 = s->slot[slot_of(sh.phase)];
      unsigned long long nb2 = 0, mb2 = 0;
      bfs_pull_big<OffT>(a, L, a.w.bm_f[fb], a.w.bm_f[fb ^ 1], a.w.list[lbuf][3], a.w.aux3[lbuf], nbig, sh,
                         grid, nb2, mb2, evisit);
      unsigned long long t0 = cta_sum_u64(nb2, sh), t1 = cta_sum_u64(mb2, sh);
      if (threadIdx.x == 0 && t0) {
        atomicAdd(&slot2.nact, t0);
        atomicAdd(&slot2.mact, t1);
      }
      if (!grid_sync(s, grid, sh, k)) return;
      const PhaseSlot& p2 = s->slot[slot_of(sh.phase - 1)];
      if (p2.nact) ovf = true;  // vertices found here are not in the online lists
      nn += p2.nact;
      mm += p2.mact;
    }
    trace_put(a.w, it, dir | (filt << 8), (long long)n_f, (long long)m_f, L, t_it);
    if (blockIdx.x == 0 && threadIdx.x == 0 && it < a.w.trace_cap) {
      a.w.trace[(long long)kTraceWords * it + 6] = (long long)t_main;  // end of the main compute phase
      a.w.trace[(long long)kTraceWords * it + 7] = (long long)nbig;    // high in-degree pull candidates
    }
    fsum += (long long)n_f;
    ++it;
    if (nn == 0) break;
    lists_ok = dir == kPush && !ovf;  // pull levels fill the bitmap, not the lists
    bm_ok = (dir == kPull);
    if (dir == kPull) fb ^= 1;
    lbuf ^= 1;
    prev_dir = dir;
    prev_n_f = n_f;
    n_f = nn;
    m_f = mm;
    m_u -= (long long)mm;
    ++L;
  }
  // statistics
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = it;
    st.push_iters = push_it;
    st.pull_iters = pull_it;
    st.ballot_iters = ballot_it;
    st.online_iters = online_it;
    st.phases = (int)(phases0 + (long long)sh.phase);
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = fsum;
    st.last_l1 = 0.0;
    s->rs.done = 1;
  }
}

const void* bfs_kernel_ptr(int off_bits) {
  return off_bits == 32 ? (const void*)bfs_kernel<int32_t> : (const void*)bfs_kernel<long long>;
}

template <class OffT>
static int run_bfs(simdx_graph* g, int32_t src, int32_t* levels, simdx_stats* stats, cudaStream_t st,
                   const int32_t* d_roots = nullptr, int nroots = 0) {
  BfsArgs<OffT> a{};
  a.n = (int)g->n;
  a.src = src;
  a.roots = d_roots;
  a.nroots = nroots;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.ioff = (const OffT*)g->in_off;
  a.iidx = g->in_idx;
  a.level = levels;
  a.m_total = g->e;
  a.w = make_work(g);
  a.k = make_knobs(g);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if (a.k.fusion == 0 && a.k.small && !a.k.stage) {
    // small frontiers on the first cluster: a cooperative launch in clusters
    const void* kern = (const void*)bfs_kernel<OffT, kPush | kPull, false, true>;
    const int grid = grid_for_cluster(g, kern, kCluster);
    if (grid >= kCluster) {
      if ((rc = launch_coop(kern, grid, args, st, kCluster)) != SIMDX_OK) return rc;
      return finish_launch(g, stats, st);
    }
    a.k.small = 0;  // no cluster fits: the grid runs every level
  }
  if (a.k.fusion == 0) {
    const void* kern = a.k.stage ? (const void*)bfs_kernel<OffT, kPush | kPull, true> : (const void*)bfs_kernel<OffT>;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    return finish_launch(g, stats, st);
  }
  // selective fusion (a launch per run of one direction) or no fusion (a
  // launch per iteration): kernels compiled for one direction each; the host
  // learns between launches whether the run ended and which direction is next
  if (capturing(st)) return SIMDX_EUNSUPPORTED;
  int want = g->cfg.direction == 2 ? kPull : kPush;
  for (int launch = 0;; ++launch) {
    const void* kern = want == kPull ? (const void*)bfs_kernel<OffT, kPull> : (const void*)bfs_kernel<OffT, kPush>;
    if (launch > 0 && (rc = prepare_resume(g, st)) != SIMDX_OK) return rc;
    if ((rc = launch_coop(kern, grid_for(g, kern), args, st)) != SIMDX_OK) return rc;
    int done = 0;
    if ((rc = read_resume(g, st, &done, &want)) != SIMDX_OK) return rc;
    if (done) return finish_launch(g, stats, st, launch + 1);
  }
}

template <class OffT>
static int launch_bfs_only(simdx_graph* g, int32_t src, int32_t* levels, cudaStream_t st) {
  BfsArgs<OffT> a{};
  a.n = (int)g->n;
  a.src = src;
  a.off = (const OffT*)g->off;
  a.idx = g->idx;
  a.ioff = (const OffT*)g->in_off;
  a.iidx = g->in_idx;
  a.level = levels;
  a.m_total = g->e;
  a.w = make_work(g);
  a.k = make_knobs(g);
  a.k.fusion = 0;  // one launch, bracketed by the caller
  const void* kern = (const void*)bfs_kernel<OffT>;
  void* args[] = {&a};
  return launch_coop(kern, grid_for(g, kern), args, st);
}

int bfs_launch_only(simdx_graph* g, int32_t src, int32_t* levels, cudaStream_t st) {
  return g->off_bits == 32 ? launch_bfs_only<int32_t>(g, src, levels, st)
                           : launch_bfs_only<long long>(g, src, levels, st);
}

// Launch the BFS kernel on caller-provided arrays and workspace views (no
// graph object): used by entry points whose workspace is not library-owned
// device memory.
int bfs_launch_raw(int off_bits, int n, long long e, const void* off, const int32_t* idx, int src,
                   int32_t* levels, const Work& w, const Knobs& k, int grid, cudaStream_t st) {
  void* args[1];
  if (off_bits == 32) {
    BfsArgs<int32_t> a{};
    a.n = n; a.src = src; a.roots = nullptr; a.nroots = 0;
    a.off = (const int32_t*)off; a.idx = idx; a.ioff = a.off; a.iidx = idx;
    a.level = levels; a.m_total = e; a.w = w; a.k = k;
    args[0] = &a;
    return launch_coop((const void*)bfs_kernel<int32_t>, grid, args, st);
  }
  BfsArgs<long long> a{};
  a.n = n; a.src = src; a.roots = nullptr; a.nroots = 0;
  a.off = (const long long*)off; a.idx = idx; a.ioff = a.off; a.iidx = idx;
  a.level = levels; a.m_total = e; a.w = w; a.k = k;
  args[0] = &a;
  return launch_coop((const void*)bfs_kernel<long long>, grid, args, st);
}

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_bfs(simdx_graph* g, int32_t src, int32_t* levels, simdx_stats* stats, void* stream) {
  if (!g || !levels || src < 0 || src >= g->n) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return g->off_bits == 32 ? run_bfs<int32_t>(g, src, levels, stats, st)
                           : run_bfs<long long>(g, src, levels, stats, st);
}

extern "C" int simdx_bfs_multi(simdx_graph* g, const int32_t* roots, int32_t k, int32_t* levels, simdx_stats* stats,
                               void* stream) {
  if (!g || !roots || !levels || k <= 0 || g->n <= 0) return SIMDX_EINVAL;
  for (int i = 0; i < k; ++i)
    if (roots[i] < 0 || roots[i] >= g->n) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool cap = capturing(st);
  if ((size_t)k > g->roots_cap) {
    // growing needs allocations, which a stream capture does not allow:
    // a captured call must follow an uncaptured one with at least k roots
    if (cap) return SIMDX_EUNSUPPORTED;
    dev_free(g->d_roots, st);
    if (g->h_roots) cudaFreeHost(g->h_roots);
    g->d_roots = nullptr;
    g->h_roots = nullptr;
    g->roots_cap = 0;
    SIMDX_CUDA(dev_alloc((void**)&g->d_roots, sizeof(int32_t) * (size_t)k, st));
    SIMDX_CUDA(cudaHostAlloc((void**)&g->h_roots, sizeof(int32_t) * (size_t)k, cudaHostAllocDefault));
    g->roots_cap = (size_t)k;
  }
  if (cap) {
    // a captured copy reads pinned memory when the graph replays: stage the
    // roots there (a replay uses the roots of the latest captured call)
    std::memcpy(g->h_roots, roots, sizeof(int32_t) * (size_t)k);
    SIMDX_CUDA(cudaMemcpyAsync(g->d_roots, g->h_roots, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st));
  } else {
    SIMDX_CUDA(cudaMemcpyAsync(g->d_roots, roots, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st));
  }
  return g->off_bits == 32 ? run_bfs<int32_t>(g, roots[0], levels, stats, st, g->d_roots, k)
                           : run_bfs<long long>(g, roots[0], levels, stats, st, g->d_roots, k);
}
