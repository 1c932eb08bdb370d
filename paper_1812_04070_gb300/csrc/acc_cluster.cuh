// acc_cluster.cuh -- small-frontier iterations on one thread-block cluster.
//
// An iteration of the persistent kernels costs a grid barrier and a chain
// of dependent global round trips whatever the size of its frontier (the
// fixed cost of a fused iteration, Sec. 5's software global barrier).  When
// the frontier is small, the iterations run on the first thread-block
// cluster alone (kCluster CTAs), with a hardware cluster barrier per
// iteration, while the other CTAs wait on a flag (bounded like the grid
// barrier).  The pieces here are shared by the BFS levels and the k-core
// decomposition's peeling:
//
//  * a frontier entry is a vertex's edge range, packed as (beg << 24) | len
//    (beg < 2^39 for any graph that fits in device memory); loc_append
//    splits a range into pieces of at most kLocChunk edges, so the slices
//    below are balanced in edges as well as entries (the k-core peeling,
//    whose small frontiers are the dense core's hubs), loc_append1 keeps one
//    entry per vertex (BFS, whose walked frontiers hold at most kLocEnterM
//    edges and are balanced enough);
//  * each CTA appends the vertices it claims to its own shared memory (one
//    shared atomic per warp and batch slot);
//  * before the barrier each CTA stores its counters into every CTA's
//    shared memory, so after it all CTAs read the same totals locally and
//    take the same decisions;
//  * CTA r walks the r-th sixteenth of the concatenated buffers, reading
//    the entries from distributed shared memory; a warp takes up to 64
//    entries (two per lane) and walks their concatenated edges.
//
// No remote atomics and no contended counters: the only cross-CTA traffic
// is the entry reads and the counter stores.
#pragma once

#include <cooperative_groups.h>

#include "acc_device.cuh"

namespace simdx {

namespace cg = cooperative_groups;

constexpr int kCluster = 16;                      // CTAs of the cluster (a non-portable size)
constexpr int kLocCap = 512;                      // entries a CTA can claim in one iteration
constexpr unsigned kLocEnterN = 4096;             // enter with at most this many frontier vertices
constexpr unsigned long long kLocEnterM = 65536;  // ... and frontier edges
constexpr unsigned kLocExitN = 6144;              // leave when the next frontier holds more
constexpr int kLocBatch = 4;                      // edges per lane in flight
constexpr long long kLocChunk = 64;               // edges per frontier entry at most
constexpr unsigned long long kLocDegMask = (1ull << 24) - 1;
constexpr unsigned long long kLocClaim = 1ull << 63;  // a claimed entry, while in registers
static_assert(kCluster <= 32 && (kCluster & (kCluster - 1)) == 0, "one lane per CTA of the cluster");

// One CTA's counters of an iteration, as stored into every CTA.
struct LocCounters {
  unsigned long long medges;  // out-edges of the CTA's claims
  unsigned long long x;       // summed (algorithm's use)
  unsigned long long y;       // minimum (algorithm's use)
  unsigned cnt;               // the CTA's entries
  unsigned flags;             // bit 0: it claimed more than kLocCap; bit 1 (rank 0): the run aborted
  unsigned z;                 // per CTA, with a prefix (algorithm's use)
  unsigned walk;              // SM clock cycles the CTA spent in the step before publishing
};

struct LocalShared {
  unsigned long long f[2][kLocCap];  // entries this CTA claimed: the current and the next frontier
  unsigned cnt[3];                   // this CTA's entries in an iteration (slots rotate over three)
  unsigned ovf[3];                   // this CTA claimed more than kLocCap
  unsigned z[3];
  unsigned stop;                     // rank 0: the run aborted (read before the barrier)
  unsigned long long medges[3];
  unsigned long long x[3];
  unsigned long long y[3];
  LocCounters all[3][kCluster];      // every CTA's counters of an iteration, stored here by that CTA
};

// The cluster's totals of one counter slot, the same in every thread.
struct LocTotals {
  unsigned n;            // entries
  unsigned long long m;  // out-edges of the claims
  unsigned long long x;  // sum of x
  unsigned long long y;  // minimum of y
  unsigned z;            // sum of z
  unsigned walk;         // the slowest CTA's cycles in the step
  unsigned ovf;          // some CTA overflowed
  unsigned stop;         // rank 0 saw the abort flag
};

__device__ __forceinline__ unsigned long long loc_pack(long long beg, long long len) {
  return ((unsigned long long)beg << 24) | (unsigned long long)(len < (long long)kLocDegMask ? len : kLocDegMask);
}

// Clears counter slot `sl` of this CTA (one thread).
__device__ __forceinline__ void loc_clear(LocalShared& ls, int sl) {
  ls.cnt[sl] = 0;
  ls.ovf[sl] = 0;
  ls.z[sl] = 0;
  ls.medges[sl] = 0;
  ls.x[sl] = 0;
  ls.y[sl] = ~0ull;
}

// The edge j (0 <= j < total) of a warp's group of up to 64 tasks: lane t
// holds tasks t and t + 32 with inclusive edge prefixes ia, ib (ib counts on
// from the first half's total ta).  Returns the task's lane and half.  Every
// lane reads both prefixes of the lane it probes and keeps the one of its
// own half (a lane's half depends on its own j).
__device__ __forceinline__ int loc_find(int ia, int ib, int ta, int j, bool& hi) {
  hi = j >= ta;
  int t = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int xa = __shfl_sync(kFull, ia, t + step - 1);
    const int xb = __shfl_sync(kFull, ib, t + step - 1);
    if ((hi ? xb : xa) <= j) t += step;
  }
  return t;
}

// The CTA (lane of the warp) that holds entry g of the concatenated buffers:
// lanes 0..kCluster-1 hold the exclusive prefix p of the CTAs' counts (lanes
// beyond hold ~0u).
__device__ __forceinline__ int loc_owner(unsigned p, unsigned g) {
  int t = 0;
#pragma unroll
  for (int step = kCluster / 2; step >= 1; step >>= 1) {
    const unsigned x = __shfl_sync(kFull, p, t + step);
    if (x <= g) t += step;
  }
  return t;
}

// Before a cluster barrier: this CTA's counters of slot `sl` go to every
// CTA of the cluster (thread c stores to CTA c), so that after the barrier
// they are read locally.  The CTA's appends are complete (__syncthreads).
__device__ __forceinline__ void loc_publish(cg::cluster_group& cl, LocalShared& ls, int sl, unsigned r,
                                            unsigned walk = 0) {
  __syncthreads();
  if (threadIdx.x < kCluster) {
    LocCounters c;
    c.medges = ls.medges[sl];
    c.x = ls.x[sl];
    c.y = ls.y[sl];
    c.cnt = ls.cnt[sl];
    c.flags = (ls.ovf[sl] ? 1u : 0u) | (r == 0 && ls.stop ? 2u : 0u);
    c.z = ls.z[sl];
    c.walk = walk;
    cl.map_shared_rank(&ls, threadIdx.x)->all[sl][r] = c;
  }
}

// After a cluster barrier: every warp reads counter slot `sl` of all CTAs
// (lane c, CTA c's copy in this CTA's shared memory).  Returns the lane's
// count and exclusive prefix of counts (lanes below kCluster; ~0u beyond),
// and the same for z, plus the cluster's totals.
__device__ __forceinline__ LocTotals loc_counts(const LocalShared& ls, int sl, unsigned& c, unsigned& p,
                                                unsigned& zc, unsigned& zp) {
  const int lane = lane_id();
  c = 0;
  zc = 0;
  unsigned long long me = 0, mx = 0, my = ~0ull;
  unsigned o = 0, x = 0, wk = 0;
  if (lane < kCluster) {
    const LocCounters& r = ls.all[sl][lane];
    c = r.cnt;
    zc = r.z;
    me = r.medges;
    mx = r.x;
    my = r.y;
    o = r.flags & 1u;
    x = r.flags & 2u;
    wk = r.walk;
  }
  unsigned incl = c, zincl = zc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, d), yz = __shfl_up_sync(kFull, zincl, d);
    if (lane >= d) {
      incl += y;
      zincl += yz;
    }
  }
  LocTotals t;
  t.n = __shfl_sync(kFull, incl, 31);
  t.z = __shfl_sync(kFull, zincl, 31);
  p = lane < kCluster ? incl - c : ~0u;
  zp = lane < kCluster ? zincl - zc : ~0u;
  t.m = warp_sum_u64(me);
  t.x = warp_sum_u64(mx);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long v = __shfl_xor_sync(kFull, my, d);
    my = v < my ? v : my;
  }
  t.y = my;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned v = __shfl_xor_sync(kFull, wk, d);
    wk = v > wk ? v : wk;
  }
  t.walk = wk;
  t.ovf = __any_sync(kFull, o != 0) ? 1u : 0u;
  t.stop = __any_sync(kFull, x != 0) ? 1u : 0u;
  return t;
}

// Writes the edge range [beg, beg + deg) as ceil(deg / kLocChunk) entries
// from position pos of buffer `buf` (counter slot `sl` flags an overflow).
__device__ __forceinline__ void loc_write(LocalShared& ls, int buf, int sl, unsigned pos, long long beg,
                                          long long deg) {
  for (long long j = 0; j < deg; j += kLocChunk, ++pos) {
    if (pos >= (unsigned)kLocCap) {
      ls.ovf[sl] = 1;
      return;
    }
    ls.f[buf][pos] = loc_pack(beg + j, deg - j < kLocChunk ? deg - j : kLocChunk);
  }
}

// One thread's edge range, appended with a shared atomic of its own.
__device__ __forceinline__ void loc_put(LocalShared& ls, int buf, int sl, long long beg, long long deg) {
  if (deg <= 0) return;
  const unsigned nch = (unsigned)((deg + kLocChunk - 1) / kLocChunk);
  loc_write(ls, buf, sl, atomicAdd(&ls.cnt[sl], nch), beg, deg);
}

// Appends each lane's claimed entry (kLocClaim set: a vertex's whole edge
// range, packed; the caller walks no range beyond kLocDegMask edges) as one
// entry: one shared atomic per warp.  Every lane of the warp calls it.
__device__ __forceinline__ void loc_append1(LocalShared& ls, int buf, int sl, unsigned long long ent) {
  const bool mine = (ent & kLocClaim) != 0;
  const unsigned mk = __ballot_sync(kFull, mine);
  if (mk == 0) return;
  const int leader = __ffs(mk) - 1;
  unsigned base = 0;
  if (lane_id() == leader) base = atomicAdd(&ls.cnt[sl], (unsigned)__popc(mk));
  base = __shfl_sync(kFull, base, leader);
  if (mine) {
    const unsigned pos = base + (unsigned)__popc(mk & lanemask_lt());
    if (pos < (unsigned)kLocCap) ls.f[buf][pos] = ent & ~kLocClaim;
    else ls.ovf[sl] = 1;
  }
}

// Appends the edge ranges of the lanes that claimed a vertex (claim set;
// deg may be 0: nothing to walk) to the CTA's buffer `buf` with counter
// slot `sl`: one shared atomic per warp.  Every lane of the warp calls it.
__device__ __forceinline__ void loc_append(LocalShared& ls, int buf, int sl, bool claim, long long beg,
                                           long long deg) {
  const unsigned nch = claim && deg > 0 ? (unsigned)((deg + kLocChunk - 1) / kLocChunk) : 0u;
  const int lane = lane_id();
  unsigned incl = nch;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const unsigned tot = __shfl_sync(kFull, incl, 31);
  if (tot == 0) return;
  unsigned base = 0;
  if (lane == 31) base = atomicAdd(&ls.cnt[sl], tot);
  base = __shfl_sync(kFull, base, 31);
  if (nch) loc_write(ls, buf, sl, base + incl - nch, beg, deg);
}

// The episode's other CTAs: thread 0 waits until the cluster has handed
// back `episodes + 1` episodes through `epoch`, bounded by the barrier
// timeout without progress (`beat` changes while the cluster works).
// Returns false (and flags the run aborted) when the wait gave up.
__device__ __forceinline__ bool loc_wait_handback(Sync* s, const Knobs& k, CtaShared& sh,
                                                  const unsigned long long* epoch, const long long* beat_p,
                                                  unsigned long long episodes) {
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long t0 = 0;
    long long beat = -1;
    unsigned spins = 0;
    while (ld_acquire_u64(epoch) < episodes + 1) {
      __nanosleep(64);
      if ((++spins & 63u) == 0) {
        if (ld_volatile_i32(&s->abort)) { ok = 0; break; }
        const unsigned long long t = globaltimer();
        const long long b = *(const volatile long long*)beat_p;
        if (t0 == 0 || b != beat) {
          t0 = t;
          beat = b;
        } else if (t - t0 > k.timeout_ns) {
          atomicExch(&s->abort, 1);
          atomicCAS(&s->err, 0, 4 /* SIMDX_EBARRIER_TIMEOUT */);
          ok = 0;
          break;
        }
      }
    }
    sh.ok = ok;
  }
  __syncthreads();
  return sh.ok != 0;
}

}  // namespace simdx
