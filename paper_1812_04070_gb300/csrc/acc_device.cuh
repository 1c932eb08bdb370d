// acc_device.cuh -- device building blocks of the ACC hot path (sm_103a).
//
// One persistent cooperative kernel per algorithm call runs every BSP
// iteration (Sec. 5, "Push-Pull based kernel fusion"; here all fusion, see
// Table 2).  The pieces shared by all algorithms live here:
//
//   * grid_sync      -- software global barrier (Sec. 5, "Software global
//                       barrier").  The grid is sized to co-residency from the
//                       occupancy calculator (the Eq. 1 analogue) and launched
//                       cooperatively, so the barrier cannot deadlock; every
//                       wait is also bounded by a %globaltimer limit, after
//                       which the run aborts with an error instead of hanging.
//   * PhaseSlot ring -- per-phase reductions (active counts, list lengths,
//                       overflow flag) folded into the barrier arrival.
//   * online filter  -- during compute, updated vertices are recorded in
//                       per-CTA bins of bounded capacity, one bin per degree
//                       class (Sec. 4, "Online filter"; threshold 64 per
//                       thread, "Overflow thresholds").  Bins are concatenated
//                       into the next task lists before the barrier.
//   * ballot filter  -- a coalesced scan of vertex metadata with warp ballots
//                       that emits sorted, duplicate-free task lists
//                       (Sec. 4, "Ballot filter"); used when a bin overflowed
//                       (JIT control, Sec. 4).
//   * class drivers  -- thread / warp / CTA work per small / medium / large
//                       task (Sec. 4, "Classification"; Sec. 3.3), plus a
//                       fourth class whose edges are split over the whole
//                       grid for the very highest degrees.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace simdx {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kClasses = 4;  // 0 thread, 1 warp, 2 CTA, 3 grid
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBallotChunk = kThreads * 32;  // largest ballot-filter chunk (vertices)
constexpr int kTraceWords = 8;                // int64 words per trace record
constexpr int kChunkBatch = kThreads * 4;     // class-3 tasks per chunk-prefix batch

// ------------------------------------------------------------ shared state
struct PhaseSlot {
  unsigned long long nact;      // vertices recorded for the next iteration
  unsigned long long mact;      // their degree sum
  unsigned long long aux0;      // algorithm-specific (u64 sum or min)
  unsigned long long aux1;
  unsigned long long aux2;
  unsigned int list_cnt[kClasses];
  unsigned int overflow;
  unsigned int flag;
  unsigned long long tclass[kClasses];  // max over CTAs of each class's duration (ns)
};

// Loop state a launch leaves for the next launch of the same run when it
// stops early (selective fusion: at a change of direction; no fusion: after
// every iteration).  The host reads `done` and `want_dir` between launches.
constexpr int kResumeWords = 32;
struct Resume {
  int active;                   // the words below continue a run
  int done;                     // the run has finished
  int want_dir;                 // direction of the next iteration (1 push, 2 pull)
  int pad;
  long long v[kResumeWords];    // algorithm loop state
};

struct Sync {
  unsigned long long arrive;    // monotonic barrier arrival counter
  int abort;                    // a wait ran out somewhere
  int err;                      // status code of the failure
  unsigned long long evisit;    // edges read by compute (statistics)
  unsigned long long pad[13];   // the polled words alone on their 128-byte line
  PhaseSlot slot[3];
  Resume rs;
  unsigned long long loc_epoch;  // small-frontier episodes handed back to the grid
  long long loc[16];             // the loop state an episode hands back
};

struct DevStats {
  int status, iterations, push_iters, pull_iters, ballot_iters, online_iters, phases, grid;
  long long edges_visited, frontier_sum;
  double last_l1;
};

struct Knobs {
  int small_max, med_max, huge_min;
  int bin_cap;          // per CTA per class (threshold per thread * threads)
  int direction;        // 0 auto, 1 push, 2 pull
  int filter;           // 0 JIT, 2 ballot only
  float alpha, beta, kalpha;
  unsigned delta;
  unsigned long long timeout_ns;
  int skip_cta, skip_phase;
  int fusion;           // 0 all iterations in one launch, 1 one launch per run of one
                        // direction, 2 one launch per iteration (Sec. 5, Table 2)
  int stage;            // stage CTA-class edge ranges in shared memory by bulk copy
  int small;            // small frontiers run on one thread-block cluster
};

// Workspace shared by all algorithms of one graph.
struct Work {
  int32_t* bins;                 // [kClasses][grid][bin_cap]
  int32_t* list[2][kClasses];    // double-buffered task lists
  uint32_t* aux3[2];             // per-entry word of the class-3 lists (set to ~0 on append)
  long long list_cap;
  int32_t* chunk_cnt;            // [chunks][kClasses] for the deterministic ballot filter
  unsigned long long* chunk_part;  // per-chunk partial sums of chunked pull tasks
  int* chunk_done;               // chunks finished per class-3 task (reset by the last)
  int* warp_start;               // [grid * kWarps + 1] first task of each warp's edge range
  uint32_t* bm_nz;               // vertices with an in-edge (pull candidates)
  uint32_t* bm_vis;              // BFS visited
  uint32_t* bm_f[2];             // BFS frontier bitmaps
  void* state;                   // per-algorithm vertex state (20 bytes / vertex)
  Sync* sync;
  DevStats* stats;
  long long* trace;              // [trace_cap][kTraceWords]
  int trace_cap;
};

// --------------------------------------------------------------- PTX bits
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Direction rules (Sec. 4.2): m > rest / alpha, decided by every thread of
// every CTA once per iteration, in single precision and multiplied out
// (double-precision division is slow on this part).  The decision only picks
// a direction; the result of the run does not depend on it.
__device__ __forceinline__ bool exceeds_share(unsigned long long m, long long rest, float alpha) {
  return (float)m * alpha > (float)rest;
}

// The global timer as the trace needs it: read by the one thread that writes
// the trace (thread 0 of CTA 0), 0 elsewhere.  A read of the global timer is
// not free, and an iteration's critical path should not pay it in every
// thread.
__device__ __forceinline__ unsigned long long trace_clock() {
  return (blockIdx.x == 0 && threadIdx.x == 0) ? globaltimer() : 0ull;
}
// Graph arrays are read-only for the whole kernel: non-coherent loads are safe
// there (and only there; state written during the kernel uses plain loads).
template <class T>
__device__ __forceinline__ T gload(const T* p) { return __ldg(p); }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------ grid barrier
// Per-CTA shared bookkeeping of the persistent loop.
struct CtaShared {
  unsigned long long phase;  // barriers passed by this CTA
  int ok;
  int bincnt[kClasses];      // online-filter bin fill per class
  int base[kClasses];
  int wcnt[kClasses][kWarps];
  unsigned long long red64[kWarps];
  double redf[kWarps];
  float redf32[kWarps];
  int bcast_i[8];
  unsigned long long bcast_u64[8];
  int scan_w[kWarps];
  int pref[kChunkBatch];     // inclusive prefix of chunk counts of a class-3 batch
};

// Every thread of every CTA calls this; returns false when the run aborted.
// Arrival is one release-add per CTA; the CTA's writes are ordered before it
// by __syncthreads + the release.  Waiting polls with acquire loads so the
// data written before other CTAs' arrivals is visible afterwards.
__device__ __forceinline__ bool grid_sync(Sync* s, unsigned grid, CtaShared& sh, const Knobs& k) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ph = sh.phase + 1;
    sh.phase = ph;
    int ok = 1;
    bool skip = (k.skip_cta == (int)blockIdx.x) && ((unsigned long long)k.skip_phase == ph);
    if (!skip) red_release_add_u64(&s->arrive, 1ull);
    const unsigned long long target = ph * (unsigned long long)grid;
    // polls with a 32 ns sleep and checks the abort word and the time limit
    // every 64 polls.  Measured on GB300: a bare loop of barriers of 608
    // CTAs takes 2.3 us each without the sleep and 2.5 us with it, but in
    // the kernels the sleeping poll runs as fast or 1-3 % faster (less
    // polling traffic while other CTAs still work)
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while (ld_acquire_u64(&s->arrive) < target) {
      __nanosleep(32);
      if ((++spins & 63u) == 0) {
        if (ld_volatile_i32(&s->abort)) { ok = 0; break; }
        unsigned long long t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > k.timeout_ns) {
          atomicExch(&s->abort, 1);
          atomicCAS(&s->err, 0, 4 /* SIMDX_EBARRIER_TIMEOUT */);
          ok = 0;
          break;
        }
      }
    }
    if (ok && ld_volatile_i32(&s->abort)) ok = 0;
    sh.ok = ok;
  }
  __syncthreads();
  return sh.ok != 0;
}

__device__ __forceinline__ int slot_of(unsigned long long phase) { return (int)(phase % 3ull); }

// Called once at the start of each phase by every CTA: CTA 0 clears the slot
// that the NEXT phase will accumulate into (nobody reads or writes it now).
__device__ __forceinline__ void clear_next_slot(Sync* s, const CtaShared& sh) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PhaseSlot& z = s->slot[slot_of(sh.phase + 1)];
    z.nact = 0; z.mact = 0; z.aux0 = 0; z.aux1 = 0; z.aux2 = 0;
    for (int c = 0; c < kClasses; ++c) {
      z.list_cnt[c] = 0;
      z.tclass[c] = 0;
    }
    z.overflow = 0; z.flag = 0;
  }
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// CTA-wide sum; result valid in every thread.  Fixed order (deterministic).
__device__ __forceinline__ unsigned long long cta_sum_u64(unsigned long long v, CtaShared& sh) {
  v = warp_sum_u64(v);
  __syncthreads();
  if (lane_id() == 0) sh.red64[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += sh.red64[w];
  return t;
}
__device__ __forceinline__ float cta_sum_f32(float v, CtaShared& sh) {
  v = warp_sum_f32(v);
  __syncthreads();
  if (lane_id() == 0) sh.redf32[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += sh.redf32[w];
  return t;
}
__device__ __forceinline__ double cta_sum_f64(double v, CtaShared& sh) {
  v = warp_sum_f64(v);
  __syncthreads();
  if (lane_id() == 0) sh.redf[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += sh.redf[w];
  return t;
}

// ----------------------------------------------------------- degree class
__device__ __forceinline__ int degree_class(long long deg, const Knobs& k) {
  return deg < k.small_max ? 0 : deg < k.med_max ? 1 : deg < k.huge_min ? 2 : 3;
}

// --------------------------------------------------------- online filter
// Record vertex u of class cls in this CTA's bin.  Warp-aggregated with
// __match_any_sync so one shared atomic serves all lanes of a class.  Entries
// beyond the bin capacity are dropped; the overflow is detected at flush.
__device__ __forceinline__ void online_record(int u, int cls, CtaShared& sh, const Work& w,
                                              const Knobs& k, unsigned grid) {
  unsigned mask = __activemask();
  unsigned peers = __match_any_sync(mask, cls);
  int leader = __ffs(peers) - 1;
  int base = 0;
  if ((int)lane_id() == leader) base = atomicAdd(&sh.bincnt[cls], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  int pos = base + __popc(peers & lanemask_lt());
  if (pos < k.bin_cap)
    w.bins[((size_t)cls * grid + blockIdx.x) * (size_t)k.bin_cap + pos] = u;
}

__device__ __forceinline__ void online_reset(CtaShared& sh) {
  if (threadIdx.x < kClasses) sh.bincnt[threadIdx.x] = 0;
}

// Append this CTA's bins to the next task lists (prefix concatenation of the
// thread bins, Sec. 3.3): one atomic per non-empty class reserves the CTA's
// range.  Must be called by all threads of the CTA.
__device__ __forceinline__ void online_flush(CtaShared& sh, const Work& w, const Knobs& k,
                                             unsigned grid, int nbuf, PhaseSlot& slot) {
  __syncthreads();
  if (threadIdx.x < kClasses) {
    int c = threadIdx.x;
    int cnt = sh.bincnt[c];
    if (cnt > k.bin_cap) {
      atomicOr(&slot.overflow, 1u);
      cnt = k.bin_cap;
    }
    int b = 0;
    if (cnt > 0) {
      b = (int)atomicAdd(&slot.list_cnt[c], (unsigned)cnt);
      if ((long long)b + cnt > w.list_cap) { atomicOr(&slot.overflow, 1u); cnt = 0; }
    }
    sh.base[c] = b;
    sh.wcnt[c][0] = cnt;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kClasses; ++c) {
    int cnt = sh.wcnt[c][0];
    const int32_t* src = w.bins + ((size_t)c * grid + blockIdx.x) * (size_t)k.bin_cap;
    int32_t* dst = w.list[nbuf][c] + sh.base[c];
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
      dst[i] = src[i];
      if (c == 3) w.aux3[nbuf][sh.base[c] + i] = 0xffffffffu;
    }
  }
}

// --------------------------------------------------------- ballot filter
// 32-vertex steps a warp takes per chunk (at most 32): as many as spread the
// n vertices over the whole grid, so that a small scan is one or two steps
// on every CTA instead of 32 dependent steps on a few.
__device__ __forceinline__ int ballot_steps(long long n, unsigned grid) {
  const long long per = (long long)grid * kThreads;
  const long long j = (n + per - 1) / per;
  return j < 1 ? 1 : (j > 32 ? 32 : (int)j);
}

// Scan vertices [0, n) in chunks of kThreads x ballot_steps (at most
// kBallotChunk); pred(v) says whether v is active and deg(v) its degree for
// the class.  Emits, per class, the active vertices of each chunk in
// increasing order (sorted, unique) into w.list[nbuf][c], reserving each
// chunk's range with one atomic per class.  `visit(v)` is called once for
// every selected vertex (by the thread that writes it) so callers can fuse
// per-vertex side effects.
template <class Pred, class Deg, class Visit>
__device__ void ballot_filter(int n, Pred pred, Deg deg, Visit visit, CtaShared& sh, const Work& w,
                              const Knobs& k, unsigned grid, int nbuf, PhaseSlot& slot) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int J = ballot_steps(n, grid);
  const long long csz = (long long)kThreads * J;
  for (long long chunk = blockIdx.x; chunk * csz < n; chunk += grid) {
    const long long wbase = chunk * csz + (long long)warp * 32 * J;
    unsigned my[kClasses] = {0u, 0u, 0u, 0u};
    for (int j = 0; j < J; ++j) {
      long long v = wbase + j * 32 + lane;
      bool act = false;
      int cls = 0;
      if (v < n && pred((int)v)) {
        act = true;
        cls = degree_class(deg((int)v), k);
      }
#pragma unroll
      for (int c = 0; c < kClasses; ++c) {
        unsigned m = __ballot_sync(kFull, act && cls == c);
        if (lane == j) my[c] = m;
      }
    }
    // per-class exclusive prefix across lanes, then across warps
    int pre[kClasses];
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      int x = __popc(my[c]);
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      pre[c] = incl - x;
      if (lane == 31) sh.wcnt[c][warp] = incl;
    }
    __syncthreads();
    if (threadIdx.x < kClasses) {
      int c = threadIdx.x, run = 0;
      for (int q = 0; q < kWarps; ++q) {
        int t = sh.wcnt[c][q];
        sh.wcnt[c][q] = run;
        run += t;
      }
      int b = 0;
      if (run > 0) b = (int)atomicAdd(&slot.list_cnt[c], (unsigned)run);
      sh.base[c] = b;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      unsigned m = my[c];
      int pos = sh.base[c] + sh.wcnt[c][warp] + pre[c];
      int32_t* dst = w.list[nbuf][c];
      while (m) {
        int b = __ffs(m) - 1;
        m &= m - 1;
        int v = (int)(wbase + lane * 32 + b);
        if (c == 3) w.aux3[nbuf][pos] = 0xffffffffu;
        dst[pos++] = v;
        visit(v);
      }
    }
    __syncthreads();
  }
}

// Ballot filter whose active set is already a bitmap (one bit per vertex):
// a lane owns one word, so no ballots are needed; output as above.
template <class Deg, class Visit>
__device__ void bitmap_filter(int n, const uint32_t* bm, Deg deg, Visit visit, CtaShared& sh,
                              const Work& w, const Knobs& k, unsigned grid, int nbuf,
                              PhaseSlot& slot) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const long long nwords = ((long long)n + 31) >> 5;
  for (long long chunk = blockIdx.x; chunk * kBallotChunk < n; chunk += grid) {
    const long long word = chunk * kThreads + (long long)warp * 32 + lane;  // 32 words per warp
    unsigned all = word < nwords ? bm[word] : 0u;
    unsigned my[kClasses] = {0u, 0u, 0u, 0u};
    for (unsigned m = all; m;) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      int v = (int)(word * 32 + b);
      my[degree_class(deg(v), k)] |= 1u << b;
    }
    int pre[kClasses];
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      int x = __popc(my[c]);
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      pre[c] = incl - x;
      if (lane == 31) sh.wcnt[c][warp] = incl;
    }
    __syncthreads();
    if (threadIdx.x < kClasses) {
      int c = threadIdx.x, run = 0;
      for (int q = 0; q < kWarps; ++q) {
        int t = sh.wcnt[c][q];
        sh.wcnt[c][q] = run;
        run += t;
      }
      int b = 0;
      if (run > 0) b = (int)atomicAdd(&slot.list_cnt[c], (unsigned)run);
      sh.base[c] = b;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      unsigned m = my[c];
      int pos = sh.base[c] + sh.wcnt[c][warp] + pre[c];
      int32_t* dst = w.list[nbuf][c];
      while (m) {
        int b = __ffs(m) - 1;
        m &= m - 1;
        int v = (int)(word * 32 + b);
        if (c == 3) w.aux3[nbuf][pos] = 0xffffffffu;
        dst[pos++] = v;
        visit(v);
      }
    }
    __syncthreads();
  }
}

// Class timing: thread 0 of each CTA folds the time its CTA spent in a degree
// class into the phase slot (max over CTAs); the trace reports it.  The
// callers pass no slot (the timing code costs 3.5 % of the grid SSSP's small
// iterations even when it runs every eighth iteration only: 86.0 against
// 83.1 ms), so the class times are 0; the PageRank pull times its phases.

struct ClassTimer {
  PhaseSlot* slot;
  unsigned long long t;
  __device__ explicit ClassTimer(PhaseSlot* s) : slot(s), t(s && threadIdx.x == 0 ? globaltimer() : 0) {}
  __device__ __forceinline__ void lap(int c) {
    if (slot && threadIdx.x == 0) {
      const unsigned long long now = globaltimer();
      atomicMax(&slot->tclass[c], now - t);
      t = now;
    }
  }
};

// ------------------------------------------------------- chunked tasks
// Inclusive prefix (in sh.pref) of the chunk counts ceil(deg / ch) of the nb
// <= kChunkBatch class-3 tasks `items`; returns the chunk size used.  With
// `spread` > 0 a batch of fewer than `spread` x ch edges (one hub, say) is cut
// into chunks of ceil(edges / spread), at least kMinChunk, so that it still
// covers `spread` CTAs.  Every CTA computes the same prefix and size.  All
// threads of the CTA call it.
constexpr long long kMinChunk = kThreads;
struct IdentityVertex {
  __device__ __forceinline__ int operator()(int v) const { return v; }
};

// `rv` maps a task id to the vertex whose CSR row it walks (the identity
// except for a batch of virtual graph copies, whose ids exceed n).
template <class OffT, class RV = IdentityVertex>
__device__ long long chunk_prefix(const int32_t* items, int nb, const OffT* off, long long ch, CtaShared& sh,
                                  RV rv = RV{}, unsigned spread = 0) {
  __syncthreads();
  const int b = threadIdx.x * 4;
  long long d[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    d[q] = 0;
    if (b + q < nb) {
      const int v = rv(items[b + q]);
      d[q] = gload(off + v + 1) - gload(off + v);
    }
  }
  if (spread) {
    const unsigned long long eb = cta_sum_u64((unsigned long long)(d[0] + d[1] + d[2] + d[3]), sh);
    const long long even = (long long)((eb + spread - 1) / spread);
    if (even < ch) ch = even > kMinChunk ? even : kMinChunk;
  }
  int x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = (int)((d[q] + ch - 1) / ch);
  const int tot = x[0] + x[1] + x[2] + x[3];
  int incl = tot;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sh.scan_w[warp] = incl;
  __syncthreads();
  int run = incl - tot;
  for (int q = 0; q < warp; ++q) run += sh.scan_w[q];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    run += x[q];
    if (b + q < nb) sh.pref[b + q] = run;
  }
  __syncthreads();
  return ch;
}

// Task of chunk kc: the smallest i with pref[i] > kc.
__device__ __forceinline__ int chunk_item(const int* pref, int nb, int kc) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (pref[mid] > kc) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Type in which a task's chunk sums are combined (FP64 for FP32 sums: a hub
// cut into hundreds of chunks would otherwise lose precision in the combine).
template <class A> struct Wide { using T = A; };
template <> struct Wide<float> { using T = double; };

__device__ __forceinline__ unsigned long long acc_bits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long acc_bits(unsigned x) { return x; }
__device__ __forceinline__ unsigned long long acc_bits(unsigned long long x) { return x; }
__device__ __forceinline__ void acc_from(unsigned long long b, float& x) { x = __uint_as_float((unsigned)b); }
__device__ __forceinline__ void acc_from(unsigned long long b, unsigned& x) { x = (unsigned)b; }
__device__ __forceinline__ void acc_from(unsigned long long b, unsigned long long& x) { x = b; }
// Add a chunk sum into a task total: FP32 sums go through FP64, other
// accumulators use the functor's own combine.
template <class F>
__device__ __forceinline__ void wide_combine(const F&, double& t, float y) { t += (double)y; }
template <class F, class A>
__device__ __forceinline__ void wide_combine(const F& f, A& t, A y) { f.combine(t, y); }

// ----------------------------------------------------- push class driver
// Visit every edge of every task in the four class lists.  F provides
//   typename F::Src;                                 per-source state
//   bool src(int v, Src& s, int cls, unsigned item); read state; false = skip
//   static Src shfl(const Src&, int lane);
//   int rv(int v);      the vertex whose CSR row task v walks (v itself except
//                       for a batch of virtual graph copies)
//   void edges(const Src (&s)[kPushBatch], const int (&v)[kPushBatch],
//              const int (&u)[kPushBatch], const long long (&p)[kPushBatch],
//              unsigned ok);      // bit q of ok: slot q holds edge (v[q] -> u[q])
// edges() receives kPushBatch edges per lane at once so it can issue all
// their loads, then all their atomics, before it needs any result.  For
// cls 1 / 2 every lane / thread of the group calls src() and it must return
// the same answer in all of them (F broadcasts).  Thread / warp / CTA tasks
// follow Sec. 3.3; class 3 tasks are cut into chunks of `ch` edges dealt
// round-robin to all CTAs (a GB300 addition for the highest degrees).
constexpr int kPushBatch = 4;

template <class F>
__device__ __forceinline__ void push_strided(F& f, const typename F::Src& s, int v, const int32_t* idx,
                                             long long beg, long long end, int lane, int width) {
  typename F::Src ss[kPushBatch];
  int vv[kPushBatch];
#pragma unroll
  for (int q = 0; q < kPushBatch; ++q) {
    ss[q] = s;
    vv[q] = v;
  }
  for (long long b = beg; b < end; b += (long long)width * kPushBatch) {
    int u[kPushBatch];
    long long pp[kPushBatch];
    unsigned ok = 0;
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q) {
      pp[q] = b + lane + (long long)q * width;
      u[q] = 0;
      if (pp[q] < end) {
        u[q] = gload(idx + pp[q]);
        ok |= 1u << q;
      }
    }
    f.edges(ss, vv, u, pp, ok);
  }
}

// ------------------------------------------- bulk-copy staging of edges
// A CTA that walks one contiguous edge range (CTA-class tasks and grid
// chunks) can stage the neighbour indices in shared memory with the bulk
// copy engine (cp.async.bulk, completion counted on an mbarrier), two
// buffers deep: while the CTA relaxes one buffer's edges the next buffer's
// copy is in flight.  Copies are 16-byte aligned and stay inside the index
// array; the unaligned head and the tail past the last whole 16 bytes are
// read from global memory directly.  Every wait is bounded: a copy that
// never completes aborts the run (the barrier then reports it) instead of
// hanging.
constexpr int kStageEdges = 2048;  // indices per buffer (8 KB)

struct __align__(128) StageShared {
  int32_t buf[2][kStageEdges];
  unsigned long long bar[2];  // mbarriers, one per buffer
  unsigned par[2];            // phase parity each buffer's next wait expects
};

struct Stager {
  StageShared* sm;      // nullptr: no staging
  Sync* sync;
  long long e_total;    // entries of the index array
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Thread 0 of the CTA, once per kernel.
__device__ __forceinline__ void stage_init(StageShared& sm) {
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.bar[b])) : "memory");
      sm.par[b] = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Thread 0: copy indices [cs, ce) (cs, ce multiples of 4) into buffer b.
__device__ __forceinline__ void stage_issue(StageShared& sm, int b, const int32_t* idx, long long cs, long long ce) {
  const unsigned bar = smem_addr(&sm.bar[b]);
  const unsigned bytes = (unsigned)((ce - cs) * 4);
  if (bytes == 0) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    return;
  }
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(sm.buf[b])), "l"(idx + cs), "r"(bytes), "r"(bar)
               : "memory");
}

// Every thread: wait for buffer b's copy (bounded), then flip its parity.
__device__ __forceinline__ void stage_wait(StageShared& sm, int b, Sync* sync) {
  const unsigned bar = smem_addr(&sm.bar[b]);
  const unsigned par = sm.par[b];
  for (int round = 0; round < 2; ++round) {
    unsigned done = 0, spins = 0;
    while (!done) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar), "r"(par)
          : "memory");
      if (!done && ++spins > (1u << 20)) break;
    }
    if (done) break;
    // the copy did not complete: abort the run, then wait once more (bounded)
    // for the copy in flight before the buffer is touched again
    if (threadIdx.x == 0 && round == 0) {
      atomicExch(&sync->abort, 1);
      atomicCAS(&sync->err, 0, 4 /* SIMDX_EBARRIER_TIMEOUT */);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.par[b] = par ^ 1u;
}

// Every thread of the CTA: the edges [beg, end) of task v (row rv), their
// indices staged through shared memory, kPushBatch per thread at a time.
template <class F>
__device__ void push_staged(F& f, const typename F::Src& s, int v, const int32_t* idx, long long beg, long long end,
                            const Stager& st) {
  StageShared& sm = *st.sm;
  const long long lim = st.e_total & ~3ll;  // copies stay inside the array
  const long long a0 = beg & ~3ll;
  const int tid = threadIdx.x;
  typename F::Src ss[kPushBatch];
  int vv[kPushBatch];
#pragma unroll
  for (int q = 0; q < kPushBatch; ++q) {
    ss[q] = s;
    vv[q] = v;
  }
  int b = 0;
  if (tid == 0) stage_issue(sm, 0, idx, a0 < lim ? a0 : lim, a0 + kStageEdges < lim ? a0 + kStageEdges : lim);
  for (long long cs = a0; cs < end; cs += kStageEdges, b ^= 1) {
    const long long nx = cs + kStageEdges;
    if (tid == 0 && nx < end)
      stage_issue(sm, b ^ 1, idx, nx < lim ? nx : lim, nx + kStageEdges < lim ? nx + kStageEdges : lim);
    stage_wait(sm, b, st.sync);
    const long long ce = cs + kStageEdges < lim ? cs + kStageEdges : (cs < lim ? lim : cs);  // staged: [cs, ce)
    const long long lo = cs < beg ? beg : cs, hi = nx < end ? nx : end;
    for (long long p0 = lo; p0 < hi; p0 += (long long)kThreads * kPushBatch) {
      int u[kPushBatch];
      long long pp[kPushBatch];
      unsigned ok = 0;
#pragma unroll
      for (int q = 0; q < kPushBatch; ++q) {
        pp[q] = p0 + tid + (long long)q * kThreads;
        u[q] = 0;
        if (pp[q] < hi) {
          u[q] = pp[q] < ce ? sm.buf[b][pp[q] - cs] : gload(idx + pp[q]);
          ok |= 1u << q;
        }
      }
      f.edges(ss, vv, u, pp, ok);
    }
    __syncthreads();  // buffer b is free for the copy issued next round
  }
}

template <class OffT, class F>
__device__ void push_classes(F& f, const OffT* off, const int32_t* idx,
                             const int32_t* const* lists, const unsigned* cnt, unsigned grid,
                             long long ch, CtaShared& sh, long long& evisit, PhaseSlot* slot = nullptr,
                             const Stager* stg = nullptr) {
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  ClassTimer tm(slot);
  // class 3: every task is cut into chunks of `ch` edges (fewer when the batch
  // would not fill the grid) and the chunks of all tasks are dealt round-robin
  // to the CTAs (edge-balanced over the grid)
  auto rvf = [&f](int v) { return f.rv(v); };
  for (unsigned b0 = 0; b0 < cnt[3]; b0 += kChunkBatch) {
    const int nb = (int)min((unsigned)kChunkBatch, cnt[3] - b0);
    const long long cb = chunk_prefix(lists[3] + b0, nb, off, ch, sh, rvf, grid);
    const int total = sh.pref[nb - 1];
    for (int kc = blockIdx.x; kc < total; kc += grid) {
      const int item = chunk_item(sh.pref, nb, kc);
      const int first = item ? sh.pref[item - 1] : 0;
      const int v = lists[3][b0 + item];
      const int rv = f.rv(v);
      const long long vb = gload(off + rv), ve = gload(off + rv + 1);
      const long long beg = vb + (long long)(kc - first) * cb;
      const long long end = beg + cb < ve ? beg + cb : ve;
      typename F::Src s;
      if (!f.src(v, s, 3, b0 + item)) continue;
      if (stg && stg->sm) push_staged(f, s, v, idx, beg, end, *stg);
      else push_strided(f, s, v, idx, beg, end, tid, kThreads);
      if (tid == 0) evisit += end - beg;
    }
  }
  tm.lap(3);
  // class 2: one CTA per task
  for (unsigned i = blockIdx.x; i < cnt[2]; i += grid) {
    int v = lists[2][i];
    typename F::Src s;
    if (!f.src(v, s, 2, i)) continue;
    const int rv = f.rv(v);
    long long beg = gload(off + rv), end = gload(off + rv + 1);
    if (stg && stg->sm) push_staged(f, s, v, idx, beg, end, *stg);
    else push_strided(f, s, v, idx, beg, end, tid, kThreads);
    if (tid == 0) evisit += end - beg;
  }
  tm.lap(2);
  // class 1: one warp per task
  {
    const unsigned gw = blockIdx.x * kWarps + warp, nw = grid * kWarps;
    for (unsigned i = gw; i < cnt[1]; i += nw) {
      int v = lists[1][i];
      typename F::Src s;
      if (!f.src(v, s, 1, i)) continue;
      const int rv = f.rv(v);
      long long beg = gload(off + rv), end = gload(off + rv + 1);
      push_strided(f, s, v, idx, beg, end, lane, 32);
      if (lane == 0) evisit += end - beg;
    }
  }
  tm.lap(1);
  // class 0: groups of up to 32 consecutive tasks per warp (fewer when the
  // list is short, so every warp gets work).  The warp walks the group's
  // concatenated edges, kPushBatch rounds of 32 edge slots at a time
  // (coalesced index loads); each slot finds its task by a binary search over
  // the warp's inclusive degree scan.
  const unsigned nw0 = grid * kWarps;
  unsigned gs = (cnt[0] + nw0 - 1) / nw0;
  gs = gs < 1 ? 1 : (gs > 32 ? 32 : gs);
  for (unsigned base = (blockIdx.x * kWarps + warp) * gs; base < cnt[0]; base += nw0 * gs) {
    const unsigned lim = base + gs < cnt[0] ? base + gs : cnt[0];
    const unsigned i = base + lane;
    int v = -1, deg = 0;
    long long beg = 0;
    typename F::Src s{};
    if (i < lim) {
      v = lists[0][i];
      if (f.src(v, s, 0, i)) {
        const int rv = f.rv(v);
        beg = gload(off + rv);
        deg = (int)(gload(off + rv + 1) - beg);
      }
    }
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - deg;
    for (int e0 = 0; e0 < total; e0 += 32 * kPushBatch) {
      typename F::Src sq[kPushBatch];
      int vq[kPushBatch], uq[kPushBatch];
      long long pq[kPushBatch];
      unsigned ok = 0;
#pragma unroll
      for (int q = 0; q < kPushBatch; ++q) {
        const int e = e0 + 32 * q + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          int t = __shfl_sync(kFull, incl, j + step - 1);
          if (t <= e) j += step;
        }
        const long long bj = __shfl_sync(kFull, beg, j);
        const int xj = __shfl_sync(kFull, excl, j);
        vq[q] = __shfl_sync(kFull, v, j);
        sq[q] = F::shfl(s, j);
        pq[q] = bj + (e - xj);
        uq[q] = 0;
        if (e < total) ok |= 1u << q;
      }
#pragma unroll
      for (int q = 0; q < kPushBatch; ++q)
        if ((ok >> q) & 1u) uq[q] = gload(idx + pq[q]);
      f.edges(sq, vq, uq, pq, ok);
    }
    evisit += deg;
  }
  tm.lap(0);
}

// ----------------------------------------------------- pull class driver
// For every task u in the class lists, combine (sum) a per-edge value over
// u's in-edges and hand the total to F:
//   typename F::Acc;  Acc zero();  void edge(Acc&, int u, int v, long long p);
//   void combine(Acc&, Acc) const;   (commutative, associative: the Combine)
//   void finish(int u, Acc total);   (called by exactly one thread per task)
// Small tasks are summed by warp_segmented_sum; warp tasks lane-strided with
// a fixed shuffle tree; CTA tasks with a fixed block tree; chunked tasks add
// their chunk sums in chunk order.  The order of every sum is therefore fixed.
template <class F, class Acc>
__device__ __forceinline__ Acc warp_sum(const F& f, Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f.combine(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Sum over the in-edges of tasks list[t_begin, t_end) (at most 32 tasks per
// window), one warp.  The warp walks the concatenated edges of a window of
// tasks in rounds of 32 edge slots, kSegUnroll rounds at a time: all index
// loads of those rounds are issued first, then all gathers, then the
// reductions, so each lane has several independent loads in flight.  Within
// a round the slots of one task are contiguous and are summed by a fixed
// shuffle tree toward the task's first slot; that partial is added to the
// task's accumulator, held by the task's own lane, in round order.  The order
// of every sum therefore depends only on the task list and the window start.
constexpr int kSegUnroll = 4;

template <class OffT, class F>
__device__ void warp_segmented_sum(F& f, const OffT* off, const int32_t* idx, const int32_t* list,
                                   unsigned t_begin, unsigned t_end, long long& evisit) {
  using Acc = typename F::Acc;
  const int lane = lane_id();
  for (unsigned t0 = t_begin; t0 < t_end; t0 += 32) {
    const unsigned i = t0 + lane;
    int u = -1, deg = 0;
    long long beg = 0;
    if (i < t_end) {
      u = list[i];
      beg = gload(off + u);
      deg = (int)(gload(off + u + 1) - beg);
    }
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - deg;
    Acc acc = f.zero();
    for (int e0 = 0; e0 < total; e0 += 32 * kSegUnroll) {
      int jq[kSegUnroll], vq[kSegUnroll], uq[kSegUnroll];
      long long pq[kSegUnroll];
#pragma unroll
      for (int q = 0; q < kSegUnroll; ++q) {
        const int e = e0 + 32 * q + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          int t = __shfl_sync(kFull, incl, j + step - 1);
          if (t <= e) j += step;
        }
        const long long bj = __shfl_sync(kFull, beg, j);
        const int xj = __shfl_sync(kFull, excl, j);
        uq[q] = __shfl_sync(kFull, u, j);
        pq[q] = bj + (e - xj);
        jq[q] = e < total ? j : 32;  // 32: no task
      }
#pragma unroll
      for (int q = 0; q < kSegUnroll; ++q) vq[q] = jq[q] < 32 ? gload(idx + pq[q]) : 0;
      Acc val[kSegUnroll];
#pragma unroll
      for (int q = 0; q < kSegUnroll; ++q) {
        val[q] = f.zero();
        if (jq[q] < 32) f.edge(val[q], uq[q], vq[q], pq[q]);
      }
#pragma unroll
      for (int q = 0; q < kSegUnroll; ++q) {
        Acc x = val[q];
        const int j = jq[q];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          Acc y = __shfl_down_sync(kFull, x, d);
          int jy = __shfl_down_sync(kFull, j, d);
          if (lane + d < 32 && jy == j) f.combine(x, y);
        }
        const int r0 = e0 + 32 * q;
        int h = excl - r0;
        h = h < 0 ? 0 : (h > 31 ? 31 : h);
        Acc part = __shfl_sync(kFull, x, h);
        if (deg > 0 && excl < r0 + 32 && incl > r0) f.combine(acc, part);
      }
    }
    if (u >= 0) {
      f.finish(u, acc);
      evisit += deg;
    }
  }
}

template <class OffT, class F>
__device__ void pull_classes(F& f, const OffT* off, const int32_t* idx, const int32_t* const* lists,
                             const unsigned* cnt, unsigned grid, typename F::Acc* red, long long ch,
                             CtaShared& sh, const Work& w, long long& evisit, PhaseSlot* slot = nullptr) {
  using Acc = typename F::Acc;
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  ClassTimer tm(slot);
  // class 3: chunks of `ch` edges dealt round-robin to the CTAs; each chunk's
  // sum goes to chunk_part, and the CTA that finishes a task's last chunk adds
  // the task's chunk sums in chunk order (fixed) and finishes the task.
  // Partials and counters are indexed across batches (gbase, b0 + item): no
  // barrier separates batches, so a finisher may still be reading while other
  // CTAs work on the next batch.
  long long gbase = 0;
  for (unsigned b0 = 0; b0 < cnt[3]; b0 += kChunkBatch) {
    const int nb = (int)min((unsigned)kChunkBatch, cnt[3] - b0);
    chunk_prefix(lists[3] + b0, nb, off, ch, sh);
    const int total = sh.pref[nb - 1];
    for (int kc = blockIdx.x; kc < total; kc += grid) {
      const int item = chunk_item(sh.pref, nb, kc);
      const int first = item ? sh.pref[item - 1] : 0;
      const int nch = sh.pref[item] - first;
      const int u = lists[3][b0 + item];
      const long long ub = gload(off + u), ue = gload(off + u + 1);
      const long long beg = ub + (long long)(kc - first) * ch;
      const long long end = beg + ch < ue ? beg + ch : ue;
      Acc a = f.zero();
#pragma unroll 4
      for (long long p = beg + tid; p < end; p += kThreads) f.edge(a, u, gload(idx + p), p);
      a = warp_sum(f, a);
      __syncthreads();
      if (lane == 0) red[warp] = a;
      __syncthreads();
      if (tid == 0) {
        Acc t = f.zero();
#pragma unroll
        for (int q = 0; q < kWarps; ++q) f.combine(t, red[q]);
        evisit += end - beg;
        if (nch == 1) {
          f.finish(u, t);
        } else {
          w.chunk_part[gbase + kc] = acc_bits(t);
          __threadfence();
          const int done = atomicAdd(&w.chunk_done[b0 + item], 1);
          if (done == nch - 1) {
            __threadfence();
            typename Wide<Acc>::T tot = (typename Wide<Acc>::T)f.zero();  // chunk sums in chunk order
            const volatile unsigned long long* part = w.chunk_part + gbase + first;
            for (int j = 0; j < nch; ++j) {
              Acc y;
              acc_from(part[j], y);
              wide_combine(f, tot, y);
            }
            w.chunk_done[b0 + item] = 0;
            f.finish(u, (Acc)tot);
          }
        }
      }
    }
    gbase += total;
  }
  tm.lap(3);
  // class 2: one CTA per task
  for (unsigned i = blockIdx.x; i < cnt[2]; i += grid) {
    int u = lists[2][i];
    long long beg = gload(off + u), end = gload(off + u + 1);
    Acc a = f.zero();
#pragma unroll 4
    for (long long p = beg + tid; p < end; p += kThreads) f.edge(a, u, gload(idx + p), p);
    a = warp_sum(f, a);
    __syncthreads();
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (tid == 0) {
      Acc t = f.zero();
#pragma unroll
      for (int q = 0; q < kWarps; ++q) f.combine(t, red[q]);
      f.finish(u, t);
      evisit += end - beg;
    }
  }
  tm.lap(2);
  {
  const unsigned gw = blockIdx.x * kWarps + warp, nw = grid * kWarps;
  for (unsigned i = gw; i < cnt[1]; i += nw) {
    int u = lists[1][i];
    long long beg = gload(off + u), end = gload(off + u + 1);
    Acc a = f.zero();
#pragma unroll 4
    for (long long p = beg + lane; p < end; p += 32) f.edge(a, u, gload(idx + p), p);
    a = warp_sum(f, a);
    if (lane == 0) {
      f.finish(u, a);
      evisit += end - beg;
    }
  }
  }
  tm.lap(1);
  // class 0: groups of up to 32 consecutive tasks per warp (fewer when the
  // list is short, so every warp gets work), walked by warp_segmented_sum
  const unsigned nw = grid * kWarps;
  unsigned gs = (cnt[0] + nw - 1) / nw;
  gs = gs < 1 ? 1 : (gs > 32 ? 32 : gs);
  for (unsigned base = (blockIdx.x * kWarps + warp) * gs; base < cnt[0]; base += nw * gs) {
    const unsigned lim = base + gs < cnt[0] ? base + gs : cnt[0];
    warp_segmented_sum<OffT>(f, off, idx, lists[0], base, lim, evisit);
  }
  tm.lap(0);
}

// ------------------------------------- deterministic (two-pass) ballot filter
// Same output as ballot_filter but globally sorted and identical run to run:
// pass 1 counts each chunk's active vertices per class; after a grid barrier
// pass 2 writes each chunk at the prefix of the counts of earlier chunks (the
// prefix-scan concatenation of Sec. 3.3, no atomics).  The caller runs
// count_pass, grid_sync, write_pass.
template <class Pred, class Cls>
__device__ void det_filter_count(int n, Pred pred, Cls cls_of, CtaShared& sh, const Work& w, unsigned grid) {
  for (long long chunk = blockIdx.x; chunk * kBallotChunk < n; chunk += grid) {
    int my[kClasses] = {0, 0, 0, 0};
    for (int j = threadIdx.x; j < kBallotChunk; j += kThreads) {
      long long v = chunk * kBallotChunk + j;
      if (v < n && pred((int)v)) my[cls_of((int)v)]++;
    }
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      int t = (int)cta_sum_u64((unsigned long long)my[c], sh);
      if (threadIdx.x == 0) w.chunk_cnt[chunk * kClasses + c] = t;
    }
  }
}

template <class Pred, class Cls>
__device__ void det_filter_write(int n, Pred pred, Cls cls_of, CtaShared& sh, const Work& w, unsigned grid,
                                 int nbuf, unsigned* totals) {
  const long long nchunks = ((long long)n + kBallotChunk - 1) / kBallotChunk;
  // totals over all chunks (every CTA computes them; fixed order)
#pragma unroll
  for (int c = 0; c < kClasses; ++c) {
    unsigned long long t = 0;
    for (long long q = threadIdx.x; q < nchunks; q += kThreads) t += (unsigned)w.chunk_cnt[q * kClasses + c];
    totals[c] = (unsigned)cta_sum_u64(t, sh);
  }
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += grid) {
    if (threadIdx.x < kClasses) sh.bcast_i[threadIdx.x] = 0;
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      unsigned long long t = 0;
      for (long long q = threadIdx.x; q < chunk; q += kThreads) t += (unsigned)w.chunk_cnt[q * kClasses + c];
      t = cta_sum_u64(t, sh);
      if (threadIdx.x == 0) sh.base[c] = (int)t;
    }
    const long long wbase = chunk * kBallotChunk + (long long)warp * 1024;
    unsigned my[kClasses] = {0u, 0u, 0u, 0u};
    for (int j = 0; j < 32; ++j) {
      long long v = wbase + j * 32 + lane;
      bool act = false;
      int cls = 0;
      if (v < n && pred((int)v)) {
        act = true;
        cls = cls_of((int)v);
      }
#pragma unroll
      for (int c = 0; c < kClasses; ++c) {
        unsigned m = __ballot_sync(kFull, act && cls == c);
        if (lane == j) my[c] = m;
      }
    }
    int pre[kClasses];
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      int x = __popc(my[c]);
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      pre[c] = incl - x;
      if (lane == 31) sh.wcnt[c][warp] = incl;
    }
    __syncthreads();
    if (threadIdx.x < kClasses) {
      int c = threadIdx.x, run = 0;
      for (int q = 0; q < kWarps; ++q) {
        int t = sh.wcnt[c][q];
        sh.wcnt[c][q] = run;
        run += t;
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
      unsigned m = my[c];
      int pos = sh.base[c] + sh.wcnt[c][warp] + pre[c];
      int32_t* dst = w.list[nbuf][c];
      while (m) {
        int b = __ffs(m) - 1;
        m &= m - 1;
        dst[pos++] = (int)(wbase + lane * 32 + b);
      }
    }
    __syncthreads();
  }
}

// Write one trace record (CTA 0 thread 0 only): flags, active vertices,
// active edges, level / bucket, and %globaltimer at the iteration's start and
// end as seen by CTA 0.
__device__ __forceinline__ void trace_put(const Work& w, int it, long long a, long long b, long long c,
                                          long long d, unsigned long long t0 = 0, unsigned long long t1 = 0) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && it < w.trace_cap) {
    long long* r = w.trace + (long long)kTraceWords * it;
    r[0] = a; r[1] = b; r[2] = c; r[3] = d;
    r[4] = (long long)t0;
    r[5] = (long long)(t1 ? t1 : globaltimer());
    r[6] = 0; r[7] = 0;
  }
}

// Trace words 6 and 7 (when a slot was timed, else 0): the slowest CTA's
// time (ns, 32 bits each) in degree
// classes 3 | 2 and 1 | 0 of the iteration's compute phase.
__device__ __forceinline__ void trace_classes(const Work& w, int it, const PhaseSlot& p) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && it < w.trace_cap) {
    auto c32 = [](unsigned long long x) { return x > 0xffffffffull ? 0xffffffffull : x; };
    long long* r = w.trace + (long long)kTraceWords * it;
    r[6] = (long long)((c32(p.tclass[3]) << 32) | c32(p.tclass[2]));
    r[7] = (long long)((c32(p.tclass[1]) << 32) | c32(p.tclass[0]));
  }
}

}  // namespace simdx
