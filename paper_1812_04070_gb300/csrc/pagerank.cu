// pagerank.cu -- PageRank as one persistent ACC kernel (Sec. 6 "PageRank";
// aggregation combine = sum, pull, all vertices active).
//
//   x_0 = 1/n
//   x_{t+1}(v) = (1-d)/n + d * ( sum_{u in N_in(v)} c_t(u) + D_t / n )
//   c_t(u) = x_t(u) / outdeg(u)      (0 for outdeg 0)
//   D_t    = sum of x_t over vertices with outdeg 0
// stopping after the first iteration with ||x_{t+1} - x_t||_1 < tol.
//
// All vertices are active in every iteration, so the ballot filter runs once
// (Sec. 4: PageRank needs the ballot filter exactly at the first iteration)
// and its sorted task lists are reused.  Vertices of in-degree < med_max form
// one list that is cut, once per run, into task-aligned ranges of equal edge
// count, one per warp (a degree prefix over the list and a binary search per
// warp); each warp walks its range with warp_segmented_sum.  Higher in-degree
// vertices keep the CTA-per-task and chunked classes.  Each vertex sums its in-neighbours'
// contributions in FP32 in a fixed order (small tasks: 32-slot rounds summed
// by a fixed shuffle tree; warp / CTA tasks: lane-strided partial sums and a
// fixed tree; chunked tasks: chunk sums added in chunk order).  The two global
// sums (L1 change and dangling rank) add one 2^-60 fixed-point integer per
// vertex, whose total does not depend on which CTA adds it or when: together
// with the deterministic task lists this makes every run bit-identical.
// One grid barrier per iteration: the sums of iteration t are read right
// after its barrier, before iteration t+1 starts.
#include "simdx_internal.h"

namespace simdx {

constexpr double kFix = 1152921504606846976.0;  // 2^60

__device__ __forceinline__ unsigned long long to_fix(double x) { return __double2ull_rn(x * kFix); }

template <class OffT>
struct PrArgs {
  int n;
  float d, tol;
  int max_iter;
  const OffT* off;   // out-edges (out-degree)
  const OffT* ioff;  // in-edges
  const int32_t* iidx;
  float* rank;
  Work w;
  Knobs k;
};

template <class OffT>
struct PrPull {
  using Acc = float;
  const float* cin;
  float* cout;
  const float* xold;
  float* xnew;
  const OffT* off;
  float base, d, dn;
  unsigned long long l1 = 0, dang = 0;  // 2^-60 fixed point, one rounding per vertex
  __device__ __forceinline__ Acc zero() const { return 0.f; }
  __device__ __forceinline__ void combine(Acc& a, Acc b) const { a += b; }
  __device__ __forceinline__ void edge(Acc& a, int, int v, long long) { a += cin[v]; }
  __device__ __forceinline__ void finish(int u, Acc sum) {
    const float xn = base + d * (sum + dn);
    xnew[u] = xn;
    const long long od = (long long)gload(off + u + 1) - (long long)gload(off + u);
    cout[u] = od > 0 ? xn / (float)od : 0.f;
    if (od == 0) dang += to_fix((double)xn);
    l1 += to_fix(fabs((double)xn - (double)xold[u]));
  }
};

template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) pagerank_kernel(PrArgs<OffT> a) {
  __shared__ CtaShared sh;
  __shared__ float red_f[kWarps];
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  float* xalt = reinterpret_cast<float*>(a.w.state);
  float* cbuf[2] = {xalt + n, xalt + 2 * (size_t)n};
  float* xbuf[2] = {a.rank, xalt};
  const OffT* off = a.off;
  const OffT* ioff = a.ioff;
  auto indeg = [ioff](int v) { return (long long)gload(ioff + v + 1) - (long long)gload(ioff + v); };
  auto all = [](int) { return true; };
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // Task classes for PageRank: vertices of in-degree 0 (class 1) only take
  // the constant teleport + dangling share; every other vertex of in-degree
  // < med_max goes to one list (class 0) that is walked edge-balanced by
  // warps; the rest keep their CTA (2) / chunked (3) classes.
  const int med_max = k.med_max, huge_min = k.huge_min;
  auto pr_class = [ioff, med_max, huge_min](int v) {
    const long long d = (long long)gload(ioff + v + 1) - (long long)gload(ioff + v);
    return d == 0 ? 1 : d < med_max ? 0 : d < huge_min ? 2 : 3;
  };
  // ---- phase 0: x_0, c_0, D_0 and the per-chunk class counts
  {
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[0];
    const float x0 = 1.0f / (float)n;
    unsigned long long dang = 0;
    for (long long v = gtid; v < n; v += gthreads) {
      const long long od = (long long)gload(off + v + 1) - (long long)gload(off + v);
      xbuf[0][v] = x0;
      cbuf[0][v] = od > 0 ? x0 / (float)od : 0.f;
      if (od == 0) dang += to_fix((double)x0);
    }
    dang = cta_sum_u64(dang, sh);
    if (threadIdx.x == 0) atomicAdd(&slot.aux0, dang);
    det_filter_count(n, all, pr_class, sh, a.w, grid);
  }
  if (!grid_sync(s, grid, sh, k)) return;
  unsigned long long Dfix = s->slot[0].aux0;
  // ---- phase 1: sorted task lists of all vertices by in-degree
  unsigned cnt[kClasses];
  clear_next_slot(s, sh);
  det_filter_write(n, all, pr_class, sh, a.w, grid, 0, cnt);
  if (!grid_sync(s, grid, sh, k)) return;
  // ---- phases 2-4: balanced, task-aligned ranges of list 0 per warp.  A task
  // weighs (in-degree + 1): zero-degree vertices still cost a slot, and they
  // come in long runs (isolated vertices), so edges alone would not balance.
  const int32_t* l0 = a.w.list[0][0];
  const unsigned c0n = cnt[0];
  long long* pre = reinterpret_cast<long long*>(xalt + 3 * (size_t)n + 2);  // [c0n + 1] task start edges
  pre = reinterpret_cast<long long*>((reinterpret_cast<uintptr_t>(pre) + 7) & ~(uintptr_t)7);
  unsigned long long* bsum = reinterpret_cast<unsigned long long*>(a.w.chunk_part);
  const long long nblk = ((long long)c0n + kBallotChunk - 1) / kBallotChunk;
  clear_next_slot(s, sh);
  for (long long b = blockIdx.x; b < nblk; b += grid) {  // block degree sums
    unsigned long long t = 0;
    for (long long q = b * kBallotChunk + threadIdx.x; q < (b + 1) * kBallotChunk && q < c0n; q += kThreads)
      t += (unsigned long long)indeg(l0[q]) + 1ull;
    t = cta_sum_u64(t, sh);
    if (threadIdx.x == 0) bsum[b] = t;
  }
  if (!grid_sync(s, grid, sh, k)) return;
  clear_next_slot(s, sh);
  unsigned long long mtot = 0;
  {
    unsigned long long t = 0;
    for (long long q = threadIdx.x; q < nblk; q += kThreads) t += bsum[q];
    mtot = cta_sum_u64(t, sh);
  }
  for (long long b = blockIdx.x; b < nblk; b += grid) {  // task start edges
    unsigned long long run = 0;
    for (long long q = threadIdx.x; q < b; q += kThreads) run += bsum[q];
    run = cta_sum_u64(run, sh);
    constexpr int kPer = kBallotChunk / kThreads;  // consecutive tasks per thread
    const long long t0 = b * kBallotChunk + (long long)threadIdx.x * kPer;
    unsigned long long mine = 0;
    for (int q = 0; q < kPer; ++q)
      if (t0 + q < c0n) mine += (unsigned long long)indeg(l0[t0 + q]) + 1ull;
    // exclusive scan of `mine` over the CTA
    unsigned long long incl = mine;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) sh.red64[warp] = incl;
    __syncthreads();
    unsigned long long ex = run + incl - mine;
    for (int q = 0; q < warp; ++q) ex += sh.red64[q];
    for (int q = 0; q < kPer; ++q)
      if (t0 + q < c0n) {
        pre[t0 + q] = (long long)ex;
        ex += (unsigned long long)indeg(l0[t0 + q]) + 1ull;
      }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pre[c0n] = (long long)mtot;
  if (!grid_sync(s, grid, sh, k)) return;
  clear_next_slot(s, sh);
  const unsigned nwarps = grid * kWarps;
  for (unsigned wv = blockIdx.x * kThreads + threadIdx.x; wv <= nwarps; wv += grid * kThreads) {
    // first task whose start edge is >= this warp's share boundary
    const long long x = (long long)((mtot * (unsigned long long)wv) / nwarps);
    unsigned lo = 0, hi = c0n;
    while (lo < hi) {
      unsigned mid = (lo + hi) >> 1;
      if (pre[mid] < x) lo = mid + 1; else hi = mid;
    }
    a.w.warp_start[wv] = wv == nwarps ? (int)c0n : (int)lo;
  }
  if (!grid_sync(s, grid, sh, k)) return;
  const unsigned my_warp = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const unsigned w_beg = (unsigned)a.w.warp_start[my_warp], w_end = (unsigned)a.w.warp_start[my_warp + 1];
  const unsigned cnt_big[kClasses] = {0u, 0u, cnt[2], cnt[3]};
  const int32_t* lists[kClasses] = {a.w.list[0][0], a.w.list[0][1], a.w.list[0][2], a.w.list[0][3]};

  const float base = (1.0f - a.d) / (float)n;
  int t = 0;
  double l1_last = 0.0;
  long long evisit = 0;
  while (true) {
    if (t >= a.max_iter) break;
    const unsigned long long t_it = globaltimer();
    // ---- compute x_{t+1}
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    PrPull<OffT> f;
    f.cin = cbuf[t & 1];
    f.cout = cbuf[(t + 1) & 1];
    f.xold = xbuf[t & 1];
    f.xnew = xbuf[(t + 1) & 1];
    f.off = off;
    f.base = base;
    f.d = a.d;
    f.dn = (float)(((double)Dfix / kFix) / (double)n);
    pull_classes<OffT>(f, ioff, a.iidx, lists, cnt_big, grid, red_f, k.huge_min, sh, a.w, evisit, &slot);
    {
      ClassTimer tm(&slot);
      warp_segmented_sum<OffT>(f, ioff, a.iidx, l0, w_beg, w_end, evisit);
      tm.lap(0);
      for (unsigned i = blockIdx.x * kThreads + threadIdx.x; i < cnt[1]; i += grid * kThreads)
        f.finish(lists[1][i], 0.f);  // in-degree 0
      tm.lap(1);
    }
    const unsigned long long l1 = cta_sum_u64(f.l1, sh);
    const unsigned long long dg = cta_sum_u64(f.dang, sh);
    if (threadIdx.x == 0) {
      atomicAdd(&slot.aux0, dg);
      atomicAdd(&slot.aux1, l1);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    Dfix = p.aux0;
    l1_last = (double)p.aux1 / kFix;
    trace_put(a.w, t, 2 | (2 << 8), n, 0, (long long)p.aux1, t_it);
    trace_classes(a.w, t, p);
    ++t;
    if (l1_last < (double)a.tol) break;
  }
  // ---- result: x_t lives in xbuf[t & 1]
  if (t & 1)
    for (long long v = gtid; v < n; v += gthreads) a.rank[v] = xalt[v];
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = t;
    st.push_iters = 0;
    st.pull_iters = t;
    st.ballot_iters = 1;
    st.online_iters = 0;
    st.phases = (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = (long long)t * n;
    st.last_l1 = l1_last;
  }
}

const void* pagerank_kernel_ptr(int off_bits) {
  return off_bits == 32 ? (const void*)pagerank_kernel<int32_t> : (const void*)pagerank_kernel<long long>;
}

template <class OffT>
static int run_pr(simdx_graph* g, float d, float tol, int max_iter, float* rank, simdx_stats* stats,
                  cudaStream_t st) {
  PrArgs<OffT> a{};
  a.n = (int)g->n;
  a.d = d;
  a.tol = tol;
  a.max_iter = max_iter;
  a.off = (const OffT*)g->off;
  a.ioff = (const OffT*)g->in_off;
  a.iidx = g->in_idx;
  a.rank = rank;
  a.w = make_work(g);
  a.k = make_knobs(g);
  const void* kern = (const void*)pagerank_kernel<OffT>;
  int grid = grid_for(g, kern);
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st);
}

}  // namespace simdx

using namespace simdx;

extern "C" int simdx_pagerank(simdx_graph* g, float damping, float l1_tol, int32_t max_iter, float* rank,
                              simdx_stats* stats, void* stream) {
  if (!g || !rank || !(damping >= 0.f && damping < 1.f) || max_iter < 0 || !(l1_tol >= 0.f))
    return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    int rc = prepare_launch(g, st);
    return rc ? rc : finish_launch(g, stats, st);
  }
  return g->off_bits == 32 ? run_pr<int32_t>(g, damping, l1_tol, max_iter, rank, stats, st)
                           : run_pr<long long>(g, damping, l1_tol, max_iter, rank, stats, st);
}
