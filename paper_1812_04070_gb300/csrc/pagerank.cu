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
// (Sec. 4: PageRank needs the ballot filter exactly at the first iteration);
// it splits the vertices into those with in-edges (list 0, vertex order) and
// those without (list 1).  Because the active set never changes, the compute
// step does not walk tasks at all: the in-edge array is cut once per run into
// equal ranges of 128-edge tiles, one range per warp, and each warp streams
// its range (each lane four consecutive edges, one 16-byte load).  A bit per
// in-edge marks the first edge of each row; rows are found from these bits,
// their rank among the marked edges indexing list 0.  Within a tile a lane
// sums its edges in order, restarting at row starts, and the sums of rows
// that cross lanes are carried by a segmented scan over the 32 lanes; the
// part of a row that crosses tiles is carried as an unevaluated FP32 pair
// (TwoSum), close to FP64 accuracy at the FP32 rate.  A row that crosses a
// warp boundary is finished by the last of its warps to arrive, which adds the
// warps' partials in warp order (FP64).  Every sum therefore has a fixed order for a
// given grid.  The two global sums (L1 change and dangling rank) are summed
// per thread in FP32, in the thread's fixed order, and each thread's share is
// added as one 2^-60 fixed-point integer, whose total does not depend on which
// CTA adds it or when: together with the deterministic lists this makes every
// run bit-identical.  One grid barrier per iteration: the sums of iteration t are
// read right after its barrier, before iteration t+1 starts.
#include <algorithm>

#include "simdx_internal.h"

namespace simdx {

constexpr double kFix = 1152921504606846976.0;  // 2^60
constexpr int kTile = 128;                       // in-edges per warp tile (4 per lane)
constexpr int kPrChunk = 2048;                   // tiles per chunk of the cost prefix (8 per thread)
constexpr int kPrRowCost = 4;                    // a row's finish costs about four in-edges

// round(x * 2^60) for a float 0 <= x < 8, from the float's exponent and
// mantissa bits (integer arithmetic: FP64 runs at a small fraction of the
// FP32 rate on this GPU, and this is done once per vertex per iteration).
// Halves round up; values below 2^-61 give 0.
__device__ __forceinline__ unsigned long long to_fix(float x) {
  const unsigned b = __float_as_uint(x);
  const int e = (int)(b >> 23) & 0xFF;
  if (e == 0) return 0ull;  // zero or subnormal
  const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
  const int sh = e - 90;  // x * 2^60 = m * 2^(e - 127 - 23 + 60)
  if (sh >= 0) return sh > 39 ? ~0ull >> 1 : m << sh;
  if (sh < -25) return 0ull;
  return (m + (1ull << (-sh - 1))) >> (-sh);
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest adds, kept apart
// from any contraction by the _rn intrinsics).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Per-run layout of the in-edge walk.
struct PrWalk {
  uint32_t* head;            // [4 * ntiles + 8] bit p: in-edge p is the first of its row; bit E marks the end
  unsigned long long* pre;   // [ntiles + 1] exclusive prefix of the tile costs
  unsigned long long* csum;  // [ceil(ntiles / kPrChunk)] tile cost per chunk of tiles
  int* tstart;               // [warps + 1] first tile of each warp's range
  double* tailp;             // [warps] partial of the row left open at the end of a warp's range
  double* headp;             // [warps] partial of the row that continues into a warp's range
  int* done;                 // [warps] arrivals for the cross-warp row ending in that warp
  unsigned long long* wtime; // [warps] SM cycles each warp's walk took (re-cut iteration)
  unsigned long long* wpre;  // [warps + 1] exclusive prefix of wtime
  int* tstart2;              // [warps + 1] the ranges cut by measured time
  long long ntiles;          // ceil(E / kTile)
  int row_cost;              // cost of finishing a row, in in-edges
  int vec4;                  // in-edge array is 16-byte aligned
};

template <class OffT>
struct PrArgs {
  int n;
  float d, tol;
  int max_iter;
  const OffT* off;   // out-edges (out-degree)
  const int32_t* idx;
  const OffT* ioff;  // in-edges
  const int32_t* iidx;
  long long e;       // in-edges
  float* rank;
  float* inv;        // [n] 1 / outdeg (0 for outdeg 0), set once per run
  // switch from pull to push (the push-tail instantiation only)
  float alpha, theta, rho;
  int recut;                // re-cut the warp ranges by measured time after this iteration (0: never)
  unsigned long long* res;  // [n] pending rank change, signed 2^-60 fixed point
  long long* push_c;        // [n] what a selected vertex sends along each out-edge (2^-60)
  PrWalk wk;
  Work w;
  Knobs k;
};

// Per-iteration view: where c_t is read and x_{t+1}, c_{t+1} are written,
// plus this thread's share of the two global sums.
template <class OffT>
struct PrPull {
  const float* cin;
  float* cout;
  const float* xold;
  float* xnew;
  float dn;                             // d * D_t / n folded with the teleport term below
  float l1 = 0.f, dang = 0.f;  // this thread's share, summed in its own fixed order
  // x_{t+1}(u) and c_{t+1}(u) from the in-neighbour sum, given 1/outdeg(u)
  // and x_t(u) already loaded (loads and stores kept apart so that several
  // rows' loads are in flight together).
  __device__ __forceinline__ void store(const PrArgs<OffT>& a, float base, int u, float sum, float iv, float xo) {
    const float xn = base + a.d * (sum + dn);
    xnew[u] = xn;
    cout[u] = xn * iv;
    if (iv == 0.f) dang += xn;
    l1 += fabsf(xn - xo);
  }
  __device__ __forceinline__ void finish(const PrArgs<OffT>& a, float base, int u, float sum) {
    store(a, base, u, sum, a.inv[u], xold[u]);
  }
};

__device__ __forceinline__ float pick4(float s0, float s1, float s2, float s3, int j) {
  return j == 0 ? s0 : j == 1 ? s1 : j == 2 ? s2 : s3;
}

struct CrossOut {
  int u;      // the row's vertex when this warp finishes it, else -1
  float sum;  // the row's total
};

// One of the warps w0..w1 covering row list0[rank] hands in its partial:
// w0, holding the row's first edge, as `tail`, every later one as `head`.
// `arrivals` counts the warps in w0..w1 with a nonempty range (an empty one
// holds a zero head partial).  The last to arrive adds the partials in warp
// order (FP64) and finishes the row.  One lane; rare, so kept out of line.
__device__ __noinline__ CrossOut pr_cross(const PrWalk* wk, const int32_t* l0, int rank, int tail, double val,
                                          int gw, int w0, int w1, int arrivals) {
  (tail ? wk->tailp : wk->headp)[gw] = val;
  __threadfence();
  const int seen = atomicAdd(wk->done + w1, 1);
  CrossOut r{-1, 0.f};
  if (seen == arrivals - 1) {
    __threadfence();
    const volatile double* tp = wk->tailp;
    const volatile double* hp = wk->headp;
    double tot = tp[w0];
    for (int j = w0 + 1; j <= w1; ++j) tot += hp[j];
    wk->done[w1] = 0;
    r.u = l0[rank];
    r.sum = (float)tot;
  }
  return r;
}

// The cross-warp rows of one warp's range: the row that continues into it
// (head) and the row left open at its end (tail), with the warps that share
// them.  Set once per run.
struct PrCross {
  int head_rank = -2, hw0 = 0, hw1 = 0, hn = 0;  // -2: the range starts with a row start
  int tail_w1 = 0, tn = 0;                       // hn, tn: arrivals
};

struct TileIn {
  float x0, x1, x2, x3;
  unsigned mw;  // the head word holding this lane's four bits
  unsigned nx;  // lane 31: the head bit just after the tile
};

template <class OffT>
__device__ __forceinline__ TileIn pr_load(const PrArgs<OffT>& a, const float* cin, int t) {
  const int lane = lane_id();
  const long long p0 = (long long)t * kTile + 4 * lane;
  const long long E = a.e;
  TileIn r;
  if (a.wk.vec4 && (long long)(t + 1) * kTile <= E) {  // a full tile (the usual case)
    const int4 q = __ldg(reinterpret_cast<const int4*>(a.iidx + p0));
    r.x0 = cin[q.x];
    r.x1 = cin[q.y];
    r.x2 = cin[q.z];
    r.x3 = cin[q.w];
  } else {
    int v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (p0 < E) v0 = gload(a.iidx + p0);
    if (p0 + 1 < E) v1 = gload(a.iidx + p0 + 1);
    if (p0 + 2 < E) v2 = gload(a.iidx + p0 + 2);
    if (p0 + 3 < E) v3 = gload(a.iidx + p0 + 3);
    r.x0 = p0 < E ? cin[v0] : 0.f;
    r.x1 = p0 + 1 < E ? cin[v1] : 0.f;
    r.x2 = p0 + 2 < E ? cin[v2] : 0.f;
    r.x3 = p0 + 3 < E ? cin[v3] : 0.f;
  }
  r.mw = a.wk.head[4 * (long long)t + (lane >> 3)];
  r.nx = lane == 31 ? (a.wk.head[4 * (long long)t + 4] & 1u) : 0u;
  return r;
}

// Sum one tile and finish the rows that end in it.  (ch, cl) (the same in
// every lane) is the partial of the row open at the tile's start, `trank` the
// number of row starts before the tile; both advance past the tile.
template <class OffT, class Pull>
__device__ __forceinline__ void pr_tile(const PrArgs<OffT>& a, Pull& f, float base, const int32_t* l0, int c0n,
                                        const TileIn& in, float& ch, float& cl, int& trank, const PrCross& cx, int gw,
                                        unsigned& end_bit) {
  const int lane = lane_id();
  if (!__any_sync(kFull, in.mw | in.nx)) {  // no row starts or ends here: the open row goes on
    float sum = ((in.x0 + in.x1) + in.x2) + in.x3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);  // same value in every lane
    float e;
    two_sum(ch, sum, ch, e);
    cl += e;
    end_bit = 0u;
    return;
  }
  const int sub = (lane & 7) * 4, wi = lane >> 3;
  const unsigned hb = (in.mw >> sub) & 0xFu;  // row starts among this lane's four edges
  const unsigned m0 = __shfl_sync(kFull, in.mw, 0), m1 = __shfl_sync(kFull, in.mw, 8);
  const unsigned m2 = __shfl_sync(kFull, in.mw, 16), m3 = __shfl_sync(kFull, in.mw, 24);
  int hp = __popc(in.mw & ((1u << sub) - 1u));  // row starts in earlier lanes of the tile
  if (wi > 0) hp += __popc(m0);
  if (wi > 1) hp += __popc(m1);
  if (wi > 2) hp += __popc(m2);
  unsigned hn = __shfl_down_sync(kFull, hb, 1) & 1u;  // a row starts right after this lane's edges
  const unsigned nx = __shfl_sync(kFull, in.nx, 31);
  if (lane == 31) hn = nx;
  // running sums, restarting at row starts
  const float s0 = in.x0;
  const float s1 = (hb & 2u) ? in.x1 : s0 + in.x1;
  const float s2 = (hb & 4u) ? in.x2 : s1 + in.x2;
  const float s3 = (hb & 8u) ? in.x3 : s2 + in.x3;
  const unsigned endm = (hb >> 1) | (hn << 3);  // bit j: edge j ends its row
  const int first = hb ? __ffs(hb) - 1 : 4;     // first row start in the lane (4: none)
  // segmented scan of the sums flowing across lanes: a lane is (pass, add),
  // and the partial entering it leaves as pass ? in + add : add
  int A = hb == 0 && hn == 0;
  float B = hn ? 0.f : s3;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float By = __shfl_up_sync(kFull, B, o);
    const int Ay = __shfl_up_sync(kFull, A, o);
    if (lane >= o) {
      if (A) B = By + B;
      A = A & Ay;
    }
  }
  int Ae = __shfl_up_sync(kFull, A, 1);
  float Be = __shfl_up_sync(kFull, B, 1);
  if (lane == 0) {
    Ae = 1;
    Be = 0.f;
  }
  const int A31 = __shfl_sync(kFull, A, 31);
  const float B31 = __shfl_sync(kFull, B, 31);
  // totals of the rows ending at each of the lane's edges: a row that began
  // in the lane ends with its running sum; the row that entered from the left
  // (ending at edge first-1) adds the partial carried into the lane
  float v0 = s0, v1 = s1, v2 = s2, v3 = s3;
  unsigned ends = endm;
  const int rb = trank + hp - 1;  // rank of the row open at the lane's start
  if (first > 0 && ((endm >> (first - 1)) & 1u)) {
    float hi = Be, lo = 0.f, e1, e2;
    if (Ae) {
      two_sum(ch, Be, hi, e1);
      lo = cl + e1;
    }
    two_sum(hi, pick4(s0, s1, s2, s3, first - 1), hi, e2);
    lo += e2;
    if (rb == cx.head_rank) {  // a row begun by an earlier warp
      ends &= ~(1u << (first - 1));
      const CrossOut c = pr_cross(&a.wk, l0, rb, 0, (double)hi + (double)lo, gw, cx.hw0, cx.hw1, cx.hn);
      if (c.u >= 0) f.finish(a, base, c.u, c.sum);
    } else {
      const float tot = hi + lo;
      v0 = first == 1 ? tot : v0;
      v1 = first == 2 ? tot : v1;
      v2 = first == 3 ? tot : v2;
      v3 = first == 4 ? tot : v3;
    }
  }
  // finish them: the rows' vertices, then their 1/outdeg and x_t, then stores
  const int r0 = rb + (int)(hb & 1u), r1 = rb + __popc(hb & 3u), r2 = rb + __popc(hb & 7u), r3 = rb + __popc(hb);
  const bool f0 = (ends & 1u) && r0 < c0n, f1 = (ends & 2u) && r1 < c0n;
  const bool f2 = (ends & 4u) && r2 < c0n, f3 = (ends & 8u) && r3 < c0n;
  int u0 = 0, u1 = 0, u2 = 0, u3 = 0;
  if (f0) u0 = l0[r0];
  if (f1) u1 = l0[r1];
  if (f2) u2 = l0[r2];
  if (f3) u3 = l0[r3];
  float i0 = 0.f, i1 = 0.f, i2 = 0.f, i3 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
  if (f0) { i0 = a.inv[u0]; o0 = f.xold[u0]; }
  if (f1) { i1 = a.inv[u1]; o1 = f.xold[u1]; }
  if (f2) { i2 = a.inv[u2]; o2 = f.xold[u2]; }
  if (f3) { i3 = a.inv[u3]; o3 = f.xold[u3]; }
  if (f0) f.store(a, base, u0, v0, i0, o0);
  if (f1) f.store(a, base, u1, v1, i1, o1);
  if (f2) f.store(a, base, u2, v2, i2, o2);
  if (f3) f.store(a, base, u3, v3, i3, o3);
  if (A31) {
    float e;
    two_sum(ch, B31, ch, e);
    cl += e;
  } else {
    ch = B31;
    cl = 0.f;
  }
  trank += __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
  end_bit = nx;
}

// Fetch the line holding p into L2 with no register waiting on it.
__device__ __forceinline__ void pr_prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// One iteration's sums over the in-edges of this warp's tile range
// [t_beg, t_end).
template <class OffT, class Pull>
__device__ __forceinline__ void pr_walk(const PrArgs<OffT>& a, Pull& f, float base, const int32_t* l0,
                                        int c0n, int gw, int t_beg, int t_end, int rank0, const PrCross& cx) {
  if (t_beg >= t_end) return;
  float ch = 0.f, cl = 0.f;  // the open row's partial, ch + cl unevaluated
  int trank = rank0;
  unsigned end_bit = 1;
  for (int t = t_beg; t < t_end; t += 2) {
    {
      // the next two tiles' in-edge indices (eight 128-byte lines) go to L2
      // while this step's gathers are in flight
      const int lane = lane_id();
      const long long p = (long long)(t + 2) * kTile + 32 * lane;
      if (lane < 8 && t + 2 + (lane >> 2) < t_end && p < a.e) pr_prefetch_l2(a.iidx + p);
    }
    const TileIn x = pr_load(a, f.cin, t);
    TileIn y{};
    const bool two = t + 1 < t_end;
    if (two) y = pr_load(a, f.cin, t + 1);
    pr_tile(a, f, base, l0, c0n, x, ch, cl, trank, cx, gw, end_bit);
    if (two) pr_tile(a, f, base, l0, c0n, y, ch, cl, trank, cx, gw, end_bit);
  }
  // the row still open at the range end continues in the next warp
  if (!end_bit && lane_id() == 0) {
    const int r = trank - 1;
    if (r < c0n) {
      const bool tail = r >= rank0;
      const CrossOut c = pr_cross(&a.wk, l0, r, tail, (double)ch + (double)cl, gw, tail ? gw : cx.hw0,
                                  tail ? cx.tail_w1 : cx.hw1, tail ? cx.tn : cx.hn);
      if (c.u >= 0) f.finish(a, base, c.u, c.sum);
    }
  }
}

// Number of leading positions q in [0, len) where pred(q) holds, pred being
// true on a prefix (32-ary search by one warp).
template <class Pred>
__device__ long long warp_partition_point(long long len, Pred pred) {
  const int lane = lane_id();
  long long lo = 0, hi = len;
  while (lo < hi) {
    const long long step = (hi - lo + 31) / 32;
    const long long q = lo + (long long)(lane + 1) * step - 1;
    const bool in = q < hi && pred(q);
    const int k = __popc(__ballot_sync(kFull, in));
    const long long nhi = lo + (long long)(k + 1) * step - 1;
    lo += (long long)k * step;
    hi = nhi < hi ? nhi : hi;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long tile_cost(const PrWalk& wk, long long t) {
  const uint32_t* h = wk.head + 4 * t;
  return (unsigned long long)kTile +
         (unsigned long long)wk.row_cost * (unsigned)(__popc(h[0]) + __popc(h[1]) + __popc(h[2]) + __popc(h[3]));
}

// ---------------------------------------------------------- push tail
// After the switch (Sec. 6 "PageRank": push once most vertices are stable)
// the run keeps ranks x (FP32, in rank) and pending changes r (signed 2^-60
// fixed point) with x* = x + (I - M)^-1 r, M the pull iteration's matrix.
// Each push iteration is two phases: a ballot scan of every vertex (it adds
// the uniform share of the dangling vertices pushed before, sums |r| for the
// stop test, and selects the vertices with |r(v)| > eps, moving r(v) into
// x(v) and fixing what v sends), then a push of the selected vertices along
// their out-edges by the degree classes, each edge one 64-bit integer add.
// Integer adds commute, and every selection and claim is made by the owner
// of the vertex, so the run is bit-identical every time.  It ends when
// ||r||_1 < tol with x + r as the result: within d / (1 - d) * tol of x*.
struct PrPush {
  struct Src {
    long long c;
  };
  unsigned long long* res;
  const long long* push_c;
  __device__ __forceinline__ bool src(int v, Src& s, int, unsigned) {
    s.c = push_c[v];
    return s.c != 0;
  }
  __device__ __forceinline__ int rv(int v) const { return v; }
  static __device__ __forceinline__ Src shfl(const Src& s, int l) {
    Src r;
    r.c = __shfl_sync(kFull, s.c, l);
    return r;
  }
  __device__ __forceinline__ void edges(const Src (&s)[kPushBatch], const int (&)[kPushBatch],
                                        const int (&u)[kPushBatch], const long long (&)[kPushBatch], unsigned ok) {
#pragma unroll
    for (int q = 0; q < kPushBatch; ++q)
      if ((ok >> q) & 1u) atomicAdd(res + u[q], (unsigned long long)s[q].c);  // no return value: a reduction
  }
};

constexpr double kUnfix = 8.67361737988403547e-19;  // 2^-60

// The push iterations.  Launched after the pull kernel of a run with the
// switch enabled; returns at once when that kernel converged by pulling
// alone (it then wrote the result and the statistics), else continues after
// its last pull iteration t, reading x_{t-1} and x_t from rank / x_alt.
template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) pagerank_push_kernel(const __grid_constant__ PrArgs<OffT> a) {
  __shared__ CtaShared sh;
  Sync* s = a.w.sync;
  if (ld_volatile_i32(&s->rs.active) == 0) return;
  const unsigned grid = gridDim.x;
  const Knobs& k = a.k;
  const int n = a.n;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  unsigned long long* res = a.res;
  long long* push_c = a.push_c;
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();
  const int pulls = (int)s->rs.v[0];
  int t = pulls;
  double l1_last = __longlong_as_double(s->rs.v[1]);
  long long evisit = 0;
  const float* xalt = reinterpret_cast<const float*>(a.w.state);
  const float* xo_p = ((t - 1) & 1) ? xalt : a.rank;
  const float* xn_p = ((t - 1) & 1) ? a.rank : xalt;
  // x = x_{t-1}, r = x_t - x_{t-1}
  clear_next_slot(s, sh);
  for (long long v = gtid; v < n; v += gthreads) {
    const float xo = xo_p[v], xn = xn_p[v];
    res[v] = (unsigned long long)((long long)to_fix(xn) - (long long)to_fix(xo));
    a.rank[v] = xo;
  }
  if (!grid_sync(s, grid, sh, k)) return;
  long long G = 0;          // uniform pending change not yet added to every r(v)
  double l1p = l1_last;     // L1 of the previous scan
  bool none = false;        // the previous scan selected no vertex
  const OffT* off = a.off;
  const double inv_n = 1.0 / (double)n;  // per-iteration scalars multiply (FP64 division is slow here)
  while (true) {
    const unsigned long long t_it = globaltimer();
    // ---- scan: add G, sum |r|, select |r| > eps and claim
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    const unsigned long long eps_fix =
        none ? 0ull : (unsigned long long)((double)a.theta * l1p * inv_n * kFix);
    unsigned long long l1acc = 0, dang = 0;
    const long long GG = G;
    auto pred = [&](int v) {
      long long rv = (long long)res[v];
      if (GG != 0) {
        rv += GG;
        res[v] = (unsigned long long)rv;
      }
      const unsigned long long av = rv < 0 ? (unsigned long long)(-rv) : (unsigned long long)rv;
      l1acc += av;
      return av > eps_fix;
    };
    auto deg = [off](int v) { return (long long)gload(off + v + 1) - (long long)gload(off + v); };
    auto visit = [&](int v) {
      const long long rv = (long long)res[v];
      res[v] = 0ull;
      a.rank[v] += (float)((double)rv * kUnfix);
      const long long od = (long long)gload(off + v + 1) - (long long)gload(off + v);
      if (od == 0) {
        dang += (unsigned long long)rv;
        push_c[v] = 0;
      } else {
        push_c[v] = llrint((double)rv * (double)a.d / (double)od);
      }
    };
    ballot_filter(n, pred, deg, visit, sh, a.w, k, grid, 1, slot);
    const unsigned long long l1s = cta_sum_u64(l1acc, sh);
    const unsigned long long ds = cta_sum_u64(dang, sh);
    if (threadIdx.x == 0) {
      atomicAdd(&slot.aux1, l1s);
      atomicAdd(&slot.aux0, ds);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    const double l1 = (double)p.aux1 * kUnfix;  // exact: kUnfix = 1 / kFix, a power of two
    unsigned cnt[kClasses];
    for (int c = 0; c < kClasses; ++c) cnt[c] = p.list_cnt[c];
    const unsigned sel = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    l1_last = l1;
    if (l1 < (double)a.tol || t >= a.max_iter) {
      // x + r (claims only moved r into x, so the sum is the state before them)
      for (long long v = gtid; v < n; v += gthreads)
        a.rank[v] += (float)((double)(long long)res[v] * kUnfix);
      trace_put(a.w, t, 1 | (2 << 8), sel, 0, (long long)p.aux1, t_it);
      break;
    }
    const long long Gn = llrint((double)a.d * (double)(long long)p.aux0 * inv_n);
    // ---- push the selected vertices' changes along their out-edges
    clear_next_slot(s, sh);
    {
      PhaseSlot& slot2 = s->slot[slot_of(sh.phase)];
      PrPush f{res, push_c};
      const int32_t* lists[kClasses] = {a.w.list[1][0], a.w.list[1][1], a.w.list[1][2], a.w.list[1][3]};
      push_classes<OffT>(f, a.off, a.idx, lists, cnt, grid, k.huge_min, sh, evisit);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    trace_put(a.w, t, 1 | (2 << 8), sel, 0, (long long)p.aux1, t_it);
    trace_classes(a.w, t, s->slot[slot_of(sh.phase - 1)]);
    G = Gn;
    none = sel == 0;
    l1p = l1;
    ++t;
  }
  const unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (!grid_sync(s, grid, sh, k)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats& st = *a.w.stats;
    st.status = 0;
    st.iterations = t;
    st.push_iters = t - pulls;
    st.pull_iters = pulls;
    st.ballot_iters = 2 + (t - pulls);  // the first pull and every push scan
    st.online_iters = 0;
    st.phases = (int)sh.phase;
    st.grid = (int)grid;
    st.edges_visited = (long long)s->evisit;
    st.frontier_sum = (long long)pulls * n;
    st.last_l1 = l1_last;
    s->rs.done = 1;
  }
}

// Second test of the switch rule: a scan for the out-edges of the vertices
// whose change exceeds eps.  Returns 1 to switch, 0 to keep pulling, -1 if
// the run aborted.  Out of line: the pull walk keeps its registers.
template <class OffT>
__device__ __noinline__ int pr_unstable_test(const PrArgs<OffT>& a, const float* xold, const float* xnew, float eps,
                                             CtaShared& sh) {
  Sync* s = a.w.sync;
  const unsigned grid = gridDim.x;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  clear_next_slot(s, sh);
  PhaseSlot& sl = s->slot[slot_of(sh.phase)];
  unsigned long long m = 0;
  for (long long v = gtid; v < a.n; v += gthreads)
    if (fabsf(xnew[v] - xold[v]) > eps) m += (unsigned long long)(gload(a.off + v + 1) - gload(a.off + v));
  m = cta_sum_u64(m, sh);
  if (threadIdx.x == 0 && m) atomicAdd(&sl.aux2, m);
  if (!grid_sync(s, grid, sh, a.k)) return -1;
  return (double)s->slot[slot_of(sh.phase - 1)].aux2 * (double)a.alpha < (double)a.e ? 1 : 0;
}

// The walk state of warp gw under the warp ranges ts (first tile of each
// warp, nwarps + 1 entries): its tile range, the rank among the rows of the
// first row starting in it, and the rows it shares with other warps.  An
// empty range writes a zero head partial (it adds nothing to a row crossing
// it).
template <class OffT>
__device__ void pr_warp_setup(const PrArgs<OffT>& a, const int* ts, long long nwarps, long long gw,
                              const int32_t* l0, int c0n, int& t_beg, int& t_end, int& rank0, PrCross& cx) {
  const PrWalk& wk = a.wk;
  const OffT* ioff = a.ioff;
  t_beg = ts[gw];
  t_end = ts[gw + 1];
  rank0 = 0;
  cx = PrCross{};
  if (t_beg >= t_end) {
    if (lane_id() == 0) wk.headp[gw] = 0.0;
    return;
  }
  auto warp_of = [ts, nwarps](long long tile) {
    return (int)warp_partition_point(nwarps, [ts, tile](long long w) { return ts[w] <= tile; }) - 1;
  };
  auto nonempty = [ts](int w0, int w1) {  // warps in [w0, w1] with a nonempty range
    int c = 0;
    for (int w = w0 + lane_id(); w <= w1; w += 32) c += ts[w] < ts[w + 1];
    return (int)warp_sum_u64((unsigned long long)c);
  };
  auto rows_before = [ioff, l0, c0n](long long x) {
    return (int)warp_partition_point(c0n, [ioff, l0, x](long long q) { return (long long)gload(ioff + l0[q]) < x; });
  };
  const long long x = (long long)t_beg * kTile;
  rank0 = rows_before(x);
  if (!((wk.head[x >> 5] >> (x & 31)) & 1u)) {
    cx.head_rank = rank0 - 1;
    const int u = l0[cx.head_rank];
    cx.hw0 = warp_of((long long)gload(ioff + u) / kTile);
    cx.hw1 = warp_of(((long long)gload(ioff + u + 1) - 1) / kTile);
    cx.hn = nonempty(cx.hw0, cx.hw1);
  }
  const long long xe = (long long)t_end * kTile;
  if (xe < a.e && !((wk.head[xe >> 5] >> (xe & 31)) & 1u)) {
    const int u = l0[rows_before(xe) - 1];
    cx.tail_w1 = warp_of(((long long)gload(ioff + u + 1) - 1) / kTile);
    cx.tn = nonempty((int)gw, cx.tail_w1);
  }
}

// Re-cut the warp ranges so that each warp's share of the measured walk
// time is equal: warp w's old range [ts[w], ts[w+1]) took wtime[w] cycles,
// spread evenly over its tiles; warp k's new range starts where the
// cumulative time reaches k / warps of the total.  Writes wk.tstart2; false
// if the run aborted.  (The summation order then follows the measured cut,
// so results may differ in the last bits from run to run.)
template <class OffT>
__device__ __noinline__ bool pr_recut_ranges(const PrArgs<OffT>& a, const int* ts, long long nwarps, CtaShared& sh) {
  const PrWalk& wk = a.wk;
  Sync* s = a.w.sync;
  const unsigned grid = gridDim.x;
  const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
  // the exclusive prefix of the warp times, by CTA 0
  clear_next_slot(s, sh);
  if (blockIdx.x == 0) {
    const long long per = (nwarps + kThreads - 1) / kThreads;
    const long long i0 = (long long)threadIdx.x * per;
    unsigned long long mine = 0;
    for (long long i = i0; i < i0 + per && i < nwarps; ++i) mine += wk.wtime[i];
    unsigned long long incl = mine;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) sh.red64[warp] = incl;
    __syncthreads();
    unsigned long long run = incl - mine;
    for (int q = 0; q < warp; ++q) run += sh.red64[q];
    for (long long i = i0; i < i0 + per && i < nwarps; ++i) {
      wk.wpre[i] = run;
      run += wk.wtime[i];
    }
    if (threadIdx.x == kThreads - 1) wk.wpre[nwarps] = run;
  }
  if (!grid_sync(s, grid, sh, a.k)) return false;
  clear_next_slot(s, sh);
  {
    const unsigned long long* pre = wk.wpre;
    const unsigned long long total = pre[nwarps];
    const unsigned long long target = total / (unsigned long long)nwarps * (unsigned long long)gw +
                                      total % (unsigned long long)nwarps * (unsigned long long)gw /
                                          (unsigned long long)nwarps;
    const long long w = warp_partition_point(nwarps, [pre, target](long long q) { return pre[q + 1] <= target; });
    int start = (int)wk.ntiles;
    if (w < nwarps) {
      const unsigned long long tw = pre[w + 1] - pre[w];  // > 0: pre[w] <= target < pre[w + 1]
      const long long ob = ts[w], oe = ts[w + 1];
      start = (int)(ob + (long long)((unsigned long long)(oe - ob) * (target - pre[w]) / tw));
    }
    if (gw == 0) start = 0;
    if (lane_id() == 0) {
      wk.tstart2[gw] = start;
      if (gw == nwarps - 1) wk.tstart2[nwarps] = (int)wk.ntiles;
    }
  }
  return grid_sync(s, grid, sh, a.k);
}

// TAIL: the instantiation that may switch to push (the pr_alpha knob); the
// pull-only kernel carries none of its registers.
// RECUT: the instantiation that re-cuts the warp ranges by measured time
// (the pr_recut knob); the default kernels carry none of its state.
template <class OffT, bool TAIL = false, bool RECUT = false>
__global__ void __launch_bounds__(kThreads, 4) pagerank_kernel(const __grid_constant__ PrArgs<OffT> a) {
  __shared__ CtaShared sh;
  const unsigned grid = gridDim.x;
  Sync* s = a.w.sync;
  const Knobs& k = a.k;
  const int n = a.n;
  const PrWalk& wk = a.wk;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long gthreads = (long long)grid * kThreads;
  const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const long long nwarps = (long long)grid * kWarps;
  float* xalt = reinterpret_cast<float*>(a.w.state);
  float* cbuf0 = xalt + n;
  float* cbuf1 = xalt + 2 * (size_t)n;
  const OffT* off = a.off;
  const OffT* ioff = a.ioff;
  auto all = [](int) { return true; };
  auto pr_class = [ioff](int v) { return gload(ioff + v + 1) == gload(ioff + v) ? 1 : 0; };
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // ---- phase 0: x_0, c_0, D_0, the per-chunk class counts; clear the row-start bits
  {
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[0];
    const float x0 = 1.0f / (float)n;
    unsigned long long dang = 0;
    for (long long v = gtid; v < n; v += gthreads) {
      const long long od = (long long)gload(off + v + 1) - (long long)gload(off + v);
      a.rank[v] = x0;
      cbuf0[v] = od > 0 ? x0 / (float)od : 0.f;
      a.inv[v] = od > 0 ? 1.0f / (float)od : 0.f;
      if (od == 0) dang += to_fix(x0);
    }
    for (long long q = gtid; q < 4 * wk.ntiles + 8; q += gthreads) wk.head[q] = 0u;
    for (long long q = gtid; q < nwarps; q += gthreads) wk.done[q] = 0;
    dang = cta_sum_u64(dang, sh);
    if (threadIdx.x == 0) atomicAdd(&slot.aux0, dang);
    det_filter_count(n, all, pr_class, sh, a.w, grid);
  }
  if (!grid_sync(s, grid, sh, k)) return;
  unsigned long long Dfix = s->slot[0].aux0;
  // ---- phase 1: list 0 (rows with in-edges) and list 1 (none), vertex order;
  // mark the first in-edge of every row, and the end of the array
  unsigned cnt[kClasses];
  clear_next_slot(s, sh);
  det_filter_write(n, all, pr_class, sh, a.w, grid, 0, cnt);
  for (long long v = gtid; v < n; v += gthreads) {
    const long long b = (long long)gload(ioff + v), e = (long long)gload(ioff + v + 1);
    if (e > b) atomicOr(wk.head + (b >> 5), 1u << (b & 31));
  }
  if (gtid == 0) atomicOr(wk.head + (a.e >> 5), 1u << (a.e & 31));
  if (!grid_sync(s, grid, sh, k)) return;
  // ---- phases 2-4: cut the tiles into one range per warp of equal cost
  // (in-edges plus row_cost per row start): chunk sums, the per-tile prefix,
  // then each warp searches the prefix for its range
  const long long ntiles = wk.ntiles;
  const long long nch = (ntiles + kPrChunk - 1) / kPrChunk;
  clear_next_slot(s, sh);
  for (long long c = blockIdx.x; c < nch; c += grid) {
    unsigned long long sum = 0;
    for (long long q = c * kPrChunk + threadIdx.x; q < (c + 1) * kPrChunk && q < ntiles; q += kThreads)
      sum += tile_cost(wk, q);
    sum = cta_sum_u64(sum, sh);
    if (threadIdx.x == 0) wk.csum[c] = sum;
  }
  if (!grid_sync(s, grid, sh, k)) return;
  clear_next_slot(s, sh);
  unsigned long long total = 0;
  {
    unsigned long long sum = 0;
    for (long long q = threadIdx.x; q < nch; q += kThreads) sum += wk.csum[q];
    total = cta_sum_u64(sum, sh);
  }
  for (long long c = blockIdx.x; c < nch; c += grid) {
    unsigned long long run = 0;
    for (long long q = threadIdx.x; q < c; q += kThreads) run += wk.csum[q];
    run = cta_sum_u64(run, sh);
    constexpr int kPer = kPrChunk / kThreads;
    const long long q0 = c * kPrChunk + (long long)threadIdx.x * kPer;
    unsigned long long mine = 0;
    for (int j = 0; j < kPer; ++j)
      if (q0 + j < ntiles) mine += tile_cost(wk, q0 + j);
    unsigned long long incl = mine;  // CTA-wide exclusive scan of `mine`
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) sh.red64[warp] = incl;
    __syncthreads();
    unsigned long long ex = run + incl - mine;
    for (int q = 0; q < warp; ++q) ex += sh.red64[q];
    for (int j = 0; j < kPer; ++j)
      if (q0 + j < ntiles) {
        wk.pre[q0 + j] = ex;
        ex += tile_cost(wk, q0 + j);
      }
    __syncthreads();
  }
  if (gtid == 0) wk.pre[ntiles] = total;
  if (!grid_sync(s, grid, sh, k)) return;
  clear_next_slot(s, sh);
  {
    const unsigned long long target = total * (unsigned long long)gw / (unsigned long long)nwarps;
    const unsigned long long* pre = wk.pre;
    const long long tb = warp_partition_point(ntiles, [pre, target](long long q) { return pre[q] < target; });
    if (lane_id() == 0) {
      wk.tstart[gw] = (int)tb;
      if (gw == nwarps - 1) wk.tstart[nwarps] = (int)ntiles;
    }
  }
  if (!grid_sync(s, grid, sh, k)) return;
  // ---- each warp: rows starting before its range and the cross-warp rows
  const int32_t* l0 = a.w.list[0][0];
  const int32_t* l1 = a.w.list[0][1];
  const int c0n = (int)cnt[0];
  int t_beg = 0, t_end = 0, rank0 = 0;
  PrCross cx;
  pr_warp_setup(a, wk.tstart, nwarps, gw, l0, c0n, t_beg, t_end, rank0, cx);
  // the zero partials of empty ranges are in place before any row sums them
  if (!grid_sync(s, grid, sh, k)) return;

  const float base = (1.0f - a.d) / (float)n;
  int t = 0;
  double l1_last = 0.0;
  bool to_push = false;
  while (true) {
    if (t >= a.max_iter) break;
    const unsigned long long t_it = globaltimer();
    // ---- compute x_{t+1}
    clear_next_slot(s, sh);
    PhaseSlot& slot = s->slot[slot_of(sh.phase)];
    PrPull<OffT> f;
    f.cin = (t & 1) ? cbuf1 : cbuf0;
    f.cout = (t & 1) ? cbuf0 : cbuf1;
    f.xold = (t & 1) ? xalt : a.rank;
    f.xnew = (t & 1) ? a.rank : xalt;
    f.dn = __ull2float_rn(Dfix) * 8.67361737988403547e-19f / (float)n;  // D_t / n (2^-60 units)
    {
      ClassTimer tm(&slot);
      const bool timed = RECUT && a.recut > 0 && t == a.recut - 1;
      const long long c0 = timed ? clock64() : 0;
      pr_walk<OffT>(a, f, base, l0, c0n, (int)gw, t_beg, t_end, rank0, cx);
      if (timed && lane_id() == 0) wk.wtime[gw] = (unsigned long long)(clock64() - c0);
      tm.lap(0);
      for (unsigned i = (unsigned)gtid; i < cnt[1]; i += (unsigned)gthreads) f.finish(a, base, l1[i], 0.f);
      tm.lap(1);
    }
    const unsigned long long l1s = cta_sum_u64(to_fix(f.l1), sh);
    const unsigned long long dg = cta_sum_u64(to_fix(f.dang), sh);
    if (threadIdx.x == 0) {
      atomicAdd(&slot.aux0, dg);
      atomicAdd(&slot.aux1, l1s);
    }
    if (!grid_sync(s, grid, sh, k)) return;
    const PhaseSlot& p = s->slot[slot_of(sh.phase - 1)];
    Dfix = p.aux0;
    const double l1_prev = l1_last;
    l1_last = (double)p.aux1 * kUnfix;  // exact: a power of two
    trace_put(a.w, t, 2 | (2 << 8), n, a.e, (long long)p.aux1, t_it);
    trace_classes(a.w, t, p);
    ++t;
    if (l1_last < (double)a.tol) break;
    if (RECUT && a.recut > 0 && t == a.recut && t < a.max_iter) {
      // ranges cut by the measured time of the last walk (the `pr_recut` knob)
      if (!pr_recut_ranges(a, wk.tstart, nwarps, sh)) return;
      pr_warp_setup(a, wk.tstart2, nwarps, gw, l0, c0n, t_beg, t_end, rank0, cx);
      if (!grid_sync(s, grid, sh, k)) return;
    }
    // switch to push (reading of Sec. 6's decision tree): first test, the
    // pull contracts slowly; only then the second, a scan for the out-edges
    // of the unstable vertices (change above theta * L1_{t-1} / n)
    if (TAIL && a.alpha > 0.f && t >= 2 && t < a.max_iter && l1_last >= (double)a.rho * l1_prev) {
      const int r = pr_unstable_test(a, f.xold, f.xnew, (float)((double)a.theta * l1_prev / (double)n), sh);
      if (r < 0) return;
      if (r) {
        to_push = true;
        break;
      }
    }
  }
  long long evisit = 0;  // in-edges this warp summed, every pull iteration
  if (lane_id() == 0 && t_beg < t_end)
    evisit = (long long)t * (min((long long)t_end * kTile, a.e) - (long long)t_beg * kTile);
  unsigned long long ev = cta_sum_u64((unsigned long long)evisit, sh);
  if (threadIdx.x == 0) atomicAdd(&s->evisit, ev);
  if (TAIL && to_push) {
    // the push kernel launched next continues from here (selective fusion:
    // a pull kernel and a push kernel, Sec. 5)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      s->rs.v[0] = t;
      s->rs.v[1] = __double_as_longlong(l1_last);
      s->rs.active = 1;
    }
    return;
  }
  // ---- result: x_t is in rank for even t, in xalt for odd t
  if (t & 1)
    for (long long v = gtid; v < n; v += gthreads) a.rank[v] = xalt[v];
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
  a.idx = g->idx;
  a.ioff = (const OffT*)g->in_off;
  a.iidx = g->in_idx;
  a.e = g->e;
  a.rank = rank;
  a.alpha = g->cfg.pr_alpha;
  a.theta = g->cfg.pr_theta;
  a.rho = g->cfg.pr_rho;
  a.recut = g->cfg.pr_recut;
  const bool tail = a.alpha > 0.f;
  // state (20 bytes per vertex): x_alt | c0 | c1 | 1/outdeg | spare; with the
  // push tail 1/outdeg moves to the spare slot, the pending changes (8 bytes)
  // take c1 and the old slot once the pulls end, and what each selected
  // vertex sends (8 bytes) takes x_alt and c0
  float* st4 = static_cast<float*>(g->state);
  a.inv = st4 + (tail ? 4 : 3) * (size_t)g->n;
  a.push_c = reinterpret_cast<long long*>(st4);
  a.res = reinterpret_cast<unsigned long long*>(st4 + 2 * (size_t)g->n);
  a.w = make_work(g);
  a.k = make_knobs(g);
  const void* kern = a.recut > 0 ? (tail ? (const void*)pagerank_kernel<OffT, true, true>
                                         : (const void*)pagerank_kernel<OffT, false, true>)
                                  : (tail ? (const void*)pagerank_kernel<OffT, true> : (const void*)pagerank_kernel<OffT>);
  int grid = grid_for(g, kern);
  // walk layout: row-start bits, tile cost prefix and chunk sums, warp
  // ranges, per-warp partials and arrival counters
  const long long ntiles = (g->e + kTile - 1) / kTile;
  const long long nw = (long long)grid * kWarps;
  const long long nch = (ntiles + kPrChunk - 1) / kPrChunk;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t head_b = up(sizeof(uint32_t) * (size_t)(4 * ntiles + 8));
  const size_t pre_b = up(sizeof(unsigned long long) * (size_t)(ntiles + 1));
  const size_t csum_b = up(sizeof(unsigned long long) * (size_t)(nch + 1));
  const size_t ts_b = up(sizeof(int) * (size_t)(nw + 1));
  const size_t part_b = up(sizeof(double) * (size_t)nw);
  const size_t wt_b = up(sizeof(unsigned long long) * (size_t)(nw + 1));
  const size_t bytes = head_b + pre_b + csum_b + ts_b + 2 * part_b + up(sizeof(int) * (size_t)nw) + 2 * wt_b + ts_b;
  if (!g->pr_ws || g->pr_bytes < bytes) {
    dev_free(g->pr_ws, st);
    g->pr_ws = nullptr;
    g->pr_bytes = 0;
    SIMDX_CUDA(dev_alloc(&g->pr_ws, bytes, st));
    g->pr_bytes = bytes;
  }
  char* base = static_cast<char*>(g->pr_ws);
  a.wk.head = reinterpret_cast<uint32_t*>(base);
  a.wk.pre = reinterpret_cast<unsigned long long*>(base + head_b);
  a.wk.csum = reinterpret_cast<unsigned long long*>(base + head_b + pre_b);
  a.wk.tstart = reinterpret_cast<int*>(base + head_b + pre_b + csum_b);
  a.wk.tailp = reinterpret_cast<double*>(base + head_b + pre_b + csum_b + ts_b);
  a.wk.headp = reinterpret_cast<double*>(base + head_b + pre_b + csum_b + ts_b + part_b);
  a.wk.done = reinterpret_cast<int*>(base + head_b + pre_b + csum_b + ts_b + 2 * part_b);
  {
    char* q = base + head_b + pre_b + csum_b + ts_b + 2 * part_b + up(sizeof(int) * (size_t)nw);
    a.wk.wtime = reinterpret_cast<unsigned long long*>(q);
    a.wk.wpre = reinterpret_cast<unsigned long long*>(q + wt_b);
    a.wk.tstart2 = reinterpret_cast<int*>(q + 2 * wt_b);
  }
  a.wk.ntiles = ntiles;
  a.wk.row_cost = g->cfg.pr_row_cost > 0 ? g->cfg.pr_row_cost : kPrRowCost;
  a.wk.vec4 = (reinterpret_cast<uintptr_t>(g->in_idx) & 15) == 0;
  int rc = prepare_launch(g, st);
  if (rc) return rc;
  void* args[] = {&a};
  if ((rc = launch_coop(kern, grid, args, st)) != SIMDX_OK) return rc;
  if (!tail) return finish_launch(g, stats, st);
  // the push kernel returns at once unless the pull kernel switched; the
  // decision stays on the device, so the call can still be captured
  const void* pk = (const void*)pagerank_push_kernel<OffT>;
  if ((rc = prepare_resume(g, st)) != SIMDX_OK) return rc;
  if ((rc = launch_coop(pk, grid_for(g, pk), args, st)) != SIMDX_OK) return rc;
  return finish_launch(g, stats, st, 2);
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
