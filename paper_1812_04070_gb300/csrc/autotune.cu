// autotune.cu -- measured choice of the knobs of simdx_config for one
// algorithm on one graph (coordinate descent, CUDA-event timing).
//
// The knobs are the degree-class thresholds and overflow threshold of the
// task lists (Sec. 4), the push/pull switch ratios (Sec. 5), the SSSP bucket
// width and the CTAs per SM of the persistent launch (Eq. 1).  None of them
// changes a BFS, SSSP or k-core result, so the tuner only compares times.
#include <algorithm>
#include <functional>
#include <vector>

#include "simdx_internal.h"

namespace {

using simdx::cuda_status;

struct Knob {
  const char* name;
  std::vector<double> values;
  void (*set)(simdx_config&, double);
  double (*get)(const simdx_config&);
};

#define SIMDX_KNOB_I(field)                                                    \
  [](simdx_config& c, double v) { c.field = (decltype(c.field))v; },            \
  [](const simdx_config& c) { return (double)c.field; }

// Knobs that apply to each algorithm, with the values tried (the current
// setting is always a candidate too).
std::vector<Knob> knobs_for(int algo) {
  std::vector<Knob> k;
  k.push_back({"ctas_per_sm", {0, 3, 2}, SIMDX_KNOB_I(ctas_per_sm)});
  if (algo == SIMDX_ALGO_PAGERANK) {  // all vertices active; no task classes
    k.push_back({"pr_row_cost", {0, 2, 8, 16, 32}, SIMDX_KNOB_I(pr_row_cost)});
    return k;
  }
  k.push_back({"small_max", {8, 16, 32, 64}, SIMDX_KNOB_I(small_max)});
  k.push_back({"med_max", {128, 256, 512, 1024, 2048}, SIMDX_KNOB_I(med_max)});
  k.push_back({"huge_min", {1024, 2048, 4096, 8192, 16384}, SIMDX_KNOB_I(huge_min)});
  k.push_back({"bin_per_thread", {16, 32, 64, 128}, SIMDX_KNOB_I(bin_per_thread)});
  if (algo == SIMDX_ALGO_BFS) {
    k.push_back({"small_frontier", {0, 1}, SIMDX_KNOB_I(small_frontier)});
    k.push_back({"alpha", {4, 7, 14, 28, 56}, SIMDX_KNOB_I(alpha)});
    k.push_back({"beta", {6, 12, 24, 48, 96}, SIMDX_KNOB_I(beta)});
  } else if (algo == SIMDX_ALGO_SSSP) {
    k.push_back({"delta", {16, 64, 256, 1024, 4096, 16384, 65536, 0}, SIMDX_KNOB_I(delta)});
  } else if (algo == SIMDX_ALGO_KCORE) {
    k.push_back({"kcore_alpha", {2, 4, 8, 16, 32}, SIMDX_KNOB_I(kcore_alpha)});
  }
  return k;
}

// Knobs of the batched calls: the bit-parallel BFS batch uses the degree
// classes and the grid; the SSSP batch adds the bins, the bucket width and
// the copies per launch; the multi-root BFS is a BFS.
std::vector<Knob> knobs_for_batch(int algo) {
  if (algo == SIMDX_ALGO_BFS_MULTI) return knobs_for(SIMDX_ALGO_BFS);
  std::vector<Knob> k;
  k.push_back({"ctas_per_sm", {0, 3, 2}, SIMDX_KNOB_I(ctas_per_sm)});
  k.push_back({"small_max", {8, 16, 32, 64}, SIMDX_KNOB_I(small_max)});
  k.push_back({"med_max", {128, 256, 512, 1024, 2048}, SIMDX_KNOB_I(med_max)});
  k.push_back({"huge_min", {1024, 2048, 4096, 8192, 16384}, SIMDX_KNOB_I(huge_min)});
  if (algo == SIMDX_ALGO_SSSP) {
    k.push_back({"bin_per_thread", {16, 32, 64, 128}, SIMDX_KNOB_I(bin_per_thread)});
    k.push_back({"delta", {16, 64, 256, 1024, 4096, 16384, 0}, SIMDX_KNOB_I(delta)});
    k.push_back({"sssp_batch_width", {8, 16, 32, 64}, SIMDX_KNOB_I(sssp_batch_width)});
    k.push_back({"batch_group", {0, 2, 4, 8, 16}, SIMDX_KNOB_I(batch_group)});
  }
  return k;
}

#undef SIMDX_KNOB_I

bool valid(const simdx_config& c) {
  return c.small_max >= 1 && c.med_max >= c.small_max && c.huge_min >= c.med_max;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

// Coordinate descent over `ks` from the graph's current knobs; `run` is one
// timed call.  Leaves the winner installed.
static int tune(simdx_graph* g, const std::vector<Knob>& ks, const std::function<int()>& run, int reps,
                void* stream, simdx_config* best, float* best_ms) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Timer tm;
  int rc = SIMDX_OK;
  // median time of `reps` runs after one untimed run; the first error otherwise
  auto measure = [&](float& ms) -> int {
    int r = run();
    if (r != SIMDX_OK) return r;
    std::vector<float> t;
    for (int i = 0; i < reps; ++i) {
      if (cudaEventRecord(tm.a, st) != cudaSuccess) return SIMDX_ECUDA;
      if ((r = run()) != SIMDX_OK) return r;
      if (cudaEventRecord(tm.b, st) != cudaSuccess) return SIMDX_ECUDA;
      cudaError_t e = cudaEventSynchronize(tm.b);
      if (e != cudaSuccess) return cuda_status(e, "cudaEventSynchronize(autotune)");
      float x = 0.f;
      cudaEventElapsedTime(&x, tm.a, tm.b);
      t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    // a run that ended in a device error (e.g. a barrier timeout) does not count
    r = simdx_graph_last_status(g, stream);
    return r;
  };
  simdx_config cur{};
  float cur_ms = 0.f;
  do {
    cudaError_t e = cudaEventCreate(&tm.a);
    if (e == cudaSuccess) e = cudaEventCreate(&tm.b);
    if (e != cudaSuccess) {
      rc = cuda_status(e, "cudaEventCreate(autotune)");
      break;
    }
    if ((rc = simdx_graph_get_config(g, &cur)) != SIMDX_OK) break;
    if ((rc = measure(cur_ms)) != SIMDX_OK) break;
    for (int pass = 0; pass < 2 && rc == SIMDX_OK; ++pass) {
      bool moved = false;
      for (const Knob& kb : ks) {
        for (double v : kb.values) {
          if (v == kb.get(cur)) continue;
          simdx_config c = cur;
          kb.set(c, v);
          if (!valid(c)) continue;
          if ((rc = simdx_graph_set_config(g, &c)) != SIMDX_OK) break;
          float ms = 0.f;
          if ((rc = measure(ms)) != SIMDX_OK) break;
          if (ms < 0.98f * cur_ms) {
            cur = c;
            cur_ms = ms;
            moved = true;
          }
        }
        if (rc != SIMDX_OK) break;
        // leave the graph on the best setting so far
        if ((rc = simdx_graph_set_config(g, &cur)) != SIMDX_OK) break;
      }
      if (!moved) break;
    }
  } while (false);
  if (rc == SIMDX_OK) rc = simdx_graph_set_config(g, &cur);
  cudaStreamSynchronize(st);
  if (rc != SIMDX_OK) return rc;
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return SIMDX_OK;
}

extern "C" int simdx_autotune(simdx_graph* g, int32_t algo, int64_t arg, int32_t reps, simdx_config* best,
                              float* best_ms, void* stream) {
  if (!g || !best || reps < 1 || reps > 64) return SIMDX_EINVAL;
  if (algo < SIMDX_ALGO_BFS || algo > SIMDX_ALGO_PAGERANK) return SIMDX_EINVAL;
  if ((algo == SIMDX_ALGO_BFS || algo == SIMDX_ALGO_SSSP) && (arg < 0 || arg >= g->n)) return SIMDX_EINVAL;
  if (algo == SIMDX_ALGO_KCORE && (arg < 0 || arg > 0x7fffffff)) return SIMDX_EINVAL;
  if (algo == SIMDX_ALGO_SSSP && !g->w) return SIMDX_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)std::max<int64_t>(g->n, 1);
  void* out = nullptr;
  void* resid = nullptr;
  SIMDX_CUDA(simdx::dev_alloc(&out, 4 * n, st));
  if (algo == SIMDX_ALGO_KCORE) {
    cudaError_t e = simdx::dev_alloc(&resid, 4 * n, st);
    if (e != cudaSuccess) {
      simdx::dev_free(out, st);
      return cuda_status(e, "dev_alloc(autotune resid)");
    }
  }
  auto run = [&]() -> int {
    switch (algo) {
      case SIMDX_ALGO_BFS: return simdx_bfs(g, (int32_t)arg, (int32_t*)out, nullptr, st);
      case SIMDX_ALGO_SSSP: return simdx_sssp(g, (int32_t)arg, (uint32_t*)out, nullptr, st);
      case SIMDX_ALGO_KCORE:
        return simdx_kcore(g, (uint32_t)arg, (uint8_t*)out, (uint32_t*)resid, nullptr, st);
      default: return simdx_pagerank(g, 0.85f, 1e-6f, 1000, (float*)out, nullptr, st);
    }
  };
  const int rc = tune(g, knobs_for(algo), run, reps, stream, best, best_ms);
  simdx::dev_free(out, st);
  simdx::dev_free(resid, st);
  cudaStreamSynchronize(st);
  return rc;
}

extern "C" int simdx_autotune_batch(simdx_graph* g, int32_t algo, const int32_t* srcs, int32_t k, int32_t reps,
                                    simdx_config* best, float* best_ms, void* stream) {
  if (!g || !best || !srcs || k <= 0 || reps < 1 || reps > 64) return SIMDX_EINVAL;
  if (algo != SIMDX_ALGO_BFS && algo != SIMDX_ALGO_SSSP && algo != SIMDX_ALGO_BFS_MULTI) return SIMDX_EINVAL;
  for (int i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return SIMDX_EINVAL;
  if (algo == SIMDX_ALGO_SSSP && !g->w) return SIMDX_EUNSUPPORTED;
  if (algo == SIMDX_ALGO_SSSP && (long long)k * g->n >= (1ll << 31) - 64) return SIMDX_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t rows = algo == SIMDX_ALGO_BFS_MULTI ? 1 : (size_t)k;
  void* out = nullptr;
  SIMDX_CUDA(simdx::dev_alloc(&out, 4 * rows * (size_t)std::max<int64_t>(g->n, 1), st));
  auto run = [&]() -> int {
    switch (algo) {
      case SIMDX_ALGO_BFS: return simdx_bfs_batch(g, srcs, k, (int32_t*)out, nullptr, st);
      case SIMDX_ALGO_SSSP: return simdx_sssp_batch(g, srcs, k, (uint32_t*)out, nullptr, st);
      default: return simdx_bfs_multi(g, srcs, k, (int32_t*)out, nullptr, st);
    }
  };
  const int rc = tune(g, knobs_for_batch(algo), run, reps, stream, best, best_ms);
  simdx::dev_free(out, st);
  cudaStreamSynchronize(st);
  return rc;
}
