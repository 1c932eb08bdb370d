// simdx_internal.h -- host-side graph object, workspace and launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/simdx.h"
#include "acc_device.cuh"

namespace simdx {
// Pinned host copy of a run's statistics plus the barrier error word (an
// aborted run never writes its statistics, so the error travels separately).
struct HostStage {
  DevStats ds;
  int err;
  int rs_done, rs_want;  // Resume::done / want_dir of the last launch (split runs)
  int pad;
  int status() const { return err ? err : ds.status; }
};
}  // namespace simdx

struct simdx_graph {
  int64_t n = 0, e = 0;
  int off_bits = 64;
  bool symmetric = true;
  bool borrowed = false;
  int device = 0;
  int num_sms = 0;
  // graph arrays (device)
  void* off = nullptr;       // CSR offsets (int32 or int64)
  int32_t* idx = nullptr;
  void* in_off = nullptr;    // CSC offsets (== off when symmetric)
  int32_t* in_idx = nullptr;
  uint32_t* w = nullptr;
  int32_t hub = 0;           // a vertex of largest degree (smallest id among them)
  long long max_deg = 0;     // its out-degree
  // knobs
  simdx_config cfg{};
  // workspace
  int grid_max = 0;          // CTAs the workspace is sized for
  int bin_cap = 0;           // entries per CTA per class
  int32_t* bins = nullptr;
  int32_t* lists = nullptr;  // [2][kClasses][list_cap]
  uint32_t* aux3 = nullptr;  // [2][list_cap]
  long long list_cap = 0;
  int32_t* chunk_cnt = nullptr;
  unsigned long long* chunk_part = nullptr;
  int* chunk_done = nullptr;
  int* warp_start = nullptr;
  unsigned long long* ms_state = nullptr;  // batched BFS masks (allocated on first use)
  int32_t* d_roots = nullptr;              // device copy of multi-root BFS roots
  int32_t* h_roots = nullptr;              // pinned staging of the roots (captured calls)
  size_t roots_cap = 0;
  void* sb_state = nullptr;                // batched SSSP lists and state (first use)
  size_t sb_bytes = 0;
  size_t sb_cap = 0;
  int sb_k = 0;
  void* pr_ws = nullptr;                   // PageRank in-edge walk layout (first use)
  size_t pr_bytes = 0;
  void* mss_state = nullptr;               // shared-edge batched SSSP state (first use)
  size_t mss_bytes = 0;
  void* mg_pack = nullptr;                 // simdx_bfs_multigraph pack with this graph first
  unsigned long long gen = 0;              // creation number (distinguishes reused addresses)
  uint32_t* bitmaps = nullptr;  // [4][words]
  void* state = nullptr;        // 20 bytes per vertex
  simdx::Sync* sync = nullptr;
  simdx::DevStats* dstats = nullptr;
  long long* trace = nullptr;
  int trace_cap = 0;
  // host side
  simdx::HostStage* h_stats = nullptr;  // pinned staging of the last run's statistics
  struct Pending {
    simdx_graph* g;
    simdx_stats* user;
  } pending[64];
  unsigned pending_head = 0;
  std::mutex mu;
};

namespace simdx {

// Convert the public knobs into the device copy.
Knobs make_knobs(const simdx_graph* g);

// Workspace views for a launch of `grid` CTAs.
Work make_work(const simdx_graph* g);

// Occupancy-based grid (the Eq. 1 analogue): resident CTAs per SM times the
// SM count, optionally clamped by cfg.ctas_per_sm.
int grid_for(const simdx_graph* g, const void* kernel);

// Reset the barrier/slot block and statistics before a launch.
int prepare_launch(simdx_graph* g, cudaStream_t st);
// Before a further launch of the same call: a fresh barrier, phase slots and
// chunk counters; the abort / error words, the edge count and the stats
// record carry over (a launch after a failed one returns at its first
// barrier, and the error stays reported).
int prepare_next_launch(simdx_graph* g, cudaStream_t st);
// Between the launches of a run split over several launches (fusion knob):
// a fresh barrier and phase slots, the resume record kept.
int prepare_resume(simdx_graph* g, cudaStream_t st);
// Wait for the stream, then report whether the run finished (or failed) and
// the direction its next launch must compute.
int read_resume(simdx_graph* g, cudaStream_t st, int* done, int* want_dir);
// The BFS kernel from src into levels, on the graph's workspace, with no
// preparation or stats (the caller brackets it).
int bfs_launch_only(simdx_graph* g, int32_t src, int32_t* levels, cudaStream_t st);

// Launch `kernel` cooperatively with `grid` CTAs of kThreads threads (in
// clusters of `cluster` CTAs when cluster > 1).
int launch_coop(const void* kernel, int grid, void** args, cudaStream_t st, int cluster = 1);
// The co-resident grid of `kernel` in clusters of `cluster` CTAs (0: none fits).
int grid_for_cluster(const simdx_graph* g, const void* kernel, int cluster);

// Enqueue the copy of device statistics into `user` (may be NULL; must be
// NULL while `st` is being captured into a CUDA graph); `launches` = kernel
// launches the call made.
int finish_launch(simdx_graph* g, simdx_stats* user, cudaStream_t st, int launches = 1);

// Whether `st` is being captured into a CUDA graph.
bool capturing(cudaStream_t st);

int cuda_status(cudaError_t e, const char* what);

// Device memory of the library comes from one stream-ordered pool per device
// that keeps the blocks it is given back (no release threshold), so graph
// creation, destruction and batch-state growth reuse memory instead of going
// to the driver each time.  dev_alloc / dev_free are ordered on `st`.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

// Batched SSSP with the sources sharing each edge read (msssp.cu).
int sssp_batch_shared(simdx_graph* g, const int32_t* srcs, int k, uint32_t* dist, simdx_stats* stats,
                      cudaStream_t st);

// Creation numbers of graph objects, and the simdx_bfs_multigraph pack a
// graph may own (freed with it).
unsigned long long next_graph_gen();
void mg_pack_free(simdx_graph* g, cudaStream_t st);

// Pinned host staging of run statistics, recycled across graphs.
HostStage* host_stage_get();
void host_stage_put(HostStage* h);

}  // namespace simdx

#define SIMDX_CUDA(call)                                             \
  do {                                                               \
    cudaError_t _e = (call);                                         \
    if (_e != cudaSuccess) return simdx::cuda_status(_e, #call);     \
  } while (0)
