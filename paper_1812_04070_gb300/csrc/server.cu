// server.cu -- continuous-batching query server (growth direction (b)).
//
// Graphs stay resident; queries (BFS from a source, SSSP from a source,
// k-core for a k) are submitted from any thread and answered asynchronously.
// One dispatcher thread runs the loop:
//   1. retire: slots whose launch finished (CUDA event) mark their tickets done;
//   2. admit: while a slot is free and queries wait, take the oldest query and
//      every waiting query compatible with it (same graph and algorithm; up
//      to 64 BFS per bit-parallel launch, up to max_sssp SSSP per virtual
//      batch, all k-core queries with the same k share one run), launch them
//      on the slot's stream, copy each query's row to its output buffer, and
//      record the slot's event.
// Queries that arrive while others run are admitted as soon as a slot frees
// up, and the slots' launches overlap on the device: each slot owns borrowed
// clones of the resident graphs (same CSR arrays, separate workspaces) and
// launches cooperative grids of 1/slots of the co-resident CTAs, so the
// kernels of all slots can be resident together.  The number of slots is
// admitted against the memory budget at creation; serving itself allocates
// nothing.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "simdx_internal.h"

namespace simdx {
const void* bfs_kernel_ptr(int off_bits);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  int graph, algo, arg;
  void* out;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<simdx_graph*> clones;  // one per resident graph
  void* d_out = nullptr;             // [max rows][max n] int32 results
  size_t row_bytes = 0;
  void* d_aux = nullptr;             // k-core residual degrees
  std::vector<Request> batch;
  bool busy = false;
};

}  // namespace

struct simdx_server {
  std::vector<simdx_graph*> graphs;
  int max_sssp = 8;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, int> status;  // ticket -> 0 pending, 1 done, < 0 -simdx_status
  uint64_t next_ticket = 1;
  bool stop = false;
  int device = 0;
  std::thread th;
  // statistics
  uint64_t launches = 0, served = 0;
};

namespace {

int launch_batch(simdx_server* s, Slot& sl) {
  const Request& r0 = sl.batch.front();
  simdx_graph* g = sl.clones[r0.graph];
  const size_t rows = sl.batch.size();
  const size_t nbytes_i32 = sizeof(int32_t) * (size_t)g->n;
  int rc = SIMDX_OK;
  std::vector<int32_t> args(rows);
  for (size_t i = 0; i < rows; ++i) args[i] = sl.batch[i].arg;
  if (r0.algo == SIMDX_ALGO_BFS) {
    rc = rows == 1 ? simdx_bfs(g, args[0], (int32_t*)sl.d_out, nullptr, sl.stream)
                   : simdx_bfs_batch(g, args.data(), (int32_t)rows, (int32_t*)sl.d_out, nullptr, sl.stream);
    for (size_t i = 0; i < rows && rc == SIMDX_OK; ++i)
      if (cudaMemcpyAsync(sl.batch[i].out, (char*)sl.d_out + i * nbytes_i32, nbytes_i32, cudaMemcpyDefault,
                          sl.stream) != cudaSuccess)
        rc = SIMDX_ECUDA;
  } else if (r0.algo == SIMDX_ALGO_SSSP) {
    rc = rows == 1 ? simdx_sssp(g, args[0], (uint32_t*)sl.d_out, nullptr, sl.stream)
                   : simdx_sssp_batch(g, args.data(), (int32_t)rows, (uint32_t*)sl.d_out, nullptr, sl.stream);
    for (size_t i = 0; i < rows && rc == SIMDX_OK; ++i)
      if (cudaMemcpyAsync(sl.batch[i].out, (char*)sl.d_out + i * nbytes_i32, nbytes_i32, cudaMemcpyDefault,
                          sl.stream) != cudaSuccess)
        rc = SIMDX_ECUDA;
  } else {
    // every query of the batch has the same k: one run answers all of them
    rc = simdx_kcore(g, (uint32_t)args[0], (uint8_t*)sl.d_out, (uint32_t*)sl.d_aux, nullptr, sl.stream);
    for (size_t i = 0; i < rows && rc == SIMDX_OK; ++i)
      if (cudaMemcpyAsync(sl.batch[i].out, sl.d_out, (size_t)g->n, cudaMemcpyDefault, sl.stream) != cudaSuccess)
        rc = SIMDX_ECUDA;
  }
  if (rc == SIMDX_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = SIMDX_ECUDA;
  return rc;
}

bool compatible(const Request& a, const Request& b) {
  if (a.graph != b.graph || a.algo != b.algo) return false;
  return a.algo != SIMDX_ALGO_KCORE || a.arg == b.arg;
}

void dispatcher(simdx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // 1. retire finished slots
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      int st = q == cudaSuccess ? 1 : -SIMDX_ECUDA;
      if (st == 1)
        for (const Request& r : sl.batch) {
          int ds = simdx_graph_last_status(sl.clones[r.graph], sl.stream);
          if (ds != SIMDX_OK) st = -ds;
        }
      for (const Request& r : sl.batch) s->status[r.ticket] = st;
      s->served += sl.batch.size();
      sl.batch.clear();
      sl.busy = false;
      progress = true;
    }
    if (progress) s->cv.notify_all();
    // 2. admit waiting queries onto free slots
    for (Slot& sl : s->slots) {
      if (sl.busy || s->queue.empty()) continue;
      Request head = s->queue.front();
      s->queue.pop_front();
      sl.batch.clear();
      sl.batch.push_back(head);
      const size_t cap = head.algo == SIMDX_ALGO_BFS ? 64 : head.algo == SIMDX_ALGO_SSSP ? (size_t)s->max_sssp : 1024;
      for (auto it = s->queue.begin(); it != s->queue.end() && sl.batch.size() < cap;) {
        if (compatible(head, *it)) {
          sl.batch.push_back(*it);
          it = s->queue.erase(it);
        } else {
          ++it;
        }
      }
      lk.unlock();
      const int rc = launch_batch(s, sl);
      lk.lock();
      if (rc != SIMDX_OK) {
        for (const Request& r : sl.batch) s->status[r.ticket] = -rc;
        sl.batch.clear();
        s->cv.notify_all();
      } else {
        sl.busy = true;
        ++s->launches;
      }
      progress = true;
    }
    if (!progress) {
      bool any_busy = false;
      for (Slot& sl : s->slots) any_busy |= sl.busy;
      // sleep until a submission arrives, or poll launches in flight
      if (any_busy)
        s->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

void free_server(simdx_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (simdx_graph* c : sl.clones)
      if (c) simdx_graph_destroy(c);
    cudaFree(sl.d_out);
    cudaFree(sl.d_aux);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

// Device bytes one slot needs for graph g (clone workspace, batch states,
// outputs), an estimate used for admission.
size_t slot_bytes(const simdx_graph* g, int max_sssp) {
  const size_t n = (size_t)g->n;
  const size_t lists = sizeof(int32_t) * 2 * 4 * std::max<size_t>(n, (size_t)g->grid_max * g->bin_cap) + 8 * n;
  const size_t bins = sizeof(int32_t) * 4 * (size_t)g->grid_max * std::max(1, g->bin_cap);
  const size_t state = 20 * n + 16 * n + 8 * ((size_t)g->e / std::max(1, g->cfg.huge_min) + n);
  const size_t ms = 24 * n;
  // batched SSSP: vertex-major distances (32 or 64 words per vertex) and two masks
  const size_t sb = g->w ? (4 * (size_t)(g->cfg.sssp_batch_width ? g->cfg.sssp_batch_width : 32) + 16) * n : 0;
  return lists + bins + state + ms + sb;
}

}  // namespace

using namespace simdx;

extern "C" {

int simdx_server_create(simdx_graph* const* gs, int32_t ng, size_t mem_budget, int32_t max_slots, int32_t max_sssp,
                        simdx_server** out) {
  if (!out || !gs || ng <= 0 || max_slots <= 0 || max_sssp <= 0) return SIMDX_EINVAL;
  *out = nullptr;
  for (int i = 0; i < ng; ++i)
    if (!gs[i] || !gs[i]->symmetric) return SIMDX_EINVAL;
  simdx_server* s = new (std::nothrow) simdx_server();
  if (!s) return SIMDX_ENOMEM;
  s->graphs.assign(gs, gs + ng);
  s->max_sssp = max_sssp;
  cudaGetDevice(&s->device);
  size_t per_slot = 0, max_n = 1;
  for (simdx_graph* g : s->graphs) {
    per_slot += slot_bytes(g, max_sssp);
    max_n = std::max<size_t>(max_n, (size_t)g->n);
  }
  per_slot += sizeof(int32_t) * max_n * (size_t)std::max(64, max_sssp) + 4 * max_n;
  int nslots = (int)std::min<size_t>((size_t)max_slots, per_slot ? mem_budget / per_slot : 0);
  int occ = 4;
  {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, bfs_kernel_ptr(gs[0]->off_bits), kThreads, 0) ==
            cudaSuccess &&
        blocks > 0)
      occ = blocks;
  }
  nslots = std::min(nslots, occ);  // every slot keeps at least one CTA per SM
  if (nslots <= 0) {
    delete s;
    return SIMDX_ENOMEM;
  }
  s->slots.resize(nslots);
  const int per_sm = std::max(1, occ / nslots);
  for (Slot& sl : s->slots) {
    int rc = SIMDX_OK;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      rc = SIMDX_ECUDA;
    sl.row_bytes = sizeof(int32_t) * max_n;
    if (rc == SIMDX_OK && cudaMalloc(&sl.d_out, sl.row_bytes * (size_t)std::max(64, max_sssp)) != cudaSuccess)
      rc = SIMDX_ENOMEM;
    if (rc == SIMDX_OK && cudaMalloc(&sl.d_aux, sizeof(uint32_t) * max_n) != cudaSuccess) rc = SIMDX_ENOMEM;
    for (simdx_graph* g : s->graphs) {
      if (rc != SIMDX_OK) break;
      simdx_csr csr{g->n, g->e, g->off_bits, g->off, g->idx};
      simdx_graph* c = nullptr;
      rc = simdx_graph_create(&csr, nullptr, g->w, SIMDX_BORROW, sl.stream, &c);
      if (rc != SIMDX_OK) break;
      sl.clones.push_back(c);
      simdx_config cfg = g->cfg;
      cfg.ctas_per_sm = per_sm;
      rc = simdx_graph_set_config(c, &cfg);
      if (rc != SIMDX_OK) break;
      // size the batch states now so that serving allocates nothing
      std::vector<int32_t> src(std::max(64, max_sssp), 0);
      rc = simdx_bfs_batch(c, src.data(), 64, (int32_t*)sl.d_out, nullptr, sl.stream);
      if (rc == SIMDX_OK && g->w)
        rc = simdx_sssp_batch(c, src.data(), max_sssp, (uint32_t*)sl.d_out, nullptr, sl.stream);
    }
    if (rc == SIMDX_OK && cudaStreamSynchronize(sl.stream) != cudaSuccess) rc = SIMDX_ECUDA;
    if (rc != SIMDX_OK) {
      free_server(s);
      return rc;
    }
  }
  s->th = std::thread(dispatcher, s);
  *out = s;
  return SIMDX_OK;
}

int simdx_server_submit(simdx_server* s, int32_t graph, int32_t algo, int32_t arg, void* out, uint64_t* ticket) {
  if (!s || !out || !ticket || graph < 0 || graph >= (int)s->graphs.size()) return SIMDX_EINVAL;
  const simdx_graph* g = s->graphs[graph];
  if (algo == SIMDX_ALGO_BFS || algo == SIMDX_ALGO_SSSP) {
    if (arg < 0 || arg >= g->n) return SIMDX_EINVAL;
    if (algo == SIMDX_ALGO_SSSP && !g->w) return SIMDX_EINVAL;
  } else if (algo != SIMDX_ALGO_KCORE || arg < 0) {
    return SIMDX_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    s->queue.push_back(Request{t, graph, algo, arg, out});
    s->status[t] = 0;
    *ticket = t;
  }
  s->cv.notify_all();
  return SIMDX_OK;
}

int simdx_server_poll(simdx_server* s, uint64_t ticket, int32_t* done) {
  if (!s || !done) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->status.find(ticket);
  if (it == s->status.end()) return SIMDX_EINVAL;
  *done = it->second != 0;
  if (it->second == 0) return SIMDX_ENOTREADY;
  const int st = it->second;
  s->status.erase(it);
  return st == 1 ? SIMDX_OK : -st;
}

int simdx_server_wait(simdx_server* s, uint64_t ticket) {
  if (!s) return SIMDX_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->status.find(ticket);
  if (it == s->status.end()) return SIMDX_EINVAL;
  s->cv.wait(lk, [&] { return s->status[ticket] != 0 || s->stop; });
  const int st = s->status[ticket];
  s->status.erase(ticket);
  return st == 1 ? SIMDX_OK : st == 0 ? SIMDX_EBUSY : -st;
}

int simdx_server_info(simdx_server* s, int32_t* slots, uint64_t* launches, uint64_t* served, uint64_t* queued) {
  if (!s) return SIMDX_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slots) *slots = (int32_t)s->slots.size();
  if (launches) *launches = s->launches;
  if (served) *served = s->served;
  if (queued) *queued = s->queue.size();
  return SIMDX_OK;
}

int simdx_server_destroy(simdx_server* s) {
  if (!s) return SIMDX_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& kv : s->status)
    if (kv.second == 0) kv.second = -SIMDX_EBUSY;
  free_server(s);
  return SIMDX_OK;
}

}  // extern "C"
