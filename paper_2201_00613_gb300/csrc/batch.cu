// batch.cu -- many fractal instances stepped together.
//
// A batch is a fixed list of (handle, buffer pair) items, possibly of
// different NBB fractals and levels.  The items are split by the tiled
// kernel's tile-row instantiation (the triangle's 27-wide rows, the Vicsek
// cross's 25-wide ones, the carpet's 64-wide ones, ...): one CA step of all
// items is one launch of the persistent batched kernel per instantiation, so
// every launch runs one specialised code path with its own CTA size and
// shared memory.  Each launch's CTAs walk a host-built schedule of (instance,
// group range) entries, cut so that every CTA gets about the same number of
// group slots (a group costs about the same whether its 32 tile lanes are
// full or not).  Launches advance up to eight steps where the items' programs
// allow (the intermediate steps stay in shared memory).  The launches of n_steps
// steps are captured once into a CUDA graph (buffers ping-ponging) and
// replayed on later calls.
#include <stdio.h>
#include <string.h>

#include <map>
#include <new>
#include <vector>

#include "squeeze_internal.cuh"

using namespace sq;

// Steps per launch of the batched kernel at most (it is instantiated for 1, 2, 4
// and 8).
constexpr uint32_t kBatchPasses = 8;

// The items of one tile-row instantiation and their launch.
struct BatchPlan {
  int kind;                 // 27, 25, 8, 16, 64 or 0 (see sq_tile_kind)
  bool life;                // every item of the plan runs B3/S23
  uint32_t passes;          // steps per launch every item's program allows (1, 2 or 4)
  TileLayout lay;           // the maxima of the items' shared-memory needs
  int threads, grid;        // CTA size; persistent grid (the same for every steps per launch)
  bool records;             // some item reads its halo from border records
  BatchWork *d_work;
  uint32_t *d_sched;
};

struct squeeze_batch {
  std::vector<squeeze_batch_item> items;
  std::vector<uint32_t *> caller_rec;  // 2 per item (records of d_buf0, d_buf1), or empty
  std::vector<BatchPlan> plans;
  int threads, ctas_per_sm;   // 0: each plan's own CTA size / the occupancy limit
  bool use_graph;
  uint32_t parity;          // 0: states are in buffer 0, 1: in buffer 1
  int device;
  unsigned char *d_arena;   // one device allocation: the tables below, then the records
  TiledDev *d_devs;
  uint8_t **d_buf0, **d_buf1;
  uint32_t *d_rec;          // border records of the items, two per item
  bool rec_valid;           // the records of the current states are written (after a run)
  cudaStream_t capture;     // stream the graphs are captured on
  std::map<uint64_t, cudaGraphExec_t> graphs;  // (n_steps, parity, records) -> executable graph
};

namespace {

void release_graphs(squeeze_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

void release(squeeze_batch *b) {
  release_graphs(b);
  b->plans.clear();
  cudaFree(b->d_arena);   // the plans' schedules, descriptions and records live in it
  if (b->capture) cudaStreamDestroy(b->capture);
  b->d_arena = nullptr;
  b->d_rec = nullptr;
  b->d_devs = nullptr;
  b->d_buf0 = b->d_buf1 = nullptr;
  b->capture = nullptr;
}

// Contiguous group ranges per CTA with about total / grid units of weight
// each (cells[i] is instance i's weight, spread evenly over its groups):
// group g of instance i starts at cum[i] + g * cells_i / groups_i and belongs
// to the CTA whose range holds that start.
void build_schedule(const std::vector<uint64_t> &cells, const std::vector<uint64_t> &groups,
                    int grid, std::vector<BatchWork> &work, std::vector<uint32_t> &start) {
  uint64_t total = 0;
  for (uint64_t c : cells) total += c;
  std::vector<uint64_t> cum(cells.size() + 1, 0);
  for (size_t i = 0; i < cells.size(); ++i) cum[i + 1] = cum[i] + cells[i];
  work.clear();
  start.assign((size_t)grid + 1, 0);
  size_t i = 0;
  for (int c = 0; c < grid; ++c) {
    start[c] = (uint32_t)work.size();
    const unsigned __int128 lo = (unsigned __int128)total * c / grid;
    const unsigned __int128 hi = (unsigned __int128)total * (c + 1) / grid;
    while (i < cells.size() && cum[i + 1] <= lo) ++i;
    for (size_t j = i; j < cells.size() && cum[j] < hi; ++j) {
      // first group whose start cell >= bound: ceil((bound - cum) * groups / cells)
      auto first_at = [&](unsigned __int128 bound) -> uint64_t {
        if (bound <= cum[j]) return 0;
        unsigned __int128 x = (bound - cum[j]) * groups[j];
        uint64_t g = (uint64_t)((x + cells[j] - 1) / cells[j]);
        return g > groups[j] ? groups[j] : g;
      };
      uint64_t g0 = first_at(lo), g1 = first_at(hi);
      if (c == grid - 1) g1 = groups[j];
      if (g0 < g1) work.push_back(BatchWork{(uint32_t)j, 1u, g0, g1});
    }
  }
  start[grid] = (uint32_t)work.size();
}

// Consecutive CTAs whose only entry is a run of one instance, each run
// starting where the previous one ends, share those groups strided instead:
// the q-th of m CTAs takes gA + q, gA + q + m, ... below gB.  The CTAs then
// step a band of neighbouring groups at a time, so the halo chunks read from
// the tiles above and below are still in L2 (used for 64-wide rows, which
// lose nothing by not handing row ends over).  Each CTA keeps its number of
// groups within one.
void stride_schedule(std::vector<BatchWork> &work, const std::vector<uint32_t> &start) {
  const size_t grid = start.size() - 1;
  size_t c = 0;
  while (c < grid) {
    if (start[c + 1] - start[c] != 1) {
      ++c;
      continue;
    }
    size_t e = c;
    while (e + 1 < grid && start[e + 2] - start[e + 1] == 1 &&
           work[start[e + 1]].instance == work[start[c]].instance &&
           work[start[e + 1]].g_first == work[start[e]].g_end)
      ++e;
    const size_t m = e - c + 1;
    if (m > 1) {
      const uint64_t gA = work[start[c]].g_first, gB = work[start[e]].g_end;
      for (size_t q = 0; q < m; ++q) {
        BatchWork &w = work[start[c + q]];
        w.g_first = gA + q;
        w.g_end = gB;
        w.g_stride = (uint32_t)m;
      }
    }
    c = e + 1;
  }
}

int setup(squeeze_batch *b) {
  release(b);
  b->rec_valid = false;
  const uint32_t count = (uint32_t)b->items.size();
  std::vector<TiledDev> devs(count);
  std::vector<TileSpec> specs(count);
  std::vector<uint8_t *> buf0(count), buf1(count);
  for (uint32_t i = 0; i < count; ++i) {
    squeeze_handle *h = b->items[i].h;
    int rc = sq_tiled_prepare(h);
    if (rc) return rc;
    rc = sq_tiled_describe(h, &devs[i], &specs[i]);
    if (rc) return rc;
    buf0[i] = b->items[i].d_buf0;
    buf1[i] = b->items[i].d_buf1;
  }
  int sms = 0;
  SQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  // One plan per instantiation, in order of first appearance.
  std::vector<int> kinds;
  for (uint32_t i = 0; i < count; ++i) {
    const int kind = sq_tile_kind(specs[i]);
    bool seen = false;
    for (int k : kinds) seen = seen || k == kind;
    if (!seen) kinds.push_back(kind);
  }
  std::vector<std::vector<BatchWork>> works;
  std::vector<std::vector<uint32_t>> starts;
  for (int kind : kinds) {
    BatchPlan p{};
    p.kind = kind;
    p.life = true;
    p.passes = kBatchPasses;
    bool first = true;
    int own_threads = 0;
    std::vector<uint32_t> idx;
    std::vector<uint64_t> weight, groups;
    for (uint32_t i = 0; i < count; ++i) {
      if (sq_tile_kind(specs[i]) != kind) continue;
      const TileSpec &sp = specs[i];
      const squeeze_handle *h = b->items[i].h;
      TileLayout l = sq_tile_layout_of(sp);
      p.lay = first ? l : sq_tile_layout_max(p.lay, l);
      first = false;
      p.life = p.life && h->rule.birth == (1u << 3) && h->rule.survive == ((1u << 2) | (1u << 3));
      p.passes = sp.passes < p.passes ? sp.passes : p.passes;
      p.records = p.records || sp.rec_words != 0;
      own_threads = sp.threads > own_threads ? sp.threads : own_threads;
      idx.push_back(i);
      // a group costs about the same whatever its fill: weigh it by its slots
      weight.push_back(sp.groups * 32ull * sp.TW * sp.TH);
      groups.push_back(sp.groups);
    }
    if (p.lay.smem > 200 * 1024) return SQUEEZE_ERR_UNSUPPORTED;
    p.threads = b->threads ? b->threads : own_threads;
    uint64_t total_groups = 0;
    for (uint64_t g : groups) total_groups += g;
    // One schedule serves every steps-per-launch kernel: it is cut for the
    // smallest of their grids, and each launches that many CTAs.
    p.grid = 0;
    for (uint32_t steps = 1; steps <= p.passes; steps *= 2) {
      const int occ = sq_batch_occupancy(p.life, kind, steps, p.threads, p.lay.smem);
      if (occ < 1) return SQUEEZE_ERR_UNSUPPORTED;
      const int per_sm = b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ;
      const uint64_t grid = (uint64_t)per_sm * sms;
      const int g = (int)(grid < total_groups ? grid : total_groups);
      p.grid = p.grid == 0 || g < p.grid ? g : p.grid;
    }
    std::vector<BatchWork> work;
    std::vector<uint32_t> start;
    build_schedule(weight, groups, p.grid, work, start);
    if (kind == 64) stride_schedule(work, start);
    for (BatchWork &w : work) w.instance = idx[w.instance];
    b->plans.push_back(p);
    works.push_back(work);
    starts.push_back(start);
  }

  // One device allocation and one copy for the batch: the items'
  // descriptions and buffer pointers, each plan's schedule, then the border
  // records (two buffers per item, of this batch alone: items may share a
  // handle, each with its own states).
  auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t off = 0;
  const size_t o_devs = off;
  off = align(off + sizeof(TiledDev) * count);
  const size_t o_buf0 = off;
  off = align(off + sizeof(uint8_t *) * count);
  const size_t o_buf1 = off;
  off = align(off + sizeof(uint8_t *) * count);
  std::vector<size_t> o_work(b->plans.size()), o_sched(b->plans.size());
  for (size_t k = 0; k < b->plans.size(); ++k) {
    o_work[k] = off;
    off = align(off + sizeof(BatchWork) * (works[k].size() ? works[k].size() : 1));
    o_sched[k] = off;
    off = align(off + sizeof(uint32_t) * starts[k].size());
  }
  const size_t table_bytes = off;
  size_t rec_total = 0;
  const bool own_rec = b->caller_rec.empty();
  for (uint32_t i = 0; i < count && own_rec; ++i)
    rec_total += 2ull * specs[i].rec_words * specs[i].tiles_x * specs[i].tiles_y;
  SQ_CUDA(cudaMalloc(&b->d_arena, table_bytes + rec_total * 4));
  unsigned char *base = b->d_arena;
  b->d_rec = rec_total ? reinterpret_cast<uint32_t *>(base + table_bytes) : nullptr;
  size_t roff = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const size_t n = (size_t)specs[i].rec_words * specs[i].tiles_x * specs[i].tiles_y;
    if (!own_rec) {   // the caller's buffers (checked at creation)
      devs[i].rec[0] = n ? b->caller_rec[2 * i] : nullptr;
      devs[i].rec[1] = n ? b->caller_rec[2 * i + 1] : nullptr;
      continue;
    }
    devs[i].rec[0] = n ? b->d_rec + roff : nullptr;          // records of buffer 0
    devs[i].rec[1] = n ? b->d_rec + roff + n : nullptr;      // and of buffer 1
    roff += 2 * n;
  }
  std::vector<unsigned char> host(table_bytes, 0);
  memcpy(host.data() + o_devs, devs.data(), sizeof(TiledDev) * count);
  memcpy(host.data() + o_buf0, buf0.data(), sizeof(uint8_t *) * count);
  memcpy(host.data() + o_buf1, buf1.data(), sizeof(uint8_t *) * count);
  for (size_t k = 0; k < b->plans.size(); ++k) {
    BatchPlan &p = b->plans[k];
    if (works[k].size())
      memcpy(host.data() + o_work[k], works[k].data(), sizeof(BatchWork) * works[k].size());
    memcpy(host.data() + o_sched[k], starts[k].data(), sizeof(uint32_t) * starts[k].size());
    p.d_work = reinterpret_cast<BatchWork *>(base + o_work[k]);
    p.d_sched = reinterpret_cast<uint32_t *>(base + o_sched[k]);
  }
  b->d_devs = reinterpret_cast<TiledDev *>(base + o_devs);
  b->d_buf0 = reinterpret_cast<uint8_t **>(base + o_buf0);
  b->d_buf1 = reinterpret_cast<uint8_t **>(base + o_buf1);
  SQ_CUDA(cudaMemcpy(base, host.data(), table_bytes, cudaMemcpyHostToDevice));
  return SQUEEZE_OK;
}

// Launches of n_steps steps: up to eight steps per launch where every plan
// can, with a launch count of n_steps' parity (each launch swaps the
// buffers; the state after an even number of steps belongs in buffer 0).
int launch_steps(squeeze_batch *b, uint64_t n_steps, bool rec_current, cudaStream_t st) {
  uint32_t passes = kBatchPasses;
  for (const BatchPlan &p : b->plans) passes = p.passes < passes ? p.passes : passes;
  uint64_t counts[4];
  sq_launch_plan(n_steps, passes, counts);
  const uint64_t total = counts[0] + counts[1] + counts[2] + counts[3];
  // Launches of several steps read their halo from border records: first
  // those of the input (one records-only launch per instantiation whose items
  // have any) unless they are current; one-step launches can gather it from
  // the states instead.
  const bool boot = !rec_current && counts[1] + counts[2] + counts[3] != 0;
  bool live = rec_current || boot;
  for (const BatchPlan &p : b->plans) {
    if (!boot || !p.records || !total) continue;
    int rc = sq_batch_launch(b->d_devs, b->d_buf0, b->d_buf1, p.d_work, p.d_sched, p.lay, p.grid,
                             p.threads, p.life, p.kind, 1, (uint32_t)(b->parity & 1u), 1, st);
    if (rc) return rc;
  }
  for (uint64_t t = 0, i = 3, used = 0; t < total; ++t) {
    while (used == counts[i]) {   // largest launches first
      --i;
      used = 0;
    }
    ++used;
    const uint32_t parity = (uint32_t)((b->parity + t) & 1u);
    const uint32_t steps = 1u << i;
    for (const BatchPlan &p : b->plans) {
      int rc = sq_batch_launch(b->d_devs, b->d_buf0, b->d_buf1, p.d_work, p.d_sched, p.lay,
                               p.grid, p.threads, p.life, p.kind, steps, parity, live ? 0 : 2,
                               st);
      if (rc) return rc;
    }
    live = true;
  }
  return SQUEEZE_OK;
}

// A batch of `count` items; d_rec (2 per item: the records of d_buf0 and of
// d_buf1, those of d_buf0 current) or null for records of the batch's own.
int create_batch(const squeeze_batch_item *items, uint32_t count, uint32_t *const *d_rec,
                 squeeze_batch **out) {
  if (!out || !items || !count) return SQUEEZE_ERR_INVALID_ARG;
  *out = nullptr;
  for (uint32_t i = 0; i < count; ++i) {
    const squeeze_batch_item &it = items[i];
    if (!it.h || !it.d_buf0 || !it.d_buf1) return SQUEEZE_ERR_INVALID_ARG;
    if (((uintptr_t)it.d_buf0 | (uintptr_t)it.d_buf1) & 15u) return SQUEEZE_ERR_INVALID_ARG;
    uint64_t n = it.h->f.cells;
    if (it.d_buf0 < it.d_buf1 ? it.d_buf0 + n > it.d_buf1 : it.d_buf1 + n > it.d_buf0)
      return SQUEEZE_ERR_INVALID_ARG;
    if (d_rec) {   // every item whose program has records needs two aligned buffers
      uint64_t bytes = 0;
      int rc = squeeze_record_bytes(it.h, &bytes);
      if (rc) return rc;
      for (int k = 0; k < 2; ++k)
        if (bytes && (!d_rec[2 * i + k] || ((uintptr_t)d_rec[2 * i + k] & 3u)))
          return SQUEEZE_ERR_INVALID_ARG;
    }
  }
  squeeze_batch *b = new (std::nothrow) squeeze_batch();
  if (!b) return SQUEEZE_ERR_OOM;
  b->items.assign(items, items + count);
  if (d_rec) b->caller_rec.assign(d_rec, d_rec + 2 * (size_t)count);
  b->threads = 0;
  b->ctas_per_sm = 0;
  b->use_graph = true;
  b->parity = 0;
  cudaError_t e = cudaGetDevice(&b->device);
  int rc = e == cudaSuccess ? setup(b) : sq_cuda_fail(e);
  if (rc) {
    release(b);
    delete b;
    return rc;
  }
  b->rec_valid = d_rec != nullptr;   // the caller wrote the records of the states in d_buf0
  *out = b;
  return SQUEEZE_OK;
}

}  // namespace

extern "C" {

int squeeze_batch_create(const squeeze_batch_item *items, uint32_t count, squeeze_batch **out) {
  return create_batch(items, count, nullptr, out);
}

int squeeze_batch_create_with_records(const squeeze_batch_item *items, uint32_t count,
                                      uint32_t *const *d_rec, squeeze_batch **out) {
  if (!d_rec) return SQUEEZE_ERR_INVALID_ARG;
  return create_batch(items, count, d_rec, out);
}

int squeeze_batch_configure(squeeze_batch *b, uint32_t threads, uint32_t ctas_per_sm,
                            int use_graph) {
  if (!b || threads % 32 || (threads && threads < 64) || threads > 384)
    return SQUEEZE_ERR_INVALID_ARG;
  if ((int)threads == b->threads && (int)ctas_per_sm == b->ctas_per_sm) {
    // same launch shape: keep the plans (and the current records)
    if (!b->graphs.empty()) SQ_CUDA(cudaDeviceSynchronize());
    release_graphs(b);
    b->use_graph = use_graph != 0;
    return SQUEEZE_OK;
  }
  SQ_CUDA(cudaDeviceSynchronize());
  b->threads = (int)threads;
  b->ctas_per_sm = (int)ctas_per_sm;
  b->use_graph = use_graph != 0;
  return setup(b);
}

int squeeze_batch_info(const squeeze_batch *b, uint32_t *grid, uint32_t *threads,
                       uint32_t *smem_bytes) {
  if (!b) return SQUEEZE_ERR_INVALID_ARG;
  uint32_t g = 0, t = 0, m = 0;
  for (const BatchPlan &p : b->plans) {
    g += (uint32_t)p.grid;
    t = (uint32_t)p.threads > t ? (uint32_t)p.threads : t;
    m = p.lay.smem > m ? p.lay.smem : m;
  }
  if (grid) *grid = g;
  if (threads) *threads = t;
  if (smem_bytes) *smem_bytes = m;
  return SQUEEZE_OK;
}

int squeeze_batch_run(squeeze_batch *b, uint64_t n_steps, void *stream) {
  if (!b) return SQUEEZE_ERR_INVALID_ARG;
  if (!n_steps) return SQUEEZE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // The records of the states are rewritten only when they are not known to
  // be current (the first run, or after squeeze_batch_states_written).
  const bool current = b->rec_valid;
  if (!b->use_graph) {
    int rc = launch_steps(b, n_steps, current, st);
    if (rc == SQUEEZE_OK) b->parity ^= (uint32_t)(n_steps & 1u);
    b->rec_valid = rc == SQUEEZE_OK;
    return rc;
  }
  const uint64_t key = (n_steps * 2 + b->parity) * 2 + (current ? 0u : 1u);
  auto found = b->graphs.find(key);
  if (found == b->graphs.end()) {
    if (!b->capture) SQ_CUDA(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SQ_CUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    int rc = launch_steps(b, n_steps, current, b->capture);
    cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return sq_cuda_fail(e);
    found = b->graphs.emplace(key, exec).first;
  }
  b->rec_valid = false;
  SQ_CUDA(cudaGraphLaunch(found->second, st));
  b->parity ^= (uint32_t)(n_steps & 1u);
  b->rec_valid = true;
  return SQUEEZE_OK;
}

int squeeze_batch_states_written(squeeze_batch *b) {
  if (!b) return SQUEEZE_ERR_INVALID_ARG;
  b->rec_valid = false;
  return SQUEEZE_OK;
}

int squeeze_batch_destroy(squeeze_batch *b) {
  if (!b) return SQUEEZE_OK;
  cudaError_t e = cudaDeviceSynchronize();
  release(b);
  delete b;
  return e == cudaSuccess ? SQUEEZE_OK : sq_cuda_fail(e);
}

}  // extern "C"
