// batch.cu -- many fractal instances stepped together.
//
// A batch is a fixed list of (handle, buffer pair) items, possibly of
// different NBB fractals and levels.  One CA step of all items is ONE launch
// of the persistent batched tiled kernel: its CTAs walk a host-built schedule
// of (instance, group range) entries, split so that every CTA gets about the
// same number of cells.  n_steps steps are captured once into a CUDA graph
// (one launch per step, buffers ping-ponging) and replayed on later calls.
#include <stdio.h>
#include <string.h>

#include <map>
#include <new>
#include <vector>

#include "squeeze_internal.cuh"

using namespace sq;

struct squeeze_batch {
  std::vector<squeeze_batch_item> items;
  TileLayout lay;
  bool life;
  int threads, grid, ctas_per_sm;
  bool use_graph;
  uint32_t parity;          // 0: states are in buffer 0, 1: in buffer 1
  int device;
  TiledDev *d_devs;
  uint8_t **d_buf0, **d_buf1;
  BatchWork *d_work;
  uint32_t *d_sched;
  cudaStream_t capture;     // stream the graphs are captured on
  std::map<uint64_t, cudaGraphExec_t> graphs;  // (n_steps, parity) -> executable graph
};

namespace {

void release_graphs(squeeze_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

void release(squeeze_batch *b) {
  release_graphs(b);
  cudaFree(b->d_devs);
  cudaFree(b->d_buf0);
  cudaFree(b->d_buf1);
  cudaFree(b->d_work);
  cudaFree(b->d_sched);
  if (b->capture) cudaStreamDestroy(b->capture);
  b->d_devs = nullptr;
  b->d_buf0 = b->d_buf1 = nullptr;
  b->d_work = nullptr;
  b->d_sched = nullptr;
  b->capture = nullptr;
}

// Contiguous group ranges per CTA with about total_cells / grid cells each:
// group g of instance i starts at cell cum[i] + g * cells_i / groups_i and
// belongs to the CTA whose cell range holds that start.
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
      if (g0 < g1) work.push_back(BatchWork{(uint32_t)j, 0u, g0, g1});
    }
  }
  start[grid] = (uint32_t)work.size();
}

int setup(squeeze_batch *b) {
  release(b);
  const uint32_t count = (uint32_t)b->items.size();
  std::vector<TiledDev> devs(count);
  std::vector<uint8_t *> buf0(count), buf1(count);
  std::vector<uint64_t> cells(count), groups(count);
  b->life = true;
  bool first = true;
  for (uint32_t i = 0; i < count; ++i) {
    squeeze_handle *h = b->items[i].h;
    int rc = sq_tiled_prepare(h);
    if (rc) return rc;
    TileSpec sp;
    rc = sq_tiled_describe(h, &devs[i], &sp);
    if (rc) return rc;
    TileLayout l = sq_tile_layout(sp.slots, sp.nhalo, sp.TH, sp.pitch);
    b->lay = first ? l : sq_tile_layout_max(b->lay, l);
    first = false;
    b->life = b->life && h->rule.birth == (1u << 3) && h->rule.survive == ((1u << 2) | (1u << 3));
    buf0[i] = b->items[i].d_buf0;
    buf1[i] = b->items[i].d_buf1;
    cells[i] = h->f.cells;
    groups[i] = sp.groups;
  }
  if (b->lay.smem > 200 * 1024) return SQUEEZE_ERR_UNSUPPORTED;
  int occ = sq_batch_occupancy(b->life, b->threads, b->lay.smem);
  if (occ < 1) return SQUEEZE_ERR_UNSUPPORTED;
  int per_sm = b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ;
  int sms = 0;
  SQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  uint64_t total_groups = 0;
  for (uint64_t g : groups) total_groups += g;
  uint64_t grid = (uint64_t)per_sm * sms;
  b->grid = (int)(grid < total_groups ? grid : total_groups);
  std::vector<BatchWork> work;
  std::vector<uint32_t> start;
  build_schedule(cells, groups, b->grid, work, start);

  SQ_CUDA(cudaMalloc(&b->d_devs, sizeof(TiledDev) * count));
  SQ_CUDA(cudaMalloc(&b->d_buf0, sizeof(uint8_t *) * count));
  SQ_CUDA(cudaMalloc(&b->d_buf1, sizeof(uint8_t *) * count));
  SQ_CUDA(cudaMalloc(&b->d_work, sizeof(BatchWork) * (work.size() ? work.size() : 1)));
  SQ_CUDA(cudaMalloc(&b->d_sched, sizeof(uint32_t) * start.size()));
  SQ_CUDA(cudaMemcpy(b->d_devs, devs.data(), sizeof(TiledDev) * count, cudaMemcpyHostToDevice));
  SQ_CUDA(cudaMemcpy(b->d_buf0, buf0.data(), sizeof(uint8_t *) * count, cudaMemcpyHostToDevice));
  SQ_CUDA(cudaMemcpy(b->d_buf1, buf1.data(), sizeof(uint8_t *) * count, cudaMemcpyHostToDevice));
  if (work.size())
    SQ_CUDA(cudaMemcpy(b->d_work, work.data(), sizeof(BatchWork) * work.size(),
                       cudaMemcpyHostToDevice));
  SQ_CUDA(cudaMemcpy(b->d_sched, start.data(), sizeof(uint32_t) * start.size(),
                     cudaMemcpyHostToDevice));
  SQ_CUDA(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  return SQUEEZE_OK;
}

int launch_steps(squeeze_batch *b, uint64_t n_steps, cudaStream_t st) {
  for (uint64_t t = 0; t < n_steps; ++t) {
    int rc = sq_batch_launch(b->d_devs, b->d_buf0, b->d_buf1, b->d_work, b->d_sched, b->lay,
                             b->grid, b->threads, b->life, (uint32_t)((b->parity + t) & 1u),
                             st);
    if (rc) return rc;
  }
  return SQUEEZE_OK;
}

}  // namespace

extern "C" {

int squeeze_batch_create(const squeeze_batch_item *items, uint32_t count, squeeze_batch **out) {
  if (!out || !items || !count) return SQUEEZE_ERR_INVALID_ARG;
  *out = nullptr;
  for (uint32_t i = 0; i < count; ++i) {
    const squeeze_batch_item &it = items[i];
    if (!it.h || !it.d_buf0 || !it.d_buf1) return SQUEEZE_ERR_INVALID_ARG;
    if (((uintptr_t)it.d_buf0 | (uintptr_t)it.d_buf1) & 15u) return SQUEEZE_ERR_INVALID_ARG;
    uint64_t n = it.h->f.cells;
    if (it.d_buf0 < it.d_buf1 ? it.d_buf0 + n > it.d_buf1 : it.d_buf1 + n > it.d_buf0)
      return SQUEEZE_ERR_INVALID_ARG;
  }
  squeeze_batch *b = new (std::nothrow) squeeze_batch();
  if (!b) return SQUEEZE_ERR_OOM;
  b->items.assign(items, items + count);
  b->threads = 288;
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
  *out = b;
  return SQUEEZE_OK;
}

int squeeze_batch_configure(squeeze_batch *b, uint32_t threads, uint32_t ctas_per_sm,
                            int use_graph) {
  if (!b || threads % 32 || threads < 64 || threads > 288) return SQUEEZE_ERR_INVALID_ARG;
  SQ_CUDA(cudaDeviceSynchronize());
  b->threads = (int)threads;
  b->ctas_per_sm = (int)ctas_per_sm;
  b->use_graph = use_graph != 0;
  return setup(b);
}

int squeeze_batch_info(const squeeze_batch *b, uint32_t *grid, uint32_t *threads,
                       uint32_t *smem_bytes) {
  if (!b) return SQUEEZE_ERR_INVALID_ARG;
  if (grid) *grid = (uint32_t)b->grid;
  if (threads) *threads = (uint32_t)b->threads;
  if (smem_bytes) *smem_bytes = b->lay.smem;
  return SQUEEZE_OK;
}

int squeeze_batch_run(squeeze_batch *b, uint64_t n_steps, void *stream) {
  if (!b) return SQUEEZE_ERR_INVALID_ARG;
  if (!n_steps) return SQUEEZE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->use_graph) {
    int rc = launch_steps(b, n_steps, st);
    if (rc == SQUEEZE_OK) b->parity ^= (uint32_t)(n_steps & 1u);
    return rc;
  }
  const uint64_t key = n_steps * 2 + b->parity;
  auto found = b->graphs.find(key);
  if (found == b->graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SQ_CUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    int rc = launch_steps(b, n_steps, b->capture);
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
  SQ_CUDA(cudaGraphLaunch(found->second, st));
  b->parity ^= (uint32_t)(n_steps & 1u);
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
