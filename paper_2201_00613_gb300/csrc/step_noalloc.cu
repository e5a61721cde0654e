// step_noalloc.cu -- squeeze_step_noalloc: one tiled step that allocates no
// memory.
//
// Some callers must not allocate device memory at all: code embedded in a
// host application or framework that owns the whole device memory budget
// (its pool has reserved nearly all HBM, so a cudaMalloc would fail or force
// it to release cached blocks), and code on a latency-critical path where the
// implicit device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable.  squeeze_create() allocates a status word and the tiled kernel
// allocates its neighbour program and adjacency table on first use, so those
// callers cannot use squeeze_step().  This entry point runs the same tiled
// kernel with all of its scratch (neighbour program, halo tables, per-tile
// adjacency table, status word) placed in one file-scope device array of
// fixed size, which every GPU that loads the library holds until exit.  With
// the runtime's lazy module loading, the array (and this library's kernel
// code) reaches a device on the first call there, when cudaGetSymbolAddress
// below loads the module: that call takes device memory, later ones do not.
//
// Host-side construction of the neighbour program uses fixed-size static host
// buffers as well, so no heap memory is requested either.
#include <stdio.h>

#include <mutex>

#include "squeeze_internal.cuh"

namespace {

using namespace sq;

// Maximum scratch of one call: status word, neighbour program, halo tables
// and the adjacency table (4 bytes per tile and halo direction).
constexpr size_t kNoallocScratchBytes = 4u << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Capacities of the static host work buffers (they bound the tile level).
constexpr uint64_t kBoxCap = 8192, kCellsCap = 1024, kSlotsCap = 1024, kHaloCap = 4096;

struct HostWork {
  int32_t inv[kBoxCap];
  uint32_t X[kCellsCap], Y[kCellsCap], refs[kSlotsCap * 8];
  uint64_t keys[kHaloCap], sorted[kHaloCap];
  uint32_t order[kHaloCap], rank[kHaloCap];
  uint16_t refs16[kSlotsCap * 8];
  uint32_t halo_off[kHaloCap];
  uint8_t halo_dir[kHaloCap];
  uint32_t chunks[5 * kHaloCap + kSlotsCap / 2 + 300];   // halo chunk and border-record tables
};

HostWork g_work;         // guarded by g_mutex
std::mutex g_mutex;
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices];  // device address of the array, per device

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

}  // namespace

extern "C" int squeeze_step_noalloc(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                                    uint32_t birth, uint32_t survive, const uint8_t *d_in,
                                    uint8_t *d_out, int *h_status, void *stream) {
  if (!d_in || !d_out || birth >= (1u << 9) || survive >= (1u << 9))
    return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_in | (uintptr_t)d_out) & 15u) return SQUEEZE_ERR_INVALID_ARG;
  FracDev f;
  int rc = sq_fill_fractal(s, k, offsets, r, f);
  if (rc) return rc;
  if (d_in < d_out ? d_in + f.cells > d_out : d_out + f.cells > d_in)
    return SQUEEZE_ERR_INVALID_ARG;  // overlapping buffers
  cudaStream_t st = (cudaStream_t)stream;

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  SQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SQUEEZE_ERR_UNSUPPORTED;
  if (!g_scratch_dev[dev]) {
    // Once per device, with that device current: the array's device address.
    // (The host-side symbol is only a stand-in and must not reach a kernel.)
    void *ptr = nullptr;
    SQ_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_scratch_dev[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *scratch = g_scratch_dev[dev];

  // The largest tile level whose program fits the static buffers and the
  // kernel's shared-memory budget (tried from the top, built in place).
  TileSpec sp;
  rc = SQUEEZE_ERR_UNSUPPORTED;
  for (int L = (int)(f.r < 16 ? f.r : 16); L >= 1; --L) {
    TileBuildSizes z;
    sq_tile_build_sizes(f, (uint32_t)L, z);
    if (z.box > kBoxCap || z.cells > kCellsCap || z.slots > kSlotsCap) continue;
    TileBuild B = {g_work.inv,   g_work.X,      g_work.Y,     g_work.refs,   g_work.keys,
                   g_work.sorted, g_work.order, g_work.rank,  g_work.refs16, g_work.halo_off,
                   g_work.halo_dir, kBoxCap,    kCellsCap,    kSlotsCap,     kHaloCap,
                   1u,            g_work.chunks};
    rc = sq_tile_build(f, (uint32_t)L, B, sp);
    if (rc == SQUEEZE_OK && sp.smem <= sq_tiled_smem_cap()) break;
    rc = SQUEEZE_ERR_UNSUPPORTED;
  }
  if (rc != SQUEEZE_OK) {
    sq_set_error_text("squeeze_step_noalloc: no tile level fits the static host buffers");
    return SQUEEZE_ERR_UNSUPPORTED;
  }

  // Scratch layout: status word | neighbour program | halo offsets and chunk
  // table | halo directions | adjacency table.
  const uint64_t tiles = (uint64_t)sp.tiles_x * sp.tiles_y;
  const uint32_t table_words = sq_tile_table_words(sp);
  const size_t off_refs = 256;
  const size_t off_hoff = align16(off_refs + (size_t)sp.slots * 16);
  const size_t off_hdir = align16(off_hoff + ((size_t)sp.nhalo + table_words) * 4);
  const size_t off_adj = align16(off_hdir + sp.nhalo);
  const uint64_t need = off_adj + (uint64_t)sp.ndirs * tiles * 4;
  if (need > kNoallocScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "squeeze_step_noalloc: level %u needs %llu bytes of scratch; the static maximum "
             "is %llu bytes",
             r, (unsigned long long)need, (unsigned long long)kNoallocScratchBytes);
    sq_set_error_text(msg);
    return SQUEEZE_ERR_UNSUPPORTED;
  }
  rc = sq_tile_launch_config(sp, dev);
  if (rc) return rc;

  // Every call rewrites the tables it reads and clears the status word; the
  // host buffers are pageable, so each copy has read them before returning.
  int *d_status = reinterpret_cast<int *>(scratch);
  uint16_t *d_refs = reinterpret_cast<uint16_t *>(scratch + off_refs);
  uint32_t *d_hoff = reinterpret_cast<uint32_t *>(scratch + off_hoff);
  uint8_t *d_hdir = scratch + off_hdir;
  uint32_t *d_adj = reinterpret_cast<uint32_t *>(scratch + off_adj);
  SQ_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  SQ_CUDA(cudaMemcpyAsync(d_refs, g_work.refs16, (size_t)sp.slots * 16, cudaMemcpyHostToDevice, st));
  if (sp.nhalo) {
    SQ_CUDA(cudaMemcpyAsync(d_hoff, g_work.halo_off, (size_t)sp.nhalo * 4, cudaMemcpyHostToDevice, st));
    if (table_words)
      SQ_CUDA(cudaMemcpyAsync(d_hoff + sp.nhalo, g_work.chunks, (size_t)table_words * 4,
                              cudaMemcpyHostToDevice, st));
    SQ_CUDA(cudaMemcpyAsync(d_hdir, g_work.halo_dir, sp.nhalo, cudaMemcpyHostToDevice, st));
  }
  Rule rule{birth, survive};
  TiledDev d = sq_tiled_dev(f, rule, sp, d_refs, d_hoff, d_hdir, d_adj, d_status);
  rc = sq_tile_build_adjacency(f, d, d_adj, st);
  if (rc == SQUEEZE_OK) rc = sq_tile_launch(d, sp, d_in, d_out, 1, st);
  if (rc) return rc;
  if (h_status) {
    SQ_CUDA(cudaStreamSynchronize(st));
    SQ_CUDA(cudaMemcpy(h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
  }
  return SQUEEZE_OK;
}
