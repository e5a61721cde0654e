// squeeze_internal.cuh -- shared device-side definitions of the CUDA library.
//
// Everything here belongs to the GPU path: the fractal descriptor passed to
// kernels by value, exact division by a runtime constant, the per-cell lambda
// and nu maps (Sec. 3.3 / 3.4 of arXiv 2201.00613) and the outer-totalistic
// rule of Sec. 4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "squeeze.h"

namespace sq {

constexpr uint8_t kHole = 0xFF;   // H_nu entry of a digit pair that is not a replica
constexpr int kMaxS = 16;          // s <= 16, so H_nu has at most 256 entries
constexpr int kMaxK = 255;
constexpr int kMaxPasses = 8;     // steps one launch of the tiled kernel can advance

// Exact unsigned 32-bit division by a runtime divisor d >= 1 with one
// multiply-high (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up variant with the add-back step).
struct FastDiv {
  uint32_t d;   // divisor
  uint32_t m;   // magic multiplier
  uint32_t l;   // ceil(log2(d)); 0 for d == 1
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 0u, 0u};
  if (d <= 1) return f;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.l = l;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d) + 1u;
  return f;
}

__host__ __device__ inline uint32_t fdiv(const FastDiv &f, uint32_t n) {
  if (f.d == 1) return n;
#ifdef __CUDA_ARCH__
  uint32_t t = __umulhi(f.m, n);
#else
  uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> 1)) >> (f.l - 1);
}

// Rule masks: a dead cell with c alive neighbours is born iff bit c of
// `birth`; an alive one survives iff bit c of `survive`.
struct Rule {
  uint32_t birth;
  uint32_t survive;
};

// Fractal descriptor handed to every kernel by value.
struct FracDev {
  uint32_t s, k, r;
  uint32_t n;          // s^r, side of the bounding box (<= 2^30)
  uint32_t W, H;       // compact columns (odd levels) and rows (even levels)
  uint64_t cells;      // k^r
  FastDiv divk, divs, divW;
  uint8_t taux[256];   // H_lambda: tau(beta) = (taux[beta], tauy[beta])
  uint8_t tauy[256];
  uint8_t hnu[256];    // H_nu[theta_y * s + theta_x] = beta, or kHole
  uint32_t nbhd;       // neighbourhood: bit (dy+1)*3+(dx+1) selects offset (dx, dy)
};

constexpr uint32_t kMoore = 0x1EFu;       // all 8 offsets
constexpr uint32_t kVonNeumann = 0xAAu;   // the 4 orthogonal offsets

// Tables staged in shared memory by the per-cell kernels.
struct SmemTables {
  uint8_t taux[256];
  uint8_t tauy[256];
  uint8_t hnu[256];
};

__device__ inline void load_tables(SmemTables &t, const FracDev &f) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    t.taux[i] = f.taux[i];
    t.tauy[i] = f.tauy[i];
    t.hnu[i] = f.hnu[i];
  }
}

// lambda (Sec. 3.3): sum over levels mu = 1..r of tau(beta_mu) * s^(mu-1),
// beta_mu the base-k digit ceil(mu/2)-1 of w_x (odd mu) or w_y (even mu).
__host__ __device__ inline void lambda_alu(const FracDev &f, const SmemTables &t, uint32_t wx,
                                           uint32_t wy, uint32_t &x, uint32_t &y) {
  uint32_t X = 0, Y = 0, scale = 1;
  for (uint32_t mu = 1; mu <= f.r; ++mu) {
    uint32_t src = (mu & 1u) ? wx : wy;
    uint32_t q = fdiv(f.divk, src);
    uint32_t beta = src - q * f.k;
    if (mu & 1u) wx = q; else wy = q;
    X += t.taux[beta] * scale;
    Y += t.tauy[beta] * scale;
    scale *= f.s;
  }
  x = X;
  y = Y;
}

// nu (Sec. 3.4): per level the base-s digit pair theta_mu selects a replica id
// through H_nu (a hole rejects the point); odd levels accumulate id *
// k^floor((mu-1)/2) on w_x, even levels on w_y.
__host__ __device__ inline bool nu_alu(const FracDev &f, const SmemTables &t, int32_t x, int32_t y,
                                       uint32_t &wx, uint32_t &wy) {
  if (x < 0 || y < 0 || (uint32_t)x >= f.n || (uint32_t)y >= f.n) return false;
  uint32_t ux = (uint32_t)x, uy = (uint32_t)y;
  uint32_t nx = 0, ny = 0, wtx = 1, wty = 1;
  for (uint32_t mu = 1; mu <= f.r; ++mu) {
    uint32_t qx = fdiv(f.divs, ux), qy = fdiv(f.divs, uy);
    uint32_t tx = ux - qx * f.s, ty = uy - qy * f.s;
    ux = qx;
    uy = qy;
    uint32_t id = t.hnu[ty * f.s + tx];
    if (id == kHole) return false;
    if (mu & 1u) {
      nx += id * wtx;
      wtx *= f.k;
    } else {
      ny += id * wty;
      wty *= f.k;
    }
  }
  wx = nx;
  wy = ny;
  return true;
}

// Compact position (nwx, nwy) of the point (dx, dy) away (|dx|, |dy| <= 1)
// from the fractal cell at compact position (wx, wy), or false for a hole or
// a point off the box.  nu of the moved point differs from the cell's own
// digits only up to the level where the carries of dx and dy stop, so the
// walk (the digit form of nu, Sec. 3.4) runs from level 1 only that far: it
// reads the cell's replica digit beta_mu, moves its offset tau(beta_mu) by the
// carries, looks up the new replica through H_nu (a hole ends the walk) and
// corrects that level's term of the compact index.
__host__ __device__ inline bool neighbour_omega(const FracDev &f, const SmemTables &t, uint32_t wx,
                                                uint32_t wy, int dx, int dy, uint32_t &nwx,
                                                uint32_t &nwy) {
  uint32_t rx = wx, ry = wy;
  nwx = wx;
  nwy = wy;
  uint64_t weight_x = 1, weight_y = 1;
  int cx = dx, cy = dy;
  for (uint32_t mu = 1; mu <= f.r; ++mu) {
    if (cx == 0 && cy == 0) return true;
    const bool odd = mu & 1u;
    uint32_t &src = odd ? rx : ry;
    const uint32_t q = fdiv(f.divk, src), beta = src - q * f.k;
    src = q;
    int xd = (int)t.taux[beta] + cx, yd = (int)t.tauy[beta] + cy;
    cx = xd < 0 ? -1 : (xd >= (int)f.s ? 1 : 0);
    cy = yd < 0 ? -1 : (yd >= (int)f.s ? 1 : 0);
    xd -= cx * (int)f.s;
    yd -= cy * (int)f.s;
    const uint32_t id = t.hnu[yd * f.s + xd];
    if (id == kHole) return false;
    const int64_t delta = (int64_t)id - (int64_t)beta;
    if (odd) {
      nwx = (uint32_t)((int64_t)nwx + delta * (int64_t)weight_x);
      weight_x *= f.k;
    } else {
      nwy = (uint32_t)((int64_t)nwy + delta * (int64_t)weight_y);
      weight_y *= f.k;
    }
  }
  return cx == 0 && cy == 0;   // a carry out of the top level leaves the box
}

__device__ __host__ inline uint32_t apply_rule(const Rule &rule, bool alive, uint32_t c) {
  return ((alive ? rule.survive : rule.birth) >> c) & 1u;
}

// SplitMix64 output number i of the stream seeded with `seed`
// (Steele, Lea, Flood, OOPSLA 2014): mix(seed + (i+1) * gamma).
__device__ __host__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __host__ inline uint8_t bernoulli_cell(uint64_t seed, uint32_t p_q24, uint32_t x,
                                                  uint32_t y) {
  uint64_t key = ((uint64_t)y << 32) | (uint64_t)x;
  return (uint8_t)((splitmix64_at(seed, key) >> 40) < (uint64_t)p_q24);
}

// Kernel-side description of a tiled-step program (see step_tiled.cu).
struct TiledDev {
  uint64_t W;                // compact row length (bytes)
  uint64_t total;            // k^r, bytes of a state buffer
  Rule rule;
  uint32_t L, TW, TH, cells, nhalo, dir_mask, slots;
  uint32_t valid;            // packed-word bits that hold a real cell (lx < TW)
  uint32_t rpw;              // tile rows per slot word: 32 / TW for TW = 8, 16, else 1
  uint32_t nwin;             // aligned 32-bit words covering one tile row
  uint32_t tiles_x, tiles_y, groups_per_band, pitch;
  uint64_t groups;
  uint32_t ndirs;
  uint32_t dir_list[9];
  uint32_t halo_start[10];   // halo slots of direction j: [halo_start[j], halo_start[j+1])
  uint64_t tiles;            // tiles_x * tiles_y
  FastDiv div_tw, div_gpb, div_tiles_x;
  const uint16_t *refs;      // slots x 8 byte offsets of the neighbour words
  const uint32_t *halo_off;  // nhalo byte offsets inside a tile
  const uint8_t *halo_dir;   // nhalo direction indices
  const uint32_t *adj;       // ndirs x tiles adjacent tile indices (~0: none)
  int *status;
  uint32_t ring_end[kMaxPasses + 1];        // halo words of rings 1..k: [0, ring_end[k])
  uint32_t ring_start[kMaxPasses - 1][10];  // words of ring k + 2 in direction j
  uint64_t wait_ns;          // a bulk-copy wait gives up after this many ns
  uint32_t fault;            // SQUEEZE_FAULT_* (test hook), normally 0
  // Halo by 16-byte chunks (64-wide rows only; 0: halo bytes one by one).
  // halo_off is followed by the chunk table: nchunks chunk offsets inside a
  // tile, nchunks + 1 cell ranges, then nhalo cells (halo word | byte << 16);
  // direction j owns chunks [chunk_start[j], chunk_start[j + 1]).
  uint32_t nchunks;
  uint32_t chunk_start[10];
  // Border records: each launch also writes, per tile, the states of its
  // cells that adjacent tiles read as halo, rec_words words per tile, segment
  // j (words [rec_seg[j], rec_seg[j+1])) holding what the tile adjacent in
  // direction j of it reads, bit i of word w = halo cell 32 w + i of that
  // segment.  The record tables after the chunk table map each record bit to
  // (exported cell | halo word << 16), each exported cell to its slot, and
  // each slot to its exported cell.  rec[0]: records of the input state (null:
  // gather the halo from the state), rec[1]: records of the output state; mode
  // 1 writes the input's records to rec[1] and nothing else.
  uint32_t rec_words;
  uint32_t rec_seg[10];
  uint32_t rec_nexp;         // exported cells: final-step words kept per group
  uint32_t *rec[2];
  uint32_t mode;
};

constexpr uint64_t kDefaultWaitNs = 2000000000ull;

// Shared-memory layout of one launch of the tiled kernel (uniform over the
// instances of a batched launch: the maxima of their needs).
struct TileLayout {
  uint32_t win_bytes;        // one word buffer (two are used)
  uint32_t hoff_bytes;       // halo offsets
  uint32_t hdir_bytes;       // halo direction indices (one byte per halo word)
  uint32_t rowa_bytes;       // per-row alignment offsets (two sets)
  uint32_t carry_bytes;      // per-row 16-byte chunk handed to the next group
  uint32_t z_bytes;          // exported final-step words of the last two groups (border records)
  uint32_t stage_bytes;      // one staging buffer (two are used)
  uint32_t smem;             // total dynamic shared memory
};

// Geometry and launch shape of a tiled-step program, independent of where its
// tables live.
struct TileSpec {
  uint32_t L, TW, TH, rpw, cells, slots, nhalo, ndirs, dir_mask;
  uint32_t passes;     // steps one launch of the program can advance: 1, 2, 4 or 8
  uint32_t ring_end[kMaxPasses + 1];  // halo words of rings 1..k: [0, ring_end[k]) (ring_end[passes] = nhalo)
  uint8_t dir_list[9];
  uint32_t halo_start[10];   // first-ring words of direction j: [halo_start[j], halo_start[j+1])
  uint32_t ring_start[kMaxPasses - 1][10];  // words of ring k + 2 in direction j: [ring_start[k][j], ring_start[k][j+1])
  uint32_t tiles_x, tiles_y, groups_per_band, pitch;
  uint32_t nchunks;          // chunk table of the halo (64-wide rows), 0 if none
  uint32_t chunk_start[10];  // chunks of direction j: [chunk_start[j], chunk_start[j+1])
  uint32_t rec_words;        // border record words per tile, 0 if none
  uint32_t rec_seg[10];      // record words read by direction j: [rec_seg[j], rec_seg[j+1])
  uint32_t rec_nexp;         // cells of a tile that its record holds
  uint64_t groups;
  size_t smem;
  int threads;
  int grid[4][2];      // persistent grid per steps-per-launch (1, 2, 4, 8) and rule (generic, B3/S23)
  int occ[4][2];       // CTAs per SM of those kernels
};

// Capacities needed to build the program of one tile level.
struct TileBuildSizes {
  uint64_t box, cells, slots, halo;
};

// Caller-provided host buffers for building a program: work arrays (inv, X,
// Y, refs, halo_key, halo_sorted, order, rank) and outputs (refs16 with
// 8 * slots entries, halo_off and halo_dir with one entry per halo slot).
struct TileBuild {
  int32_t *inv;
  uint32_t *X, *Y, *refs;
  uint64_t *halo_key, *halo_sorted;
  uint32_t *order, *rank;
  uint16_t *refs16;
  uint32_t *halo_off;
  uint8_t *halo_dir;
  uint64_t box_cap, cells_cap, slots_cap, halo_cap;
  // Steps per launch the program is built for (1, 2, 4 or 8): for P > 1 the halo
  // rings 2..P are built too, and references for rings 1..P-1 (refs and
  // refs16 then need (slots + halo_cap) * 8 entries).
  uint32_t passes;
  // Optional: the halo's chunk table (64-wide rows) and the border-record
  // tables, at most 5 * halo_cap + slots_cap / 2 + 300 words (layout as in
  // TiledDev); null builds a program without them.
  uint32_t *chunks;
};

// One entry of a batched launch's schedule: CTA c processes entries
// [sched_start[c], sched_start[c + 1]), each the groups g_first, g_first +
// g_stride, ... below g_end of one instance.
struct BatchWork {
  uint32_t instance;
  uint32_t g_stride;
  uint64_t g_first, g_end;
};

inline unsigned grid_for(uint64_t items, unsigned block, unsigned cap = 152u * 16u) {
  uint64_t g = (items + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace sq

// ---- host-side internals shared between translation units ------------------

struct TiledProgram;  // defined in step_tiled.cu

struct squeeze_handle {
  sq::FracDev f;
  sq::Rule rule;
  int *d_status;             // device status word (SQUEEZE_OK / DEVICE_*)
  int device;                // CUDA device the tables live on
  uint32_t tiled_level;      // 0 = not chosen yet
  TiledProgram *tiled;       // lazily built neighbour program of the tiled kernel
  uint64_t wait_ns;          // device wait limit of the tiled kernels (0: default)
  uint32_t fault;            // fault-injection flags (tests only)
  int last_kind;             // kind the last squeeze_step ran (0 before the first)
  uint64_t last_launches;    // kernel launches of that call
  uint64_t last_counts[4];   // of which 1, 2, 4 and 8 steps per launch
  uint32_t max_passes;       // steps per launch at most (0: the default choice)
};

// Error plumbing and descriptor validation (handle.cu).
int sq_cuda_fail(cudaError_t e);
// Allow a kernel `bytes` of dynamic shared memory on the current device
// (raised only; see handle.cu).
cudaError_t sq_allow_smem(const void *fn, size_t bytes);
void sq_set_error_text(const char *text);
int sq_fill_fractal(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r, sq::FracDev &f);
#define SQ_CUDA(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return sq_cuda_fail(e_);   \
  } while (0)

// Launchers implemented in the kernel translation units.
int sq_launch_lambda(const squeeze_handle *h, const uint64_t *omega, int32_t *xy,
                     uint64_t count, cudaStream_t st);
int sq_launch_nu(const squeeze_handle *h, const int32_t *xy, uint64_t *omega, uint64_t count,
                 cudaStream_t st);
int sq_launch_init(const squeeze_handle *h, uint8_t *state, uint64_t seed, uint32_t p_q24,
                   cudaStream_t st);
int sq_launch_step_alu(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                       cudaStream_t st);
int sq_tiled_prepare(squeeze_handle *h);
// One launch of the handle's tiled program: steps = 1, 2, 4 or 8, at most the
// passes the program was built for (sq_tiled_passes); `last`: no later launch
// of the call reads the border records of its output.
int sq_launch_step_tiled(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                         uint32_t steps, bool last, cudaStream_t st);
// Border records of a squeeze_step call's input, before its tiled launches,
// when some launch advances several steps (multi); *launches = 1 if a
// records-only launch was made.
int sq_tiled_begin(const squeeze_handle *h, const uint8_t *in, bool multi, cudaStream_t st,
                   int *launches);
uint32_t sq_tiled_passes(const squeeze_handle *h);
// Launches of n steps at up to `passes` steps each: counts[i] launches of
// 2^i steps (i = 0..3), with a launch count of n's parity (every launch swaps
// the buffers; the result belongs in buffer n & 1).
void sq_launch_plan(uint64_t n, uint32_t passes, uint64_t *counts);
void sq_tiled_free(TiledProgram *p);
int sq_tiled_default_level(const squeeze_handle *h);
int sq_tiled_default_level_for(const sq::FracDev &f);
size_t sq_tiled_smem_cap();
void sq_tile_build_sizes(const sq::FracDev &f, uint32_t L, sq::TileBuildSizes &z);
int sq_tile_build(const sq::FracDev &f, uint32_t L, const sq::TileBuild &B, sq::TileSpec &sp);
int sq_tile_launch_config(sq::TileSpec &sp, int device);
sq::TiledDev sq_tiled_dev(const sq::FracDev &f, const sq::Rule &rule, const sq::TileSpec &sp,
                          const uint16_t *refs, const uint32_t *halo_off,
                          const uint8_t *halo_dir, const uint32_t *adj, int *status);
sq::TileLayout sq_tile_layout(uint32_t slots, uint32_t nhalo, uint32_t TH, uint32_t pitch,
                              uint32_t table_words = 0, uint32_t z_words = 0);
// Shared-memory layout of a program (its tables and record buffers included).
sq::TileLayout sq_tile_layout_of(const sq::TileSpec &sp);
// Words of a program's halo chunk table (0 when it has none).
uint32_t sq_tile_table_words(const sq::TileSpec &sp);
sq::TileLayout sq_tile_layout_max(const sq::TileLayout &a, const sq::TileLayout &b);
int sq_tile_build_adjacency(const sq::FracDev &f, const sq::TiledDev &d, uint32_t *adj,
                            cudaStream_t st);
// One launch of the tiled kernel: steps = 1, 2, 4 or 8 (at most the program's passes).
int sq_tile_launch(const sq::TiledDev &d, const sq::TileSpec &sp, const uint8_t *in,
                   uint8_t *out, uint32_t steps, cudaStream_t st);
// The handle's prepared tiled program (sq_tiled_prepare first).
int sq_tiled_describe(const squeeze_handle *h, sq::TiledDev *d, sq::TileSpec *sp);
// Tile-row instantiation of a program: 8 or 16 (rows sharing a slot word),
// 27, 25 or 64 (their own instantiations), 0 (width taken at run time).
int sq_tile_kind(const sq::TileSpec &sp);
// CTAs per SM of the batched kernel instance for this shape (0 if it cannot
// run); steps = 1 or 2 per launch.
int sq_batch_occupancy(bool life, int kind, uint32_t steps, int threads, uint32_t smem);
int sq_batch_launch(const sq::TiledDev *d_devs, uint8_t *const *d_buf0, uint8_t *const *d_buf1,
                    const sq::BatchWork *d_work, const uint32_t *d_sched,
                    const sq::TileLayout &lay, int grid, int threads, bool life, int kind,
                    uint32_t steps, uint32_t parity, uint32_t mode, cudaStream_t st);
bool sq_tiled_level_fits(const squeeze_handle *h, uint32_t level);
int sq_launch_step_tc(const squeeze_handle *h, const uint8_t *in, uint8_t *out, cudaStream_t st);
int sq_launch_map_tc(const squeeze_handle *h, int direction, const void *in, void *out,
                     uint64_t count, cudaStream_t st);
int sq_launch_bb_init(const squeeze_handle *h, uint8_t *grid, uint64_t seed, uint32_t p_q24,
                      cudaStream_t st);
int sq_launch_bb_step(const squeeze_handle *h, const uint8_t *in, uint8_t *out, cudaStream_t st);
int sq_launch_heat_step(const squeeze_handle *h, const float *in, float *out, float alpha,
                        cudaStream_t st);
int sq_launch_ising(const squeeze_handle *h, uint8_t *state, uint64_t n_sweeps, uint64_t seed,
                    double temperature, cudaStream_t st);
int sq_launch_lambda_step(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                          cudaStream_t st);
int sq_launch_bb_gather(const squeeze_handle *h, const uint8_t *grid, uint8_t *state,
                        cudaStream_t st);
