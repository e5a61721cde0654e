// step_tiled.cu -- the bit-sliced tile kernel for one neighbourhood step.
//
// Self-similarity (Sec. 3: every level-L sub-replica of an NBB fractal is a
// translated copy of the level-L fractal) means the compact -> expanded map
// restricted to one level-L sub-replica ("tile", k^L cells) is the same for
// every tile up to a translation.  So is the neighbour relation between cells
// of one tile: the lambda / 8-neighbour / nu exploration of Sec. 3.2 is run
// once, on the host, for the level-L fractal, and stored as a table of up to
// 8 local neighbour references per local cell.  A neighbour that falls in an
// adjacent level-L block is a "halo" reference (direction, local cell there);
// whether that block is a tile, a hole or off the box is decided once per
// handle on the device by a carry walk over each tile's higher replica digits
// (the digit-level form of nu, Sec. 3.4, which stops at the first level
// without a carry) and kept as an adjacency table.
//
// A CTA owns a group of up to 32 tiles lying side by side in compact x.  TMA
// bulk copies stage their rows in shared memory; each lane packs one tile row
// (<= 32 cells) into a 32-bit word and a 5-stage shuffle butterfly transposes
// the warp's 32 words, so that bit i of a word is the state of one local cell
// in tile i.  The rule then runs on whole words with a bit-sliced adder (32
// cells per bitwise operation); the inverse transpose and an unaligned,
// merged unpack return the bytes to the staging rows, and TMA bulk stores
// write them back.  Rows 8 or 16 cells wide share a word (4 or 2 rows per
// word); rows 64 cells wide take two words.  A launch of several steps reads
// its halo from border records, a few words per tile that the previous launch
// wrote for its neighbours; a one-step launch can instead read the halo bytes
// from the state (single bytes, or for 64-wide rows, whose tiles start on
// 64-byte boundaries, 16-byte chunks of the adjacent tiles).
//
// Bit order of a packed row word: bit 8b + j holds tile-row byte 4j + b (the
// order the pack produces for free); the neighbour program is built in that
// order, with slot p = 32 * ly + (8 * (lx & 3) + (lx >> 2)) for one row per
// word (rows sharing a word or split over two words extend lx accordingly).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tile2d.cuh"

struct TiledProgram {
  sq::TileSpec spec;
  uint16_t *d_refs;         // 8 x slots byte offsets of the neighbour words
  uint32_t *d_halo_off;     // nhalo byte offsets inside a tile (ly * W + lx)
  uint8_t *d_halo_dir;      // nhalo indices into dir_list
  uint32_t *d_adj;          // ndirs x tiles: adjacent tile index, or ~0 (hole / off the box)
  // Border records: tiles x rec_words words each, one per state buffer of a
  // squeeze_step call; rec_cur is the one of the next launch's input (the
  // launches of a call alternate, like the buffers).
  uint32_t *d_rec[2];
  int rec_cur;
  bool rec_live;            // d_rec[rec_cur] holds the records of the next launch's input
};

namespace sq {
namespace {

// ---- host side: the level-L neighbour program ------------------------------

// The instantiation for a program: rows shared by slot words (rpw 4 or 2) and
// rows of two slot words (width 64) have their own, as have the common widths
// 27 (triangle) and 25 (Vicsek); steps per launch 1, 2, 4 or 8.
template <bool kLife, int kT>
const void *tiled_kernel_of(uint32_t TW, uint32_t rpw) {
  if (rpw == 4) return (const void *)step_tiled_kernel<kLife, 8, kT>;
  if (rpw == 2) return (const void *)step_tiled_kernel<kLife, 16, kT>;
  if (TW == 64) return (const void *)step_tiled_kernel<kLife, 64, kT>;
  if (TW == 27) return (const void *)step_tiled_kernel<kLife, 27, kT>;
  if (TW == 25) return (const void *)step_tiled_kernel<kLife, 25, kT>;
  return (const void *)step_tiled_kernel<kLife, 0, kT>;
}

const void *tiled_kernel_for(bool life, uint32_t TW, uint32_t rpw, uint32_t steps) {
  if (steps == 8) return life ? tiled_kernel_of<true, 8>(TW, rpw) : tiled_kernel_of<false, 8>(TW, rpw);
  if (steps == 4) return life ? tiled_kernel_of<true, 4>(TW, rpw) : tiled_kernel_of<false, 4>(TW, rpw);
  if (steps == 2) return life ? tiled_kernel_of<true, 2>(TW, rpw) : tiled_kernel_of<false, 2>(TW, rpw);
  return life ? tiled_kernel_of<true, 1>(TW, rpw) : tiled_kernel_of<false, 1>(TW, rpw);
}

int steps_index(uint32_t steps) { return steps == 8 ? 3 : (steps == 4 ? 2 : (steps == 2 ? 1 : 0)); }


uint64_t ipow(uint64_t b, uint32_t e) {
  uint64_t p = 1;
  while (e--) p *= b;
  return p;
}

}  // namespace
}  // namespace sq

using namespace sq;

static uint32_t layout_total(const TileLayout &l) {
  return 2 * l.win_bytes + l.hoff_bytes + l.hdir_bytes + 16 + l.rowa_bytes + l.carry_bytes +
         l.z_bytes + 2 * l.stage_bytes;
}

// Word buffer: slots, halo words, the zero word and 9 per-direction masks.
TileLayout sq_tile_layout(uint32_t slots, uint32_t nhalo, uint32_t TH, uint32_t pitch,
                          uint32_t table_words, uint32_t z_words) {
  TileLayout l;
  l.win_bytes = (uint32_t)((((size_t)slots + nhalo + 1 + 9) * 4 + 15) & ~(size_t)15);
  l.hoff_bytes = (uint32_t)((((size_t)nhalo + table_words) * 4 + 15) & ~(size_t)15);
  l.hdir_bytes = (uint32_t)(((size_t)nhalo + 15) & ~(size_t)15);
  l.rowa_bytes = (uint32_t)(((size_t)2 * TH + 15) & ~(size_t)15);
  l.carry_bytes = 16u * TH;
  l.z_bytes = (uint32_t)(((size_t)z_words * 4 + 15) & ~(size_t)15);
  // + slack: the last lane's whole-word reads and writes of the last row run up
  // to 8 bytes past it (a 27-wide row: 9 words from a 4-byte boundary below a
  // row start at most 15 bytes into the pitch, and 32 * 27 + 15 <= pitch)
  l.stage_bytes = (uint32_t)((size_t)TH * pitch + 16);
  l.smem = layout_total(l);
  return l;
}

// Words of the chunk table (kept in shared memory) and of the record tables
// (read through the cache), which follow the halo offsets in device memory.
static uint32_t chunk_table_words(const TileSpec &sp) {
  return sp.nchunks ? 2u * sp.nchunks + 1u + sp.nhalo : 0u;
}

uint32_t sq_tile_table_words(const TileSpec &sp) {
  return chunk_table_words(sp) +
         (sp.rec_words ? 32u * sp.rec_words + sp.rec_nexp + (sp.slots + 1u) / 2u : 0u);
}

TileLayout sq_tile_layout_of(const TileSpec &sp) {
  return sq_tile_layout(sp.slots, sp.nhalo, sp.TH, sp.pitch, chunk_table_words(sp),
                        2u * sp.rec_nexp);
}

TileLayout sq_tile_layout_max(const TileLayout &a, const TileLayout &b) {
  TileLayout l;
  l.win_bytes = a.win_bytes > b.win_bytes ? a.win_bytes : b.win_bytes;
  l.hoff_bytes = a.hoff_bytes > b.hoff_bytes ? a.hoff_bytes : b.hoff_bytes;
  l.hdir_bytes = a.hdir_bytes > b.hdir_bytes ? a.hdir_bytes : b.hdir_bytes;
  l.rowa_bytes = a.rowa_bytes > b.rowa_bytes ? a.rowa_bytes : b.rowa_bytes;
  l.carry_bytes = a.carry_bytes > b.carry_bytes ? a.carry_bytes : b.carry_bytes;
  l.z_bytes = a.z_bytes > b.z_bytes ? a.z_bytes : b.z_bytes;
  l.stage_bytes = a.stage_bytes > b.stage_bytes ? a.stage_bytes : b.stage_bytes;
  l.smem = layout_total(l);
  return l;
}

namespace sq {
namespace {

size_t smem_for(uint32_t slots, uint32_t nhalo, uint32_t TH, uint32_t pitch) {
  return sq_tile_layout(slots, nhalo, TH, pitch).smem;
}

// Staging row: up to 15 bytes of alignment offset + 32 tiles + one spare chunk.
uint32_t pitch_for(uint32_t TW) { return (32u * TW + 15u + 15u) / 16u * 16u; }

// Slot of local cell lx inside its row word (the pack's bit order).
inline uint32_t lane_of(uint32_t lx) { return 8u * (lx & 3u) + (lx >> 2); }

// Tile rows that share one slot word: 32 / TW for the power-of-two widths 8 and
// 16 when TH is a multiple of it (such rows start at multiples of TW, so the
// kernel reads and writes them as whole aligned words), else 1.
uint32_t rows_per_word(uint32_t TW, uint32_t TH) {
  if ((TW == 8 || TW == 16) && TH % (32 / TW) == 0) return 32 / TW;
  return 1;
}

// Slot word index of local cell c of a TW-wide tile: its slot row times 32
// plus its lane (rpw tile rows per slot row, or two slot rows per tile row
// when wpr = 2).
uint32_t tile_slot_of(uint32_t c, uint32_t TW, uint32_t rpw, uint32_t wpr) {
  if (wpr == 2) return (c / TW * 2u + c % TW / 32u) * 32u + lane_of(c % TW % 32u);
  return (c / TW / rpw) * 32u + lane_of((c / TW % rpw) * TW + c % TW);
}

// Local lambda of the level-L fractal: compact (lx, ly) -> expanded (X, Y).
void local_lambda(const FracDev &f, uint32_t L, uint32_t lx, uint32_t ly, uint32_t &X,
                  uint32_t &Y) {
  X = Y = 0;
  uint32_t scale = 1;
  for (uint32_t mu = 1; mu <= L; ++mu) {
    uint32_t &src = (mu & 1u) ? lx : ly;
    uint32_t beta = src % f.k;
    src /= f.k;
    X += f.taux[beta] * scale;
    Y += f.tauy[beta] * scale;
    scale *= f.s;
  }
}

}  // namespace
}  // namespace sq

using namespace sq;


TiledDev sq_tiled_dev(const FracDev &f, const Rule &rule, const TileSpec &sp,
                      const uint16_t *refs, const uint32_t *halo_off, const uint8_t *halo_dir,
                      const uint32_t *adj, int *status) {
  TiledDev d;
  memset(&d, 0, sizeof(d));
  d.W = f.W;
  d.total = f.cells;
  d.rule = rule;
  d.L = sp.L;
  d.TW = sp.TW;
  d.TH = sp.TH;
  d.cells = sp.cells;
  d.slots = sp.slots;
  d.nhalo = sp.nhalo;
  d.nwin = (3u + sp.TW + 3u) / 4u;
  d.valid = 0;
  for (uint32_t lx = 0; lx < sp.rpw * sp.TW && lx < 32; ++lx) d.valid |= 1u << lane_of(lx);
  d.rpw = sp.rpw;
  d.dir_mask = sp.dir_mask;
  d.ndirs = sp.ndirs;
  for (int i = 0; i < 9; ++i) d.dir_list[i] = sp.dir_list[i];
  for (int i = 0; i < 10; ++i) d.halo_start[i] = sp.halo_start[i];
  d.tiles_x = sp.tiles_x;
  d.tiles_y = sp.tiles_y;
  d.tiles = (uint64_t)sp.tiles_x * sp.tiles_y;
  d.groups_per_band = sp.groups_per_band;
  d.pitch = sp.pitch;
  d.groups = sp.groups;
  d.div_tw = make_fastdiv(sp.TW);
  d.div_gpb = make_fastdiv(sp.groups_per_band);
  d.div_tiles_x = make_fastdiv(sp.tiles_x);
  d.refs = refs;
  d.halo_off = halo_off;
  d.halo_dir = halo_dir;
  d.adj = adj;
  d.status = status;
  d.wait_ns = kDefaultWaitNs;
  d.fault = 0;
  for (int i = 0; i <= kMaxPasses; ++i) d.ring_end[i] = sp.ring_end[i];
  for (int k = 0; k < kMaxPasses - 1; ++k)
    for (int i = 0; i < 10; ++i) d.ring_start[k][i] = sp.ring_start[k][i];
  d.nchunks = sp.nchunks;
  for (int i = 0; i < 10; ++i) d.chunk_start[i] = sp.chunk_start[i];
  d.rec_words = sp.rec_words;
  for (int i = 0; i < 10; ++i) d.rec_seg[i] = sp.rec_seg[i];
  d.rec_nexp = sp.rec_nexp;
  d.rec[0] = d.rec[1] = nullptr;
  d.mode = 0;
  return d;
}

void sq_tiled_free(TiledProgram *p) {
  if (!p) return;
  cudaFree(p->d_refs);
  cudaFree(p->d_halo_off);
  cudaFree(p->d_halo_dir);
  cudaFree(p->d_adj);
  cudaFree(p->d_rec[0]);
  cudaFree(p->d_rec[1]);
  delete p;
}

uint32_t count_halo(const FracDev &f, uint32_t L);

bool sq_tiled_level_fits(const squeeze_handle *h, uint32_t level) {
  const uint64_t TW = ipow(h->f.k, (level + 1) / 2), TH = ipow(h->f.k, level / 2);
  const uint64_t side = ipow(h->f.s, level);
  if (level < 1 || level > h->f.r || (TW > 32 && TW != 64) || TH > 4096 || side * side > (1ull << 24))
    return false;
  // the program's shared memory must fit one CTA
  const uint32_t slots = (uint32_t)TH * (TW == 64 ? 64u : 32u);
  return smem_for(slots, count_halo(h->f, level), (uint32_t)TH, pitch_for((uint32_t)TW)) <=
         kTiledSmemLimit;
}

// Largest level whose tile rows fit one 32-bit word and whose shared memory
// stays within kTiledSmemCap (so that several CTAs share an SM).
int sq_tiled_default_level(const squeeze_handle *h) { return sq_tiled_default_level_for(h->f); }

// Number of distinct halo words of the one-step level-L program (the first
// ring), which decides the tile level; the handle then builds as many passes
// as fit the same shared-memory budget.
uint32_t count_halo(const FracDev &f, uint32_t L) {
  TileBuildSizes z;
  sq_tile_build_sizes(f, L, z);
  std::vector<int32_t> inv(z.box);
  std::vector<uint32_t> X(z.cells), Y(z.cells), refs((z.slots + z.halo) * 8), order(z.halo),
      rank(z.halo);
  std::vector<uint64_t> keys(z.halo), sorted(z.halo);
  std::vector<uint16_t> refs16((z.slots + z.halo) * 8);
  std::vector<uint32_t> halo_off(z.halo);
  std::vector<uint8_t> halo_dir(z.halo);
  TileBuild B = {inv.data(), X.data(), Y.data(), refs.data(), keys.data(), sorted.data(),
                 order.data(), rank.data(), refs16.data(), halo_off.data(), halo_dir.data(),
                 z.box, z.cells, z.slots, z.halo, 1u};
  TileSpec sp;
  if (sq_tile_build(f, L, B, sp) != SQUEEZE_OK) return 0xFFFFu;   // too large to build
  return sp.nhalo;
}

size_t sq_tiled_smem_cap() { return kTiledSmemCap; }

int sq_tiled_default_level_for(const FracDev &f) {
  int best = -1;
  for (uint32_t L = 1; L <= f.r; ++L) {
    uint64_t TW = ipow(f.k, (L + 1) / 2), TH = ipow(f.k, L / 2), side = ipow(f.s, L);
    if ((TW > 32 && TW != 64) || TH > 4096 || side * side > (1ull << 24)) break;
    uint32_t slots = (uint32_t)TH * (TW == 64 ? 64 : 32);
    size_t sm = smem_for(slots, count_halo(f, L), (uint32_t)TH, pitch_for((uint32_t)TW));
    if (sm <= kTiledSmemCap) best = (int)L;
  }
  return best;
}

void sq_tile_build_sizes(const FracDev &f, uint32_t L, TileBuildSizes &z) {
  uint64_t TW = ipow(f.k, (L + 1) / 2), TH = ipow(f.k, L / 2), side = ipow(f.s, L);
  z.box = side * side;
  z.cells = TW * TH;
  z.slots = TH * (TW == 64 ? 64 : 32);
  z.halo = 8 * z.cells;
}

// The halo's chunk table for 64-wide rows.  A tile starts on a multiple of 64
// bytes and W is a multiple of 64, so the halo cell at offset o of an adjacent
// tile lies in the 16-byte chunk o & ~15 of it, at byte o & 15.  Per
// direction: its distinct chunks in increasing order, and per chunk its cells
// in increasing halo-word order (so ring by ring).  out = chunk offsets |
// nchunks + 1 cell ranges | nhalo cells (halo word | byte << 16).
static void build_chunks(uint32_t nhalo, const uint32_t *halo_off, const uint8_t *halo_dir,
                         TileSpec &sp, uint32_t *out) {
  std::vector<uint32_t> coff, cstart, cells;
  for (uint32_t j = 0; j <= sp.ndirs; ++j) {
    sp.chunk_start[j] = (uint32_t)coff.size();
    if (j == sp.ndirs) break;
    std::vector<uint32_t> mine;   // chunk offsets of direction j
    for (uint32_t h = 0; h < nhalo; ++h)
      if (halo_dir[h] == j) mine.push_back(halo_off[h] & ~15u);
    std::sort(mine.begin(), mine.end());
    mine.erase(std::unique(mine.begin(), mine.end()), mine.end());
    for (uint32_t c : mine) {
      coff.push_back(c);
      cstart.push_back((uint32_t)cells.size());
      for (uint32_t h = 0; h < nhalo; ++h)
        if (halo_dir[h] == j && (halo_off[h] & ~15u) == c)
          cells.push_back(h | ((halo_off[h] & 15u) << 16));
    }
  }
  for (uint32_t j = sp.ndirs + 1; j < 10; ++j) sp.chunk_start[j] = (uint32_t)coff.size();
  cstart.push_back((uint32_t)cells.size());
  sp.nchunks = (uint32_t)coff.size();
  uint32_t *o = out;
  for (uint32_t v : coff) *o++ = v;
  for (uint32_t v : cstart) *o++ = v;
  for (uint32_t v : cells) *o++ = v;
}

// The border-record tables.  Segment j of a tile's record holds, in
// halo-word order, the states of the tile's cells that the tile adjacent to it
// in direction j reads as its direction-j halo (the halo words h with
// halo_dir[h] == j, all rings): ceil(n_j / 32) words from rec_seg[j].  The
// cells a record names, its exported cells, are numbered e = 0 .. rec_nexp-1
// in order of first use; a launch keeps the final-step words of those slots
// only.  out = record bits (32 per record word: e | halo word << 16, or ~0 to
// pad a segment's last word) | the slot of each exported cell | per slot its
// export number or 0xFFFF (16 bits each, two per word).
static void build_records(uint64_t W, uint32_t TW, uint32_t rpw, uint32_t wpr, uint32_t slots,
                          uint32_t nhalo, const uint32_t *halo_off, const uint8_t *halo_dir,
                          TileSpec &sp, uint32_t *out) {
  std::vector<uint32_t> exp_of(slots, 0xFFFFu), exp_slot;
  uint32_t words = 0;
  for (uint32_t j = 0; j < sp.ndirs; ++j) {
    sp.rec_seg[j] = words;
    uint32_t n = 0;
    for (uint32_t h = 0; h < nhalo; ++h)
      if (halo_dir[h] == j) {
        const uint32_t lc = (uint32_t)(halo_off[h] / W) * TW + (uint32_t)(halo_off[h] % W);
        const uint32_t s = tile_slot_of(lc, TW, rpw, wpr);
        if (exp_of[s] == 0xFFFFu) {
          exp_of[s] = (uint32_t)exp_slot.size();
          exp_slot.push_back(s);
        }
        out[32u * words + n++] = exp_of[s] | (h << 16);
      }
    const uint32_t used = (n + 31u) / 32u;
    for (uint32_t i = n; i < 32u * used; ++i) out[32u * words + i] = 0xFFFFFFFFu;
    words += used;
  }
  for (uint32_t j = sp.ndirs; j < 10; ++j) sp.rec_seg[j] = words;
  sp.rec_words = words;
  sp.rec_nexp = (uint32_t)exp_slot.size();
  uint32_t *o = out + 32u * words;
  for (uint32_t s : exp_slot) *o++ = s;
  for (uint32_t s = 0; s < slots; s += 2)
    *o++ = exp_of[s] | ((s + 1 < slots ? exp_of[s + 1] : 0xFFFFu) << 16);
}

// Host construction of the level-L neighbour program (see the file comment):
// local lambda and its inverse over the level-L box, 8 references per slot
// (local slot, halo word or the zero word), halo words sorted by direction.
//
// With B.passes = P > 1 (2, 4 or 8) the program also serves launches that run up to P
// steps: ring 1 of halo cells (the cells of adjacent blocks that neighbour the
// tile's cells), ring 2 (their neighbours outside the tile and ring 1), ...,
// ring P are built, and rings 1 .. P-1 get references of their own, so that a
// launch can advance the tile and rings 1..P-t by step t in shared memory
// and the tile alone by step P.  Halo words are numbered ring by ring, each
// ring sorted by direction: ring k is [ring_end[k-1], ring_end[k]); a launch
// of fewer steps reads the first rings only.  Word array: slots | rings |
// zero word | 9 words of per-direction "adjacent tile exists" masks.
int sq_tile_build(const FracDev &f, uint32_t L, const TileBuild &B, TileSpec &sp) {
  if (L == 0 || L > f.r) return SQUEEZE_ERR_UNSUPPORTED;
  uint64_t TW64 = ipow(f.k, (L + 1) / 2), TH64 = ipow(f.k, L / 2);
  // a tile row must fit one slot word, or be exactly two (width 64)
  if ((TW64 > 32 && TW64 != 64) || TH64 > 4096) return SQUEEZE_ERR_UNSUPPORTED;
  uint32_t TW = (uint32_t)TW64, TH = (uint32_t)TH64;
  // Narrow power-of-two rows share a slot word: 32 / TW tile rows per word;
  // 64-wide rows take two words (left and right half).
  const uint32_t rpw = rows_per_word(TW, TH), wpr = TW == 64 ? 2u : 1u;
  uint32_t cells = TW * TH, side = (uint32_t)ipow(f.s, L), slots = TH * wpr / rpw * 32;
  if ((uint64_t)side * side > B.box_cap || cells > B.cells_cap || slots > B.slots_cap)
    return SQUEEZE_ERR_UNSUPPORTED;
  if ((uint64_t)TH * f.W > 0xFFFFFFFFull) return SQUEEZE_ERR_UNSUPPORTED;

  int32_t *inv = B.inv;
  for (uint64_t i = 0; i < (uint64_t)side * side; ++i) inv[i] = -1;
  for (uint32_t c = 0; c < cells; ++c) {
    local_lambda(f, L, c % TW, c / TW, B.X[c], B.Y[c]);
    inv[(size_t)B.Y[c] * side + B.X[c]] = (int32_t)c;
  }
  auto slot_of = [&](uint32_t c) { return tile_slot_of(c, TW, rpw, wpr); };
  const uint32_t kNone = 0xFFFFFFFFu, kFull = 0xFFFFFFFEu, kFar = 0xFFFFFFFDu;
  uint32_t *refs = B.refs;
  uint32_t nhalo = 0;
  // Reference to the point (qx, qy) of the expanded plane, relative to the
  // tile's own level-L box: a local slot, slots + a halo index (a halo cell is
  // registered on first sight), kNone for a hole, kFull when the halo list
  // is full, or kFar for a point beyond the 8 adjacent boxes (a ring deeper
  // than the box is wide).
  auto ref_of = [&](int64_t qx, int64_t qy) -> uint32_t {
    if (qx < -(int64_t)side || qy < -(int64_t)side || qx >= 2 * (int64_t)side ||
        qy >= 2 * (int64_t)side)
      return kFar;
    const int bx = qx < 0 ? -1 : (qx >= side ? 1 : 0), by = qy < 0 ? -1 : (qy >= side ? 1 : 0);
    const int64_t lxp = qx - (int64_t)bx * side, lyp = qy - (int64_t)by * side;
    const int32_t target = inv[(size_t)lyp * side + lxp];
    if (target < 0) return kNone;
    if (bx == 0 && by == 0) return slot_of((uint32_t)target);
    // (direction << 32) | local cell in the adjacent block
    const uint64_t key = ((uint64_t)((by + 1) * 3 + (bx + 1)) << 32) | (uint32_t)target;
    uint32_t i = 0;
    while (i < nhalo && B.halo_key[i] != key) ++i;
    if (i == nhalo) {
      if (nhalo == B.halo_cap) return kFull;
      B.halo_key[nhalo++] = key;
    }
    return slots + i;
  };
  // The 8 references of the cell at (px, py); an offset outside the
  // neighbourhood refers to the zero word, like a hole.
  auto fill_refs = [&](int64_t px, int64_t py, uint32_t *row) -> bool {
    int k8 = 0;
    for (int d = 0; d < 9; ++d) {
      if (d == 4) continue;
      uint32_t ref = kNone;
      if ((f.nbhd >> d) & 1u) ref = ref_of(px + d % 3 - 1, py + d / 3 - 1);
      if (ref == kFull || ref == kFar) return false;
      row[k8++] = ref;
    }
    return true;
  };
  for (size_t i = 0; i < (size_t)slots * 8; ++i) refs[i] = kNone;   // slots without a cell
  for (uint32_t c = 0; c < cells; ++c)
    if (!fill_refs(B.X[c], B.Y[c], refs + (size_t)slot_of(c) * 8)) return SQUEEZE_ERR_UNSUPPORTED;
  const uint32_t P = B.passes == 8 ? 8u : (B.passes == 4 ? 4u : (B.passes == 2 ? 2u : 1u));
  uint32_t ends[kMaxPasses + 1] = {0, nhalo};
  for (uint32_t k = 1; k < P; ++k) {
    // References of ring k (its neighbours outside the tile and rings 1..k
    // make up ring k + 1).
    for (uint32_t i = ends[k - 1]; i < ends[k]; ++i) {
      const uint64_t key = B.halo_key[i];
      const uint32_t d = (uint32_t)(key >> 32), t = (uint32_t)key;
      const int64_t px = (int64_t)B.X[t] + ((int)(d % 3) - 1) * (int64_t)side;
      const int64_t py = (int64_t)B.Y[t] + ((int)(d / 3) - 1) * (int64_t)side;
      if (!fill_refs(px, py, refs + (size_t)(slots + i) * 8)) return SQUEEZE_ERR_UNSUPPORTED;
    }
    ends[k + 1] = nhalo;
  }
  for (uint32_t k = P + 1; k <= (uint32_t)kMaxPasses; ++k) ends[k] = nhalo;
  // Sort each ring by direction (then local cell) and renumber within it.
  for (uint32_t i = 0; i < nhalo; ++i) B.order[i] = i;
  auto by_key = [&](uint32_t x, uint32_t y) { return B.halo_key[x] < B.halo_key[y]; };
  for (uint32_t k = 1; k <= P; ++k) std::sort(B.order + ends[k - 1], B.order + ends[k], by_key);
  for (uint32_t i = 0; i < nhalo; ++i) B.rank[B.order[i]] = i;
  uint64_t *sorted = B.halo_sorted;
  for (uint32_t i = 0; i < nhalo; ++i) sorted[B.rank[i]] = B.halo_key[i];
  // References are byte offsets into the word array, 8 per slot (16 bytes);
  // rows of the first ring follow the slots' rows in their sorted order.
  const uint32_t zero = slots + nhalo;
  if (((uint64_t)zero + 1 + 9) * 4 > 0xFFFFu) return SQUEEZE_ERR_UNSUPPORTED;
  auto enc = [&](uint32_t r) -> uint16_t {
    if (r == kNone) return (uint16_t)(4u * zero);
    return (uint16_t)(4u * (r < slots ? r : slots + B.rank[r - slots]));
  };
  for (uint32_t c = 0; c < slots; ++c)
    for (uint32_t d = 0; d < 8; ++d) B.refs16[(size_t)c * 8 + d] = enc(refs[(size_t)c * 8 + d]);
  for (uint32_t i = 0; i < ends[P - 1]; ++i)   // rings with references, in sorted order
    for (uint32_t d = 0; d < 8; ++d)
      B.refs16[(size_t)(slots + B.rank[i]) * 8 + d] = enc(refs[(size_t)(slots + i) * 8 + d]);
  uint32_t dir_mask = 0;
  for (uint32_t i = 0; i < nhalo; ++i) dir_mask |= 1u << (uint32_t)(sorted[i] >> 32);
  memset(&sp, 0, sizeof(sp));
  uint8_t dir_index[9] = {0};
  for (uint32_t d = 0; d < 9; ++d)
    if ((dir_mask >> d) & 1u) {
      dir_index[d] = (uint8_t)sp.ndirs;
      sp.dir_list[sp.ndirs++] = (uint8_t)d;
    }
  // per ring and direction: the range of its words ([ends[k-1], ends[k]) sorted by direction)
  uint32_t *starts[kMaxPasses];
  starts[0] = sp.halo_start;
  for (int k = 1; k < kMaxPasses; ++k) starts[k] = sp.ring_start[k - 1];
  for (uint32_t k = 0; k < (uint32_t)kMaxPasses; ++k)
    for (uint32_t j = 0; j < 10; ++j) starts[k][j] = ends[k];
  for (uint32_t i = 0; i < nhalo; ++i) {
    uint32_t d = (uint32_t)(sorted[i] >> 32), lc = (uint32_t)sorted[i];
    B.halo_dir[i] = dir_index[d];
    B.halo_off[i] = (lc / TW) * f.W + lc % TW;
    uint32_t k = 0;
    while (i >= ends[k + 1]) ++k;
    starts[k][dir_index[d] + 1] = i + 1;
  }
  for (uint32_t k = 0; k < (uint32_t)kMaxPasses; ++k)
    for (uint32_t j = 1; j <= 9; ++j)
      if (starts[k][j] < starts[k][j - 1]) starts[k][j] = starts[k][j - 1];
  sp.L = L;
  sp.TW = TW;
  sp.TH = TH;
  sp.rpw = rpw;
  sp.cells = cells;
  sp.slots = slots;
  sp.nhalo = nhalo;
  sp.passes = P;
  for (uint32_t k = 0; k <= (uint32_t)kMaxPasses; ++k) sp.ring_end[k] = ends[k];
  sp.dir_mask = dir_mask;
  sp.tiles_x = f.W / TW;
  sp.tiles_y = f.H / TH;
  sp.groups_per_band = (sp.tiles_x + 31) / 32;
  sp.groups = (uint64_t)sp.groups_per_band * sp.tiles_y;
  sp.pitch = pitch_for(TW);
  if (B.chunks && nhalo) {
    if (TW == 64) build_chunks(nhalo, B.halo_off, B.halo_dir, sp, B.chunks);
    build_records(f.W, TW, rpw, wpr, slots, nhalo, B.halo_off, B.halo_dir, sp,
                  B.chunks + chunk_table_words(sp));
  }
  sp.smem = sq_tile_layout_of(sp).smem;
  if (sp.groups >= (1ull << 32) || sp.smem > kTiledSmemLimit) return SQUEEZE_ERR_UNSUPPORTED;
  // Whole warps, one tile row per warp per pass: pick 6..12 warps to balance TH rows.
  // Shared slot words: two slot rows per warp, 4..8 warps.
  int best_w = 8;
  if (wpr > 1) {
    // two tile rows (four slot rows) per warp and pass
    best_w = (int)((TH + 1) / 2) < 4 ? 4 : ((int)((TH + 1) / 2) > 8 ? 8 : (int)((TH + 1) / 2));
  } else if (rpw > 1) {
    const int vr = (int)(TH / rpw);
    best_w = (vr + 1) / 2 < 4 ? 4 : ((vr + 1) / 2 > 8 ? 8 : (vr + 1) / 2);
  } else {
    for (int w = 12; w >= 6; --w)
      if ((TH + w - 1) / w * w - TH < (TH + best_w - 1) / best_w * best_w - TH) best_w = w;
  }
  sp.threads = 32 * best_w;
  return SQUEEZE_OK;
}

// Shared-memory opt-in and the persistent grid (CTAs per SM x SMs), per
// instantiation (the generic-rule kernel may fit fewer CTAs per SM).
int sq_tile_launch_config(TileSpec &sp, int device) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return sq_cuda_fail(e);
  for (uint32_t steps = 1; steps <= sp.passes; steps *= 2)
    for (int life = 0; life < 2; ++life) {
      const void *fn = tiled_kernel_for(life != 0, sp.TW, sp.rpw, steps);
      e = sq_allow_smem(fn, sp.smem);
      int n = 0;
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, sp.threads, sp.smem);
      if (e != cudaSuccess) return sq_cuda_fail(e);
      if (n < 1) return SQUEEZE_ERR_UNSUPPORTED;
      const uint64_t grid = (uint64_t)n * sms;
      sp.grid[steps_index(steps)][life] = (int)(grid < sp.groups ? grid : sp.groups);
      sp.occ[steps_index(steps)][life] = n;
    }
  return SQUEEZE_OK;
}

int sq_tile_build_adjacency(const FracDev &f, const TiledDev &d, uint32_t *adj, cudaStream_t st) {
  uint64_t n = (uint64_t)d.ndirs * d.tiles;
  if (!n) return SQUEEZE_OK;
  build_adjacency_kernel<<<grid_for(n, 256), 256, 0, st>>>(f, d, adj);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_tile_launch(const TiledDev &d, const TileSpec &sp, const uint8_t *in, uint8_t *out,
                   uint32_t steps, cudaStream_t st) {
  if (((uintptr_t)in | (uintptr_t)out) & 15u) return SQUEEZE_ERR_INVALID_ARG;
  if ((steps != 1 && steps != 2 && steps != 4 && steps != 8) || steps > sp.passes)
    return SQUEEZE_ERR_INVALID_ARG;
  if (sp.TW == 64 && sp.nhalo && !sp.nchunks) return SQUEEZE_ERR_INVALID_ARG;  // no chunk table
  if ((d.rec[0] || d.rec[1]) && !sp.rec_words) return SQUEEZE_ERR_INVALID_ARG;
  // several steps per launch read the halo from the input's records only
  if (steps > 1 && sp.rec_words && (d.mode != 0 || !d.rec[0])) return SQUEEZE_ERR_INVALID_ARG;
  bool life = d.rule.birth == (1u << 3) && d.rule.survive == ((1u << 2) | (1u << 3));
  TiledDev dd = d;
  TileLayout lay = sq_tile_layout_of(sp);
  void *args[] = {&dd, &lay, &in, &out};
  const int grid = sp.grid[steps_index(steps)][life ? 1 : 0];
  SQ_CUDA(cudaLaunchKernel(tiled_kernel_for(life, sp.TW, sp.rpw, steps), dim3(grid),
                           dim3(sp.threads), args, sp.smem, st));
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_tiled_prepare(squeeze_handle *h) {
  if (h->tiled) return SQUEEZE_OK;
  const FracDev &f = h->f;
  uint32_t L = h->tiled_level ? h->tiled_level : (uint32_t)sq_tiled_default_level(h);
  if ((int)L <= 0 || L > f.r) return SQUEEZE_ERR_UNSUPPORTED;
  if (!sq_tiled_level_fits(h, L)) return SQUEEZE_ERR_UNSUPPORTED;
  TileBuildSizes z;
  sq_tile_build_sizes(f, L, z);
  if (z.box > (1ull << 28)) return SQUEEZE_ERR_UNSUPPORTED;
  std::vector<int32_t> inv(z.box);
  std::vector<uint32_t> X(z.cells), Y(z.cells), refs((z.slots + z.halo) * 8), order(z.halo),
      rank(z.halo);
  std::vector<uint64_t> keys(z.halo), sorted(z.halo);
  std::vector<uint16_t> refs16((z.slots + z.halo) * 8);
  std::vector<uint32_t> halo_off(z.halo), chunks(5 * z.halo + z.slots / 2 + 300);
  std::vector<uint8_t> halo_dir(z.halo);
  TileBuild B = {inv.data(), X.data(), Y.data(), refs.data(), keys.data(), sorted.data(),
                 order.data(), rank.data(), refs16.data(), halo_off.data(), halo_dir.data(),
                 z.box, z.cells, z.slots, z.halo, kTiledPasses, chunks.data()};
  TiledProgram *p = new TiledProgram;
  memset(p, 0, sizeof(*p));
  // Steps per launch: by default the most (8, 4, 2) whose program builds and
  // whose kernel keeps the CTAs per SM of the one-step kernel, or 3 if that
  // has more (its shared memory grows with the halo rings; with the halo read
  // from border records eight steps at 3 CTAs per SM beat four at 4 by 30 %
  // for the triangle and Vicsek, and tie for the carpet); with
  // squeeze_set_max_steps_per_launch the most up to that limit that build.
  int rc = SQUEEZE_ERR_UNSUPPORTED, occ1 = 0;
  {
    B.passes = 1;
    TileSpec one;
    rc = sq_tile_build(f, L, B, one);
    if (rc == SQUEEZE_OK) rc = sq_tile_launch_config(one, h->device);
    if (rc == SQUEEZE_OK) occ1 = one.occ[0][1] < 3 ? one.occ[0][1] : 3;
  }
  for (uint32_t passes = h->max_passes ? h->max_passes : kTiledPasses; rc == SQUEEZE_OK; passes /= 2) {
    B.passes = passes;
    rc = sq_tile_build(f, L, B, p->spec);
    if (rc == SQUEEZE_OK) rc = sq_tile_launch_config(p->spec, h->device);
    if (passes == 1) break;
    if (rc == SQUEEZE_OK &&
        (h->max_passes || p->spec.occ[steps_index(p->spec.passes)][1] >= occ1))
      break;
    rc = SQUEEZE_OK;   // try fewer steps per launch
  }
  if (rc != SQUEEZE_OK) {
    delete p;
    return rc;
  }
  const TileSpec &sp = p->spec;
  uint32_t nhalo = sp.nhalo, tw = sq_tile_table_words(sp);
  // slots, then the rings with references (1 .. passes - 1)
  const size_t ref_bytes = (size_t)(sp.slots + sp.ring_end[sp.passes - 1]) * 16;
  cudaError_t e = cudaMalloc(&p->d_refs, ref_bytes);
  // halo offsets, then the chunk table (if any)
  if (e == cudaSuccess) e = cudaMalloc(&p->d_halo_off, ((size_t)nhalo + tw + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_halo_dir, (nhalo ? nhalo : 1));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_refs, refs16.data(), ref_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nhalo)
    e = cudaMemcpy(p->d_halo_off, halo_off.data(), nhalo * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && tw)
    e = cudaMemcpy(p->d_halo_off + nhalo, chunks.data(), (size_t)tw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nhalo)
    e = cudaMemcpy(p->d_halo_dir, halo_dir.data(), nhalo, cudaMemcpyHostToDevice);
  uint64_t tiles = (uint64_t)sp.tiles_x * sp.tiles_y;
  if (e == cudaSuccess && sp.ndirs) e = cudaMalloc(&p->d_adj, (size_t)sp.ndirs * tiles * 4);
  if (e != cudaSuccess) {
    sq_tiled_free(p);
    return sq_cuda_fail(e);
  }
  TiledDev d = sq_tiled_dev(f, h->rule, sp, p->d_refs, p->d_halo_off, p->d_halo_dir, p->d_adj,
                            h->d_status);
  rc = sq_tile_build_adjacency(f, d, p->d_adj, 0);
  if (rc == SQUEEZE_OK) {
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = sq_cuda_fail(e);
  }
  if (rc != SQUEEZE_OK) {
    sq_tiled_free(p);
    return rc;
  }
  h->tiled = p;
  h->tiled_level = L;
  return SQUEEZE_OK;
}

int sq_launch_step_tiled(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                         uint32_t steps, bool last, cudaStream_t st) {
  TiledProgram *p = h->tiled;
  if (!p) return SQUEEZE_ERR_INVALID_ARG;
  TiledDev d = sq_tiled_dev(h->f, h->rule, p->spec, p->d_refs, p->d_halo_off, p->d_halo_dir,
                            p->d_adj, h->d_status);
  if (h->wait_ns) d.wait_ns = h->wait_ns;
  d.fault = h->fault;
  if (p->spec.rec_words) {   // records of the input (else gathered), and of the output
    d.rec[0] = p->rec_live ? p->d_rec[p->rec_cur] : nullptr;
    d.rec[1] = last ? nullptr : p->d_rec[p->rec_cur ^ 1];
  }
  const int rc = sq_tile_launch(d, p->spec, in, out, steps, st);
  if (rc == SQUEEZE_OK) {
    p->rec_cur ^= 1;
    p->rec_live = p->spec.rec_words != 0 && !last;
  }
  return rc;
}

// Before the launches of a squeeze_step call: the border records of its input
// when a launch of several steps will read them (one records-only launch);
// one-step launches gather the halo from the state instead (and write the
// records of their output, which later launches of the call read).
int sq_tiled_begin(const squeeze_handle *h, const uint8_t *in, bool multi, cudaStream_t st,
                   int *launches) {
  TiledProgram *p = h->tiled;
  *launches = 0;
  if (!p || !p->spec.rec_words) return SQUEEZE_OK;
  // the record buffers, on the first squeeze_step (a batch keeps its own)
  const size_t rec_bytes = (size_t)p->spec.rec_words * p->spec.tiles_x * p->spec.tiles_y * 4;
  for (int i = 0; i < 2; ++i)
    if (!p->d_rec[i]) SQ_CUDA(cudaMalloc(&p->d_rec[i], rec_bytes));
  p->rec_cur = 0;
  p->rec_live = false;
  if (!multi) return SQUEEZE_OK;
  TiledDev d = sq_tiled_dev(h->f, h->rule, p->spec, p->d_refs, p->d_halo_off, p->d_halo_dir,
                            p->d_adj, h->d_status);
  if (h->wait_ns) d.wait_ns = h->wait_ns;
  d.fault = h->fault;
  d.rec[1] = p->d_rec[0];
  d.mode = 1;
  *launches = 1;
  const int rc = sq_tile_launch(d, p->spec, in, const_cast<uint8_t *>(in), 1, st);
  p->rec_live = rc == SQUEEZE_OK;
  return rc;
}

uint32_t sq_tiled_passes(const squeeze_handle *h) { return h->tiled ? h->tiled->spec.passes : 1u; }

void sq_launch_plan(uint64_t n, uint32_t passes, uint64_t *counts) {
  uint64_t left = n;
  for (int i = 3; i >= 0; --i) {
    const uint64_t size = 1ull << i;
    counts[i] = size <= passes ? left / size : 0;
    left -= counts[i] * size;
  }
  // Launches must have the parity of n (= that of the one-step launches):
  // split the smallest multi-step launch in two when they do not.
  if ((counts[1] + counts[2] + counts[3]) & 1u) {
    for (int i = 1; i <= 3; ++i)
      if (counts[i]) {
        counts[i] -= 1;
        counts[i - 1] += 2;
        break;
      }
  }
}

int sq_tiled_describe(const squeeze_handle *h, TiledDev *d, TileSpec *sp) {
  const TiledProgram *p = h->tiled;
  if (!p) return SQUEEZE_ERR_INVALID_ARG;
  *d = sq_tiled_dev(h->f, h->rule, p->spec, p->d_refs, p->d_halo_off, p->d_halo_dir, p->d_adj,
                    h->d_status);
  if (h->wait_ns) d->wait_ns = h->wait_ns;
  d->fault = h->fault;
  *sp = p->spec;
  return SQUEEZE_OK;
}

int sq_tile_kind(const TileSpec &sp) {
  if (sp.rpw == 4) return 8;
  if (sp.rpw == 2) return 16;
  if (sp.TW == 27 || sp.TW == 25 || sp.TW == 64) return (int)sp.TW;
  return 0;
}
