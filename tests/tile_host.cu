// tile_host.cu -- test support: the host-built neighbour program of the tiled
// step (step_tiled.cu), exported so that a CPU emulation of one step can run
// on it and be compared with the oracle.  No CUDA calls are made.
#include "step_tiled.cu"

int sq_cuda_fail(cudaError_t) { return SQUEEZE_ERR_CUDA; }   // never reached: no CUDA calls here
cudaError_t sq_allow_smem(const void *, size_t) { return cudaSuccess; }
void sq_set_error_text(const char *) {}

namespace {

// The kernel-side descriptor of a level-r fractal (the fields the builder reads).
bool fill(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t nbhd, FracDev &f) {
  memset(&f, 0, sizeof(f));
  f.s = s;
  f.k = k;
  f.r = r;
  f.n = (uint32_t)ipow(s, r);
  f.W = (uint32_t)ipow(k, (r + 1) / 2);
  f.H = (uint32_t)ipow(k, r / 2);
  f.cells = (uint64_t)f.W * f.H;
  f.divk = make_fastdiv(k);
  f.divs = make_fastdiv(s);
  f.divW = make_fastdiv(f.W);
  f.nbhd = nbhd;
  memset(f.hnu, kHole, sizeof(f.hnu));
  for (uint32_t b = 0; b < k; ++b) {
    if (off[2 * b] >= s || off[2 * b + 1] >= s) return false;
    f.taux[b] = off[2 * b];
    f.tauy[b] = off[2 * b + 1];
    f.hnu[off[2 * b + 1] * s + off[2 * b]] = (uint8_t)b;
  }
  return true;
}

}  // namespace

extern "C" {

// Capacities of the program arrays: cells, slots, halo entries.
int tile_sizes(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L, uint64_t *out) {
  FracDev f;
  if (!fill(s, k, off, r, kMoore, f)) return SQUEEZE_ERR_INVALID_ARG;
  TileBuildSizes z;
  sq_tile_build_sizes(f, L, z);
  out[0] = z.cells;
  out[1] = z.slots;
  out[2] = z.halo;
  return SQUEEZE_OK;
}

// The level-L program for up to `passes` steps per launch (1, 2, 4 or 8): info
// = (TW, TH, rpw, wpr, cells, slots, nhalo, ndirs, passes, ring_end[0..8]); per
// local cell its slot and local expanded position; per slot (and per halo word
// of rings 1 .. passes-1 after them) 8 byte offsets into the word array
// (slots, then halo words ring by ring, then a zero word); per halo word its
// offset from the adjacent tile's base and its direction index into
// dir_list.  refs16 needs (slots + halo) * 8 entries.
int tile_program(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L,
                 uint32_t nbhd, uint32_t passes, uint32_t *info, uint32_t *slot, uint32_t *X,
                 uint32_t *Y, uint16_t *refs16, uint32_t *halo_off, uint8_t *halo_dir,
                 uint8_t *dir_list) {
  FracDev f;
  if (!fill(s, k, off, r, nbhd, f)) return SQUEEZE_ERR_INVALID_ARG;
  TileBuildSizes z;
  sq_tile_build_sizes(f, L, z);
  std::vector<int32_t> inv(z.box);
  std::vector<uint32_t> vX(z.cells), vY(z.cells), refs((z.slots + z.halo) * 8), order(z.halo),
      rank(z.halo);
  std::vector<uint64_t> key(z.halo), sorted(z.halo);
  TileBuild B;
  B.inv = inv.data();
  B.X = vX.data();
  B.Y = vY.data();
  B.refs = refs.data();
  B.halo_key = key.data();
  B.halo_sorted = sorted.data();
  B.order = order.data();
  B.rank = rank.data();
  B.refs16 = refs16;
  B.halo_off = halo_off;
  B.halo_dir = halo_dir;
  B.box_cap = z.box;
  B.cells_cap = z.cells;
  B.slots_cap = z.slots;
  B.halo_cap = z.halo;
  B.passes = passes;
  std::vector<uint32_t> chunks(5 * z.halo + z.slots / 2 + 300);
  B.chunks = chunks.data();
  TileSpec sp;
  const int rc = sq_tile_build(f, L, B, sp);
  if (rc) return rc;
  const uint32_t wpr = sp.TW == 64 ? 2u : 1u;
  const uint32_t v[9] = {sp.TW, sp.TH, sp.rpw, wpr, sp.cells, sp.slots, sp.nhalo, sp.ndirs,
                         sp.passes};
  memcpy(info, v, sizeof(v));
  memcpy(info + 9, sp.ring_end, sizeof(sp.ring_end));   // kMaxPasses + 1 entries
  for (uint32_t c = 0; c < sp.cells; ++c) {
    slot[c] = tile_slot_of(c, sp.TW, sp.rpw, wpr);
    X[c] = vX[c];
    Y[c] = vY[c];
  }
  memcpy(dir_list, sp.dir_list, 9);
  return SQUEEZE_OK;
}

// The halo chunk table (64-wide rows only) and the border-record tables of
// the level-L program: info = (nchunks, chunk_start[0..9], rec_words,
// rec_seg[0..9], rec_nexp); table = nchunks chunk offsets, nchunks + 1 cell
// ranges, nhalo cells (halo word | byte << 16) -- absent for other widths --
// then 32 * rec_words record bits (exported cell | halo word << 16, or ~0),
// rec_nexp exported slots and the export number of every slot (16 bits, two
// per word): 5 * halo + slots / 2 + 300 words at most; halo_off and halo_dir
// as in tile_program.
int tile_chunks(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L,
                uint32_t nbhd, uint32_t passes, uint32_t *info, uint32_t *table,
                uint32_t *halo_off, uint8_t *halo_dir) {
  FracDev f;
  if (!fill(s, k, off, r, nbhd, f)) return SQUEEZE_ERR_INVALID_ARG;
  TileBuildSizes z;
  sq_tile_build_sizes(f, L, z);
  std::vector<int32_t> inv(z.box);
  std::vector<uint32_t> vX(z.cells), vY(z.cells), refs((z.slots + z.halo) * 8), order(z.halo),
      rank(z.halo);
  std::vector<uint64_t> key(z.halo), sorted(z.halo);
  std::vector<uint16_t> refs16((z.slots + z.halo) * 8);
  TileBuild B = {inv.data(), vX.data(),  vY.data(),  refs.data(), key.data(),  sorted.data(),
                 order.data(), rank.data(), refs16.data(), halo_off, halo_dir, z.box,
                 z.cells,      z.slots,     z.halo,        passes,   table};
  TileSpec sp;
  const int rc = sq_tile_build(f, L, B, sp);
  if (rc) return rc;
  info[0] = sp.nchunks;
  memcpy(info + 1, sp.chunk_start, sizeof(sp.chunk_start));
  info[11] = sp.rec_words;
  memcpy(info + 12, sp.rec_seg, sizeof(sp.rec_seg));
  info[22] = sp.rec_nexp;
  return SQUEEZE_OK;
}

// The tile adjacent to every tile (tx, ty) of the level-r fractal in
// direction d = (dy+1)*3 + (dx+1), by the kernel's carry walk:
// out[ty * tiles_x + tx] = nty * tiles_x + ntx, or UINT32_MAX for none.
int tile_adjacency(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L, uint32_t d,
                   uint32_t *out) {
  FracDev f;
  if (!fill(s, k, off, r, kMoore, f)) return SQUEEZE_ERR_INVALID_ARG;
  const uint32_t TW = (uint32_t)ipow(k, (L + 1) / 2), TH = (uint32_t)ipow(k, L / 2);
  const uint32_t tiles_x = f.W / TW, tiles_y = f.H / TH;
  for (uint32_t ty = 0; ty < tiles_y; ++ty)
    for (uint32_t tx = 0; tx < tiles_x; ++tx) {
      uint32_t ntx, nty, v = ~0u;
      if (adjacent_tile(f, L, f.taux, f.tauy, f.hnu, tx, ty, (int)(d % 3) - 1, (int)(d / 3) - 1,
                        ntx, nty))
        v = nty * tiles_x + ntx;
      out[(size_t)ty * tiles_x + tx] = v;
    }
  return SQUEEZE_OK;
}

}  // extern "C"
