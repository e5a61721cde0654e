// tile3_host.cu -- test support: the host-built program of the 3-D tile
// kernel (tile3d.cu) and the adjacent tiles by the kernel's rule (lambda of a
// tile's first cell moved by one block, nu back), exported so that a CPU
// emulation of one step can run on them and be compared with the 3-D oracle.
// No CUDA calls are made.
#include "tile3d.cu"

int sq_cuda_fail(cudaError_t) { return SQUEEZE_ERR_CUDA; }   // never reached: no CUDA calls here
cudaError_t sq_allow_smem(const void *, size_t) { return cudaSuccess; }

namespace {

bool fill(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t nbhd, Frac3Dev &f) {
  memset(&f, 0, sizeof(f));
  f.s = s;
  f.k = k;
  f.r = r;
  f.n = (uint32_t)ipow3(s, r);
  f.Wx = (uint32_t)ipow3(k, (r + 2) / 3);
  f.Wy = (uint32_t)ipow3(k, (r + 1) / 3);
  f.Wz = (uint32_t)ipow3(k, r / 3);
  f.cells = (uint64_t)f.Wx * f.Wy * f.Wz;
  f.plane = (uint64_t)f.Wx * f.Wy;
  f.divk = sq::make_fastdiv(k);
  f.divs = sq::make_fastdiv(s);
  f.divWx = sq::make_fastdiv(f.Wx);
  f.divWy = sq::make_fastdiv(f.Wy);
  f.nbhd = nbhd;
  memset(f.hnu, kHole, sizeof(f.hnu));
  for (uint32_t b = 0; b < k; ++b) {
    const uint8_t x = off[3 * b], y = off[3 * b + 1], z = off[3 * b + 2];
    if (x >= s || y >= s || z >= s) return false;
    f.tau[0][b] = x;
    f.tau[1][b] = y;
    f.tau[2][b] = z;
    f.hnu[(z * s + y) * s + x] = (uint8_t)b;
  }
  return true;
}

}  // namespace

extern "C" {

// info = (TX, TY, TZ, slots, nhalo, ndirs, default level); refs16: slots x 32
// byte offsets into the word array (slots, halo words, zero word); halo_off:
// offsets from the adjacent tile's first cell; dir_list: the program's
// directions d = (dz+1)*9 + (dy+1)*3 + (dx+1); halo_start: 28 entries.
int tile3_program(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L,
                  uint32_t nbhd, uint32_t *info, uint16_t *refs16, uint64_t refs_cap,
                  uint32_t *halo_off, uint64_t halo_cap, uint8_t *dir_list,
                  uint32_t *halo_start) {
  Frac3Dev f;
  if (!fill(s, k, off, r, nbhd, f)) return SQUEEZE_ERR_INVALID_ARG;
  std::vector<uint16_t> refs;
  std::vector<uint32_t> hoff;
  std::vector<uint8_t> dirs;
  uint32_t nhalo = 0, slots = 0;
  const int rc = sq3_tile_build(f, L, refs, hoff, dirs, halo_start, nhalo, slots);
  if (rc) return rc;
  if (refs.size() > refs_cap || nhalo > halo_cap) return SQUEEZE_ERR_INVALID_ARG;
  uint32_t TX, TY, TZ, sl;
  uint64_t box;
  sq3_tile_shape(f, L, TX, TY, TZ, sl, box);
  const uint32_t v[7] = {TX, TY, TZ, slots, nhalo, (uint32_t)dirs.size(),
                         sq3_tile_default_level(f)};
  memcpy(info, v, sizeof(v));
  memcpy(refs16, refs.data(), refs.size() * 2);
  memcpy(halo_off, hoff.data(), hoff.size() * 4);
  memcpy(dir_list, dirs.data(), dirs.size());
  return SQUEEZE_OK;
}

// The tile next to every tile in direction d, by the kernel's rule:
// out[tile] = adjacent tile index, or UINT32_MAX.
int tile3_adjacency(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t L,
                    uint32_t d, uint32_t *out) {
  Frac3Dev f;
  if (!fill(s, k, off, r, kMoore26, f)) return SQUEEZE_ERR_INVALID_ARG;
  uint32_t TX, TY, TZ, slots;
  uint64_t box;
  if (!sq3_tile_shape(f, L, TX, TY, TZ, slots, box)) return SQUEEZE_ERR_UNSUPPORTED;
  Tables3 t;
  memcpy(t.tau, f.tau, sizeof(t.tau));
  memcpy(t.hnu, f.hnu, sizeof(t.hnu));
  const uint32_t side = (uint32_t)ipow3(s, L);
  const uint32_t tiles_x = f.Wx / TX, tiles_y = f.Wy / TY, tiles_z = f.Wz / TZ;
  for (uint32_t tz = 0; tz < tiles_z; ++tz)
    for (uint32_t ty = 0; ty < tiles_y; ++ty)
      for (uint32_t tx = 0; tx < tiles_x; ++tx) {
        uint32_t x, y, z, v = ~0u;
        lambda3(f, t, tx * TX, ty * TY, tz * TZ, x, y, z);
        const int64_t qx = (int64_t)x + ((int)(d % 3) - 1) * (int64_t)side;
        const int64_t qy = (int64_t)y + ((int)((d / 3) % 3) - 1) * (int64_t)side;
        const int64_t qz = (int64_t)z + ((int)(d / 9) - 1) * (int64_t)side;
        uint64_t om;
        if (nu3(f, t, (int32_t)qx, (int32_t)qy, (int32_t)qz, om)) {
          uint32_t wx, wy, wz;
          split3(f, om, wx, wy, wz);
          v = ((wz / TZ) * tiles_y + wy / TY) * tiles_x + wx / TX;
        }
        out[((size_t)tz * tiles_y + ty) * tiles_x + tx] = v;
      }
  return SQUEEZE_OK;
}

}  // extern "C"
