// nbb3d_host.cu -- test support: the per-cell functions of the 3-D step
// (nbb3d.cuh, all host-callable) run on the CPU, so that their index
// arithmetic can be compared with the oracle without a GPU.  The loop in
// h3_step is the body of step3_kernel, one compact cell per iteration.
#include "nbb3d.cu"

int sq_cuda_fail(cudaError_t) { return SQUEEZE_ERR_CUDA; }   // never reached: no CUDA calls here
cudaError_t sq_allow_smem(const void *, size_t) { return cudaSuccess; }
// The tile kernel (tile3d.cu) is not part of this host library; the step
// entry point that would reach it is never called here.
bool sq3_tile_shape(const Frac3Dev &, uint32_t, uint32_t &, uint32_t &, uint32_t &, uint32_t &,
                    uint64_t &) {
  return false;
}
uint32_t sq3_tile_default_level(const Frac3Dev &) { return 0; }
int sq3_tile_prepare(const Frac3Dev &, uint32_t, int, Tile3Program **) {
  return SQUEEZE_ERR_UNSUPPORTED;
}
void sq3_tile_free(Tile3Program *) {}
int sq3_tile_launch(const Tile3Program *, uint32_t, uint32_t, int *, const uint8_t *, uint8_t *,
                    cudaStream_t) {
  return SQUEEZE_ERR_UNSUPPORTED;
}

namespace {
void tables_of(const Frac3Dev &f, Tables3 &t) {
  memcpy(t.tau, f.tau, sizeof(t.tau));
  memcpy(t.hnu, f.hnu, sizeof(t.hnu));
}
}  // namespace

extern "C" {

int h3_info(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint64_t *info) {
  Frac3Dev f;
  const int rc = fill3(s, k, off, r, f);
  if (rc) return rc;
  info[0] = f.cells;
  info[1] = f.Wx;
  info[2] = f.Wy;
  info[3] = f.Wz;
  info[4] = f.n;
  return SQUEEZE_OK;
}

int h3_lambda(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const uint64_t *om,
              int32_t *xyz, uint64_t count) {
  Frac3Dev f;
  const int rc = fill3(s, k, off, r, f);
  if (rc) return rc;
  Tables3 t;
  tables_of(f, t);
  for (uint64_t i = 0; i < count; ++i) {
    int32_t X = -1, Y = -1, Z = -1;
    if (om[i] < f.cells) {
      uint32_t wx, wy, wz, x, y, z;
      sq3::split3(f, om[i], wx, wy, wz);
      sq3::lambda3(f, t, wx, wy, wz, x, y, z);
      X = (int32_t)x;
      Y = (int32_t)y;
      Z = (int32_t)z;
    }
    xyz[3 * i] = X;
    xyz[3 * i + 1] = Y;
    xyz[3 * i + 2] = Z;
  }
  return SQUEEZE_OK;
}

int h3_nu(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const int32_t *xyz, uint64_t *om,
          uint64_t count) {
  Frac3Dev f;
  const int rc = fill3(s, k, off, r, f);
  if (rc) return rc;
  Tables3 t;
  tables_of(f, t);
  for (uint64_t i = 0; i < count; ++i) {
    uint64_t o;
    om[i] = sq3::nu3(f, t, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], o) ? o : ~0ull;
  }
  return SQUEEZE_OK;
}

// The compact index of each of the 27 offsets d = (dz+1)*9 + (dy+1)*3 + (dx+1)
// of every cell in `which`, found by the neighbour walk (UINT64_MAX for a
// hole, a point off the box and the cell itself): out[27 * i + d].
int h3_neighbours(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const uint64_t *which,
                  uint64_t count, uint64_t *out) {
  Frac3Dev f;
  const int rc = fill3(s, k, off, r, f);
  if (rc) return rc;
  Tables3 t;
  tables_of(f, t);
  for (uint64_t i = 0; i < count; ++i) {
    const uint64_t omega = which[i];
    uint32_t wx, wy, wz;
    sq3::split3(f, omega, wx, wy, wz);
    const sq3::Cell3 c = sq3::cell3(f, t, wx, wy, wz);
    for (int d = 0; d < 27; ++d) {
      int64_t delta;
      const bool ok = d != 13 && f.r > 0 &&
                      sq3::neighbour3(f, t, c, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1, delta);
      out[27 * i + d] = ok ? omega + (uint64_t)delta : ~0ull;
    }
  }
  return SQUEEZE_OK;
}

// Next state of the cells listed in `which` (every cell when which is NULL);
// *bad counts neighbour indices past the state.
int h3_step(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, uint32_t nbhd, uint32_t birth,
            uint32_t survive, const uint8_t *in, uint8_t *out, const uint64_t *which,
            uint64_t count, uint64_t *bad) {
  Frac3Dev f;
  const int rc = fill3(s, k, off, r, f);
  if (rc) return rc;
  f.nbhd = nbhd;
  f.birth = birth;
  f.survive = survive;
  Tables3 t;
  tables_of(f, t);
  const uint64_t n = which ? count : f.cells;
  *bad = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t omega = which ? which[i] : i;
    uint32_t wx, wy, wz;
    sq3::split3(f, omega, wx, wy, wz);
    const sq3::Cell3 c = sq3::cell3(f, t, wx, wy, wz);
    uint32_t cnt = 0;
    if (f.r > 0) {
      for (int d = 0; d < 27; ++d) {
        if (d == 13 || !((f.nbhd >> d) & 1u)) continue;
        int64_t delta;
        if (!sq3::neighbour3(f, t, c, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1, delta)) continue;
        const uint64_t nb = omega + (uint64_t)delta;
        if (nb < f.cells) cnt += in[nb] & 1u;
        else ++*bad;
      }
    }
    const bool alive = in[omega] & 1u;
    out[which ? i : omega] = (uint8_t)((((alive ? f.survive : f.birth) >> cnt) & 1u));
  }
  return SQUEEZE_OK;
}

}  // extern "C"
