// maps_host.cu -- test support: the per-cell lambda, nu and neighbour walk of
// the two-dimensional kernels (squeeze_internal.cuh; host-callable) run on
// the CPU, so that they can be compared with the oracle without a GPU.
#include <string.h>

#include "squeeze_internal.cuh"

using namespace sq;

namespace {

bool fill(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, FracDev &f, SmemTables &t) {
  memset(&f, 0, sizeof(f));
  uint64_t n = 1, W = 1, H = 1;
  for (uint32_t i = 0; i < r; ++i) n *= s;
  for (uint32_t i = 0; i < (r + 1) / 2; ++i) W *= k;
  for (uint32_t i = 0; i < r / 2; ++i) H *= k;
  if (n > (1ull << 30) || W > 0xFFFFFFFFull || H > 0xFFFFFFFFull) return false;
  f.s = s;
  f.k = k;
  f.r = r;
  f.n = (uint32_t)n;
  f.W = (uint32_t)W;
  f.H = (uint32_t)H;
  f.cells = W * H;
  f.divk = make_fastdiv(k);
  f.divs = make_fastdiv(s);
  f.divW = make_fastdiv((uint32_t)W);
  f.nbhd = kMoore;
  memset(f.hnu, kHole, sizeof(f.hnu));
  for (uint32_t b = 0; b < k; ++b) {
    f.taux[b] = off[2 * b];
    f.tauy[b] = off[2 * b + 1];
    f.hnu[off[2 * b + 1] * s + off[2 * b]] = (uint8_t)b;
  }
  memcpy(t.taux, f.taux, 256);
  memcpy(t.tauy, f.tauy, 256);
  memcpy(t.hnu, f.hnu, 256);
  return true;
}

}  // namespace

extern "C" {

int h2_lambda(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const uint64_t *om,
              int64_t *xy, uint64_t count) {
  FracDev f;
  SmemTables t;
  if (!fill(s, k, off, r, f, t)) return SQUEEZE_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < count; ++i) {
    xy[2 * i] = xy[2 * i + 1] = -1;
    if (om[i] >= f.cells) continue;
    uint32_t x, y;
    lambda_alu(f, t, (uint32_t)(om[i] % f.W), (uint32_t)(om[i] / f.W), x, y);
    xy[2 * i] = x;
    xy[2 * i + 1] = y;
  }
  return SQUEEZE_OK;
}

int h2_nu(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const int64_t *xy, uint64_t *om,
          uint64_t count) {
  FracDev f;
  SmemTables t;
  if (!fill(s, k, off, r, f, t)) return SQUEEZE_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < count; ++i) {
    uint32_t wx, wy;
    const int64_t x = xy[2 * i], y = xy[2 * i + 1];
    const bool in32 = x >= INT32_MIN && x <= INT32_MAX && y >= INT32_MIN && y <= INT32_MAX;
    om[i] = in32 && nu_alu(f, t, (int32_t)x, (int32_t)y, wx, wy) ? (uint64_t)wy * f.W + wx : ~0ull;
  }
  return SQUEEZE_OK;
}

// Compact index of each of the 9 offsets d = (dy+1)*3 + (dx+1) of each cell
// by the carry walk (UINT64_MAX for a hole, a point off the box, the cell).
int h2_neighbours(uint32_t s, uint32_t k, const uint8_t *off, uint32_t r, const uint64_t *om,
                  uint64_t count, uint64_t *out) {
  FracDev f;
  SmemTables t;
  if (!fill(s, k, off, r, f, t)) return SQUEEZE_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < count; ++i)
    for (int d = 0; d < 9; ++d) {
      uint32_t nx, ny;
      const bool ok = d != 4 && neighbour_omega(f, t, (uint32_t)(om[i] % f.W),
                                                (uint32_t)(om[i] / f.W), d % 3 - 1, d / 3 - 1, nx, ny);
      out[9 * i + d] = ok ? (uint64_t)ny * f.W + nx : ~0ull;
    }
  return SQUEEZE_OK;
}

}  // extern "C"
