// bitslice.cuh -- warp-wide 32 x 32 bit transposes and carry-save adders
// shared by the bit-sliced tile kernels (planar and three-dimensional).
//
// A tile kernel packs one tile row per lane into a 32-bit word and transposes
// the warp's 32 words, so that bit t of a word is the state of one local cell
// in tile t; every logical operation then updates 32 tiles at once.
#pragma once

#include <stdint.h>

namespace sq {

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

// 32x32 bit transposes across a warp: on return lane j holds the word whose
// bit i was bit j of lane i's input.  Five butterfly stages; keep[] / rot[]
// are the per-lane masks and rotations of each stage (see make_transpose).
// kN independent transposes with their shuffle stages interleaved.  The two
// byte-granular stages (distance 16 and 8) are single byte permutes with
// per-lane selectors keep[0], keep[1]; the bit-granular ones rotate the
// partner's word and merge under a per-lane mask.
template <int kN>
__device__ __forceinline__ void transpose32_n(uint32_t *x, const uint32_t *keep,
                                              const uint32_t *rot) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    uint32_t y[kN];
#pragma unroll
    for (int k = 0; k < kN; ++k) y[k] = __shfl_xor_sync(0xFFFFFFFFu, x[k], 16 >> s);
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      if (s < 2) {
        x[k] = __byte_perm(x[k], y[k], keep[s]);
      } else {
        uint32_t t = __funnelshift_l(y[k], y[k], rot[s]);
        x[k] = (x[k] & keep[s]) | (t & ~keep[s]);
      }
    }
  }
}

__device__ __forceinline__ void make_transpose(unsigned lane, uint32_t *keep, uint32_t *rot) {
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    uint32_t j = 16u >> s;
    bool upper = lane & j;
    keep[s] = upper ? ~m[s] : m[s];
    rot[s] = upper ? 32u - j : j;
  }
  // Byte-permute selectors: the lower lane of a pair keeps its own low
  // half (byte) and takes the partner's low half up; the upper lane takes the
  // partner's high half down and keeps its own high half.
  keep[0] = (lane & 16u) ? 0x3276u : 0x5410u;
  keep[1] = (lane & 8u) ? 0x3715u : 0x6240u;
}

}  // namespace sq
