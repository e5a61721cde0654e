// tile3d.cu -- the bit-sliced tile kernel for three-dimensional NBB fractals.
//
// The planar tile kernel (step_tiled.cu) carried over to a third axis.  Every
// level-L sub-replica of a 3-D NBB fractal (a "tile", k^L cells) is a
// translated copy of the level-L fractal, so the lambda / 26-neighbour / nu
// exploration is the same inside every tile: the host runs it once per
// fractal and level and stores, per local cell, 26 references into a word
// array (local cells, halo cells of the 26 adjacent level-L blocks, or a zero
// word).  Which block lies next to a tile in each direction (a tile, a hole
// or off the box) is found once per handle on the device, from lambda of the
// tile's first cell moved by one block and nu back.
//
// In the compact layout (levels cycling x -> y -> z) a tile is a TX x TY x TZ
// brick: TX = k^ceil(L/3) contiguous bytes per row, TY * TZ rows.  A CTA owns
// a group of up to 32 tiles side by side in compact x, so each of its rows is
// one contiguous segment of 32 * TX bytes.  Each lane loads its tile's rows
// straight from global memory (TX = 8 or 16 cells, 32 / TX rows per 32-bit
// word), a warp transpose turns them into words whose bit t is a local cell
// of tile t, the rule runs on whole words (a carry-save adder over 26
// neighbour words, then the birth / survive masks), and the inverse
// transpose gives the rows back, which each lane stores as whole words.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bitslice.cuh"
#include "nbb3d.cuh"

using sq::FastDiv;
using sq::fdiv;

// Kernel-side description of a level-L program.
struct Tile3Dev {
  uint64_t Wx, plane, total;       // compact row length, W_x * W_y, cells
  uint32_t TX, TY, TZ, rows, VR, slots, nhalo, ndirs;
  uint32_t tiles_x, tiles_y, groups_per_band, pad_;
  uint64_t tiles, groups;
  FastDiv div_gpb, div_tiles_x, div_tiles_y, div_ty;
  uint32_t halo_start[28];         // halo words of direction j: [halo_start[j], halo_start[j+1])
  uint32_t nact;                   // counts with a birth or survive bit
  uint32_t act[27];                // count | 0x100 if it gives birth | 0x200 if it survives
  const uint16_t *refs;            // 32 per slot (26 used): byte offsets into the word array
  const uint32_t *halo_off;        // nhalo offsets from the adjacent tile's first cell
  const uint32_t *adj;             // ndirs x tiles: adjacent tile, or ~0 (hole / off the box)
  int *status;
};

struct Tile3Program {
  Tile3Dev dev;                    // device pointers and geometry (status set per launch)
  uint32_t L, smem, threads;
  int grid;
  uint16_t *d_refs;
  uint32_t *d_halo_off;
  uint32_t *d_adj;
};

namespace sq3 {
namespace {

constexpr int kT3Threads = 256;
constexpr uint32_t kMaxSlots = 4096;       // refs table <= 256 KB
constexpr size_t kT3SmemCap = 48 * 1024;

__device__ __forceinline__ void flag(int *status, int code) { atomicCAS(status, 0, code); }

// Full adder on bit planes: returns the sum, leaves the carry in `c`.
__device__ __forceinline__ uint32_t fa(uint32_t a, uint32_t b, uint32_t d, uint32_t &c) {
  c = sq::maj3(a, b, d);
  return a ^ b ^ d;
}

// Count of 26 one-bit inputs per bit position, as 5 bit planes (carry-save
// adder tree: 21 full adders and 2 half adders).
__device__ __forceinline__ void count26(const uint32_t *x, uint32_t *cnt) {
  uint32_t w1[10], w2[13], w4[6], w8[3];
#pragma unroll
  for (int i = 0; i < 8; ++i) w1[i] = fa(x[3 * i], x[3 * i + 1], x[3 * i + 2], w2[i]);
  w1[8] = x[24];
  w1[9] = x[25];
  // weight 1: 10 -> 4 -> 2 -> 1
  uint32_t a1[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) a1[i] = fa(w1[3 * i], w1[3 * i + 1], w1[3 * i + 2], w2[8 + i]);
  a1[3] = w1[9];
  uint32_t b1 = fa(a1[0], a1[1], a1[2], w2[11]);
  cnt[0] = b1 ^ a1[3];
  w2[12] = b1 & a1[3];
  // weight 2: 13 -> 5 -> 3 -> 1
  uint32_t a2[5];
#pragma unroll
  for (int i = 0; i < 4; ++i) a2[i] = fa(w2[3 * i], w2[3 * i + 1], w2[3 * i + 2], w4[i]);
  a2[4] = w2[12];
  uint32_t b2 = fa(a2[0], a2[1], a2[2], w4[4]);
  cnt[1] = fa(b2, a2[3], a2[4], w4[5]);
  // weight 4: 6 -> 2 -> 1
  uint32_t a4[2];
  a4[0] = fa(w4[0], w4[1], w4[2], w8[0]);
  a4[1] = fa(w4[3], w4[4], w4[5], w8[1]);
  cnt[2] = a4[0] ^ a4[1];
  w8[2] = a4[0] & a4[1];
  // weight 8 and 16
  cnt[3] = fa(w8[0], w8[1], w8[2], cnt[4]);
}

// Next state of 32 cells: `self` alive bits, 26 neighbour words.
__device__ __forceinline__ uint32_t rule26(const Tile3Dev &p, uint32_t self, const uint32_t *x) {
  uint32_t c[5];
  count26(x, c);
  uint32_t next = 0;
  for (uint32_t i = 0; i < p.nact; ++i) {
    const uint32_t a = p.act[i], n = a & 0xFFu;
    uint32_t miss = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) miss |= c[b] ^ (((n >> b) & 1u) ? 0xFFFFFFFFu : 0u);
    const uint32_t eq = ~miss;
    const uint32_t who = (a & 0x100u) ? ((a & 0x200u) ? 0xFFFFFFFFu : ~self) : self;
    next |= eq & who;
  }
  return next;
}

// First byte of tile t (~0 for t = ~0).
__device__ __forceinline__ uint64_t tile_base3(const Tile3Dev &p, uint32_t t) {
  if (t == ~0u) return ~0ull;
  const uint32_t band = fdiv(p.div_tiles_x, t), tx = t - band * p.tiles_x;
  const uint32_t tz = fdiv(p.div_tiles_y, band), ty = band - tz * p.tiles_y;
  return (uint64_t)tz * p.TZ * p.plane + (uint64_t)ty * p.TY * p.Wx + (uint64_t)tx * p.TX;
}

// Byte offset of tile row r (r = lz * TY + ly) from the tile's first byte.
__device__ __forceinline__ uint64_t row_offset3(const Tile3Dev &p, uint32_t r) {
  const uint32_t lz = fdiv(p.div_ty, r), ly = r - lz * p.TY;
  return (uint64_t)lz * p.plane + (uint64_t)ly * p.Wx;
}

// One step: CTA c of the persistent grid takes groups [c G / grid, (c+1) G / grid).
// kTX = 8 or 16 cells per tile row; kRPW = 32 / kTX rows share a slot word.
template <int kTX>
__global__ void __launch_bounds__(kT3Threads) tile3_kernel(Tile3Dev p, const uint8_t *__restrict__ in,
                                                           uint8_t *__restrict__ out) {
  extern __shared__ __align__(16) uint32_t words[];   // slots | halo | zero word
  constexpr uint32_t kRPW = 32u / (uint32_t)kTX;
  constexpr int kR = 2;                               // slot rows in flight per warp
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t keep[5], rot[5];
  sq::make_transpose(lane, keep, rot);
  if (threadIdx.x == 0) words[p.slots + p.nhalo] = 0u;
  const uint64_t g0 = (uint64_t)blockIdx.x * p.groups / gridDim.x;
  const uint64_t g1 = (uint64_t)(blockIdx.x + 1) * p.groups / gridDim.x;
  for (uint64_t g = g0; g < g1; ++g) {
    const uint32_t band = fdiv(p.div_gpb, (uint32_t)g);
    const uint32_t tx0 = ((uint32_t)g - band * p.groups_per_band) * 32u;
    const uint32_t ntiles = min(32u, p.tiles_x - tx0);
    const uint32_t tz = fdiv(p.div_tiles_y, band), ty = band - tz * p.tiles_y;
    const uint64_t base = (uint64_t)tz * p.TZ * p.plane + (uint64_t)ty * p.TY * p.Wx +
                          (uint64_t)(tx0 + lane) * kTX;   // this lane's tile
    const bool live = lane < ntiles;
    __syncthreads();   // the previous group's rule pass is done with the words
    // Pack: lane = tile; bit 8b + j of a row word <- byte 4j + b of the row,
    // the kRPW rows of a slot word in consecutive 4-bit (TX = 16) or 2-bit
    // (TX = 8) fields; then lane = local cell, bit = tile.
    for (uint32_t v0 = warp; v0 < p.VR; v0 += kR * nw) {
      uint32_t acc[kR];
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t v = v0 + (uint32_t)k * nw;
        acc[k] = 0;
        if (v < p.VR && live) {
#pragma unroll
          for (uint32_t i = 0; i < kRPW; ++i) {
            const uint64_t a = base + row_offset3(p, v * kRPW + i);
            uint32_t w;
            if constexpr (kTX == 16) {
              const uint4 q = __ldg(reinterpret_cast<const uint4 *>(in + a));
              w = (q.x & 0x01010101u) | ((q.y & 0x01010101u) << 1) |
                  ((q.z & 0x01010101u) << 2) | ((q.w & 0x01010101u) << 3);
            } else {
              const uint2 q = __ldg(reinterpret_cast<const uint2 *>(in + a));
              w = (q.x & 0x01010101u) | ((q.y & 0x01010101u) << 1);
            }
            acc[k] |= w << (i * (uint32_t)(kTX / 4));
          }
        }
      }
      sq::transpose32_n<kR>(acc, keep, rot);
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t v = v0 + (uint32_t)k * nw;
        if (v < p.VR) words[v * 32u + lane] = acc[k];
      }
    }
    // Halo words, direction j per warp: bit `lane` = the halo cell of this
    // lane's adjacent tile in direction j (dead for a hole or off the box).
    const uint32_t tile0 = (tz * p.tiles_y + ty) * p.tiles_x + tx0;
    for (uint32_t j = warp; j < p.ndirs; j += nw) {
      const uint32_t t = live ? __ldg(p.adj + (uint64_t)j * p.tiles + tile0 + lane) : ~0u;
      const uint64_t tb = tile_base3(p, t);
      for (uint32_t h = p.halo_start[j]; h < p.halo_start[j + 1]; ++h) {
        bool alive = false;
        if (tb != ~0ull) {
          const uint64_t a = tb + __ldg(p.halo_off + h);
          if (a < p.total) alive = __ldg(in + a) & 1u;
          else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
        }
        const uint32_t wd = __ballot_sync(0xFFFFFFFFu, alive);
        if (lane == 0) words[p.slots + h] = wd;
      }
    }
    __syncthreads();   // all words in place
    // Rule, inverse transpose, and the rows back to global memory.
    const unsigned char *wb = reinterpret_cast<const unsigned char *>(words);
    for (uint32_t v0 = warp; v0 < p.VR; v0 += kR * nw) {
      uint32_t y[kR];
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t v = v0 + (uint32_t)k * nw;
        y[k] = 0;
        if (v < p.VR) {
          const uint32_t c = v * 32u + lane;
          const uint4 *r4 = reinterpret_cast<const uint4 *>(p.refs) + (size_t)c * 4u;
          uint32_t x[26];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 rr = __ldg(r4 + q);
            const uint32_t rw[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i0 = 8 * q + 2 * e, i1 = i0 + 1;
              if (i0 < 26)
                x[i0] = *reinterpret_cast<const uint32_t *>(wb + __byte_perm(rw[e], 0, 0x4410));
              if (i1 < 26)
                x[i1] = *reinterpret_cast<const uint32_t *>(wb + __byte_perm(rw[e], 0, 0x4432));
            }
          }
          y[k] = rule26(p, words[c], x);
        }
      }
      sq::transpose32_n<kR>(y, keep, rot);
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t v = v0 + (uint32_t)k * nw;
        if (v < p.VR && live) {
#pragma unroll
          for (uint32_t i = 0; i < kRPW; ++i) {
            const uint32_t w = y[k] >> (i * (uint32_t)(kTX / 4));
            const uint64_t a = base + row_offset3(p, v * kRPW + i);
            if constexpr (kTX == 16) {
              *reinterpret_cast<uint4 *>(out + a) =
                  make_uint4(w & 0x01010101u, (w >> 1) & 0x01010101u, (w >> 2) & 0x01010101u,
                             (w >> 3) & 0x01010101u);
            } else {
              *reinterpret_cast<uint2 *>(out + a) =
                  make_uint2(w & 0x01010101u, (w >> 1) & 0x01010101u);
            }
          }
        }
      }
    }
  }
}

// One thread per (direction, tile): the tile next to tile t in direction
// dir_list[j], from lambda of the tile's first cell moved by one level-L
// block and nu back (the block's same local point is its first cell when the
// block is a tile).
__global__ void tile3_adjacency_kernel(Frac3Dev f, Tile3Dev p, uint32_t L, uint32_t side,
                                       const uint8_t *__restrict__ dir_list,
                                       uint32_t *__restrict__ adj) {
  __shared__ Tables3 t;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    t.tau[0][i] = f.tau[0][i];
    t.tau[1][i] = f.tau[1][i];
    t.tau[2][i] = f.tau[2][i];
  }
  for (int i = threadIdx.x; i < 512; i += blockDim.x) t.hnu[i] = f.hnu[i];
  __syncthreads();
  const uint64_t n = (uint64_t)p.ndirs * p.tiles;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(i / p.tiles);
    const uint32_t tile = (uint32_t)(i - (uint64_t)j * p.tiles);
    const uint32_t band = tile / p.tiles_x, tx = tile - band * p.tiles_x;
    const uint32_t tz = band / p.tiles_y, ty = band - tz * p.tiles_y;
    uint32_t x, y, z;
    lambda3(f, t, tx * p.TX, ty * p.TY, tz * p.TZ, x, y, z);
    const uint32_t d = dir_list[j];
    const int64_t qx = (int64_t)x + ((int)(d % 3) - 1) * (int64_t)side;
    const int64_t qy = (int64_t)y + ((int)((d / 3) % 3) - 1) * (int64_t)side;
    const int64_t qz = (int64_t)z + ((int)(d / 9) - 1) * (int64_t)side;
    uint32_t r = ~0u;
    uint64_t om;
    if (qx >= 0 && qy >= 0 && qz >= 0 && qx < f.n && qy < f.n && qz < f.n &&
        nu3(f, t, (int32_t)qx, (int32_t)qy, (int32_t)qz, om)) {
      uint32_t wx, wy, wz;
      split3(f, om, wx, wy, wz);
      r = ((wz / p.TZ) * p.tiles_y + wy / p.TY) * p.tiles_x + wx / p.TX;
    }
    adj[i] = r;
  }
}

uint64_t ipow3(uint64_t b, uint32_t e) {
  uint64_t v = 1;
  while (e--) v *= b;
  return v;
}

}  // namespace
}  // namespace sq3

using namespace sq3;

// Sizes of the level-L program of a 3-D fractal (cells, slots, box points),
// or false when the tile kernel cannot take this level: tile rows of 8 or
// 16 cells only (32 / TX rows share a slot word), W_x a multiple of 16 (every
// row of a group then starts on a 16-byte boundary), at most kMaxSlots slots.
bool sq3_tile_shape(const Frac3Dev &f, uint32_t L, uint32_t &TX, uint32_t &TY, uint32_t &TZ,
                    uint32_t &slots, uint64_t &box) {
  if (L == 0 || L > f.r) return false;
  const uint64_t tx = ipow3(f.k, (L + 2) / 3), ty = ipow3(f.k, (L + 1) / 3),
                 tz = ipow3(f.k, L / 3), side = ipow3(f.s, L);
  if (tx != 8 && tx != 16) return false;
  const uint64_t rows = ty * tz, rpw = 32 / tx;
  if (rows % rpw || rows / rpw * 32 > kMaxSlots || f.Wx % 16) return false;
  if (side * side * side > (1ull << 24)) return false;
  if ((uint64_t)tz * f.plane > 0xFFFFFFFFull) return false;   // halo offsets fit 32 bits
  TX = (uint32_t)tx;
  TY = (uint32_t)ty;
  TZ = (uint32_t)tz;
  slots = (uint32_t)(rows / rpw * 32);
  box = side * side * side;
  return true;
}

// Host construction of the level-L program: local lambda over the level-L box
// (levels cycling over the compact axes), its inverse, 26 references per
// local cell (zero word where the neighbour is a hole or outside the
// neighbourhood), halo cells keyed by (direction, local cell in the adjacent
// block) and sorted by direction.  refs16: slots x 32 byte offsets.
int sq3_tile_build(const Frac3Dev &f, uint32_t L, std::vector<uint16_t> &refs16,
                   std::vector<uint32_t> &halo_off, std::vector<uint8_t> &dir_list,
                   uint32_t *halo_start, uint32_t &nhalo_out, uint32_t &slots_out) {
  uint32_t TX, TY, TZ, slots;
  uint64_t box;
  if (!sq3_tile_shape(f, L, TX, TY, TZ, slots, box)) return SQUEEZE_ERR_UNSUPPORTED;
  const uint32_t side = (uint32_t)ipow3(f.s, L), cells = TX * TY * TZ, rpw = 32 / TX;
  Frac3Dev fl = f;   // the level-L fractal: lambda of local coordinates
  fl.r = L;
  Tables3 t;
  memcpy(t.tau, f.tau, sizeof(t.tau));
  memcpy(t.hnu, f.hnu, sizeof(t.hnu));
  std::vector<int32_t> inv(box, -1);
  std::vector<uint32_t> X(cells), Y(cells), Z(cells);
  for (uint32_t c = 0; c < cells; ++c) {
    const uint32_t lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    lambda3(fl, t, lx, ly, lz, X[c], Y[c], Z[c]);
    inv[((size_t)Z[c] * side + Y[c]) * side + X[c]] = (int32_t)c;
  }
  // slot of local cell c: its row r = c / TX shares slot word r / rpw with
  // rpw - 1 other rows; bit order of the pack (byte 4j + b -> bit 8b + j)
  auto slot_of = [&](uint32_t c) {
    const uint32_t r = c / TX, pos = (r % rpw) * TX + c % TX;
    return (r / rpw) * 32u + 8u * (pos & 3u) + (pos >> 2);
  };
  const uint32_t kNone = 0xFFFFFFFFu;
  std::vector<uint32_t> refs((size_t)slots * 32, kNone);
  std::vector<uint64_t> keys;
  for (uint32_t c = 0; c < cells; ++c) {
    int k26 = 0;
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;
      uint32_t ref = kNone;
      if ((f.nbhd >> d) & 1u) {
        const int64_t q[3] = {(int64_t)X[c] + d % 3 - 1, (int64_t)Y[c] + (d / 3) % 3 - 1,
                              (int64_t)Z[c] + d / 9 - 1};
        int bl[3];
        int64_t loc[3];
        for (int a = 0; a < 3; ++a) {
          bl[a] = q[a] < 0 ? -1 : (q[a] >= side ? 1 : 0);
          loc[a] = q[a] - (int64_t)bl[a] * side;
        }
        const int32_t target = inv[((size_t)loc[2] * side + loc[1]) * side + loc[0]];
        if (target >= 0) {
          if (!bl[0] && !bl[1] && !bl[2]) {
            ref = slot_of((uint32_t)target);
          } else {
            const uint64_t key = ((uint64_t)((bl[2] + 1) * 9 + (bl[1] + 1) * 3 + (bl[0] + 1)) << 32) |
                                 (uint32_t)target;
            size_t i = 0;
            while (i < keys.size() && keys[i] != key) ++i;
            if (i == keys.size()) keys.push_back(key);
            ref = slots + (uint32_t)i;
          }
        }
      }
      refs[(size_t)slot_of(c) * 32 + k26++] = ref;
    }
  }
  const uint32_t nhalo = (uint32_t)keys.size();
  std::vector<uint32_t> order(nhalo), rank(nhalo);
  for (uint32_t i = 0; i < nhalo; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
  for (uint32_t i = 0; i < nhalo; ++i) rank[order[i]] = i;
  const uint32_t zero = slots + nhalo;
  if (((uint64_t)zero + 1) * 4 > 0xFFFFu) return SQUEEZE_ERR_UNSUPPORTED;
  refs16.assign((size_t)slots * 32, (uint16_t)(4u * zero));
  for (size_t i = 0; i < refs.size(); ++i) {
    const uint32_t r = refs[i];
    if (r != kNone) refs16[i] = (uint16_t)(4u * (r < slots ? r : slots + rank[r - slots]));
  }
  uint8_t dir_index[27];
  uint32_t dir_mask = 0;
  for (uint32_t i = 0; i < nhalo; ++i) dir_mask |= 1u << (uint32_t)(keys[i] >> 32);
  dir_list.clear();
  for (uint32_t d = 0; d < 27; ++d)
    if ((dir_mask >> d) & 1u) {
      dir_index[d] = (uint8_t)dir_list.size();
      dir_list.push_back((uint8_t)d);
    }
  halo_off.assign(nhalo, 0);
  for (uint32_t j = 0; j < 28; ++j) halo_start[j] = 0;
  for (uint32_t i = 0; i < nhalo; ++i) {
    const uint64_t key = keys[order[i]];
    const uint32_t d = (uint32_t)(key >> 32), lc = (uint32_t)key;
    const uint32_t lx = lc % TX, ly = (lc / TX) % TY, lz = lc / (TX * TY);
    halo_off[i] = (uint32_t)((uint64_t)lz * f.plane + (uint64_t)ly * f.Wx + lx);
    halo_start[dir_index[d] + 1] = i + 1;
  }
  for (uint32_t j = 1; j < 28; ++j)
    if (halo_start[j] < halo_start[j - 1]) halo_start[j] = halo_start[j - 1];
  nhalo_out = nhalo;
  slots_out = slots;
  return SQUEEZE_OK;
}

uint32_t sq3_tile_default_level(const Frac3Dev &f) {
  for (uint32_t L = f.r; L >= 1; --L) {
    uint32_t TX, TY, TZ, slots;
    uint64_t box;
    if (sq3_tile_shape(f, L, TX, TY, TZ, slots, box) && slots <= 1024) return L;
  }
  return 0;
}

void sq3_tile_free(Tile3Program *p) {
  if (!p) return;
  cudaFree(p->d_refs);
  cudaFree(p->d_halo_off);
  cudaFree(p->d_adj);
  delete p;
}

// Build the level-L program of a 3-D handle on its device: tables, adjacency,
// launch shape.  Returns UNSUPPORTED for a level the tile kernel cannot take.
int sq3_tile_prepare(const Frac3Dev &f, uint32_t L, int device, Tile3Program **out) {
  *out = nullptr;
  std::vector<uint16_t> refs16;
  std::vector<uint32_t> halo_off;
  std::vector<uint8_t> dir_list;
  uint32_t halo_start[28], nhalo = 0, slots = 0;
  int rc = sq3_tile_build(f, L, refs16, halo_off, dir_list, halo_start, nhalo, slots);
  if (rc) return rc;
  uint32_t TX, TY, TZ, sl;
  uint64_t box;
  sq3_tile_shape(f, L, TX, TY, TZ, sl, box);
  const uint32_t smem = (uint32_t)(((size_t)slots + nhalo + 1) * 4);
  if (smem > kT3SmemCap) return SQUEEZE_ERR_UNSUPPORTED;
  Tile3Program *p = new (std::nothrow) Tile3Program;
  if (!p) return SQUEEZE_ERR_OOM;
  memset(p, 0, sizeof(*p));
  Tile3Dev &d = p->dev;
  d.Wx = f.Wx;
  d.plane = f.plane;
  d.total = f.cells;
  d.TX = TX;
  d.TY = TY;
  d.TZ = TZ;
  d.rows = TY * TZ;
  d.VR = d.rows / (32 / TX);
  d.slots = slots;
  d.nhalo = nhalo;
  d.ndirs = (uint32_t)dir_list.size();
  d.tiles_x = f.Wx / TX;
  d.tiles_y = f.Wy / TY;
  d.groups_per_band = (d.tiles_x + 31) / 32;
  d.tiles = (uint64_t)d.tiles_x * d.tiles_y * (f.Wz / TZ);
  d.groups = (uint64_t)d.groups_per_band * d.tiles_y * (f.Wz / TZ);
  if (d.tiles >= (1ull << 32) || d.groups >= (1ull << 32)) {
    delete p;
    return SQUEEZE_ERR_UNSUPPORTED;
  }
  d.div_gpb = sq::make_fastdiv(d.groups_per_band);
  d.div_tiles_x = sq::make_fastdiv(d.tiles_x);
  d.div_tiles_y = sq::make_fastdiv(d.tiles_y);
  d.div_ty = sq::make_fastdiv(TY);
  memcpy(d.halo_start, halo_start, sizeof(d.halo_start));
  p->L = L;
  p->smem = smem;
  p->threads = kT3Threads;
  cudaError_t e = cudaMalloc(&p->d_refs, refs16.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_halo_off, (nhalo ? nhalo : 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_adj, (d.ndirs ? d.ndirs : 1) * d.tiles * 4);
  uint8_t *d_dirs = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_dirs, 32);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_refs, refs16.data(), refs16.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nhalo)
    e = cudaMemcpy(p->d_halo_off, halo_off.data(), nhalo * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d.ndirs)
    e = cudaMemcpy(d_dirs, dir_list.data(), d.ndirs, cudaMemcpyHostToDevice);
  d.refs = p->d_refs;
  d.halo_off = p->d_halo_off;
  d.adj = p->d_adj;
  if (e == cudaSuccess && d.ndirs) {
    tile3_adjacency_kernel<<<sq::grid_for((uint64_t)d.ndirs * d.tiles, 256), 256>>>(
        f, d, L, (uint32_t)ipow3(f.s, L), d_dirs, p->d_adj);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(d_dirs);
  const void *fn = TX == 16 ? (const void *)tile3_kernel<16> : (const void *)tile3_kernel<8>;
  int n = 0, sms = 0;
  if (e == cudaSuccess)
    e = sq_allow_smem(fn, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kT3Threads, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess || n < 1) {
    sq3_tile_free(p);
    return e != cudaSuccess ? sq_cuda_fail(e) : SQUEEZE_ERR_UNSUPPORTED;
  }
  const uint64_t grid = (uint64_t)n * sms;
  p->grid = (int)(grid < d.groups ? grid : d.groups);
  *out = p;
  return SQUEEZE_OK;
}

// One step through the program: rule masks and status of the handle.
int sq3_tile_launch(const Tile3Program *p, uint32_t birth, uint32_t survive, int *status,
                    const uint8_t *in, uint8_t *out, cudaStream_t st) {
  if (((uintptr_t)in | (uintptr_t)out) & 15u) return SQUEEZE_ERR_INVALID_ARG;
  Tile3Dev d = p->dev;
  d.status = status;
  d.nact = 0;
  for (uint32_t n = 0; n <= 26; ++n) {
    const uint32_t b = (birth >> n) & 1u, s = (survive >> n) & 1u;
    if (b | s) d.act[d.nact++] = n | (b << 8) | (s << 9);
  }
  if (p->dev.TX == 16)
    tile3_kernel<16><<<p->grid, p->threads, p->smem, st>>>(d, in, out);
  else
    tile3_kernel<8><<<p->grid, p->threads, p->smem, st>>>(d, in, out);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}
