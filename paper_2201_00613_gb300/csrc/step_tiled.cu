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
// whether that block is a tile, a hole or off the box is decided per tile on
// the device by a carry walk over the tile's higher replica digits (the
// digit-level form of nu, Sec. 3.4), which stops at the first level without
// a carry.
//
// A CTA owns a group of up to 32 tiles lying side by side in compact x.  It
// stages their bytes in shared memory, transposes them so that bit i of word
// c is the state of local cell c in tile i, runs the rule on whole words with
// a bit-sliced adder (32 cells per bitwise operation), transposes back and
// writes the group's bytes.  Reads and writes of the compact buffers are
// coalesced 16-byte accesses; only halo bytes are single-byte loads.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "squeeze_internal.cuh"

struct TiledProgram {
  uint32_t L, TW, TH, cells, nhalo;
  uint32_t dir_mask;        // bit d set when some halo slot uses direction d
  uint32_t tiles_x, tiles_y, groups_per_band;
  uint64_t groups;
  uint32_t pitch;           // bytes per staging row
  size_t smem;
  int grid;
  uint16_t *d_refs;         // cells x 8 local references
  uint64_t *d_halo_off;     // nhalo byte offsets inside a tile (ly * W + lx)
  uint8_t *d_halo_dir;      // nhalo directions, (dy + 1) * 3 + (dx + 1)
};

namespace sq {
namespace {

constexpr int kTiledThreads = 256;
constexpr int kTiledWarps = kTiledThreads / 32;
constexpr size_t kTiledSmemCap = 48 * 1024;

struct TiledDev {
  FracDev f;
  Rule rule;
  uint32_t L, TW, TH, cells, nhalo, dir_mask;
  uint32_t tiles_x, tiles_y, groups_per_band, pitch;
  uint64_t groups;
  FastDiv div_tw, div_gpb;
  const uint16_t *refs;
  const uint64_t *halo_off;
  const uint8_t *halo_dir;
  int *status;
};

__device__ __forceinline__ void flag(int *status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

// Outer-totalistic rule on 32 cells at once: n[0..7] are the neighbour bits.
__device__ __forceinline__ uint32_t rule_word(const Rule &rule, uint32_t self, const uint32_t *n) {
  uint32_t s0 = n[0] ^ n[1] ^ n[2], c0 = maj3(n[0], n[1], n[2]);
  uint32_t s1 = n[3] ^ n[4] ^ n[5], c1 = maj3(n[3], n[4], n[5]);
  uint32_t s2 = n[6] ^ n[7], c2 = n[6] & n[7];
  uint32_t b0 = s0 ^ s1 ^ s2, c3 = maj3(s0, s1, s2);
  uint32_t t = c0 ^ c1 ^ c2, u = maj3(c0, c1, c2);
  uint32_t b1 = t ^ c3, v = t & c3;
  uint32_t b2 = u ^ v, b3 = u & v;
  uint32_t next = 0, any = rule.birth | rule.survive;
#pragma unroll
  for (uint32_t c = 0; c <= 8; ++c) {
    if (!((any >> c) & 1u)) continue;
    uint32_t e = ((c & 1u) ? b0 : ~b0) & ((c & 2u) ? b1 : ~b1) & ((c & 4u) ? b2 : ~b2) &
                 ((c & 8u) ? b3 : ~b3);
    bool bb = (rule.birth >> c) & 1u, ss = (rule.survive >> c) & 1u;
    next |= bb && ss ? e : (bb ? (e & ~self) : (e & self));
  }
  return next;
}

// Carry walk: the level-L block adjacent to tile (tx, ty) in direction
// (dx, dy), as a tile (ntx, nty), or false for a hole / off the box.
__device__ bool adjacent_tile(const TiledDev &p, const uint8_t *taux, const uint8_t *tauy,
                              const uint8_t *hnu, uint32_t tx, uint32_t ty, int dx, int dy,
                              uint32_t &ntx, uint32_t &nty) {
  const FracDev &f = p.f;
  int cx = dx, cy = dy;
  uint32_t qx = tx, qy = ty, pwx = 1, pwy = 1;
  int64_t ax = tx, ay = ty;
  for (uint32_t mu = p.L + 1; mu <= f.r && (cx | cy); ++mu) {
    bool odd = mu & 1u;
    uint32_t src = odd ? qx : qy;
    uint32_t q = fdiv(f.divk, src);
    uint32_t beta = src - q * f.k;
    if (odd) qx = q; else qy = q;
    int ox = (int)taux[beta] + cx, oy = (int)tauy[beta] + cy;
    cx = ox < 0 ? -1 : (ox >= (int)f.s ? 1 : 0);
    cy = oy < 0 ? -1 : (oy >= (int)f.s ? 1 : 0);
    ox -= cx * (int)f.s;
    oy -= cy * (int)f.s;
    uint32_t nb = hnu[oy * f.s + ox];
    if (nb == kHole) return false;
    int64_t delta = (int64_t)nb - (int64_t)beta;
    if (odd) {
      ax += delta * pwx;
      pwx *= f.k;
    } else {
      ay += delta * pwy;
      pwy *= f.k;
    }
  }
  if (cx | cy) return false;  // carried past the top level: off the box
  ntx = (uint32_t)ax;
  nty = (uint32_t)ay;
  return true;
}

__global__ void __launch_bounds__(kTiledThreads) step_tiled_kernel(TiledDev p,
                                                                   const uint8_t *__restrict__ in,
                                                                   uint8_t *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t cells = p.cells, nhalo = p.nhalo;
  // Shared-memory carve-up (all offsets multiples of 16 bytes).
  uint16_t *refs = reinterpret_cast<uint16_t *>(smem);                       // cells * 8
  size_t off = ((size_t)cells * 16 + 15) & ~(size_t)15;
  uint32_t *win = reinterpret_cast<uint32_t *>(smem + off);                  // cells + nhalo + 1
  off += (((size_t)cells + nhalo + 1) * 4 + 15) & ~(size_t)15;
  uint32_t *wout = reinterpret_cast<uint32_t *>(smem + off);                 // cells
  off += ((size_t)cells * 4 + 15) & ~(size_t)15;
  uint64_t *adj = reinterpret_cast<uint64_t *>(smem + off);                  // 9 * 32
  off += 9 * 32 * 8;
  uint32_t *row_a = reinterpret_cast<uint32_t *>(smem + off);                // TH
  off += ((size_t)p.TH * 4 + 15) & ~(size_t)15;
  uint8_t *tab = smem + off;                                                 // 3 * 256
  off += 3 * 256;
  uint8_t *stage = smem + off;                                               // TH * pitch

  const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t i = tid; i < cells * 8; i += blockDim.x) refs[i] = p.refs[i];
  for (uint32_t i = tid; i < 256; i += blockDim.x) {
    tab[i] = p.f.taux[i];
    tab[256 + i] = p.f.tauy[i];
    tab[512 + i] = p.f.hnu[i];
  }
  if (tid == 0) win[cells + nhalo] = 0u;  // the "no neighbour" word
  const uint64_t total = p.f.cells, W = p.f.W;

  for (uint64_t g = blockIdx.x; g < p.groups; g += gridDim.x) {
    const uint32_t ty = fdiv(p.div_gpb, (uint32_t)g);  // groups < 2^32 checked on the host
    const uint32_t tx0 = ((uint32_t)g - ty * p.groups_per_band) * 32u;
    const uint32_t ntiles = min(32u, p.tiles_x - tx0);
    const uint32_t seg = ntiles * p.TW;  // bytes of this group in one compact row

    // Phase 1: stage the group's rows (16-byte aligned chunks) with cp.async;
    // warp 0 also resolves each tile's adjacent blocks.
    for (uint32_t ly = tid; ly < p.TH; ly += blockDim.x) {
      uint64_t S = ((uint64_t)ty * p.TH + ly) * W + (uint64_t)tx0 * p.TW;
      row_a[ly] = (uint32_t)(S & 15u);
    }
    __syncthreads();
    const uint32_t nchunk = (15u + seg + 15u) / 16u;
    for (uint32_t i = tid; i < p.TH * nchunk; i += blockDim.x) {
      uint32_t ly = i / nchunk, c = i - ly * nchunk;
      uint64_t S = ((uint64_t)ty * p.TH + ly) * W + (uint64_t)tx0 * p.TW;
      uint64_t A = (S & ~(uint64_t)15) + 16ull * c;
      if (A >= S + seg) continue;
      uint8_t *dst = stage + (size_t)ly * p.pitch + 16u * c;
      if (A + 16 <= total) {
        uint32_t sdst = (uint32_t)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst), "l"(in + A));
      } else {
        for (uint32_t b = 0; b < 16; ++b) dst[b] = A + b < total ? in[A + b] : 0;
      }
    }
    if (warp == 0) {
      uint32_t tx = tx0 + lane;
#pragma unroll 1
      for (int d = 0; d < 9; ++d) {
        uint64_t base = ~0ull;
        if (((p.dir_mask >> d) & 1u) && lane < ntiles) {
          uint32_t ntx, nty;
          if (adjacent_tile(p, tab, tab + 256, tab + 512, tx, ty, d % 3 - 1, d / 3 - 1, ntx, nty))
            base = (uint64_t)nty * p.TH * W + (uint64_t)ntx * p.TW;
        }
        adj[d * 32 + lane] = base;
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    // Phase 2: transpose bytes -> words (bit i = tile i) and gather halo words.
    for (uint32_t c = warp; c < cells; c += kTiledWarps) {
      uint32_t ly = fdiv(p.div_tw, c), lx = c - ly * p.TW;
      bool alive = false;
      if (lane < ntiles) alive = stage[(size_t)ly * p.pitch + row_a[ly] + lane * p.TW + lx] != 0;
      uint32_t word = __ballot_sync(0xFFFFFFFFu, alive);
      if (lane == 0) win[c] = word;
    }
    for (uint32_t h = warp; h < nhalo; h += kTiledWarps) {
      uint64_t base = adj[p.halo_dir[h] * 32u + lane];
      bool alive = false;
      if (base != ~0ull) {
        uint64_t a = base + p.halo_off[h];
        if (a < total) alive = in[a] != 0;
        else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
      }
      uint32_t word = __ballot_sync(0xFFFFFFFFu, alive);
      if (lane == 0) win[cells + h] = word;
    }
    __syncthreads();

    // Phase 3: the rule on whole words.
    for (uint32_t c = tid; c < cells; c += blockDim.x) {
      uint4 rr = reinterpret_cast<const uint4 *>(refs)[c];
      uint32_t n[8];
      n[0] = win[rr.x & 0xFFFFu];
      n[1] = win[rr.x >> 16];
      n[2] = win[rr.y & 0xFFFFu];
      n[3] = win[rr.y >> 16];
      n[4] = win[rr.z & 0xFFFFu];
      n[5] = win[rr.z >> 16];
      n[6] = win[rr.w & 0xFFFFu];
      n[7] = win[rr.w >> 16];
      wout[c] = rule_word(p.rule, win[c], n);
    }
    __syncthreads();

    // Phase 4: transpose words -> bytes into the staging rows.
    for (uint32_t c = warp; c < cells; c += kTiledWarps) {
      uint32_t ly = fdiv(p.div_tw, c), lx = c - ly * p.TW;
      uint32_t word = wout[c];
      if (lane < ntiles)
        stage[(size_t)ly * p.pitch + row_a[ly] + lane * p.TW + lx] = (uint8_t)((word >> lane) & 1u);
    }
    __syncthreads();

    // Phase 5: write the group's bytes; partial 16-byte chunks at the two ends
    // of a row segment are written byte by byte (they border other groups).
    for (uint32_t i = tid; i < p.TH * nchunk; i += blockDim.x) {
      uint32_t ly = i / nchunk, c = i - ly * nchunk;
      uint64_t S = ((uint64_t)ty * p.TH + ly) * W + (uint64_t)tx0 * p.TW;
      uint64_t A = (S & ~(uint64_t)15) + 16ull * c;
      if (A >= S + seg) continue;
      const uint8_t *src = stage + (size_t)ly * p.pitch + 16u * c;
      if (A >= S && A + 16 <= S + seg) {
        *reinterpret_cast<uint4 *>(out + A) = *reinterpret_cast<const uint4 *>(src);
      } else {
        for (uint32_t b = 0; b < 16; ++b)
          if (A + b >= S && A + b < S + seg) out[A + b] = src[b];
      }
    }
    __syncthreads();
  }
}

// ---- host side: the level-L neighbour program ------------------------------

uint64_t ipow(uint64_t b, uint32_t e) {
  uint64_t p = 1;
  while (e--) p *= b;
  return p;
}

size_t smem_for(uint32_t cells, uint32_t nhalo, uint32_t TH, uint32_t pitch) {
  size_t off = ((size_t)cells * 16 + 15) & ~(size_t)15;
  off += (((size_t)cells + nhalo + 1) * 4 + 15) & ~(size_t)15;
  off += ((size_t)cells * 4 + 15) & ~(size_t)15;
  off += 9 * 32 * 8;
  off += ((size_t)TH * 4 + 15) & ~(size_t)15;
  off += 3 * 256;
  off += (size_t)TH * pitch;
  return off;
}

uint32_t pitch_for(uint32_t TW) { return ((32u * TW + 30u) / 16u + 1u) * 16u; }

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

void sq_tiled_free(TiledProgram *p) {
  if (!p) return;
  cudaFree(p->d_refs);
  cudaFree(p->d_halo_off);
  cudaFree(p->d_halo_dir);
  delete p;
}

int sq_tiled_default_level(const squeeze_handle *h) {
  const FracDev &f = h->f;
  int best = -1;
  for (uint32_t L = 1; L <= f.r; ++L) {
    uint64_t cells = ipow(f.k, L);
    if (cells > 16384) break;
    uint32_t TW = (uint32_t)ipow(f.k, (L + 1) / 2), TH = (uint32_t)ipow(f.k, L / 2);
    // halo slots are bounded by the perimeter cells times 3
    size_t sm = smem_for((uint32_t)cells, 12u * (uint32_t)ipow(f.s, L) + 8u, TH, pitch_for(TW));
    if (sm <= kTiledSmemCap) best = (int)L;
  }
  return best;
}

int sq_tiled_prepare(squeeze_handle *h) {
  if (h->tiled) return SQUEEZE_OK;
  const FracDev &f = h->f;
  uint32_t L = h->tiled_level ? h->tiled_level : (uint32_t)sq_tiled_default_level(h);
  if ((int)L <= 0 || L > f.r) return SQUEEZE_ERR_UNSUPPORTED;
  uint32_t TW = (uint32_t)ipow(f.k, (L + 1) / 2), TH = (uint32_t)ipow(f.k, L / 2);
  uint32_t cells = TW * TH, side = (uint32_t)ipow(f.s, L);
  if ((uint64_t)side * side > (1ull << 28)) return SQUEEZE_ERR_UNSUPPORTED;

  // Local lambda and its inverse over the level-L box.
  std::vector<int32_t> inv((size_t)side * side, -1);
  std::vector<uint32_t> X(cells), Y(cells);
  for (uint32_t c = 0; c < cells; ++c) {
    local_lambda(f, L, c % TW, c / TW, X[c], Y[c]);
    inv[(size_t)Y[c] * side + X[c]] = (int32_t)c;
  }
  // Neighbour references: local cell, halo slot, or the zero word.
  std::vector<uint32_t> refs((size_t)cells * 8);
  std::vector<uint64_t> halo_key;  // (dir << 32) | local cell in the adjacent block
  const uint32_t kNone = 0xFFFFFFFFu;
  for (uint32_t c = 0; c < cells; ++c) {
    int slot = 0;
    for (int d = 0; d < 9; ++d) {
      if (d == 4) continue;
      int64_t qx = (int64_t)X[c] + d % 3 - 1, qy = (int64_t)Y[c] + d / 3 - 1;
      int bx = qx < 0 ? -1 : (qx >= side ? 1 : 0), by = qy < 0 ? -1 : (qy >= side ? 1 : 0);
      int64_t lxp = qx - (int64_t)bx * side, lyp = qy - (int64_t)by * side;
      int32_t target = inv[(size_t)lyp * side + lxp];
      uint32_t ref = kNone;
      if (target >= 0) {
        if (bx == 0 && by == 0) {
          ref = (uint32_t)target;
        } else {
          uint64_t key = ((uint64_t)((by + 1) * 3 + (bx + 1)) << 32) | (uint32_t)target;
          size_t i = 0;
          while (i < halo_key.size() && halo_key[i] != key) ++i;
          if (i == halo_key.size()) halo_key.push_back(key);
          ref = cells + (uint32_t)i;
        }
      }
      refs[(size_t)c * 8 + slot++] = ref;
    }
  }
  uint32_t nhalo = (uint32_t)halo_key.size();
  if ((uint64_t)cells + nhalo + 1 > 0xFFFFu) return SQUEEZE_ERR_UNSUPPORTED;
  std::vector<uint16_t> refs16((size_t)cells * 8);
  for (size_t i = 0; i < refs.size(); ++i)
    refs16[i] = (uint16_t)(refs[i] == kNone ? cells + nhalo : refs[i]);
  std::vector<uint64_t> halo_off(nhalo);
  std::vector<uint8_t> halo_dir(nhalo);
  uint32_t dir_mask = 0;
  for (uint32_t i = 0; i < nhalo; ++i) {
    uint32_t d = (uint32_t)(halo_key[i] >> 32), lc = (uint32_t)halo_key[i];
    halo_dir[i] = (uint8_t)d;
    halo_off[i] = (uint64_t)(lc / TW) * f.W + lc % TW;
    dir_mask |= 1u << d;
  }

  TiledProgram *p = new TiledProgram;
  memset(p, 0, sizeof(*p));
  p->L = L;
  p->TW = TW;
  p->TH = TH;
  p->cells = cells;
  p->nhalo = nhalo;
  p->dir_mask = dir_mask;
  p->tiles_x = f.W / TW;
  p->tiles_y = f.H / TH;
  p->groups_per_band = (p->tiles_x + 31) / 32;
  p->groups = (uint64_t)p->groups_per_band * p->tiles_y;
  p->pitch = pitch_for(TW);
  p->smem = smem_for(cells, nhalo, TH, p->pitch);
  if (p->groups >= (1ull << 32)) {
    delete p;
    return SQUEEZE_ERR_UNSUPPORTED;
  }
  cudaError_t e = cudaMalloc(&p->d_refs, refs16.size() * 2);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_halo_off, (nhalo ? nhalo : 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_halo_dir, (nhalo ? nhalo : 1));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_refs, refs16.data(), refs16.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nhalo)
    e = cudaMemcpy(p->d_halo_off, halo_off.data(), nhalo * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nhalo)
    e = cudaMemcpy(p->d_halo_dir, halo_dir.data(), nhalo, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p->smem);
  int per_sm = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tiled_kernel, kTiledThreads,
                                                      p->smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    sq_tiled_free(p);
    return sq_cuda_fail(e);
  }
  if (per_sm < 1) {
    sq_tiled_free(p);
    return SQUEEZE_ERR_UNSUPPORTED;
  }
  uint64_t grid = (uint64_t)per_sm * sms;
  p->grid = (int)(grid < p->groups ? grid : p->groups);
  h->tiled = p;
  h->tiled_level = L;
  return SQUEEZE_OK;
}

int sq_launch_step_tiled(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                         cudaStream_t st) {
  const TiledProgram *p = h->tiled;
  if (!p) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)in | (uintptr_t)out) & 15u) return SQUEEZE_ERR_INVALID_ARG;
  TiledDev d;
  d.f = h->f;
  d.rule = h->rule;
  d.L = p->L;
  d.TW = p->TW;
  d.TH = p->TH;
  d.cells = p->cells;
  d.nhalo = p->nhalo;
  d.dir_mask = p->dir_mask;
  d.tiles_x = p->tiles_x;
  d.tiles_y = p->tiles_y;
  d.groups_per_band = p->groups_per_band;
  d.pitch = p->pitch;
  d.groups = p->groups;
  d.div_tw = make_fastdiv(p->TW);
  d.div_gpb = make_fastdiv(p->groups_per_band);
  d.refs = p->d_refs;
  d.halo_off = p->d_halo_off;
  d.halo_dir = p->d_halo_dir;
  d.status = h->d_status;
  step_tiled_kernel<<<p->grid, kTiledThreads, p->smem, st>>>(d, in, out);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}
