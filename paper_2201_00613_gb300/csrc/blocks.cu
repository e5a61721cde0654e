// blocks.cu -- block-level Squeeze (Sec. 3.5): the state stored as rho x rho
// expanded micro-boxes.
//
// With rho = s^b, the level-r fractal is the level-(r - b) fractal of level-b
// blocks.  The block-level layout keeps the compact order at level r_b = r - b
// (W_b = k^ceil(r_b / 2) columns, row-major) and stores each block as its
// rho x rho expanded micro-box, holes included (as 0): k^(r - b) * rho^2
// bytes (Sec. 3.5; r_b = r - log_s rho).  A cell's neighbours inside its own
// block are direct; those across the block border are found through the 8
// neighbouring blocks, which nu at block level (Sec. 3.4 on the level-r_b
// fractal, as a carry walk from the block's digits) gives once per block.
// The step stages each block with a one-cell ring in shared memory and
// applies the rule there.  rho = 1 is the compact layout.
#include "squeeze_internal.cuh"

namespace sq {
namespace {

constexpr uint32_t kMaxRho = 32;          // largest micro-box side
constexpr int kBlockThreads = 256;
constexpr uint32_t kMaxBlocksPerCta = 28;  // neighbour tables in shared memory
constexpr uint32_t kTileBytes = 2048;      // micro-boxes with their rings, per CTA pass

struct BlockDev {
  FracDev fb;                 // the level-r_b fractal of blocks
  uint32_t b, rho, rho2;      // block level, micro-box side, cells per block
  uint32_t bpc;               // blocks per CTA pass
  FastDiv div_rho, div_rho2, div_side, div_side2;   // rho, rho^2, rho + 2, (rho + 2)^2
  uint32_t nbhd;              // the cell neighbourhood (the block lookups always use Moore)
  uint8_t mask[kMaxRho * kMaxRho];  // micro-box membership (level-b pattern), row-major
};

// For d = 0..8, the block at offset (d % 3 - 1, d / 3 - 1) from block omega
// (in block units): omega itself for d = 4, ~0 for a hole or off the box.
// The carry walk of nu from omega's own digits stops at the first level
// without a carry.
__device__ inline uint32_t neighbour_block(const FracDev &fb, const SmemTables &t, uint64_t omega,
                                          int d) {
  if (d == 4) return (uint32_t)omega;
  const uint32_t wy = fdiv(fb.divW, (uint32_t)omega), wx = (uint32_t)omega - wy * fb.W;
  uint32_t nx, ny;
  if (!neighbour_omega(fb, t, wx, wy, d % 3 - 1, d / 3 - 1, nx, ny)) return ~0u;
  return ny * fb.W + nx;
}

__global__ void __launch_bounds__(kBlockThreads) block_step_kernel(BlockDev B, Rule rule,
                                                                  const uint8_t *__restrict__ in,
                                                                  uint8_t *__restrict__ out) {
  __shared__ SmemTables t;
  __shared__ uint32_t nb[kMaxBlocksPerCta][9];
  __shared__ uint8_t m[kMaxRho * kMaxRho];
  // each block's micro-box with a one-cell ring from its neighbours, (rho + 2)^2 bytes
  __shared__ uint8_t tile[kTileBytes];
  load_tables(t, B.fb);
  for (uint32_t i = threadIdx.x; i < B.rho2; i += blockDim.x) m[i] = B.mask[i];
  const uint64_t nblocks = B.fb.cells;
  const uint32_t rho = B.rho, rho2 = B.rho2, bpc = B.bpc, side = rho + 2, side2 = side * side;
  const uint32_t nbhd = B.nbhd;
  for (uint64_t base = (uint64_t)blockIdx.x * bpc; base < nblocks;
       base += (uint64_t)gridDim.x * bpc) {
    __syncthreads();  // tables loaded / previous pass done with nb and the tiles
    if (threadIdx.x < bpc * 9) {
      const uint32_t j = threadIdx.x / 9, d = threadIdx.x % 9;
      nb[j][d] = base + j < nblocks ? neighbour_block(B.fb, t, base + j, (int)d) : ~0u;
    }
    __syncthreads();
    // Fill the tiles: consecutive threads take consecutive bytes of a tile row.
    for (uint32_t c = threadIdx.x; c < bpc * side2; c += blockDim.x) {
      const uint32_t j = fdiv(B.div_side2, c), e = c - j * side2;
      const uint32_t ty = fdiv(B.div_side, e), tx = e - ty * side;
      const int qx = (int)tx - 1, qy = (int)ty - 1;
      const int bx = qx < 0 ? -1 : (qx >= (int)rho ? 1 : 0);
      const int by = qy < 0 ? -1 : (qy >= (int)rho ? 1 : 0);
      const uint32_t nbo = base + j < nblocks ? nb[j][(by + 1) * 3 + (bx + 1)] : ~0u;
      uint8_t v = 0;
      if (nbo != ~0u) {
        const uint32_t q = (uint32_t)((qy - by * (int)rho) * (int)rho + (qx - bx * (int)rho));
        v = in[(uint64_t)nbo * rho2 + q] & 1u;
      }
      tile[c] = v;
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < bpc * rho2; c += blockDim.x) {
      const uint32_t j = fdiv(B.div_rho2, c), cell = c - j * rho2;
      const uint64_t omega = base + j;
      if (omega >= nblocks) break;
      const uint32_t ly = fdiv(B.div_rho, cell), lx = cell - ly * rho;
      const uint8_t *w = tile + j * side2 + ly * side + lx;   // the 3 x 3 window's top-left
      uint32_t count;
      if (nbhd == kMoore) {
        count = w[0] + w[1] + w[2] + w[side] + w[side + 2] + w[2 * side] + w[2 * side + 1] +
                w[2 * side + 2];
      } else {
        count = 0;
#pragma unroll
        for (int d = 0; d < 9; ++d)
          if (d != 4 && ((nbhd >> d) & 1u)) count += w[(d / 3) * side + d % 3];
      }
      out[omega * rho2 + cell] =
          m[cell] ? (uint8_t)apply_rule(rule, w[side + 1], count) : (uint8_t)0;
    }
  }
}

// Seeded Bernoulli start in block layout, keyed by expanded position exactly
// as squeeze_init_bernoulli; micro-box holes are 0.
__global__ void __launch_bounds__(kBlockThreads) block_init_kernel(BlockDev B, uint8_t *out,
                                                                  uint64_t seed, uint32_t p_q24) {
  __shared__ SmemTables t;
  load_tables(t, B.fb);
  __syncthreads();
  const uint64_t total = B.fb.cells * B.rho2;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t omega = i / B.rho2;
    const uint32_t cell = (uint32_t)(i - omega * B.rho2);
    uint8_t v = 0;
    if (B.mask[cell]) {
      const uint32_t wy = fdiv(B.fb.divW, (uint32_t)omega), wx = (uint32_t)omega - wy * B.fb.W;
      uint32_t X, Y;
      lambda_alu(B.fb, t, wx, wy, X, Y);
      v = bernoulli_cell(seed, p_q24, X * B.rho + cell % B.rho, Y * B.rho + cell / B.rho);
    }
    out[i] = v;
  }
}

// Compact state (level r) from the block layout: cell omega of the level-r
// fractal sits at lambda(omega); its block is nu (block level) of that
// position divided by rho, and its place in the micro-box the remainder.
__global__ void __launch_bounds__(kBlockThreads) block_gather_kernel(FracDev f, BlockDev B,
                                                                    const uint8_t *__restrict__ in,
                                                                    uint8_t *__restrict__ out) {
  __shared__ SmemTables t, tb;
  load_tables(t, f);
  load_tables(tb, B.fb);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t wy = (uint32_t)(i / f.W), wx = (uint32_t)(i - (uint64_t)wy * f.W);
    uint32_t x, y, bx, by;
    lambda_alu(f, t, wx, wy, x, y);
    uint8_t v = 0;
    if (nu_alu(B.fb, tb, (int32_t)(x / B.rho), (int32_t)(y / B.rho), bx, by))
      v = in[((uint64_t)by * B.fb.W + bx) * B.rho2 + (y % B.rho) * B.rho + x % B.rho] & 1u;
    out[i] = v;
  }
}

// Block-level descriptor for level b of handle h (b <= r, s^b <= kMaxRho).
int make_block_dev(const squeeze_handle *h, uint32_t b, BlockDev &B) {
  const FracDev &f = h->f;
  if (b > f.r) return SQUEEZE_ERR_INVALID_ARG;
  uint64_t rho = 1;
  for (uint32_t i = 0; i < b; ++i) rho *= f.s;
  if (rho > kMaxRho) return SQUEEZE_ERR_UNSUPPORTED;
  uint8_t offsets[2 * 256];
  for (uint32_t i = 0; i < f.k; ++i) {
    offsets[2 * i] = f.taux[i];
    offsets[2 * i + 1] = f.tauy[i];
  }
  memset(&B, 0, sizeof(B));
  int rc = sq_fill_fractal(f.s, f.k, offsets, f.r - b, B.fb);
  if (rc) return rc;
  if (B.fb.cells >= (1ull << 32)) return SQUEEZE_ERR_UNSUPPORTED;   // block indices are 32-bit
  B.b = b;
  B.nbhd = f.nbhd;
  B.rho = (uint32_t)rho;
  B.rho2 = (uint32_t)(rho * rho);
  // as many blocks per pass as their tiles fit (<= 28: one neighbour lookup per thread)
  uint32_t bpc = kTileBytes / ((B.rho + 2) * (B.rho + 2));
  B.bpc = bpc < 1 ? 1 : (bpc > kMaxBlocksPerCta ? kMaxBlocksPerCta : bpc);
  B.div_rho = make_fastdiv(B.rho);
  B.div_rho2 = make_fastdiv(B.rho2);
  B.div_side = make_fastdiv(B.rho + 2);
  B.div_side2 = make_fastdiv((B.rho + 2) * (B.rho + 2));
  if ((uint64_t)B.bpc * (B.rho + 2) * (B.rho + 2) > kTileBytes) return SQUEEZE_ERR_UNSUPPORTED;
  // micro-box membership: every base-s digit pair of (x, y) below level b is an offset
  for (uint32_t y = 0; y < rho; ++y)
    for (uint32_t x = 0; x < rho; ++x) {
      bool member = true;
      for (uint32_t i = 0, ux = x, uy = y; i < b; ++i, ux /= f.s, uy /= f.s)
        member = member && f.hnu[(uy % f.s) * f.s + ux % f.s] != kHole;
      B.mask[y * rho + x] = member ? 1 : 0;
    }
  return SQUEEZE_OK;
}

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" {

int squeeze_block_bytes(const squeeze_handle *h, uint32_t b, uint64_t *bytes) {
  if (!h || !bytes) return SQUEEZE_ERR_INVALID_ARG;
  BlockDev B;
  int rc = make_block_dev(h, b, B);
  if (rc) return rc;
  *bytes = B.fb.cells * B.rho2;
  return SQUEEZE_OK;
}

int squeeze_block_init(const squeeze_handle *h, uint32_t b, uint8_t *d_blocks, uint64_t seed,
                       uint32_t p_q24, void *stream) {
  if (!h || !d_blocks || p_q24 > (1u << 24)) return SQUEEZE_ERR_INVALID_ARG;
  BlockDev B;
  int rc = make_block_dev(h, b, B);
  if (rc) return rc;
  block_init_kernel<<<grid_for(B.fb.cells * B.rho2, kBlockThreads), kBlockThreads, 0,
                      (cudaStream_t)stream>>>(B, d_blocks, seed, p_q24);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int squeeze_block_step(const squeeze_handle *h, uint32_t b, uint8_t *d_blocks0,
                       uint8_t *d_blocks1, uint64_t n_steps, void *stream) {
  if (!h || !d_blocks0 || !d_blocks1 || d_blocks0 == d_blocks1) return SQUEEZE_ERR_INVALID_ARG;
  BlockDev B;
  int rc = make_block_dev(h, b, B);
  if (rc) return rc;
  const uint64_t passes = (B.fb.cells + B.bpc - 1) / B.bpc;
  const unsigned grid = grid_for(passes * kBlockThreads, kBlockThreads);
  uint8_t *a = d_blocks0, *c = d_blocks1;
  for (uint64_t s = 0; s < n_steps; ++s) {
    block_step_kernel<<<grid, kBlockThreads, 0, (cudaStream_t)stream>>>(B, h->rule, a, c);
    SQ_CUDA(cudaGetLastError());
    uint8_t *tmp = a;
    a = c;
    c = tmp;
  }
  return SQUEEZE_OK;
}

int squeeze_block_to_compact(const squeeze_handle *h, uint32_t b, const uint8_t *d_blocks,
                             uint8_t *d_state, void *stream) {
  if (!h || !d_blocks || !d_state) return SQUEEZE_ERR_INVALID_ARG;
  BlockDev B;
  int rc = make_block_dev(h, b, B);
  if (rc) return rc;
  block_gather_kernel<<<grid_for(h->f.cells, kBlockThreads), kBlockThreads, 0,
                        (cudaStream_t)stream>>>(h->f, B, d_blocks, d_state);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

}  // extern "C"
