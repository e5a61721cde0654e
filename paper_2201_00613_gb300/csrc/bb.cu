// bb.cu -- expanded bounding-box comparator (Sec. 4, approach "BB").
//
// The whole n x n box is stored, one byte per cell: bit 0 = alive, bit 1 =
// fractal cell.  Holes are marked once at initialisation (value 0) and never
// change, so the step needs no per-cell digit test: a hole simply contributes
// no alive neighbour and is written back as 0.  One thread handles a 16-byte
// column chunk over a strip of rows and computes the neighbour counts of 16
// cells at a time with byte-wise (SWAR) arithmetic.
#include "squeeze_internal.cuh"

namespace sq {
namespace {

constexpr int kBBRows = 64;      // rows per thread strip
constexpr int kBBRing = 8;       // rows in a thread's shared-memory ring (up to 6 in flight)
constexpr int kBBThreads = 256;  // 16-byte chunks per block along a row

__global__ void bb_init_kernel(FracDev f, uint8_t *__restrict__ grid, uint64_t seed,
                               uint32_t p_q24) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  uint64_t total = (uint64_t)f.n * f.n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t y = (uint32_t)(i / f.n), x = (uint32_t)(i - (uint64_t)y * f.n);
    uint32_t ux = x, uy = y;
    bool member = true;
    for (uint32_t mu = 1; mu <= f.r && member; ++mu) {
      uint32_t qx = fdiv(f.divs, ux), qy = fdiv(f.divs, uy);
      member = t.hnu[(uy - qy * f.s) * f.s + (ux - qx * f.s)] != kHole;
      ux = qx;
      uy = qy;
    }
    grid[i] = member ? (uint8_t)(2u | bernoulli_cell(seed, p_q24, x, y)) : (uint8_t)0;
  }
}

// Generic byte-per-thread step (any n, any neighbourhood mask).
__global__ void bb_step_simple(uint32_t n, Rule rule, uint32_t nbhd, const uint8_t *__restrict__ in,
                               uint8_t *__restrict__ out) {
  uint64_t total = (uint64_t)n * n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t y = (uint32_t)(i / n), x = (uint32_t)(i - (uint64_t)y * n);
    uint8_t v = in[i];
    if (!(v & 2)) {
      out[i] = 0;
      continue;
    }
    uint32_t c = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if ((!dx && !dy) || !((nbhd >> ((dy + 1) * 3 + (dx + 1))) & 1u)) continue;
        int64_t qx = (int64_t)x + dx, qy = (int64_t)y + dy;
        if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
        c += in[(uint64_t)qy * n + qx] & 1u;
      }
    out[i] = (uint8_t)(2u | apply_rule(rule, v & 1u, c));
  }
}

// Byte-wise "equals c" over 4 counts in [0, 8]: 0x01 in each byte whose count is c.
__device__ __forceinline__ uint32_t bytes_eq(uint32_t cnt, uint32_t c) {
  uint32_t x = cnt ^ (c * 0x01010101u);  // each byte <= 0x0F
  return (~(x + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
}

// Next alive bits (0x01 per byte) of 4 cells with neighbour counts cnt and
// alive bits `alive`.  kLife: B3/S23 is "count | alive == 3" (a count of 3,
// or 2 with the cell alive); otherwise the masks are evaluated count by count.
template <bool kLife>
__device__ __forceinline__ uint32_t swar_rule(Rule rule, uint32_t cnt, uint32_t alive) {
  if (kLife) return bytes_eq(cnt | alive, 3u);
  uint32_t next = 0;
  uint32_t any = rule.birth | rule.survive;
#pragma unroll
  for (uint32_t c = 0; c <= 8; ++c) {
    if (!((any >> c) & 1u)) continue;
    uint32_t e = bytes_eq(cnt, c);
    bool b = (rule.birth >> c) & 1u, s = (rule.survive >> c) & 1u;
    next |= b && s ? e : (b ? (e & ~alive) : (e & alive));
  }
  return next;
}

struct Row16 {
  uint32_t h[4];  // horizontal 3-sums of the alive bits (one count per byte)
};

__device__ __forceinline__ void make_row(const uint4 &v, uint32_t left, uint32_t right, Row16 &o) {
  uint32_t a[4] = {v.x & 0x01010101u, v.y & 0x01010101u, v.z & 0x01010101u, v.w & 0x01010101u};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t lw = j ? (a[j - 1] >> 24) : (left & 1u);
    uint32_t rw = j < 3 ? (a[j + 1] << 24) : ((right & 1u) << 24);
    uint32_t L = (a[j] << 8) | lw;
    uint32_t R = (a[j] >> 8) | rw;
    o.h[j] = a[j] + L + R;
  }
}

// Asynchronous 16-byte global -> shared copies (cp.async, tracked per thread
// in commit groups; no registers are held while a copy is in flight).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int kN>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kN) : "memory");
}

// SWAR step; requires n % 16 == 0.  Block: kBBThreads consecutive 16-byte
// chunks of a row; grid.y: strips of kBBRows rows.  Every thread streams its
// column of chunks through a ring of kBBRing rows in shared memory with
// cp.async, so up to kBBRing - 2 rows of loads are in flight per thread
// without holding registers; the warp's edge lanes also stream the chunk just
// outside the warp for the edge byte.  A thread reads only its own ring
// slots, so no barrier is needed.  The horizontal 3-sums of the rows above,
// at and below the row computed roll through registers.  Each row is read
// (kBBRows + 2) / kBBRows times (3 % more than once).
template <bool kLife>
__global__ void __launch_bounds__(kBBThreads) bb_step_swar(uint32_t n, Rule rule,
                                                           const uint8_t *__restrict__ in,
                                                           uint8_t *__restrict__ out) {
  __shared__ __align__(16) uint4 ring[kBBRing][kBBThreads];
  __shared__ __align__(16) uint4 edge[kBBRing][kBBThreads / 32][2];
  const uint32_t nchunks = n / 16;
  const uint32_t chunk = blockIdx.x * kBBThreads + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const int64_t y0 = (int64_t)blockIdx.y * kBBRows;
  const int64_t y_last = y0 + kBBRows;   // the strip's last neighbour row
  // Row y into ring slot `slot` (zeros off the box, past the row, or past the
  // strip's rows), as one commit group.
  auto issue = [&](int64_t y, int slot) {
    const bool in_box = y >= 0 && y < (int64_t)n && y <= y_last;
    const uint8_t *row = in + (uint64_t)(in_box ? y : 0) * n;
    uint4 *dst = &ring[slot][threadIdx.x];
    if (in_box && chunk < nchunks) cp_async16(dst, row + (uint64_t)chunk * 16);
    else *dst = make_uint4(0, 0, 0, 0);
    if (lane == 0) {
      uint4 *e = &edge[slot][warp][0];
      if (in_box && chunk > 0 && chunk < nchunks) cp_async16(e, row + (uint64_t)(chunk - 1) * 16);
      else *e = make_uint4(0, 0, 0, 0);
    }
    if (lane == 31) {
      uint4 *e = &edge[slot][warp][1];
      if (in_box && chunk + 1 < nchunks) cp_async16(e, row + (uint64_t)(chunk + 1) * 16);
      else *e = make_uint4(0, 0, 0, 0);
    }
    cp_async_commit();
  };
  // Horizontal sums of the row in `slot` (edge bytes from the neighbouring
  // lanes, or from the edge chunks for the warp's edge lanes).
  auto sums = [&](int slot, uint4 &v, Row16 &o) {
    v = ring[slot][threadIdx.x];
    uint32_t left = __shfl_up_sync(0xFFFFFFFFu, v.w >> 24, 1);
    uint32_t right = __shfl_down_sync(0xFFFFFFFFu, v.x, 1) & 0xFFu;
    if (lane == 0) left = edge[slot][warp][0].w >> 24;
    if (lane == 31) right = edge[slot][warp][1].x & 0xFFu;
    make_row(v, left, right, o);
  };
  // row y0 - 1 + k -> slot k % kBBRing
#pragma unroll
  for (int k = 0; k < kBBRing; ++k) issue(y0 - 1 + k, k);
  cp_async_wait<kBBRing - 2>();   // rows y0 - 1 and y0 have landed
  Row16 up, cur;
  uint4 vup, vcur;
  sums(0, vup, up);
  sums(1, vcur, cur);
  for (int i0 = 0; i0 < kBBRows; i0 += kBBRing) {
#pragma unroll
    for (int k = 0; k < kBBRing; ++k) {
      const int64_t y = y0 + i0 + k;
      if (y >= n) break;  // uniform across the block
      cp_async_wait<kBBRing - 3>();   // row y + 1 has landed
      Row16 dn;
      uint4 vnext;
      sums((k + 2) % kBBRing, vnext, dn);
      issue(y - 1 + kBBRing, k % kBBRing);   // the slot of row y - 1 is free now
      if (chunk < nchunks) {
        const uint32_t w[4] = {vcur.x, vcur.y, vcur.z, vcur.w};
        uint32_t o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t alive = w[j] & 0x01010101u;
          const uint32_t cnt = up.h[j] + dn.h[j] + cur.h[j] - alive;
          const uint32_t next = swar_rule<kLife>(rule, cnt, alive);
          o[j] = (w[j] & 0x02020202u) | (next & (w[j] >> 1) & 0x01010101u);
        }
        reinterpret_cast<uint4 *>(out + (uint64_t)y * n)[chunk] = make_uint4(o[0], o[1], o[2], o[3]);
      }
      up = cur;
      cur = dn;
      vcur = vnext;
    }
  }
  cp_async_wait<0>();   // nothing left in flight when the block ends
}

__global__ void bb_gather_kernel(FracDev f, const uint8_t *__restrict__ grid,
                                 uint8_t *__restrict__ state) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wy = (uint32_t)(i / f.W), wx = (uint32_t)(i - (uint64_t)wy * f.W);
    uint32_t x, y;
    lambda_alu(f, t, wx, wy, x, y);
    state[i] = grid[(uint64_t)y * f.n + x] & 1u;
  }
}

// The lambda(omega) approach (Sec. 2, the compact thread grid over expanded
// memory): one thread per compact index omega finds its cell with lambda, reads
// its 8 Moore neighbours directly in the box (holes hold 0, points off the box
// are skipped) and writes its new state at the same place of the second box.
// No nu is needed, but the memory is the whole box; holes are never written.
__global__ void lambda_step_kernel(FracDev f, Rule rule, const uint8_t *__restrict__ in,
                                   uint8_t *__restrict__ out) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  const uint32_t n = f.n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy, x, y;
    if (i < (1ull << 32)) {
      wy = fdiv(f.divW, (uint32_t)i);
      wx = (uint32_t)i - wy * f.W;
    } else {
      wy = (uint32_t)(i / f.W);
      wx = (uint32_t)(i - (uint64_t)wy * f.W);
    }
    lambda_alu(f, t, wx, wy, x, y);
    uint32_t c = 0;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      if (d == 4 || !((f.nbhd >> d) & 1u)) continue;
      const int64_t qx = (int64_t)x + d % 3 - 1, qy = (int64_t)y + d / 3 - 1;
      if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
      c += in[(uint64_t)qy * n + (uint64_t)qx] & 1u;
    }
    const uint64_t at = (uint64_t)y * n + x;
    out[at] = (uint8_t)(2u | apply_rule(rule, in[at] & 1u, c));
  }
}

}  // namespace
}  // namespace sq

using namespace sq;

int sq_launch_bb_init(const squeeze_handle *h, uint8_t *grid, uint64_t seed, uint32_t p_q24,
                      cudaStream_t st) {
  uint64_t total = (uint64_t)h->f.n * h->f.n;
  bb_init_kernel<<<grid_for(total, 256), 256, 0, st>>>(h->f, grid, seed, p_q24);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_bb_step(const squeeze_handle *h, const uint8_t *in, uint8_t *out, cudaStream_t st) {
  uint32_t n = h->f.n;
  if (h->f.nbhd == kMoore && n % 16 == 0 && ((uintptr_t)in % 16 == 0) &&
      ((uintptr_t)out % 16 == 0)) {
    uint32_t nchunks = n / 16;
    dim3 grid((nchunks + kBBThreads - 1) / kBBThreads, (n + kBBRows - 1) / kBBRows);
    const bool life = h->rule.birth == (1u << 3) && h->rule.survive == ((1u << 2) | (1u << 3));
    if (life) bb_step_swar<true><<<grid, kBBThreads, 0, st>>>(n, h->rule, in, out);
    else bb_step_swar<false><<<grid, kBBThreads, 0, st>>>(n, h->rule, in, out);
  } else {
    uint64_t total = (uint64_t)n * n;
    bb_step_simple<<<grid_for(total, 256), 256, 0, st>>>(n, h->rule, h->f.nbhd, in, out);
  }
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_bb_gather(const squeeze_handle *h, const uint8_t *grid, uint8_t *state,
                        cudaStream_t st) {
  bb_gather_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(h->f, grid, state);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_lambda_step(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                          cudaStream_t st) {
  lambda_step_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(h->f, h->rule, in, out);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}
