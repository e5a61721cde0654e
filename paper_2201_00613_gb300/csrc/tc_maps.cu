// tc_maps.cu -- tensor-core (tcgen05) forms of the lambda / nu sums (Sec. 3.6).
//
// Both maps end in a sum of small integer digits times level weights:
//   lambda (Sec. 3.3):  x = sum_mu tau_x(beta_mu) s^(mu-1),  y = sum_mu tau_y(beta_mu) s^(mu-1)
//   nu (Sec. 3.4):      omega = sum_mu id_mu w_mu,  w_mu = k^((mu-1)/2) for odd mu and
//                       W k^((mu-2)/2) for even mu (omega = w_y W + w_x, row-major compact)
// A CTA of 128 threads computes the digits of 128 points on the integer ALU and
// stages them as the rows of a bf16 matrix A (128 x K, K-major) in shared memory;
// digits are below 256 and so exact in bf16.  The weights sit in a bf16 matrix B
// whose columns are their radix-256 limbs (each limb < 256, exact).  One thread
// issues tcgen05.mma kind::f16 with fp32 accumulation into tensor memory, so
// column l of D holds sum_mu digit_mu * limb_l(w_mu).
//
// Exactness bound: r <= 30 (s^r <= 2^30 with s >= 2), digits <= 254 (k <= 255)
// and limbs <= 255, so every column sum is at most 30 * 254 * 255 < 2^21, far
// below 2^24: every partial sum the tensor core forms is an integer that fp32
// holds exactly, whatever the order of accumulation.  The epilogue reads D
// back (tcgen05.ld) and recombines sum_l D_l 2^(8 l) in 64-bit integers.
//
// Tile shapes: M = 128 points, N = 16 columns (two groups of 8 limbs), K = 64:
//   lambda  columns 0..31 tau_x of levels 1..r, 32..63 tau_y; D columns 0..3 are
//           the limbs of x, 4..7 those of y.
//   nu      two points per row: columns 0..31 the replica ids of the first,
//           32..63 those of the second; D columns 0..7 / 8..15 their omegas.
// The per-cell step stages lambda of 128 cells (one MMA chain) and then its
// 8 Moore neighbours as 4 such neighbour pairs (four chains), gathers the
// neighbours that nu accepted and applies the rule, as the ALU step does.
#include "squeeze_internal.cuh"

namespace sq {
namespace {

constexpr uint32_t kRows = 128;   // points per tile (MMA M)
constexpr uint32_t kN = 16;       // D columns (MMA N)
constexpr uint32_t kK = 64;       // digit columns of every A tile
constexpr uint32_t kTileBytes = kRows * kK * 2;   // one A tile, 16 KiB
constexpr uint32_t kBBytes = kN * kK * 2;         // one B matrix, 2 KiB
enum Mode { kLambda = 0, kNu = 1, kStep = 2 };

// Shared-memory carve-up (bytes from a 128-byte aligned base): the A tiles
// (one for the maps; four for the step, where the lambda tile is reused as
// neighbour pair 0 once its MMA has completed), the two B matrices, the
// tables, the mbarrier, the tensor-memory address and the abort flag.
__host__ __device__ constexpr uint32_t a_tiles(int mode) { return mode == kStep ? 4u : 1u; }
__host__ __device__ constexpr uint32_t off_b(int mode) { return a_tiles(mode) * kTileBytes; }
__host__ __device__ constexpr uint32_t off_tables(int mode) { return off_b(mode) + 2 * kBBytes; }
__host__ __device__ constexpr uint32_t off_mbar(int mode) { return off_tables(mode) + 1536; }
__host__ __device__ constexpr uint32_t smem_bytes(int mode) { return off_mbar(mode) + 16 + 128; }
// Tensor-memory columns: D of lambda at column 0; in the step, neighbour pair
// p at 16 + 16 p (80 columns, rounded up to the allocation's power of two).
__host__ __device__ constexpr uint32_t tmem_cols(int mode) { return mode == kStep ? 128u : 32u; }

// Instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((kN >> 3) << 17) | ((kRows >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of the 16-byte piece (row, k-block kb) of a K-major tile with no
// swizzle: 8-row x 16-byte core matrices, adjacent along K (128 bytes apart),
// 8-row groups K * 16 bytes apart.
__device__ __forceinline__ uint32_t cm_off(uint32_t row, uint32_t kb) {
  return (row >> 3) * (kK * 16u) + kb * 128u + (row & 7u) * 16u;
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29: the K step between core matrices), stride byte
// offset >> 4 (bits 32-45: the step between 8-row groups), descriptor version
// 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((kK * 16u) >> 4) << 32) | (1ull << 46);
}

// bf16 bit pattern of an integer v < 256 (8 significant bits: exact).  The
// staged tables hold these patterns; a hole of H_nu is stored as -0.0 (0x8000),
// an exact zero for the MMA that the digit loop still tells apart.
constexpr uint32_t kHoleBf16 = 0x8000u;
__device__ __forceinline__ uint32_t bf16_of(uint32_t v) {
  return __float_as_uint((float)v) >> 16;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Make this thread's generic shared-memory stores visible to the tensor core
// (async proxy), then a CTA barrier ordered with the tcgen05 operations.
__device__ __forceinline__ void sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
}

// D[128 x 16] (fp32, tensor memory) = A[128 x 64] . B[16 x 64]^T: four K = 16 MMAs.
__device__ __forceinline__ void mma_chain(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr) {
#pragma unroll
  for (uint32_t ks = 0; ks < kK / 16; ++ks) {
    const uint64_t a = sdesc(a_addr + ks * 256u), b = sdesc(b_addr + ks * 256u);
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(ks));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(mbar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for an mbarrier phase: false after ~2 s.
__device__ __forceinline__ bool mbar_wait_2s(uint64_t *m, uint32_t parity) {
  if (mbar_test(m, parity)) return true;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (!mbar_test(m, parity)) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 2000000000ull) return false;
  }
  return true;
}

// 16 consecutive fp32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// sum_l D[first + l] 2^(8 l) over `limbs` columns (each an exact fp32 integer).
__device__ __forceinline__ uint64_t limbs_to_u64(const uint32_t (&v)[16], int first, int limbs) {
  uint64_t o = 0;
#pragma unroll
  for (int l = 0; l < 8; ++l)
    if (l < limbs) o += (uint64_t)(uint32_t)__uint_as_float(v[first + l]) << (8 * l);
  return o;
}

__device__ __forceinline__ void store_half(uint8_t *tile, uint32_t row, uint32_t kb0,
                                           const uint32_t (&w)[16]) {
#pragma unroll
  for (uint32_t b = 0; b < 4; ++b)
    *reinterpret_cast<uint4 *>(tile + cm_off(row, kb0 + b)) =
        make_uint4(w[4 * b], w[4 * b + 1], w[4 * b + 2], w[4 * b + 3]);
}

// Row `row` of the lambda tile: tau_x digits in columns 0..31, tau_y in 32..63.
__device__ __forceinline__ void lambda_row(const FracDev &f, const uint16_t *taux,
                                           const uint16_t *tauy, uint32_t wx, uint32_t wy,
                                           uint8_t *tile, uint32_t row) {
  uint32_t px[16], py[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) px[i] = py[i] = 0;
#pragma unroll
  for (uint32_t c = 0; c < 32; ++c) {   // c = mu - 1
    if (c < f.r) {
      uint32_t &src = (c & 1u) ? wy : wx;   // odd levels take w_x's digits
      const uint32_t q = fdiv(f.divk, src), beta = src - q * f.k;
      src = q;
      px[c >> 1] |= (uint32_t)taux[beta] << (16u * (c & 1u));
      py[c >> 1] |= (uint32_t)tauy[beta] << (16u * (c & 1u));
    }
  }
  store_half(tile, row, 0, px);
  store_half(tile, row, 4, py);
}

// Half `half` of row `row` of a nu tile: the replica ids of (x, y) per level.
// Returns whether (x, y) is a fractal cell (in the box and no hole digit).
__device__ __forceinline__ bool nu_row(const FracDev &f, const uint16_t *hnu, int32_t x,
                                       int32_t y, uint8_t *tile, uint32_t row, uint32_t half) {
  bool ok = x >= 0 && y >= 0 && (uint32_t)x < f.n && (uint32_t)y < f.n;
  uint32_t ux = ok ? (uint32_t)x : 0u, uy = ok ? (uint32_t)y : 0u;
  uint32_t p[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) p[i] = 0;
#pragma unroll
  for (uint32_t c = 0; c < 32; ++c) {
    if (c < f.r) {
      const uint32_t qx = fdiv(f.divs, ux), qy = fdiv(f.divs, uy);
      const uint32_t id = hnu[(uy - qy * f.s) * f.s + (ux - qx * f.s)];
      ux = qx;
      uy = qy;
      ok = ok && id != kHoleBf16;
      p[c >> 1] |= id << (16u * (c & 1u));
    }
  }
  store_half(tile, row, 4 * half, p);
  return ok;
}

__device__ __forceinline__ uint64_t ipow64(uint64_t b, uint32_t e) {
  uint64_t v = 1;
  for (uint32_t i = 0; i < e; ++i) v *= b;
  return v;
}

__device__ __forceinline__ void put_bf16(uint8_t *tile, uint32_t row, uint32_t col, uint32_t v) {
  *reinterpret_cast<uint16_t *>(tile + cm_off(row, col >> 3) + (col & 7u) * 2u) =
      (uint16_t)bf16_of(v);
}

// B matrices (16 x 64, K-major): row n holds one radix-256 limb of the weights.
//   lambda: rows 0..3 limbs of s^c against columns c = 0..31 (x half), rows
//           4..7 the same limbs against columns 32..63 (y half).
//   nu:     rows 0..7 limbs of w_(c+1) against columns c = 0..31, rows 8..15
//           the same against columns 32..63 (second point of the row).
__device__ void build_weights(const FracDev &f, uint8_t *b_lam, uint8_t *b_nu) {
  for (uint32_t i = threadIdx.x; i < kN * kK; i += blockDim.x) {
    const uint32_t n = i / kK, c = i % kK, half = c >> 5, level = c & 31u;
    uint32_t lam = 0, nu = 0;
    if (level < f.r) {
      if (n < 8 && (n >> 2) == half)
        lam = (uint32_t)(ipow64(f.s, level) >> (8u * (n & 3u))) & 255u;
      if ((n >> 3) == half) {
        const uint32_t mu = level + 1;
        const uint64_t w = (mu & 1u) ? ipow64(f.k, (mu - 1) / 2)
                                     : (uint64_t)f.W * ipow64(f.k, (mu - 2) / 2);
        nu = (uint32_t)(w >> (8u * (n & 7u))) & 255u;
      }
    }
    put_bf16(b_lam, n, c, lam);
    put_bf16(b_nu, n, c, nu);
  }
}

__device__ __forceinline__ void flag(int *status, int code) { atomicCAS(status, 0, code); }

template <int kMode>
__global__ void __launch_bounds__(128) tc_kernel(FracDev f, Rule rule, const void *in_,
                                                 void *out_, uint64_t count, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
  uint16_t *taux = reinterpret_cast<uint16_t *>(sm + off_tables(kMode));
  uint16_t *tauy = taux + 256, *hnu = taux + 512;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + off_mbar(kMode));
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + off_mbar(kMode) + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + off_mbar(kMode) + 12);
  uint8_t *tile0 = sm, *b_lam_p = sm + off_b(kMode), *b_nu_p = b_lam_p + kBBytes;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;

  for (uint32_t i = tid; i < 256; i += blockDim.x) {
    taux[i] = (uint16_t)bf16_of(f.taux[i]);
    tauy[i] = (uint16_t)bf16_of(f.tauy[i]);
    hnu[i] = f.hnu[i] == kHole ? (uint16_t)kHoleBf16 : (uint16_t)bf16_of(f.hnu[i]);
  }
  build_weights(f, b_lam_p, b_nu_p);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(tmem_cols(kMode)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_for_mma();
  const uint32_t tmem = *tslot;
  const uint32_t lane_addr = tmem + ((warp * 32u) << 16);   // this warp's 32 lanes
  const uint32_t a0 = saddr(tile0), b_lam = saddr(b_lam_p), b_nu = saddr(b_nu_p);
  uint32_t phase = 0;
  bool pending = false;   // an MMA chain was committed and not yet seen complete

  // Thread 0 waits (bounded) for the committed chain; the CTA barrier then
  // hands the completion to the other threads, which sleep in the barrier
  // instead of polling the mbarrier.
  auto wait_mma = [&]() {
    if (tid == 0) {
      if (mbar_wait_2s(mbar, phase)) {
        pending = false;
      } else {
        flag(status, SQUEEZE_ERR_DEVICE_TIMEOUT);
        *abort_flag = 1;
      }
    }
    phase ^= 1u;
    fence_before();
    __syncthreads();
    fence_after();
  };

  const uint32_t per_tile = kMode == kNu ? 2 * kRows : kRows;
  const uint64_t tiles = (count + per_tile - 1) / per_tile;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    if (kMode == kNu) {
      const int2 *xy = static_cast<const int2 *>(in_);
      uint64_t *omega = static_cast<uint64_t *>(out_);
      const uint64_t i0 = tile * per_tile + tid, i1 = i0 + kRows;
      const int2 p0 = i0 < count ? xy[i0] : make_int2(-1, -1);
      const int2 p1 = i1 < count ? xy[i1] : make_int2(-1, -1);
      const bool ok0 = nu_row(f, hnu, p0.x, p0.y, tile0, tid, 0);
      const bool ok1 = nu_row(f, hnu, p1.x, p1.y, tile0, tid, 1);
      sync_for_mma();
      if (*abort_flag) break;
      if (tid == 0) {
        mma_chain(tmem, a0, b_nu);
        mma_commit(mbar);
      }
      pending = true;
      wait_mma();
      uint32_t v[16];
      tmem_ld16(lane_addr, v);
      if (i0 < count) omega[i0] = ok0 ? limbs_to_u64(v, 0, 8) : ~0ull;
      if (i1 < count) omega[i1] = ok1 ? limbs_to_u64(v, 8, 8) : ~0ull;
      continue;
    }
    // lambda of this tile's 128 points (map mode: the given omegas; step: the cells)
    const uint64_t i = tile * kRows + tid;
    uint64_t o = kMode == kLambda ? (i < count ? static_cast<const uint64_t *>(in_)[i] : ~0ull)
                                  : i;
    const bool valid = i < count && o < f.cells;
    uint32_t wx = 0, wy = 0;
    if (valid) {
      if (o < (1ull << 32)) {
        wy = fdiv(f.divW, (uint32_t)o);
        wx = (uint32_t)o - wy * f.W;
      } else {
        wy = (uint32_t)(o / f.W);
        wx = (uint32_t)(o - (uint64_t)wy * f.W);
      }
    }
    lambda_row(f, taux, tauy, wx, wy, tile0, tid);
    sync_for_mma();
    if (*abort_flag) break;
    if (tid == 0) {
      mma_chain(tmem, a0, b_lam);
      mma_commit(mbar);
    }
    pending = true;
    wait_mma();
    uint32_t v[16];
    tmem_ld16(lane_addr, v);
    const uint32_t x = (uint32_t)limbs_to_u64(v, 0, 4), y = (uint32_t)limbs_to_u64(v, 4, 4);
    if (kMode == kLambda) {
      if (i < count)
        reinterpret_cast<int2 *>(out_)[i] =
            valid ? make_int2((int32_t)x, (int32_t)y) : make_int2(-1, -1);
      continue;
    }
    // step: the 8 Moore neighbours as 4 pairs (nu tile p holds neighbours 2p,
    // 2p+1; tile 0 is free again: the lambda MMA has completed)
    uint32_t okmask = 0;
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t d = j < 4 ? j : j + 1;   // skip the centre of the 3 x 3 block
      const int32_t qx = (int32_t)x + (int32_t)(d % 3) - 1, qy = (int32_t)y + (int32_t)(d / 3) - 1;
      const bool ok = nu_row(f, hnu, qx, qy, tile0 + (j >> 1) * kTileBytes, tid, j & 1u);
      okmask |= (ok && ((f.nbhd >> d) & 1u) ? 1u : 0u) << j;
    }
    sync_for_mma();
    if (*abort_flag) break;
    if (tid == 0) {
#pragma unroll
      for (uint32_t p = 0; p < 4; ++p) mma_chain(tmem + 16u + 16u * p, a0 + p * kTileBytes, b_nu);
      mma_commit(mbar);
    }
    pending = true;
    wait_mma();
    const uint8_t *in = static_cast<const uint8_t *>(in_);
    uint32_t c = 0;
#pragma unroll
    for (uint32_t p = 0; p < 4; ++p) {
      tmem_ld16(lane_addr + 16u + 16u * p, v);
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        if (valid && ((okmask >> (2 * p + h)) & 1u)) {
          const uint64_t w = limbs_to_u64(v, 8 * h, 8);
          if (w < f.cells) c += in[w] & 1u;
          else flag(status, SQUEEZE_ERR_DEVICE_BOUNDS);
        }
      }
    }
    if (valid) static_cast<uint8_t *>(out_)[i] = (uint8_t)apply_rule(rule, in[i] & 1u, c);
  }
  // A chain that timed out may still be in flight: give it one more bounded
  // wait before the tensor memory is released.
  if (pending && tid == 0) mbar_wait_2s(mbar, phase ^ 1u);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols(kMode)));
}

template <int kMode>
int launch_tc(const squeeze_handle *h, const void *in, void *out, uint64_t count,
              cudaStream_t st) {
  if (!count) return SQUEEZE_OK;
  const void *fn = (const void *)tc_kernel<kMode>;
  const int smem = (int)smem_bytes(kMode);
  SQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int sms = 0, sm_smem = 0, reserved = 0;
  SQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  SQ_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
  SQ_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, h->device));
  // Resident CTAs per SM, from the shared-memory footprint, capped at 8 and so
  // that their tensor-memory allocations fit the SM's 512 columns together.
  // (The runtime's occupancy query reports one CTA per SM for these kernels,
  // which halves the throughput; the grid is sized here instead.)
  const int by_smem = sm_smem / (smem + reserved);
  const int tmem_cap = (int)(512u / tmem_cols(kMode));
  int per_sm = by_smem < tmem_cap ? by_smem : tmem_cap;
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  const uint64_t per_tile = kMode == kNu ? 2 * kRows : kRows;
  const uint64_t tiles = (count + per_tile - 1) / per_tile;
  const uint64_t cap = (uint64_t)per_sm * sms;
  const uint64_t grid = tiles < cap ? tiles : cap;
  tc_kernel<kMode><<<(unsigned)grid, kRows, smem, st>>>(h->f, h->rule, in, out, count,
                                                        h->d_status);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

}  // namespace
}  // namespace sq

using namespace sq;

int sq_launch_step_tc(const squeeze_handle *h, const uint8_t *in, uint8_t *out, cudaStream_t st) {
  return launch_tc<kStep>(h, in, out, h->f.cells, st);
}

int sq_launch_map_tc(const squeeze_handle *h, int direction, const void *in, void *out,
                     uint64_t count, cudaStream_t st) {
  return direction == 0 ? launch_tc<kLambda>(h, in, out, count, st)
                        : launch_tc<kNu>(h, in, out, count, st);
}
