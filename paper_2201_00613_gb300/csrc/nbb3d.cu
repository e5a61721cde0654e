// nbb3d.cu -- the compact step on three-dimensional NBB fractals, and its C ABI.
//
// One thread per compact cell: its compact coordinates, the level-1 replica
// id shared by all neighbour walks, up to 26 neighbours found by the carry
// walk of nu (holes and points off the box are dead), and the
// outer-totalistic rule into the second buffer.  The per-cell arithmetic is
// in nbb3d.cuh.
#include <string.h>

#include <new>

#include "nbb3d.cuh"

using sq3::Frac3Dev;
using sq3::Tables3;
using sq::grid_for;

struct squeeze_3d_handle {
  Frac3Dev f;
  int *d_status;   // device status word (SQUEEZE_OK / DEVICE_*)
  int device;
  int tiled_level;        // -1: the default level; 0: the per-cell kernel only; else L
  Tile3Program *tiled;    // the tile kernel's program, built on the first step
};

namespace {

constexpr int kThreads = 256;

__device__ inline void load_tables3(Tables3 &t, const Frac3Dev &f) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    t.tau[0][i] = f.tau[0][i];
    t.tau[1][i] = f.tau[1][i];
    t.tau[2][i] = f.tau[2][i];
  }
  for (int i = threadIdx.x; i < 512; i += blockDim.x) t.hnu[i] = f.hnu[i];
}

__global__ void __launch_bounds__(kThreads) step3_kernel(Frac3Dev f, const uint8_t *__restrict__ in,
                                                         uint8_t *__restrict__ out, int *status) {
  __shared__ Tables3 t;
  load_tables3(t, f);
  __syncthreads();
  for (uint64_t omega = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; omega < f.cells;
       omega += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy, wz;
    sq3::split3(f, omega, wx, wy, wz);
    const sq3::Cell3 c = sq3::cell3(f, t, wx, wy, wz);
    uint32_t count = 0;
    if (f.r > 0) {
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        if (d == 13 || !((f.nbhd >> d) & 1u)) continue;
        int64_t delta;
        if (!sq3::neighbour3(f, t, c, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1, delta)) continue;
        const uint64_t nb = omega + (uint64_t)delta;
        if (nb < f.cells) count += in[nb] & 1u;
        else atomicCAS(status, 0, SQUEEZE_ERR_DEVICE_BOUNDS);
      }
    }
    const bool alive = in[omega] & 1u;
    out[omega] = (uint8_t)((((alive ? f.survive : f.birth) >> count) & 1u));
  }
}

__global__ void init3_kernel(uint64_t cells, uint64_t seed, uint32_t p_q24, uint8_t *state) {
  for (uint64_t omega = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; omega < cells;
       omega += (uint64_t)gridDim.x * blockDim.x)
    state[omega] = (uint8_t)((sq::splitmix64_at(seed, omega) >> 40) < (uint64_t)p_q24);
}

__global__ void lambda3_kernel(Frac3Dev f, const uint64_t *__restrict__ omega,
                               int32_t *__restrict__ xyz, uint64_t count) {
  __shared__ Tables3 t;
  load_tables3(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t om = omega[i];
    int32_t X = -1, Y = -1, Z = -1;
    if (om < f.cells) {
      uint32_t wx, wy, wz, x, y, z;
      sq3::split3(f, om, wx, wy, wz);
      sq3::lambda3(f, t, wx, wy, wz, x, y, z);
      X = (int32_t)x;
      Y = (int32_t)y;
      Z = (int32_t)z;
    }
    xyz[3 * i] = X;
    xyz[3 * i + 1] = Y;
    xyz[3 * i + 2] = Z;
  }
}

__global__ void nu3_kernel(Frac3Dev f, const int32_t *__restrict__ xyz, uint64_t *__restrict__ omega,
                           uint64_t count) {
  __shared__ Tables3 t;
  load_tables3(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t om;
    omega[i] = sq3::nu3(f, t, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], om) ? om : ~0ull;
  }
}

bool pow_fits(uint64_t base, uint32_t e, uint64_t limit, uint64_t &out) {
  uint64_t p = 1;
  for (uint32_t i = 0; i < e; ++i) {
    if (p > limit / base) return false;
    p *= base;
  }
  out = p;
  return true;
}

// Validate a 3-D descriptor and fill the kernel-side tables (no device work).
int fill3(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r, Frac3Dev &f) {
  if (!offsets || s < 2 || s > (uint32_t)sq3::kMaxS) return SQUEEZE_ERR_INVALID_ARG;
  if (k < 1 || k > s * s * s || k > (uint32_t)sq3::kMaxK) return SQUEEZE_ERR_INVALID_ARG;
  memset(&f, 0, sizeof(f));
  uint64_t n, cells, Wx, Wy, Wz;
  const uint32_t lx = (r + 2) / 3, ly = (r + 1) / 3, lz = r / 3;
  if (!pow_fits(s, r, 1ull << 30, n) || !pow_fits(k, r, 1ull << 40, cells))
    return SQUEEZE_ERR_INVALID_ARG;
  if (!pow_fits(k, lx, 0xFFFFFFFFull, Wx) || !pow_fits(k, ly, 0xFFFFFFFFull, Wy) ||
      !pow_fits(k, lz, 0xFFFFFFFFull, Wz) || Wy * Wz > 0xFFFFFFFFull)
    return SQUEEZE_ERR_INVALID_ARG;
  memset(f.hnu, sq3::kHole, sizeof(f.hnu));
  for (uint32_t b = 0; b < k; ++b) {
    const uint8_t x = offsets[3 * b], y = offsets[3 * b + 1], z = offsets[3 * b + 2];
    if (x >= s || y >= s || z >= s) return SQUEEZE_ERR_INVALID_ARG;
    uint8_t &slot = f.hnu[(z * s + y) * s + x];
    if (slot != sq3::kHole) return SQUEEZE_ERR_INVALID_ARG;   // repeated offset
    slot = (uint8_t)b;
    f.tau[0][b] = x;
    f.tau[1][b] = y;
    f.tau[2][b] = z;
  }
  f.s = s;
  f.k = k;
  f.r = r;
  f.n = (uint32_t)n;
  f.Wx = (uint32_t)Wx;
  f.Wy = (uint32_t)Wy;
  f.Wz = (uint32_t)Wz;
  f.cells = cells;
  f.plane = Wx * Wy;
  f.divk = sq::make_fastdiv(k);
  f.divs = sq::make_fastdiv(s);
  f.divWx = sq::make_fastdiv((uint32_t)Wx);
  f.divWy = sq::make_fastdiv((uint32_t)Wy);
  f.nbhd = sq3::kMoore26;
  f.birth = 1u << 5;                  // B5/S45
  f.survive = (1u << 4) | (1u << 5);
  return SQUEEZE_OK;
}

}  // namespace

extern "C" {

int squeeze_3d_create(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                      squeeze_3d_handle **out) {
  if (!out) return SQUEEZE_ERR_INVALID_ARG;
  *out = nullptr;
  Frac3Dev f;
  const int rc = fill3(s, k, offsets, r, f);
  if (rc) return rc;
  squeeze_3d_handle *h = new (std::nothrow) squeeze_3d_handle;
  if (!h) return SQUEEZE_ERR_OOM;
  memset(h, 0, sizeof(*h));
  h->tiled_level = -1;
  h->f = f;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return sq_cuda_fail(e);
  }
  *out = h;
  return SQUEEZE_OK;
}

int squeeze_3d_destroy(squeeze_3d_handle *h) {
  if (!h) return SQUEEZE_OK;
  cudaError_t e = cudaDeviceSynchronize();
  sq3_tile_free(h->tiled);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return e == cudaSuccess ? SQUEEZE_OK : sq_cuda_fail(e);
}

int squeeze_3d_info(const squeeze_3d_handle *h, uint64_t *n_cells, uint64_t *wx, uint64_t *wy,
                    uint64_t *wz, uint64_t *side) {
  if (!h) return SQUEEZE_ERR_INVALID_ARG;
  if (n_cells) *n_cells = h->f.cells;
  if (wx) *wx = h->f.Wx;
  if (wy) *wy = h->f.Wy;
  if (wz) *wz = h->f.Wz;
  if (side) *side = h->f.n;
  return SQUEEZE_OK;
}

int squeeze_3d_set_rule(squeeze_3d_handle *h, uint32_t birth, uint32_t survive) {
  if (!h || birth >= (1u << 27) || survive >= (1u << 27)) return SQUEEZE_ERR_INVALID_ARG;
  h->f.birth = birth;
  h->f.survive = survive;
  return SQUEEZE_OK;
}

int squeeze_3d_set_neighbourhood(squeeze_3d_handle *h, uint32_t mask) {
  if (!h || mask >= (1u << 27) || (mask & (1u << 13))) return SQUEEZE_ERR_INVALID_ARG;
  h->f.nbhd = mask;
  if (h->tiled) {   // the program's references depend on the neighbourhood
    const cudaError_t e = cudaDeviceSynchronize();
    sq3_tile_free(h->tiled);
    h->tiled = nullptr;
    if (e != cudaSuccess) return sq_cuda_fail(e);
  }
  return SQUEEZE_OK;
}

int squeeze_3d_lambda(const squeeze_3d_handle *h, const uint64_t *d_omega, int32_t *d_xyz,
                      uint64_t count, void *stream) {
  if (!h || (count && (!d_omega || !d_xyz))) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_omega & 7u) || ((uintptr_t)d_xyz & 3u)) return SQUEEZE_ERR_INVALID_ARG;
  if (!count) return SQUEEZE_OK;
  lambda3_kernel<<<grid_for(count, kThreads), kThreads, 0, (cudaStream_t)stream>>>(h->f, d_omega,
                                                                                  d_xyz, count);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int squeeze_3d_nu(const squeeze_3d_handle *h, const int32_t *d_xyz, uint64_t *d_omega,
                  uint64_t count, void *stream) {
  if (!h || (count && (!d_omega || !d_xyz))) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_omega & 7u) || ((uintptr_t)d_xyz & 3u)) return SQUEEZE_ERR_INVALID_ARG;
  if (!count) return SQUEEZE_OK;
  nu3_kernel<<<grid_for(count, kThreads), kThreads, 0, (cudaStream_t)stream>>>(h->f, d_xyz,
                                                                              d_omega, count);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int squeeze_3d_init_bernoulli(const squeeze_3d_handle *h, uint8_t *d_state, uint64_t seed,
                              uint32_t p_q24, void *stream) {
  if (!h || !d_state || p_q24 > (1u << 24)) return SQUEEZE_ERR_INVALID_ARG;
  init3_kernel<<<grid_for(h->f.cells, kThreads), kThreads, 0, (cudaStream_t)stream>>>(
      h->f.cells, seed, p_q24, d_state);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

// The level the tile kernel runs at for this handle, or 0 for the per-cell kernel.
static uint32_t tiled_level_of(const squeeze_3d_handle *h) {
  if (h->tiled_level == 0) return 0;
  return h->tiled_level > 0 ? (uint32_t)h->tiled_level : sq3_tile_default_level(h->f);
}

int squeeze_3d_step(squeeze_3d_handle *h, uint8_t *d_buf0, uint8_t *d_buf1, uint64_t n_steps,
                    void *stream) {
  if (!h || !d_buf0 || !d_buf1 || d_buf0 == d_buf1) return SQUEEZE_ERR_INVALID_ARG;
  if (!n_steps) return SQUEEZE_OK;
  uint8_t *a = d_buf0, *b = d_buf1;
  const uint32_t L = tiled_level_of(h);
  if (L && !(((uintptr_t)d_buf0 | (uintptr_t)d_buf1) & 15u)) {
    if (!h->tiled) {
      const int rc = sq3_tile_prepare(h->f, L, h->device, &h->tiled);
      if (rc && (rc != SQUEEZE_ERR_UNSUPPORTED || h->tiled_level > 0)) return rc;
    }
    if (h->tiled) {
      for (uint64_t i = 0; i < n_steps; ++i) {
        const int rc = sq3_tile_launch(h->tiled, h->f.birth, h->f.survive, h->d_status, a, b,
                                       (cudaStream_t)stream);
        if (rc) return rc;
        uint8_t *tmp = a;
        a = b;
        b = tmp;
      }
      return SQUEEZE_OK;
    }
  }
  const unsigned grid = grid_for(h->f.cells, kThreads);
  for (uint64_t i = 0; i < n_steps; ++i) {
    step3_kernel<<<grid, kThreads, 0, (cudaStream_t)stream>>>(h->f, a, b, h->d_status);
    SQ_CUDA(cudaGetLastError());
    uint8_t *tmp = a;
    a = b;
    b = tmp;
  }
  return SQUEEZE_OK;
}

int squeeze_3d_set_tiled_level(squeeze_3d_handle *h, uint32_t level) {
  if (!h || level > h->f.r) return SQUEEZE_ERR_INVALID_ARG;
  if (level) {
    uint32_t TX, TY, TZ, slots;
    uint64_t box;
    if (!sq3_tile_shape(h->f, level, TX, TY, TZ, slots, box)) return SQUEEZE_ERR_UNSUPPORTED;
  }
  if (h->tiled) {
    const cudaError_t e = cudaDeviceSynchronize();
    sq3_tile_free(h->tiled);
    h->tiled = nullptr;
    if (e != cudaSuccess) return sq_cuda_fail(e);
  }
  h->tiled_level = (int)level;
  return SQUEEZE_OK;
}

int squeeze_3d_tiled_level(const squeeze_3d_handle *h) {
  if (!h) return SQUEEZE_ERR_INVALID_ARG;
  return (int)tiled_level_of(h);
}

int squeeze_3d_device_status(squeeze_3d_handle *h, int *status) {
  if (!h || !status) return SQUEEZE_ERR_INVALID_ARG;
  SQ_CUDA(cudaDeviceSynchronize());
  int v = 0;
  SQ_CUDA(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  SQ_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
  *status = v;
  return SQUEEZE_OK;
}

}  // extern "C"
