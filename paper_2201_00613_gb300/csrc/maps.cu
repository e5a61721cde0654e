// maps.cu -- per-element kernels with the integer-ALU maps:
//   * lambda and nu over arrays (Sec. 3.3, Sec. 3.4),
//   * the seeded Bernoulli initial state keyed by expanded position,
//   * the per-cell step: one thread per compact index omega runs one lambda,
//     forms the 8 Moore neighbours in a virtual expanded space, maps each back
//     with nu (holes and points off the box are dead) and applies the rule
//     into the second buffer (Sec. 3.2 neighbourhood exploration, Sec. 4).
#include <math.h>

#include "squeeze_internal.cuh"

namespace sq {
namespace {

// Split a linear compact index into (w_x, w_y), row-major with W columns.
__device__ inline void split_omega(const FracDev &f, uint64_t omega, uint32_t &wx, uint32_t &wy) {
  if (omega < (1ull << 32)) {
    uint32_t o = (uint32_t)omega;
    wy = fdiv(f.divW, o);
    wx = o - wy * f.W;
  } else {
    wy = (uint32_t)(omega / f.W);
    wx = (uint32_t)(omega - (uint64_t)wy * f.W);
  }
}

__global__ void lambda_kernel(FracDev f, const uint64_t *__restrict__ omega,
                              int32_t *__restrict__ xy, uint64_t count) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t o = omega[i];
    int2 out = make_int2(-1, -1);
    if (o < f.cells) {
      uint32_t wx, wy, x, y;
      split_omega(f, o, wx, wy);
      lambda_alu(f, t, wx, wy, x, y);
      out = make_int2((int32_t)x, (int32_t)y);
    }
    reinterpret_cast<int2 *>(xy)[i] = out;
  }
}

__global__ void nu_kernel(FracDev f, const int32_t *__restrict__ xy, uint64_t *__restrict__ omega,
                          uint64_t count) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    int2 p = reinterpret_cast<const int2 *>(xy)[i];
    uint32_t wx, wy;
    omega[i] = nu_alu(f, t, p.x, p.y, wx, wy) ? (uint64_t)wy * f.W + wx : ~0ull;
  }
}

__global__ void init_kernel(FracDev f, uint8_t *__restrict__ state, uint64_t seed,
                            uint32_t p_q24) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy, x, y;
    split_omega(f, i, wx, wy);
    lambda_alu(f, t, wx, wy, x, y);
    state[i] = bernoulli_cell(seed, p_q24, x, y);
  }
}

__global__ void step_alu_kernel(FracDev f, Rule rule, const uint8_t *__restrict__ in,
                                uint8_t *__restrict__ out) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy, x, y;
    split_omega(f, i, wx, wy);
    lambda_alu(f, t, wx, wy, x, y);
    uint32_t c = 0;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      if (d == 4 || !((f.nbhd >> d) & 1u)) continue;
      int32_t qx = (int32_t)x + d % 3 - 1, qy = (int32_t)y + d / 3 - 1;
      uint32_t nx, ny;
      if (nu_alu(f, t, qx, qy, nx, ny)) c += in[(uint64_t)ny * f.W + nx] & 1u;
    }
    out[i] = (uint8_t)apply_rule(rule, in[i] & 1u, c);
  }
}

// Explicit heat diffusion on the fractal graph (Sec. 1 names PDE solvers
// among the uses of the compact maps): one thread per compact cell finds its
// neighbours (the handle's neighbourhood) by the carry walk of nu from its own
// digits (neighbour_omega); holes and points off the box have no edge.  u'(p) = u(p) + alpha * sum over
// neighbours q of (u(q) - u(p)), in fp32.
__global__ void heat_step_kernel(FracDev f, float alpha, const float *__restrict__ in,
                                 float *__restrict__ out) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy;
    split_omega(f, i, wx, wy);
    const float u = in[i];
    float flow = 0.0f;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      if (d == 4 || !((f.nbhd >> d) & 1u)) continue;
      uint32_t nx, ny;
      if (neighbour_omega(f, t, wx, wy, d % 3 - 1, d / 3 - 1, nx, ny))
        flow += in[(uint64_t)ny * f.W + nx] - u;
    }
    out[i] = u + alpha * flow;
  }
}

// Ising spins on the fractal graph (Sec. 1 names spin-model simulations): one
// half-sweep of checkerboard Metropolis updates, in place.  Spin +1 where bit
// 0 is set; cells with (x + y) % 2 == parity update from their neighbours
// (the mask joins only cells of the other parity, so nothing they read
// changes); dE / 2 = s * (sum of neighbour spins); the spin flips iff
// dE <= 0 or (draw >> 40) < thr[dE / 2], the draw being output number
// y * 2^32 + x of the SplitMix64 stream seeded with this half-sweep's seed.
struct IsingThr {
  uint32_t thr[9];   // floor(exp(-2 e / T) * 2^24) for dE / 2 = e = 1..8; thr[0] unused
};

__global__ void ising_half_kernel(FracDev f, uint8_t *__restrict__ state, uint32_t parity,
                                  uint64_t half_seed, IsingThr T) {
  __shared__ SmemTables t;
  load_tables(t, f);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < f.cells;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t wx, wy, x, y;
    split_omega(f, i, wx, wy);
    lambda_alu(f, t, wx, wy, x, y);
    if (((x + y) & 1u) != parity) continue;
    int h = 0;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      if (d == 4 || !((f.nbhd >> d) & 1u)) continue;
      uint32_t nx, ny;
      if (neighbour_omega(f, t, wx, wy, d % 3 - 1, d / 3 - 1, nx, ny))
        h += (state[(uint64_t)ny * f.W + nx] & 1u) ? 1 : -1;
    }
    const uint8_t v = state[i];
    const int e2 = ((v & 1u) ? 1 : -1) * h;
    bool flip = e2 <= 0;
    if (!flip) {
      const uint64_t draw = splitmix64_at(half_seed, ((uint64_t)y << 32) | x);
      flip = (draw >> 40) < (uint64_t)T.thr[e2];
    }
    if (flip) state[i] = (uint8_t)((v & 1u) ^ 1u);
  }
}

}  // namespace
}  // namespace sq

using namespace sq;

int sq_launch_lambda(const squeeze_handle *h, const uint64_t *omega, int32_t *xy, uint64_t count,
                     cudaStream_t st) {
  lambda_kernel<<<grid_for(count, 256), 256, 0, st>>>(h->f, omega, xy, count);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_nu(const squeeze_handle *h, const int32_t *xy, uint64_t *omega, uint64_t count,
                 cudaStream_t st) {
  nu_kernel<<<grid_for(count, 256), 256, 0, st>>>(h->f, xy, omega, count);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_init(const squeeze_handle *h, uint8_t *state, uint64_t seed, uint32_t p_q24,
                   cudaStream_t st) {
  init_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(h->f, state, seed, p_q24);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_step_alu(const squeeze_handle *h, const uint8_t *in, uint8_t *out,
                       cudaStream_t st) {
  step_alu_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(h->f, h->rule, in, out);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_heat_step(const squeeze_handle *h, const float *in, float *out, float alpha,
                        cudaStream_t st) {
  heat_step_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(h->f, alpha, in, out);
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}

int sq_launch_ising(const squeeze_handle *h, uint8_t *state, uint64_t n_sweeps, uint64_t seed,
                    double temperature, cudaStream_t st) {
  IsingThr T;
  T.thr[0] = 1u << 24;
  for (int e = 1; e <= 8; ++e)
    T.thr[e] = temperature > 0.0 ? (uint32_t)floor(exp(-(2.0 * e) / temperature) * 16777216.0) : 0u;
  for (uint64_t t = 0; t < 2 * n_sweeps; ++t) {
    ising_half_kernel<<<grid_for(h->f.cells, 256), 256, 0, st>>>(
        h->f, state, (uint32_t)(t & 1u), splitmix64_at(seed, t), T);
    SQ_CUDA(cudaGetLastError());
  }
  return SQUEEZE_OK;
}
