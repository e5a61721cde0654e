// handle.cu -- descriptor validation, per-fractal tables and the C-ABI
// entry points that dispatch to the kernels.
//
// The per-fractal tables are the two look-up tables of the paper: H_lambda
// (replica id -> offset, Sec. 3.3, Eq. tau) and H_nu (digit pair -> replica id,
// Sec. 3.4), the latter widened to s*s entries with a hole marker.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "squeeze_internal.cuh"

namespace {

thread_local char g_last_cuda_error[256] = "";

bool fits_pow(uint64_t base, uint32_t e, uint64_t limit, uint64_t *out) {
  uint64_t p = 1;
  for (uint32_t i = 0; i < e; ++i) {
    if (p > limit / base) return false;
    p *= base;
  }
  *out = p;
  return p <= limit;
}

int check_handle(const squeeze_handle *h) { return h ? SQUEEZE_OK : SQUEEZE_ERR_INVALID_ARG; }

}  // namespace

// Validate an NBB descriptor and fill the kernel-side tables (no device work).
int sq_fill_fractal(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r, sq::FracDev &f) {
  if (!offsets) return SQUEEZE_ERR_INVALID_ARG;
  if (s < 2 || s > (uint32_t)sq::kMaxS) return SQUEEZE_ERR_INVALID_ARG;
  if (k < 1 || k > s * s || k > (uint32_t)sq::kMaxK) return SQUEEZE_ERR_INVALID_ARG;
  if (r > 62) return SQUEEZE_ERR_INVALID_ARG;
  uint64_t n, W, H;
  if (!fits_pow(s, r, 1ull << 30, &n)) return SQUEEZE_ERR_INVALID_ARG;
  if (!fits_pow(k, (r + 1) / 2, 0xFFFFFFFFull, &W)) return SQUEEZE_ERR_INVALID_ARG;
  if (!fits_pow(k, r / 2, 0xFFFFFFFFull, &H)) return SQUEEZE_ERR_INVALID_ARG;
  memset(&f, 0, sizeof(f));
  f.s = s;
  f.k = k;
  f.r = r;
  f.n = (uint32_t)n;
  f.W = (uint32_t)W;
  f.H = (uint32_t)H;
  f.cells = W * H;
  f.divk = sq::make_fastdiv(k);
  f.divs = sq::make_fastdiv(s);
  f.divW = sq::make_fastdiv((uint32_t)W);
  f.nbhd = sq::kMoore;
  memset(f.hnu, sq::kHole, sizeof(f.hnu));
  for (uint32_t b = 0; b < k; ++b) {
    uint32_t tx = offsets[2 * b], ty = offsets[2 * b + 1];
    if (tx >= s || ty >= s || f.hnu[ty * s + tx] != sq::kHole)
      return SQUEEZE_ERR_INVALID_ARG;  // offset out of range or repeated
    f.taux[b] = (uint8_t)tx;
    f.tauy[b] = (uint8_t)ty;
    f.hnu[ty * s + tx] = (uint8_t)b;
  }
  return SQUEEZE_OK;
}

void sq_set_error_text(const char *text) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s", text);
}

// The dynamic shared memory a kernel may use is an attribute of the function
// (per device), shared by every handle and batch that launches it: it is only
// ever raised, so that a program with less shared memory does not lower it
// under a program with more that launches the same kernel.
cudaError_t sq_allow_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> allowed;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = allowed[std::make_pair(dev, fn)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int sq_cuda_fail(cudaError_t e) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e),
           cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SQUEEZE_ERR_OOM : SQUEEZE_ERR_CUDA;
}

extern "C" {

const char *squeeze_status_string(int status) {
  switch (status) {
    case SQUEEZE_OK: return "ok";
    case SQUEEZE_ERR_INVALID_ARG: return "invalid argument";
    case SQUEEZE_ERR_UNSUPPORTED: return "unsupported on this build or device";
    case SQUEEZE_ERR_OOM: return "out of memory";
    case SQUEEZE_ERR_CUDA: return "CUDA runtime error";
    case SQUEEZE_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case SQUEEZE_ERR_DEVICE_BOUNDS: return "device-side bounds check failed";
    case SQUEEZE_ERR_IO: return "file could not be read or written, or is damaged";
    case SQUEEZE_ERR_DEVICE_UNSAFE:
      return "a timed-out bulk copy never landed; later launches on this context are unsafe";
    default: return "unknown status";
  }
}

const char *squeeze_last_cuda_error(void) { return g_last_cuda_error; }

int squeeze_create(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                   squeeze_handle **out) {
  if (!out) return SQUEEZE_ERR_INVALID_ARG;
  *out = nullptr;
  sq::FracDev f;
  int rc = sq_fill_fractal(s, k, offsets, r, f);
  if (rc) return rc;
  squeeze_handle *h = new (std::nothrow) squeeze_handle;
  if (!h) return SQUEEZE_ERR_OOM;
  memset(h, 0, sizeof(*h));
  h->f = f;
  h->rule.birth = 1u << 3;
  h->rule.survive = (1u << 2) | (1u << 3);
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

int squeeze_destroy(squeeze_handle *h) {
  if (!h) return SQUEEZE_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (h->tiled) sq_tiled_free(h->tiled);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return e == cudaSuccess ? SQUEEZE_OK : sq_cuda_fail(e);
}

int squeeze_info(const squeeze_handle *h, uint64_t *n_cells, uint64_t *width, uint64_t *height,
                 uint64_t *side) {
  if (check_handle(h)) return SQUEEZE_ERR_INVALID_ARG;
  if (n_cells) *n_cells = h->f.cells;
  if (width) *width = h->f.W;
  if (height) *height = h->f.H;
  if (side) *side = h->f.n;
  return SQUEEZE_OK;
}

int squeeze_set_rule(squeeze_handle *h, uint32_t birth, uint32_t survive) {
  if (check_handle(h) || birth >= (1u << 9) || survive >= (1u << 9))
    return SQUEEZE_ERR_INVALID_ARG;
  h->rule.birth = birth;
  h->rule.survive = survive;
  return SQUEEZE_OK;
}

int squeeze_set_neighbourhood(squeeze_handle *h, uint32_t mask) {
  if (check_handle(h) || mask >= (1u << 9) || (mask & (1u << 4))) return SQUEEZE_ERR_INVALID_ARG;
  if (mask == h->f.nbhd) return SQUEEZE_OK;
  if (h->tiled) {  // the tiled program holds the neighbour references: rebuild it
    cudaError_t e = cudaDeviceSynchronize();
    sq_tiled_free(h->tiled);
    h->tiled = nullptr;
    if (e != cudaSuccess) return sq_cuda_fail(e);
  }
  h->f.nbhd = mask;
  return SQUEEZE_OK;
}

int squeeze_lambda(const squeeze_handle *h, const uint64_t *d_omega, int32_t *d_xy,
                   uint64_t count, void *stream) {
  if (check_handle(h) || (count && (!d_omega || !d_xy))) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_omega | (uintptr_t)d_xy) & 7u) return SQUEEZE_ERR_INVALID_ARG;
  if (!count) return SQUEEZE_OK;
  return sq_launch_lambda(h, d_omega, d_xy, count, (cudaStream_t)stream);
}

int squeeze_nu(const squeeze_handle *h, const int32_t *d_xy, uint64_t *d_omega, uint64_t count,
               void *stream) {
  if (check_handle(h) || (count && (!d_omega || !d_xy))) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_omega | (uintptr_t)d_xy) & 7u) return SQUEEZE_ERR_INVALID_ARG;
  if (!count) return SQUEEZE_OK;
  return sq_launch_nu(h, d_xy, d_omega, count, (cudaStream_t)stream);
}

int squeeze_map_tc(const squeeze_handle *h, int direction, const void *d_in, void *d_out,
                   uint64_t count, int kind, void *stream) {
  if (check_handle(h) || (direction != 0 && direction != 1) || (count && (!d_in || !d_out)))
    return SQUEEZE_ERR_INVALID_ARG;
  if (kind == SQUEEZE_MAP_TC_I8) return SQUEEZE_ERR_UNSUPPORTED;
  if (kind != SQUEEZE_MAP_TC_BF16) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_in | (uintptr_t)d_out) & 7u) return SQUEEZE_ERR_INVALID_ARG;
  if (!count) return SQUEEZE_OK;
  return sq_launch_map_tc(h, direction, d_in, d_out, count, (cudaStream_t)stream);
}

int squeeze_init_bernoulli(const squeeze_handle *h, uint8_t *d_state, uint64_t seed,
                           uint32_t p_q24, void *stream) {
  if (check_handle(h) || !d_state || p_q24 > (1u << 24)) return SQUEEZE_ERR_INVALID_ARG;
  return sq_launch_init(h, d_state, seed, p_q24, (cudaStream_t)stream);
}

int squeeze_tiled_level(const squeeze_handle *h) {
  if (check_handle(h)) return SQUEEZE_ERR_INVALID_ARG;
  if (h->tiled_level) return (int)h->tiled_level;
  return sq_tiled_default_level(h);
}

int squeeze_set_tiled_level(squeeze_handle *h, uint32_t level) {
  if (check_handle(h) || level == 0 || level > h->f.r) return SQUEEZE_ERR_INVALID_ARG;
  if (!sq_tiled_level_fits(h, level)) return SQUEEZE_ERR_UNSUPPORTED;
  if (h->tiled && h->tiled_level != level) {
    cudaError_t e = cudaDeviceSynchronize();
    sq_tiled_free(h->tiled);
    h->tiled = nullptr;
    if (e != cudaSuccess) return sq_cuda_fail(e);
  }
  h->tiled_level = level;
  return SQUEEZE_OK;
}

int squeeze_step(squeeze_handle *h, uint8_t *d_buf0, uint8_t *d_buf1, uint64_t n_steps, int kind,
                 void *stream) {
  if (check_handle(h) || !d_buf0 || !d_buf1) return SQUEEZE_ERR_INVALID_ARG;
  uint64_t bytes = h->f.cells;
  if (d_buf0 < d_buf1 ? d_buf0 + bytes > d_buf1 : d_buf1 + bytes > d_buf0)
    return SQUEEZE_ERR_INVALID_ARG;  // overlapping buffers
  if (kind == SQUEEZE_MAP_TC_I8) return SQUEEZE_ERR_UNSUPPORTED;
  if (kind < SQUEEZE_STEP_AUTO || kind > SQUEEZE_MAP_TC_BF16) return SQUEEZE_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  bool aligned = (((uintptr_t)d_buf0 | (uintptr_t)d_buf1) & 15u) == 0;
  if (kind == SQUEEZE_STEP_AUTO)
    kind = aligned && (h->tiled_level || sq_tiled_default_level(h) > 0) ? SQUEEZE_STEP_TILED
                                                                        : SQUEEZE_MAP_ALU;
  if (kind == SQUEEZE_STEP_TILED && !aligned) return SQUEEZE_ERR_INVALID_ARG;
  if (kind == SQUEEZE_STEP_TILED) {
    int rc = sq_tiled_prepare(h);
    if (rc) return rc;
  }
  h->last_kind = kind;
  // The tiled kernel runs up to eight steps per launch where its program
  // allows (sq_launch_plan: launches of 8, 4, 2 and 1 steps whose count has
  // the parity of n_steps, since every launch swaps the buffers and the
  // result belongs in d_buf[n_steps & 1]).
  uint64_t counts[4] = {n_steps, 0, 0, 0};
  if (kind == SQUEEZE_STEP_TILED) sq_launch_plan(n_steps, sq_tiled_passes(h), counts);
  const uint64_t total = counts[0] + counts[1] + counts[2] + counts[3];
  // the border records of the input first (one extra launch) when a launch of
  // several steps will read them
  int extra = 0;
  if (kind == SQUEEZE_STEP_TILED && total) {
    const int rc = sq_tiled_begin(h, d_buf0, counts[1] + counts[2] + counts[3] != 0, st, &extra);
    if (rc) return rc;
  }
  uint8_t *a = d_buf0, *b = d_buf1;
  for (uint64_t t = 0, i = 3, used = 0; t < total; ++t) {
    while (used == counts[i]) {   // largest launches first
      --i;
      used = 0;
    }
    ++used;
    const uint32_t steps = 1u << i;
    int rc;
    switch (kind) {
      case SQUEEZE_STEP_TILED: rc = sq_launch_step_tiled(h, a, b, steps, t + 1 == total, st); break;
      case SQUEEZE_MAP_TC_BF16: rc = sq_launch_step_tc(h, a, b, st); break;
      default: rc = sq_launch_step_alu(h, a, b, st); break;
    }
    if (rc) return rc;
    uint8_t *tmp = a;
    a = b;
    b = tmp;
  }
  h->last_launches = total + (uint64_t)extra;
  for (int i = 0; i < 4; ++i) h->last_counts[i] = counts[i];
  return SQUEEZE_OK;
}

int squeeze_step_host(squeeze_handle *h, const uint8_t *h_in, uint8_t *h_out, uint8_t *d_buf0,
                      uint8_t *d_buf1, uint64_t n_steps, int kind, void *stream) {
  if (check_handle(h) || !h_in || !h_out) return SQUEEZE_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SQ_CUDA(cudaMemcpyAsync(d_buf0, h_in, h->f.cells, cudaMemcpyHostToDevice, st));
  int rc = squeeze_step(h, d_buf0, d_buf1, n_steps, kind, st);
  if (rc) return rc;
  const uint8_t *res = (n_steps & 1) ? d_buf1 : d_buf0;
  SQ_CUDA(cudaMemcpyAsync(h_out, res, h->f.cells, cudaMemcpyDeviceToHost, st));
  SQ_CUDA(cudaStreamSynchronize(st));
  return SQUEEZE_OK;
}

int squeeze_bb_init(const squeeze_handle *h, uint8_t *d_grid, uint64_t seed, uint32_t p_q24,
                    void *stream) {
  if (check_handle(h) || !d_grid || p_q24 > (1u << 24)) return SQUEEZE_ERR_INVALID_ARG;
  return sq_launch_bb_init(h, d_grid, seed, p_q24, (cudaStream_t)stream);
}

int squeeze_bb_step(const squeeze_handle *h, uint8_t *d_grid0, uint8_t *d_grid1, uint64_t n_steps,
                    void *stream) {
  if (check_handle(h) || !d_grid0 || !d_grid1) return SQUEEZE_ERR_INVALID_ARG;
  uint8_t *a = d_grid0, *b = d_grid1;
  for (uint64_t t = 0; t < n_steps; ++t) {
    int rc = sq_launch_bb_step(h, a, b, (cudaStream_t)stream);
    if (rc) return rc;
    uint8_t *tmp = a;
    a = b;
    b = tmp;
  }
  return SQUEEZE_OK;
}

int squeeze_heat_step(const squeeze_handle *h, float *d_u0, float *d_u1, uint64_t n_steps,
                      float alpha, void *stream) {
  if (check_handle(h) || !d_u0 || !d_u1 || d_u0 == d_u1) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_u0 | (uintptr_t)d_u1) & 3u) return SQUEEZE_ERR_INVALID_ARG;
  const uint64_t n = h->f.cells;
  if (d_u0 < d_u1 ? d_u0 + n > d_u1 : d_u1 + n > d_u0) return SQUEEZE_ERR_INVALID_ARG;
  float *a = d_u0, *b = d_u1;
  for (uint64_t t = 0; t < n_steps; ++t) {
    int rc = sq_launch_heat_step(h, a, b, alpha, (cudaStream_t)stream);
    if (rc) return rc;
    float *tmp = a;
    a = b;
    b = tmp;
  }
  return SQUEEZE_OK;
}

int squeeze_ising_sweep(const squeeze_handle *h, uint8_t *d_state, uint64_t n_sweeps,
                        uint64_t seed, double temperature, void *stream) {
  if (check_handle(h) || !d_state || !(temperature >= 0.0)) return SQUEEZE_ERR_INVALID_ARG;
  // checkerboard updates need a neighbourhood that joins opposite parities only
  if (h->f.nbhd & ~sq::kVonNeumann) return SQUEEZE_ERR_UNSUPPORTED;
  return sq_launch_ising(h, d_state, n_sweeps, seed, temperature, (cudaStream_t)stream);
}

int squeeze_lambda_step(const squeeze_handle *h, uint8_t *d_grid0, uint8_t *d_grid1,
                        uint64_t n_steps, void *stream) {
  if (check_handle(h) || !d_grid0 || !d_grid1 || d_grid0 == d_grid1) return SQUEEZE_ERR_INVALID_ARG;
  uint8_t *a = d_grid0, *b = d_grid1;
  for (uint64_t t = 0; t < n_steps; ++t) {
    int rc = sq_launch_lambda_step(h, a, b, (cudaStream_t)stream);
    if (rc) return rc;
    uint8_t *tmp = a;
    a = b;
    b = tmp;
  }
  return SQUEEZE_OK;
}

int squeeze_bb_to_compact(const squeeze_handle *h, const uint8_t *d_grid, uint8_t *d_state,
                          void *stream) {
  if (check_handle(h) || !d_grid || !d_state) return SQUEEZE_ERR_INVALID_ARG;
  return sq_launch_bb_gather(h, d_grid, d_state, (cudaStream_t)stream);
}

int squeeze_last_step_info(const squeeze_handle *h, int *kind, uint64_t *launches,
                           uint64_t *by_steps) {
  if (check_handle(h)) return SQUEEZE_ERR_INVALID_ARG;
  if (kind) *kind = h->last_kind;
  if (launches) *launches = h->last_launches;
  if (by_steps)
    for (int i = 0; i < 4; ++i) by_steps[i] = h->last_counts[i];
  return SQUEEZE_OK;
}

int squeeze_record_bytes(squeeze_handle *h, uint64_t *bytes) {
  if (check_handle(h) || !bytes) return SQUEEZE_ERR_INVALID_ARG;
  *bytes = 0;
  int rc = sq_tiled_prepare(h);
  if (rc) return rc;
  sq::TiledDev d;
  sq::TileSpec sp;
  rc = sq_tiled_describe(h, &d, &sp);
  if (rc) return rc;
  *bytes = (uint64_t)sp.rec_words * sp.tiles_x * sp.tiles_y * 4;
  return SQUEEZE_OK;
}

int squeeze_write_records(squeeze_handle *h, const uint8_t *d_state, uint32_t *d_rec,
                          void *stream) {
  if (check_handle(h) || !d_state || !d_rec) return SQUEEZE_ERR_INVALID_ARG;
  if (((uintptr_t)d_state & 15u) || ((uintptr_t)d_rec & 3u)) return SQUEEZE_ERR_INVALID_ARG;
  int rc = sq_tiled_prepare(h);
  if (rc) return rc;
  sq::TiledDev d;
  sq::TileSpec sp;
  rc = sq_tiled_describe(h, &d, &sp);
  if (rc || !sp.rec_words) return rc;
  d.rec[0] = nullptr;
  d.rec[1] = d_rec;   // the records-only launch writes the input's records here
  d.mode = 1;
  return sq_tile_launch(d, sp, d_state, const_cast<uint8_t *>(d_state), 1, (cudaStream_t)stream);
}

int squeeze_set_max_steps_per_launch(squeeze_handle *h, uint32_t steps) {
  if (check_handle(h) || (steps != 0 && steps != 1 && steps != 2 && steps != 4 && steps != 8))
    return SQUEEZE_ERR_INVALID_ARG;
  if (h->tiled && steps != h->max_passes) {   // rebuilt on the next step
    cudaError_t e = cudaDeviceSynchronize();
    sq_tiled_free(h->tiled);
    h->tiled = nullptr;
    if (e != cudaSuccess) return sq_cuda_fail(e);
  }
  h->max_passes = steps;
  return SQUEEZE_OK;
}

int squeeze_set_wait_limit(squeeze_handle *h, uint64_t ns) {
  if (check_handle(h) || (ns && (ns < 1000ull || ns > 10000000000ull)))
    return SQUEEZE_ERR_INVALID_ARG;
  h->wait_ns = ns;
  return SQUEEZE_OK;
}

int squeeze_set_fault_injection(squeeze_handle *h, uint32_t flags) {
  if (check_handle(h) || (flags & ~SQUEEZE_FAULT_WITHHOLD_LOADS)) return SQUEEZE_ERR_INVALID_ARG;
  h->fault = flags;
  return SQUEEZE_OK;
}

int squeeze_device_status(squeeze_handle *h, int *status) {
  if (check_handle(h) || !status) return SQUEEZE_ERR_INVALID_ARG;
  SQ_CUDA(cudaDeviceSynchronize());
  int v = 0;
  SQ_CUDA(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  SQ_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
  *status = v;
  return SQUEEZE_OK;
}

}  // extern "C"
