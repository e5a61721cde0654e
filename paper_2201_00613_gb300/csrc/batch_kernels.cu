// batch_kernels.cu -- the batched planar step's kernel instantiations (one
// per tile-row width, rule kind and steps per launch) and their launches; the
// schedule and the C ABI are in batch.cu, the device code in tile2d.cuh.
#include "tile2d.cuh"

namespace sq {
namespace {

// The batched kernel of one tile-row instantiation (see tiled_kernel_for).
template <bool kLife, int kT>
const void *batch_kernel_of(int kind) {
  switch (kind) {
    case 27: return (const void *)step_batch_kernel<kLife, 27, kT>;
    case 25: return (const void *)step_batch_kernel<kLife, 25, kT>;
    case 8: return (const void *)step_batch_kernel<kLife, 8, kT>;
    case 16: return (const void *)step_batch_kernel<kLife, 16, kT>;
    case 64: return (const void *)step_batch_kernel<kLife, 64, kT>;
    default: return (const void *)step_batch_kernel<kLife, 0, kT>;
  }
}

const void *batch_kernel_for(bool life, int kind, uint32_t steps) {
  if (steps == 8) return life ? batch_kernel_of<true, 8>(kind) : batch_kernel_of<false, 8>(kind);
  if (steps == 4) return life ? batch_kernel_of<true, 4>(kind) : batch_kernel_of<false, 4>(kind);
  if (steps == 2) return life ? batch_kernel_of<true, 2>(kind) : batch_kernel_of<false, 2>(kind);
  return life ? batch_kernel_of<true, 1>(kind) : batch_kernel_of<false, 1>(kind);
}

}  // namespace
}  // namespace sq

using namespace sq;

int sq_batch_occupancy(bool life, int kind, uint32_t steps, int threads, uint32_t smem) {
  const void *fn = batch_kernel_for(life, kind, steps);
  if (sq_allow_smem(fn, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) return 0;
  return n;
}

int sq_batch_launch(const TiledDev *d_devs, uint8_t *const *d_buf0, uint8_t *const *d_buf1,
                    const BatchWork *d_work, const uint32_t *d_sched, const TileLayout &lay,
                    int grid, int threads, bool life, int kind, uint32_t steps, uint32_t parity,
                    uint32_t mode, cudaStream_t st) {
  TileLayout l = lay;
  void *args[] = {&d_devs, &d_buf0, &d_buf1, &d_work, &d_sched, &l, &parity, &mode};
  SQ_CUDA(cudaLaunchKernel(batch_kernel_for(life, kind, steps), dim3(grid), dim3(threads), args,
                           l.smem, st));
  SQ_CUDA(cudaGetLastError());
  return SQUEEZE_OK;
}
