// batch_host.cu -- test support: the batched step's work schedule
// (build_schedule in batch.cu, host code) exported for a CPU test.  The
// library functions batch.cu calls elsewhere are stubbed: the test reaches
// none of them.
#include "batch.cu"

int sq_cuda_fail(cudaError_t) { return SQUEEZE_ERR_CUDA; }
cudaError_t sq_allow_smem(const void *, size_t) { return cudaSuccess; }
extern "C" int squeeze_record_bytes(squeeze_handle *, uint64_t *) { return SQUEEZE_ERR_UNSUPPORTED; }
int sq_tiled_prepare(squeeze_handle *) { return SQUEEZE_ERR_UNSUPPORTED; }
int sq_tiled_describe(const squeeze_handle *, sq::TiledDev *, sq::TileSpec *) {
  return SQUEEZE_ERR_UNSUPPORTED;
}
sq::TileLayout sq_tile_layout(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t) { return sq::TileLayout{}; }
uint32_t sq_tile_table_words(const sq::TileSpec &) { return 0; }
sq::TileLayout sq_tile_layout_of(const sq::TileSpec &) { return sq::TileLayout{}; }
sq::TileLayout sq_tile_layout_max(const sq::TileLayout &a, const sq::TileLayout &) { return a; }
int sq_tile_kind(const sq::TileSpec &) { return 0; }
void sq_launch_plan(uint64_t, uint32_t, uint64_t *counts) {
  for (int i = 0; i < 4; ++i) counts[i] = 0;
}
int sq_batch_occupancy(bool, int, uint32_t, int, uint32_t) { return 0; }
int sq_batch_launch(const sq::TiledDev *, uint8_t *const *, uint8_t *const *, const sq::BatchWork *,
                    const uint32_t *, const sq::TileLayout &, int, int, bool, int, uint32_t,
                    uint32_t, uint32_t, cudaStream_t) {
  return SQUEEZE_ERR_UNSUPPORTED;
}

extern "C" {

// Schedule of `count` instances over `grid` CTAs (strided as for 64-wide
// rows when `strided` is set).  Returns the number of entries (instance, first
// group, end group, stride) written to work[4 * e ..], or -1 when more than
// `cap` would be needed; start receives grid + 1 offsets.
int64_t batch_schedule(const uint64_t *cells, const uint64_t *groups, uint32_t count, int grid,
                       int strided, uint64_t *work, uint64_t cap, uint32_t *start) {
  std::vector<uint64_t> c(cells, cells + count), g(groups, groups + count);
  std::vector<sq::BatchWork> w;
  std::vector<uint32_t> st;
  build_schedule(c, g, grid, w, st);
  if (strided) stride_schedule(w, st);
  if (w.size() > cap) return -1;
  for (size_t e = 0; e < w.size(); ++e) {
    work[4 * e] = w[e].instance;
    work[4 * e + 1] = w[e].g_first;
    work[4 * e + 2] = w[e].g_end;
    work[4 * e + 3] = w[e].g_stride;
  }
  for (size_t i = 0; i < st.size(); ++i) start[i] = st[i];
  return (int64_t)w.size();
}

}  // extern "C"
