// recon_2d.cu -- instantiations of the reconstruction kernel for d = 2.
#include "recon.cuh"
#include "recon_pair.cuh"

namespace cteno {

cudaError_t launch_recon_2d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s) {
  // the characteristic reconstruction runs in the variable-per-lane schedule only
  if (a.characteristic && !(block >= kLaneSchedule && block < kStagedCells)) return cudaErrorInvalidValue;
  if (block == kHaloLanes || block == kHaloLanes + 1) {  // gather-staged lane schedule (mixed)
    if (!fp32) return cudaErrorInvalidValue;  // mixed path only
    const bool one = block == kHaloLanes + 1;  // one tile per block, single stage
#define CTENO_HALO(R, SC) \
  (one ? launch_recon_halo<2, R, SC, true>(a, s) : launch_recon_halo<2, R, SC, false>(a, s))
    if (degree == 2 && scheme == 0) CTENO_HALO(2, 0);
    if (degree == 2 && scheme == 1) CTENO_HALO(2, 1);
    if (degree == 3 && scheme == 0) CTENO_HALO(3, 0);
    if (degree == 3 && scheme == 1) CTENO_HALO(3, 1);
#undef CTENO_HALO
    return cudaSuccess;
  }
  {
    int warps = 0, stages = 0;
    pair_launch(block, &warps, &stages);
    if (warps) {  // streamed schedule, two lanes per cell (mixed)
      if (!fp32) return cudaErrorInvalidValue;  // mixed path only
#define CTENO_PAIR(R, SC) \
  (stages == 3 ? launch_recon_pair<2, R, SC, 3>(a, warps, s) : launch_recon_pair<2, R, SC, 2>(a, warps, s))
      if (degree == 2 && scheme == 0) CTENO_PAIR(2, 0);
      if (degree == 2 && scheme == 1) CTENO_PAIR(2, 1);
      if (degree == 3 && scheme == 0) CTENO_PAIR(3, 0);
      if (degree == 3 && scheme == 1) CTENO_PAIR(3, 1);
#undef CTENO_PAIR
      return cudaSuccess;
    }
  }
  if (block > kStreamCells && block <= kStreamCells + 8) {  // streamed thread-per-cell schedule (mixed)
    if (!fp32) return cudaErrorInvalidValue;  // mixed path only
    const int warps = block - kStreamCells;
    if (degree == 2 && scheme == 0) launch_recon_stream_cells<2, 2, 0>(a, warps, s);
    if (degree == 2 && scheme == 1) launch_recon_stream_cells<2, 2, 1>(a, warps, s);
    if (degree == 3 && scheme == 0) launch_recon_stream_cells<2, 3, 0>(a, warps, s);
    if (degree == 3 && scheme == 1) launch_recon_stream_cells<2, 3, 1>(a, warps, s);
    return cudaSuccess;
  }
  {
    int warps = 0, stages = 0;
    stream_launch(block, &warps, &stages);
    if (warps) {  // streamed lane schedule (mixed)
      if (!fp32) return cudaErrorInvalidValue;  // mixed path only
#define CTENO_STREAM(R, SC) \
  (stages == 3 ? launch_recon_stream<2, R, SC, 3>(a, warps, s) : launch_recon_stream<2, R, SC, 2>(a, warps, s))
      if (degree == 2 && scheme == 0) CTENO_STREAM(2, 0);
      if (degree == 2 && scheme == 1) CTENO_STREAM(2, 1);
      if (degree == 3 && scheme == 0) CTENO_STREAM(3, 0);
      if (degree == 3 && scheme == 1) CTENO_STREAM(3, 1);
#undef CTENO_STREAM
      return cudaSuccess;
    }
  }
  if (block >= kStagedCells) {  // staged persistent schedules (mixed path; the launch value is
                                // validated by the caller)
    const bool lanes = block >= kStagedLanes;
    const int threads = block - (lanes ? kStagedLanes : kStagedCells);
    if (!fp32) return cudaErrorInvalidValue;  // mixed path only
#define CTENO_STAGED(R, SC) \
  (lanes ? launch_recon_staged<2, R, float, SC, true>(a, threads, s) : launch_recon_staged<2, R, float, SC, false>(a, threads, s))
    if (degree == 2 && scheme == 0) CTENO_STAGED(2, 0);
    if (degree == 2 && scheme == 1) CTENO_STAGED(2, 1);
    if (degree == 3 && scheme == 0) CTENO_STAGED(3, 0);
    if (degree == 3 && scheme == 1) CTENO_STAGED(3, 1);
#undef CTENO_STAGED
    return cudaSuccess;
  }
  if (block >= kLaneSchedule) {  // variable-per-lane schedule, block - kLaneSchedule threads
    const int threads = block - kLaneSchedule, cpw = 32 / (2 + 2);
    const int64_t cells_per_block = (int64_t)(threads / 32) * cpw;
    const unsigned grid = (unsigned)((a.N + cells_per_block - 1) / cells_per_block);
#define CTENO_LANES(R, T, SC)                                                                   \
  (a.characteristic ? launch_stage_kernel(recon_lanes_kernel<2, R, T, SC, true>, grid, threads, 0, s, a) \
                    : launch_stage_kernel(recon_lanes_kernel<2, R, T, SC, false>, grid, threads, 0, s, a))
    if (degree == 2 && fp32 && scheme == 0) CTENO_LANES(2, float, 0);
    if (degree == 2 && fp32 && scheme == 1) CTENO_LANES(2, float, 1);
    if (degree == 3 && fp32 && scheme == 0) CTENO_LANES(3, float, 0);
    if (degree == 3 && fp32 && scheme == 1) CTENO_LANES(3, float, 1);
    if (degree == 2 && !fp32 && scheme == 0) CTENO_LANES(2, double, 0);
    if (degree == 2 && !fp32 && scheme == 1) CTENO_LANES(2, double, 1);
    if (degree == 3 && !fp32 && scheme == 0) CTENO_LANES(3, double, 0);
    if (degree == 3 && !fp32 && scheme == 1) CTENO_LANES(3, double, 1);
#undef CTENO_LANES
    return cudaSuccess;
  }
  const bool capped = block < 0;  // register-capped variant (FP32 only)
  if (capped) block = -block;
  const unsigned grid = (unsigned)((a.N + block - 1) / block);
#define CTENO_RECON(R, T, SC, MB) launch_stage_kernel(recon_kernel<2, R, T, SC, MB>, grid, block, 0, s, a)
  if (degree == 2 && fp32 && scheme == 0) { if (capped) CTENO_RECON(2, float, 0, 8); else CTENO_RECON(2, float, 0, 0); }
  if (degree == 2 && fp32 && scheme == 1) { if (capped) CTENO_RECON(2, float, 1, 8); else CTENO_RECON(2, float, 1, 0); }
  if (degree == 3 && fp32 && scheme == 0) { if (capped) CTENO_RECON(3, float, 0, 8); else CTENO_RECON(3, float, 0, 0); }
  if (degree == 3 && fp32 && scheme == 1) { if (capped) CTENO_RECON(3, float, 1, 8); else CTENO_RECON(3, float, 1, 0); }
  if (degree == 2 && !fp32 && scheme == 0) CTENO_RECON(2, double, 0, 0);
  if (degree == 2 && !fp32 && scheme == 1) CTENO_RECON(2, double, 1, 0);
  if (degree == 3 && !fp32 && scheme == 0) CTENO_RECON(3, double, 0, 0);
  if (degree == 3 && !fp32 && scheme == 1) CTENO_RECON(3, double, 1, 0);
#undef CTENO_RECON
  return cudaSuccess;
}

cudaError_t upload_recon_tables_2d(int degree, const Tables &t, cudaStream_t s) {
  return upload_recon_tables(2, degree, t, s);
}

}  // namespace cteno
