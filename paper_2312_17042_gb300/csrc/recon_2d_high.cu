// recon_2d_high.cu -- instantiations of the reconstruction of central degrees 4 to 6 (2D).
#include "recon_high.cuh"

namespace cteno {

cudaError_t launch_recon_2d_high(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s) {
  if (block >= kHighOcc + 32 && block <= kHighOcc + 256 && block % 32 == 0) {  // the 64-register build
    if (!fp32 || a.characteristic) return cudaErrorInvalidValue;
    const int threads = block - kHighOcc;
    const unsigned grid = (unsigned)((a.N + (threads / 32) * 8 - 1) / ((threads / 32) * 8));
#define CTENO_OCC(R, SC) launch_stage_kernel(recon_high_kernel_occ<R, SC>, grid, threads, 0, s, a)
    if (degree == 4 && scheme == 0) CTENO_OCC(4, 0);
    if (degree == 4 && scheme == 1) CTENO_OCC(4, 1);
    if (degree == 5 && scheme == 0) CTENO_OCC(5, 0);
    if (degree == 5 && scheme == 1) CTENO_OCC(5, 1);
    if (degree == 6 && scheme == 0) CTENO_OCC(6, 0);
    if (degree == 6 && scheme == 1) CTENO_OCC(6, 1);
#undef CTENO_OCC
    return cudaSuccess;
  }
  if (block < kLaneSchedule + 32 || block > kLaneSchedule + 256 || block % 32) return cudaErrorInvalidValue;
  const int threads = block - kLaneSchedule;
  const int64_t cells_per_block = (int64_t)(threads / 32) * 8;
  const unsigned grid = (unsigned)((a.N + cells_per_block - 1) / cells_per_block);
#define CTENO_HIGH(R, T, SC)                                                              \
  (a.characteristic ? launch_stage_kernel(recon_high_kernel<R, T, SC, true>, grid, threads, 0, s, a) \
                    : launch_stage_kernel(recon_high_kernel<R, T, SC, false>, grid, threads, 0, s, a))
  if (degree == 4 && fp32 && scheme == 0) CTENO_HIGH(4, float, 0);
  if (degree == 4 && fp32 && scheme == 1) CTENO_HIGH(4, float, 1);
  if (degree == 5 && fp32 && scheme == 0) CTENO_HIGH(5, float, 0);
  if (degree == 5 && fp32 && scheme == 1) CTENO_HIGH(5, float, 1);
  if (degree == 6 && fp32 && scheme == 0) CTENO_HIGH(6, float, 0);
  if (degree == 6 && fp32 && scheme == 1) CTENO_HIGH(6, float, 1);
  if (degree == 4 && !fp32 && scheme == 0) CTENO_HIGH(4, double, 0);
  if (degree == 4 && !fp32 && scheme == 1) CTENO_HIGH(4, double, 1);
  if (degree == 5 && !fp32 && scheme == 0) CTENO_HIGH(5, double, 0);
  if (degree == 5 && !fp32 && scheme == 1) CTENO_HIGH(5, double, 1);
  if (degree == 6 && !fp32 && scheme == 0) CTENO_HIGH(6, double, 0);
  if (degree == 6 && !fp32 && scheme == 1) CTENO_HIGH(6, double, 1);
#undef CTENO_HIGH
  return cudaSuccess;
}

cudaError_t upload_recon_tables_2d_high(int degree, const Tables &t, cudaStream_t s) {
  if (degree == 4) return upload_high_tables<4>(t, s);
  if (degree == 5) return upload_high_tables<5>(t, s);
  if (degree == 6) return upload_high_tables<6>(t, s);
  return cudaErrorInvalidValue;
}

}  // namespace cteno
