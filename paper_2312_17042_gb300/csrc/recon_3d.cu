// recon_3d.cu -- instantiations of the reconstruction kernel for d = 3.
#include "recon.cuh"

namespace cteno {

void launch_recon_3d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s) {
  const unsigned grid = (unsigned)((a.N + block - 1) / block);
#define CTENO_RECON(R, T, SC) recon_kernel<3, R, T, SC><<<grid, block, 0, s>>>(a)
  if (degree == 2 && fp32 && scheme == 0) CTENO_RECON(2, float, 0);
  if (degree == 2 && fp32 && scheme == 1) CTENO_RECON(2, float, 1);
  if (degree == 2 && !fp32 && scheme == 0) CTENO_RECON(2, double, 0);
  if (degree == 2 && !fp32 && scheme == 1) CTENO_RECON(2, double, 1);
  if (degree == 3 && fp32 && scheme == 0) CTENO_RECON(3, float, 0);
  if (degree == 3 && fp32 && scheme == 1) CTENO_RECON(3, float, 1);
  if (degree == 3 && !fp32 && scheme == 0) CTENO_RECON(3, double, 0);
  if (degree == 3 && !fp32 && scheme == 1) CTENO_RECON(3, double, 1);
#undef CTENO_RECON
}

cudaError_t upload_recon_tables_3d(int degree, const Tables &t, cudaStream_t s) {
  return upload_recon_tables(3, degree, t, s);
}

}  // namespace cteno
