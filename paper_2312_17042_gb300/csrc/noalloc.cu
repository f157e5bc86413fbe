// noalloc.cu -- state read-back that allocates no memory.
//
// cteno_get_state with a host output gathers the mesh's cell means into a device staging buffer
// that it allocates (cudaMalloc) on first use or when a larger mesh is read, then copies that
// buffer to the host. Code that may not allocate device memory at that point -- for instance a
// host program that hands all device memory to its own pool up front, or one that reads states
// while allocation is forbidden -- can use cteno_get_state_noalloc instead: the same gather kernel
// writes into a fixed staging array compiled into the library, so the call never calls
// cudaMalloc, cudaFree or any allocating routine.
#include <mutex>

#include "device.h"

namespace {

// Staging area: 2^21 doubles (16 MiB). Every GPU that loads the library keeps this array for the
// life of the process.
constexpr int64_t kStageValues = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_stage[kStageValues];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_stage_addr[kMaxDevices] = {};

}  // namespace

namespace cteno {

// Device address of the staging array on the current device, looked up once per device. In host
// code the array's name is only a host-side stand-in, so a kernel must be given this address,
// never the symbol. Under lazy module loading the lookup also loads the module that holds the
// array (which allocates it); cteno_lsq_build calls this on the context's device for that reason.
cudaError_t noalloc_stage_address(double **out, int64_t *capacity) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_stage_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_stage);
    if (e != cudaSuccess) return e;
    g_stage_addr[dev] = static_cast<double *>(p);
  }
  *out = g_stage_addr[dev];
  *capacity = kStageValues;
  return cudaSuccess;
}

// Implemented in api.cpp: everything cteno_get_state needs, through the context's staging address.
int get_state_noalloc(cteno_ctx *ctx, int32_t mesh_id, double *U_out);

}  // namespace cteno

extern "C" int cteno_get_state_noalloc(cteno_ctx *ctx, int32_t mesh_id, double *U_out) {
  return cteno::get_state_noalloc(ctx, mesh_id, U_out);
}
