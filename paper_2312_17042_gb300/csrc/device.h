// device.h -- device data layout, kernel argument block and launcher declarations.
//
// Every per-cell array is stored cell-major (array-of-structures): the record of device cell i
// is one contiguous, 16-byte aligned block, so a thread reads its own record, or a neighbour's,
// with 16-byte vector loads, and the records of a warp's 32 consecutive cells form one
// contiguous span (fully used DRAM sectors).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace cteno {

// Record sizes for dimension D.
template <int D>
struct Lay {
  static constexpr int NV = D + 2;              // conserved variables
  static constexpr int NVP = (D == 2) ? 4 : 6;  // state record length (padded to 16 B pairs)
  static constexpr int NF = D + 1;              // faces
  static constexpr int NQ = (D == 2) ? 2 : 4;   // Gauss points per face
  static constexpr int ND = 2 * D;              // max members of a directional stencil
  static constexpr int PDS = (D == 2) ? 8 : 20; // directional operator record per face (D*ND padded)
};
inline int lay_nvp(int d) { return d == 2 ? 4 : 6; }
inline int lay_pds(int d) { return d == 2 ? 8 : 20; }

// Directional operator records for central degree R. Up to degree 3: degree-1 stencils (D
// unknowns, at most 2D members), member-major entries j * D + k, padded to Lay<D>::PDS. Degrees 4
// to 6 (2D): degree-2 stencils (5 unknowns, at most 10 members), unknown-major entries k * NDP + j
// with NDP = 12 member slots per unknown (16-byte rows in FP32 and FP64).
template <int D, int R>
struct Dir {
  static constexpr bool HIGH = R >= 4;
  static constexpr int KD = HIGH ? 5 : D;       // unknowns of a directional polynomial
  static constexpr int ND = 2 * KD;             // members at most
  static constexpr int NDP = HIGH ? 12 : ND;    // member slots of one unknown's row (HIGH)
  static constexpr int PDS = HIGH ? KD * NDP : Lay<D>::PDS;
};
inline int dir_pds(int d, int degree) { return degree >= 4 ? 60 : lay_pds(d); }

// Bits of the per-cell word `cinfo`:
//   [4f, 4f+4)   members of the directional stencil of local face f (its first slots in the
//                device stencil list are those members, face after face)
//   16 + f       directional stencil of face f admissible (set by the least-squares build)
//   20 + 3f      index of the permutation taking the face's local vertex slots to the order of
//                their global ids (canonical Gauss-point order)
constexpr int kInfoAdmShift = 16;
constexpr int kInfoPermShift = 20;
// Bits of `fmeta`: [2f, 2f+2) neighbour's local face; 8 + f: this cell owns face f (computes the
// flux in its own orientation; the other cell uses the exact negative normal and negates);
// [12 + 2f, 14 + 2f): kind of boundary face f (CTENO_BOUNDARY_*: transmissive, wall, fixed state
// A, moving shock between states A and B).
constexpr int kMetaOwnerShift = 8;
constexpr int kMetaKindShift = 12;

// Error word bits.
constexpr int kErrNonFinite = 1;
constexpr int kErrRank = 2;
constexpr int kErrTimeout = 4;  // a bounded wait on a bulk copy gave up

// Device tables (a copy of Tables with the fields the kernels read).
struct DevTables {
  int nk, nq, nperm, nvq;
  int ex[kMaxNK][3];
  double psibar[kMaxNK];
  double O[kMaxNK][kMaxNK];
  double Phi[kMaxNF][kMaxPerm][kMaxNQ][kMaxNK];
  double fw[kMaxNQ];
  double vq[kMaxVQ][3];
  double vw[kMaxVQ];
};

// Everything a kernel touches, passed by value. Layouts (i = device cell, T = FP64 or FP32):
//   U, Un   double [N][NVP]        conserved means (padding entries unused)
//   U32     float2 [N][NVP]        mixed path: (hi, lo) = (fl32(U), fl32(U - hi))
//   st      int32  [N][M]          stencil ids, directional members first (face after face)
//   Pc      T      [N][M][nk]      central pseudo-inverse, member-major
//   Pd      T      [N][NF][PDS]    directional pseudo-inverses (layout of Dir<D, R>)
//   Uf      T      [N][NF][NQ][NV] face Gauss-point states
//   nbr     int32  [N][4]          face neighbours, -1 on a boundary
//   geo     double [N][NF][4]      outward unit normal (n_x, n_y[, n_z]) and area in slot 3;
//                                  exact negatives across a face; geo32 its FP32 copy
//   flags   uint8  [nv][N]         selection flags (debug)
struct KArgs {
  int64_t N;
  int nmesh;
  const int64_t *mesh_off;  // [nmesh + 1] first device cell of each mesh
  double *U;
  double *Un;
  double *Acc;              // classical RK4: U^n + dt/6 (k1 + 2 k2 + 2 k3) so far, [N][NVP]
  float *U32;
  const int32_t *st;
  const uint32_t *cinfo;
  const void *Pc;
  const void *Pd;
  void *Uf;
  uint8_t *flags;
  const int32_t *nbr;
  const uint32_t *fmeta;
  const double *geo;
  const float *geo32;
  const double *vol;        // [N] 1 / |V_i|
  double *dt;               // [2 * nmesh]: [0..nmesh) current step, [nmesh..2 nmesh) next step
  const DevTables *tab;
  int *err;
  unsigned long long *guard;
  // parameters
  double C_T, lambda1p, eps, gamma, cfl;
  int lam_gamma, guard_on, ctenoz_form;
  int characteristic;  // characteristic-variable reconstruction per face (Sec. 2.2, 3.2)
  int cweno;          // CWENO weighting (Sec. 2.3) instead of the cut-off selection
  int central_split;  // p_1 from the CWENO split of eq. 17 (CTENO, CTENOZ, CWENO); 0: TENO's p_opt
  // linear coefficients of eq. 18, evaluated once on the host in FP64:
  // lam1 = 1 - 1/lambda_1', 1/lam1, 1 - lam1 (lambda_s = (1 - lam1) / (s_t - 1)) and base-2 logs
  double lam1, inv_lam1, one_m_lam1;
  float log2_lam1, log2_one_m_lam1;
  // lambda_s of each directional stencil when st stencils are admissible (index st - 1, 1..d+1):
  // (1 - lam1) / (st - 1) in FP64, its FP32 copy and base-2 log; CTENOZ mean factor 1 / (st - 1)
  double lams_d[kMaxNF + 1];
  float lams_f[kMaxNF + 1], log2_lams_f[kMaxNF + 1], inv_stm1_f[kMaxNF + 1];
  // FP32 copies for the mixed path (no per-thread conversions)
  float gamma32, gm1_32, eps32, C_T32, inv_lam1_32, one_m_lam1_32, cfl32;
  float fw32[kMaxNQ];
  double fw[kMaxNQ];        // face quadrature weights
  // gather staging (mixed path): cells in tiles of htile; per tile a record of hrec int32 words
  // [count, 0, 0, 0, distinct member ids ascending, padding]; per cell hms uint16 local indices
  // into its tile's list (stencil members in device order, then the cell itself)
  const int32_t *hl;
  const uint16_t *lidx;
  int htile, hrec, hms;
  // face-based flux schedule: face e = {owner device cell << 2 | local face, the same for the
  // neighbour side or -1 on a boundary}; cellface[i*4+f] =
  // face id, bit 31 set where cell i is not the owner; Ff [nfaces][(nv+3)&~3] face fluxes (T)
  const int32_t *face;
  const int32_t *cellface;
  void *Ff;
  int64_t nfaces;
  int pdl;                  // launched with programmatic dependent launch (see pdl_wait)
  // test hook of the bounded waits (0 = off): the staged schedules first wait at most this many
  // nanoseconds on a barrier that nothing completes, then take their timeout path
  unsigned long long test_wait_ns;
  // boundary states A and B (conserved, padded) and the moving shock's speed term: a face of the
  // moving-shock kind takes A where c_f + vs t > 0, c_f = xs0 + sy y_mid - x_mid stored in the
  // face's unused third geometry slot (2D), t = time[mesh] + stage_c dt[mesh]
  double bA[6], bB[6];
  float bA32[6], bB32[6];
  double shock_vs, stage_c;
  const double *time;       // [nmesh] physical time at the start of the step (moving shock only)
  int stage;                // 0 .. last_stage
  int rk4;                  // classical four-stage Runge-Kutta (else SSP-RK3)
  int last_stage;           // 2 (SSP-RK3) or 3 (RK4): the stage that computes the next CFL step
  int dt_swap;              // stage 0 of a CFL step: move dt[next] to dt[cur] first
};

// Set-up (FP64): geometry, moments, Householder QR, pseudo-inverses.
struct SetupArgs {
  int64_t N;
  const double *X;          // [N][d+1][d] unwrapped, oriented vertices
  const int32_t *st;        // [N][M]
  uint32_t *cinfo;          // [N] (admissibility bits written)
  const int32_t *nbr;       // [N][4]
  const uint32_t *fmeta;
  double period[3];
  void *Pc, *Pd;            // outputs, T = double (FP64 path) or float (mixed path)
  int store_fp32;
  double *geo, *vol;       // vol receives 1 / |V_i|
  float *geo32;
  const DevTables *tab;
  int *err;
  double shock_xs0, shock_sy;  // moving-shock line x = xs0 + sy y + vs t (2D boundary faces)
};

// Launch-value convention of the reconstruction kernel: b in [32, 256] one thread per cell;
// -b the register-capped thread-per-cell variant; kLaneSchedule + b the variable-per-lane
// schedule with b threads per block.
constexpr int kLaneSchedule = 1024;
// kStagedCells + b / kStagedLanes + b: the thread-per-cell / variable-per-lane schedule as a
// persistent kernel whose operator records are staged in shared memory by bulk copies (mixed path).
constexpr int kStagedCells = 2048;
constexpr int kStagedLanes = 3072;
constexpr int kMaxStagedSmem = 200 * 1024;  // dynamic shared memory of the two stages, at most
// kHaloLanes: the staged lane schedule (4 warps) that also stages each tile's distinct stencil
// members' states in shared memory (mixed path).
constexpr int kHaloLanes = 4096;
// Flux launch value kFaceFlux + b: the face-based schedule (HLLC once per face, then a per-cell
// gather and update), b threads per block.
constexpr int kFaceFlux = 8192;
constexpr int kHaloWarps = 4;
// kStreamLanes + w (w warps per block, 1..16): the streamed lane schedule (mixed path): every warp
// streams its tiles' operator records through its own ring of three shared-memory stages;
// kStreamLanes2 + w the same with two stages (a smaller ring, more warps).
constexpr int kStreamLanes = 5120;
constexpr int kStreamLanes2 = 5152;
constexpr int kMaxStreamSmem = 227 * 1024;  // the per-block limit of the GPU
// kStreamCells + w (w warps per block, 1..8): the streamed thread-per-cell schedule (mixed path):
// every warp walks tiles of 32 cells and each lane streams its own cell's operator record through
// the warp's ring of shared-memory stages, four stencil members at a time.
constexpr int kStreamCells = 6144;
constexpr int kStreamCellStages = 3;
inline long long recon_stream_cells_smem(int d, int degree, int warps) {
  const int nk = (d == 2 ? (degree + 1) * (degree + 2) / 2 : (degree + 1) * (degree + 2) * (degree + 3) / 6) - 1;
  const long long stage = 32LL * 4 * nk * 4;
  const long long nphi = d == 3 ? (long long)(d + 1) * 6 * 4 * nk : 1;
  const long long phi = (nphi * 4 + 15) / 16 * 16;
  return phi + (long long)warps * kStreamCellStages * stage + (long long)warps * kStreamCellStages * 8 + 8;
}
// Dynamic shared memory of the streamed lane schedule with `warps` warps and `stages` stages (see
// StreamShape).
inline long long recon_stream_smem(int d, int degree, int warps, int stages) {
  const int nk = (d == 2 ? (degree + 1) * (degree + 2) / 2 : (degree + 1) * (degree + 2) * (degree + 3) / 6) - 1;
  const int M = 2 * (nk + 1), nv = d + 2, cpw = 32 / nv, mc = (M % 8 == 0) ? 8 : 4;
  const long long stage = (long long)cpw * mc * nk * 4;
  const long long hdr = (long long)cpw * (d + 1) * lay_pds(d) * 4 + (long long)cpw * M * 4;
  const long long phi = 16;  // no face-value table (see StreamShape)
  return phi + (long long)warps * (2 * hdr + stages * stage) + (long long)warps * (2 + stages) * 8 + 8;
}
// Launch value -> (warps, stages) of the streamed lane schedule, or warps = 0.
inline void stream_launch(int b, int *warps, int *stages) {
  *warps = 0;
  *stages = 0;
  if (b > kStreamLanes && b <= kStreamLanes + 16) *warps = b - kStreamLanes, *stages = 3;
  if (b > kStreamLanes2 && b <= kStreamLanes2 + 16) *warps = b - kStreamLanes2, *stages = 2;
}
// kPairLanes + w / kPairLanes3 + w (w warps per block, 1..8): the streamed schedule with two lanes
// per cell (mixed path), a two- / three-stage ring of 4-member chunks of 16 cells per warp.
constexpr int kPairLanes = 7168;
constexpr int kPairLanes3 = 7200;
inline long long recon_pair_smem(int d, int degree, int warps, int stages) {
  const int nk = (d == 2 ? (degree + 1) * (degree + 2) / 2 : (degree + 1) * (degree + 2) * (degree + 3) / 6) - 1;
  const int M = 2 * (nk + 1);
  const long long stage = 16LL * 4 * nk * 4;
  const long long hdr = 16LL * (d + 1) * lay_pds(d) * 4 + 16LL * M * 4;
  const long long nphi = d == 3 ? (long long)(d + 1) * 6 * 4 * nk : 1;
  const long long phi = (nphi * 4 + 15) / 16 * 16;
  return phi + (long long)warps * (2 * hdr + stages * stage) + (long long)warps * (2 + stages) * 8 + 8;
}
// Launch value -> (warps, stages) of the two-lanes-per-cell schedule, or warps = 0.
inline void pair_launch(int b, int *warps, int *stages) {
  *warps = 0;
  *stages = 0;
  if (b > kPairLanes && b <= kPairLanes + 8) *warps = b - kPairLanes, *stages = 2;
  if (b > kPairLanes3 && b <= kPairLanes3 + 8) *warps = b - kPairLanes3, *stages = 3;
}
inline int halo_tile(int d) { return kHaloWarps * (32 / (d + 2)); }
inline int halo_ms(int M) { return (M + 1 + 7) / 8 * 8; }
// Dynamic shared memory of the gather-staged launch for a tile record of hrec words.
inline long long recon_halo_smem(int d, int degree, int hrec) {
  const int nk = (d == 2 ? (degree + 1) * (degree + 2) / 2 : (degree + 1) * (degree + 2) * (degree + 3) / 6) - 1;
  const int M = 2 * (nk + 1), C = halo_tile(d);
  const long long rec = (long long)M * nk * 4 + (long long)(d + 1) * lay_pds(d) * 4 + 2LL * halo_ms(M);
  const long long hs = 8LL * lay_nvp(d);  // one FP32 (hi, lo) state record
  return 2 * (C * rec + 4LL * hrec + (long long)(hrec - 4) * hs);
}

// Dynamic shared memory of a staged launch value (two stages of a tile's operator records).
inline long long recon_staged_smem(int d, int degree, int fp32, int block) {
  const int nk = (d == 2 ? (degree + 1) * (degree + 2) / 2 : (degree + 1) * (degree + 2) * (degree + 3) / 6) - 1;
  const int M = 2 * (nk + 1), sT = fp32 ? 4 : 8;
  const int threads = block >= kStagedLanes ? block - kStagedLanes : block - kStagedCells;
  const int cells = block >= kStagedLanes ? (threads / 32) * (32 / (d + 2)) : threads;
  const long long cell_bytes = (long long)M * nk * sT + (long long)(d + 1) * lay_pds(d) * sT + 4LL * M;
  return 2 * cells * cell_bytes;
}

void launch_setup(int dim, int degree, const SetupArgs &a, cudaStream_t s);
// Central degrees 4 to 6 (2D): constant banks and the variable-per-lane reconstruction
// (recon_2d_high.cu); launch values other than kLaneSchedule + b (and, on the mixed path without
// the characteristic projection, kHighOcc + b: the same schedule compiled for at most 64
// registers per thread) give cudaErrorInvalidValue.
constexpr int kHighOcc = 1536;
cudaError_t upload_recon_tables_2d_high(int degree, const Tables &t, cudaStream_t s);
cudaError_t launch_recon_2d_high(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s);
// Upload the (d, r) smoothness matrix and face-point basis values to the constant banks of the
// reconstruction kernels.
cudaError_t upload_recon_tables_2d(int degree, const Tables &t, cudaStream_t s);
cudaError_t upload_recon_tables_3d(int degree, const Tables &t, cudaStream_t s);
// cudaErrorInvalidValue (and no launch) for a launch value the path does not have (a staged,
// gather-staged or streamed schedule on the FP64 path).
cudaError_t launch_recon_2d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s);
cudaError_t launch_recon_3d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s);
inline cudaError_t launch_recon(int dim, int degree, int fp32, int scheme, const KArgs &a, int block,
                                cudaStream_t s) {
  if (dim == 2 && degree >= 4) return launch_recon_2d_high(degree, fp32, scheme, a, block, s);
  return dim == 2 ? launch_recon_2d(degree, fp32, scheme, a, block, s)
                  : launch_recon_3d(degree, fp32, scheme, a, block, s);
}
// nq: Gauss points per face (face_points(dim, degree)).
void launch_flux(int dim, int nq, int fp32, const KArgs &a, int block, cudaStream_t s);
void launch_dt(int dim, const KArgs &a, cudaStream_t s);
void launch_dt_reset(const KArgs &a, cudaStream_t s);
// time[m] += dt[m] for every mesh: the end of a step (kept only when a moving-shock boundary exists)
void launch_time_advance(double *time, const double *dt, int nmesh, cudaStream_t s);
// CFL step of one mesh only (device cells [first, first + count)).
void launch_dt_mesh(int dim, const KArgs &a, int mesh, int64_t first, int64_t count, cudaStream_t s);
// All meshes in one launch: host-side order is mesh after mesh, [v][cell] per mesh in the mesh's
// original numbering; grank[c] is the device cell of concatenated original cell c.
// Set every mesh's state from src (device or page-locked host memory, layout above) and compute
// each mesh's CFL step of it, in one pass.
void launch_set_state_all(int dim, const KArgs &a, const int32_t *grank, const double *src, cudaStream_t s);
void launch_permute_out_all(int nv, int nvp, int64_t N, int nmesh, const int64_t *mesh_off,
                            const int32_t *grank, const double *U, double *dst, cudaStream_t s);
void launch_permute_in(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                       const double *src, double *U, float *U32, cudaStream_t s);
void launch_permute_out(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                        const double *U, double *dst, cudaStream_t s);
// Load the kernel of launch_permute_out on the current device (lazy module loading).
cudaError_t preload_permute_out();
// Device address, on the current device, of the staging array of the allocation-free read-back
// (noalloc.cu) and its capacity in doubles.
cudaError_t noalloc_stage_address(double **out, int64_t *capacity);

// 16-byte vector access to records (the records are 16-byte aligned by construction).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void unpack(const float4 &x, float *o) {
    o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  }
  __device__ __forceinline__ static float4 pack(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void unpack(const double2 &x, double *o) {
    o[0] = x.x; o[1] = x.y;
  }
  __device__ __forceinline__ static double2 pack(const double *o) { return make_double2(o[0], o[1]); }
};

// Load / store COUNT (a multiple of 16 / sizeof(T)) consecutive values from / to a 16-byte
// aligned address. Global loads (SH = false) go through the read-only path: use them only on data
// the kernel does not write; SH = true reads a shared-memory copy.
template <typename T, int COUNT, bool SH = false>
__device__ __forceinline__ void load16(const T *__restrict__ src, T *dst) {
  using V = Vec16<T>;
  static_assert(COUNT % V::n == 0, "record not a multiple of 16 bytes");
#pragma unroll
  for (int c = 0; c < COUNT / V::n; ++c) {
    if constexpr (SH)
      V::unpack(reinterpret_cast<const typename V::type *>(src)[c], dst + c * V::n);
    else
      V::unpack(__ldg(reinterpret_cast<const typename V::type *>(src) + c), dst + c * V::n);
  }
}
#ifdef __CUDACC__
// Programmatic dependent launch of the stage kernels: the next kernel of the stream is launched
// as this kernel's blocks exit (before its completion has been processed) and runs its prologue
// that does not depend on it (barrier set-up, basis tables, the first bulk copies of operator
// records); pdl_wait then holds each thread, before its first access to data that the previous
// kernel produces or still reads, until that kernel has completed and its writes are visible.
// No kernel triggers its dependents early: measured, blocks of the next kernel that start
// during a kernel's work hold SM resources it needs (6-13 % slower steps).
__device__ __forceinline__ void pdl_wait(const KArgs &a) {
  if (a.pdl) asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Launch a stage kernel, with the programmatic-serialisation attribute when a.pdl is set.
inline void launch_stage_kernel(void (*kern)(KArgs), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                                const KArgs &a) {
  if (!a.pdl) {
    kern<<<grid, block, smem, s>>>(a);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, a);
}

// Streamed operator records (read once per cell): 16-byte read-only global loads that do not
// allocate in L1 (kept for the reused neighbour means) and ask L2 for 256-byte blocks (the next
// chunks of the same record arrive with the first miss).
template <typename T, int COUNT>
__device__ __forceinline__ void load16_stream(const T *__restrict__ src, T *dst) {
  static_assert(COUNT % (16 / sizeof(T)) == 0, "record not a multiple of 16 bytes");
#pragma unroll
  for (int c = 0; c < COUNT * (int)sizeof(T) / 16; ++c) {
    if constexpr (sizeof(T) == 4) {
      float4 x;
      asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
          : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
          : "l"(reinterpret_cast<const float4 *>(src) + c));
      dst[4 * c] = x.x; dst[4 * c + 1] = x.y; dst[4 * c + 2] = x.z; dst[4 * c + 3] = x.w;
    } else {
      double2 x;
      asm("ld.global.nc.L1::no_allocate.L2::256B.v2.f64 {%0, %1}, [%2];"
          : "=d"(x.x), "=d"(x.y)
          : "l"(reinterpret_cast<const double2 *>(src) + c));
      dst[2 * c] = x.x; dst[2 * c + 1] = x.y;
    }
  }
}
template <bool SH>
__device__ __forceinline__ int4 load_i4(const int32_t *__restrict__ src) {
  if constexpr (SH) return *reinterpret_cast<const int4 *>(src);
  else return __ldg(reinterpret_cast<const int4 *>(src));
}
template <bool SH>
__device__ __forceinline__ int32_t load_i1(const int32_t *__restrict__ src) {
  if constexpr (SH) return *src;
  else return __ldg(src);
}
#endif
template <typename T, int COUNT>
__device__ __forceinline__ void store16(T *__restrict__ dstp, const T *src) {
  using V = Vec16<T>;
  static_assert(COUNT % V::n == 0, "record not a multiple of 16 bytes");
#pragma unroll
  for (int c = 0; c < COUNT / V::n; ++c)
    reinterpret_cast<typename V::type *>(dstp)[c] = V::pack(src + c * V::n);
}

}  // namespace cteno
