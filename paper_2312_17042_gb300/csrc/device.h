// device.h -- device buffers, kernel argument block and launcher declarations.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace cteno {

// Bits of the per-cell word `cinfo`:
//   [4f, 4f+4)   members of the directional stencil of local face f (its first slots in the
//                device stencil list are those members, face after face)
//   16 + f       directional stencil of face f admissible (set by the least-squares build)
//   20 + 3f      index of the permutation taking the face's local vertex slots to the order of
//                their global ids (canonical Gauss-point order)
constexpr int kInfoAdmShift = 16;
constexpr int kInfoPermShift = 20;
// Bits of `fmeta`: [2f, 2f+2) neighbour's local face; 8 + f: this cell owns face f (computes the
// flux in its own orientation; the other cell uses the exact negative normal and negates).
constexpr int kMetaOwnerShift = 8;

// Error word bits.
constexpr int kErrNonFinite = 1;
constexpr int kErrRank = 2;

// Device tables (a copy of Tables with the fields the kernels read).
struct DevTables {
  int nk, nq, nperm, nvq;
  int ex[kMaxNK][3];
  double psibar[kMaxNK];
  double O[kMaxNK][kMaxNK];
  double Phi[kMaxNF][kMaxPerm][kMaxNQ][kMaxNK];
  double fw[kMaxNQ];
  double vq[8][3];
  double vw[8];
};

// Everything a kernel touches, passed by value. Arrays are structure-of-arrays over the N cells
// in device order: element e of cell c is base[e * N + c].
struct KArgs {
  int64_t N;
  int nmesh;
  const int64_t *mesh_off;  // [nmesh + 1] first device cell of each mesh
  // state
  double *U;                // [nv][N] FP64 cell means of the current stage
  double *Un;               // [nv][N] U^n, start of the step
  float *U32;               // [nv][N] float2 (hi, lo) split of U: hi = fl32(U), lo = fl32(U - hi)
  // stencils and least-squares operators
  const int32_t *st;        // [M][N] device stencil ids (directional members first)
  const uint32_t *cinfo;    // [N]
  const void *Pc;           // [nk][M][N] central pseudo-inverse (T)
  const void *Pd;           // [nf][d][2d][N] directional pseudo-inverses (T)
  void *Uf;                 // [nf][nq][nv][N] face Gauss-point states (T)
  uint8_t *flags;           // [nv][N] selection flags, or null
  // faces and geometry
  const int32_t *nbr;       // [nf][N] neighbour device id, -1 on a boundary
  const uint32_t *fmeta;    // [N]
  const double *fn;         // [nf][d][N] outward unit normal (exact negative across a face)
  const double *fa;         // [nf][N] face area
  const float *fn32;        // FP32 copies (mixed path)
  const float *fa32;
  const double *vol;        // [N]
  double *dt;               // [2 * nmesh]: [0..nmesh) current step, [nmesh..2 nmesh) next step
  const DevTables *tab;
  int *err;
  unsigned long long *guard;
  // parameters
  double C_T, lambda1p, eps, gamma, cfl;
  int lam_gamma, guard_on;
  int stage;                // 0, 1, 2
  int dt_swap;              // stage 0 of a CFL step: move dt[next] to dt[cur] first
};

// Set-up (FP64): geometry, moments, Householder QR, pseudo-inverses.
struct SetupArgs {
  int64_t N;
  const double *X;          // [N][d+1][d] unwrapped, oriented vertices
  const int32_t *st;        // [M][N]
  uint32_t *cinfo;          // [N] (admissibility bits written)
  const int32_t *nbr;       // [nf][N]
  const uint32_t *fmeta;
  double period[3];
  void *Pc, *Pd;            // outputs, T = double (FP64 path) or float (mixed path)
  int store_fp32;
  double *fn, *fa, *vol;
  float *fn32, *fa32;
  const DevTables *tab;
  int *err;
};

void launch_setup(int dim, int degree, const SetupArgs &a, cudaStream_t s);
void launch_flux(int dim, int fp32, const KArgs &a, int block, cudaStream_t s);
void launch_dt(int dim, const KArgs &a, cudaStream_t s);
void launch_dt_reset(const KArgs &a, cudaStream_t s);
void launch_permute_in(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                       const double *src, double *U, float *U32, cudaStream_t s);
void launch_permute_out(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                        const double *U, double *dst, cudaStream_t s);

}  // namespace cteno

namespace cteno {
void launch_recon_2d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s);
void launch_recon_3d(int degree, int fp32, int scheme, const KArgs &a, int block, cudaStream_t s);
inline void launch_recon(int dim, int degree, int fp32, int scheme, const KArgs &a, int block,
                         cudaStream_t s) {
  if (dim == 2) launch_recon_2d(degree, fp32, scheme, a, block, s);
  else launch_recon_3d(degree, fp32, scheme, a, block, s);
}
}  // namespace cteno
