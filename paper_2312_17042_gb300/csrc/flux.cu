// flux.cu -- per-cell flux gather, residual and SSP-RK3 update (paper eq. 2, Sec. 2.7), the
// CFL time step, and the state permutation kernels.
//
// Every cell computes the HLLC flux (eqs. 24-29) at the Gauss points of its own faces, so no
// atomics are needed. A face is evaluated in the orientation of its owner on both sides, with
// the same operands in the same order and a normal that is the exact negative of the other
// side's, so the two cells obtain bit-identical fluxes and the update is exactly conservative.
#include <cfloat>

#include "device.h"

namespace cteno {
namespace {

template <int D, typename T>
__device__ __forceinline__ void physical_flux(const T *u, const T *n, T p, T un, T *F) {
  F[0] = u[0] * un;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = u[1 + j] * un + p * n[j];
  F[D + 1] = (u[D + 1] + p) * un;
}

// HLLC flux through a face with unit normal n from state uL (inside) to uR (outside). Wave
// speeds of eq. 25 with the Roe averages of eq. 26 (full averaged velocity in the sound speed),
// contact speed and star pressure of eq. 28, star states of eq. 29 in vector form.
template <int D, typename T>
__device__ __forceinline__ void hllc(const T *uL, const T *uR, const T *n, T g, T *F) {
  constexpr int NV = D + 2;
  const T rL = uL[0], rR = uR[0];
  const T iL = (T)1 / rL, iR = (T)1 / rR;
  T vL[D], vR[D], unL = 0, unR = 0, kL = 0, kR = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vL[j] = uL[1 + j] * iL;
    vR[j] = uR[1 + j] * iR;
    unL += vL[j] * n[j];
    unR += vR[j] * n[j];
    kL += vL[j] * uL[1 + j];
    kR += vR[j] * uR[1 + j];
  }
  const T pL = (g - (T)1) * (uL[NV - 1] - (T)0.5 * kL);
  const T pR = (g - (T)1) * (uR[NV - 1] - (T)0.5 * kR);
  const T cL = sqrt(g * pL * iL), cR = sqrt(g * pR * iR);
  const T HL = (uL[NV - 1] + pL) * iL, HR = (uR[NV - 1] + pR) * iR;
  const T Dr = sqrt(rR * iL);
  const T idn = (T)1 / ((T)1 + Dr);
  T ut2 = 0, utn = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const T ut = (vL[j] + vR[j] * Dr) * idn;
    ut2 += ut * ut;
    utn += ut * n[j];
  }
  const T Ht = (HL + HR * Dr) * idn;
  const T ct = sqrt((g - (T)1) * (Ht - (T)0.5 * ut2));
  const T SL = fmin(unL - cL, utn - ct);
  const T SR = fmax(unR + cR, utn + ct);
  const T SM = (rR * unR * (SR - unR) - rL * unL * (SL - unL) + pL - pR) /
               (rR * (SR - unR) - rL * (SL - unL));
  if (SL > (T)0) {
    physical_flux<D, T>(uL, n, pL, unL, F);
  } else if (SM > (T)0) {
    const T ps = rL * (unL - SL) * (unL - SM) + pL;
    const T fct = (T)1 / (SL - SM), a = SL - unL;
    physical_flux<D, T>(uL, n, pL, unL, F);
    F[0] += SL * (rL * a * fct - uL[0]);
#pragma unroll
    for (int j = 0; j < D; ++j) F[1 + j] += SL * ((a * uL[1 + j] + (ps - pL) * n[j]) * fct - uL[1 + j]);
    F[NV - 1] += SL * ((a * uL[NV - 1] - pL * unL + ps * SM) * fct - uL[NV - 1]);
  } else if (SR > (T)0) {
    const T ps = rL * (unL - SL) * (unL - SM) + pL;
    const T fct = (T)1 / (SR - SM), a = SR - unR;
    physical_flux<D, T>(uR, n, pR, unR, F);
    F[0] += SR * (rR * a * fct - uR[0]);
#pragma unroll
    for (int j = 0; j < D; ++j) F[1 + j] += SR * ((a * uR[1 + j] + (ps - pR) * n[j]) * fct - uR[1 + j]);
    F[NV - 1] += SR * ((a * uR[NV - 1] - pR * unR + ps * SM) * fct - uR[NV - 1]);
  } else {
    physical_flux<D, T>(uR, n, pR, unR, F);
  }
}

__device__ __forceinline__ int mesh_of(const KArgs &a, int64_t i) {
  int lo = 0, hi = a.nmesh - 1;
  while (lo < hi) {  // last mesh whose offset <= i
    const int mid = (lo + hi + 1) >> 1;
    if (a.mesh_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Order-preserving map of a non-negative double onto unsigned 64-bit (for an atomic minimum).
__device__ __forceinline__ void atomic_min_pos(double *addr, double v) {
  atomicMin((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Local CFL step of one cell: |V_i| / sum_f |A_f| (|u_i . n_f| + c_i).
template <int D>
__device__ __forceinline__ double local_dt(const KArgs &a, int64_t i, const double *u) {
  const int64_t N = a.N;
  const double ir = 1.0 / u[0];
  double ke = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) ke += u[1 + j] * u[1 + j];
  const double p = (a.gamma - 1.0) * (u[D + 1] - 0.5 * ke * ir);
  const double c = sqrt(a.gamma * p * ir);
  double s = 0.0;
#pragma unroll
  for (int f = 0; f < D + 1; ++f) {
    double un = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) un += u[1 + j] * ir * a.fn[(f * D + j) * N + i];
    s += a.fa[f * N + i] * (fabs(un) + c);
  }
  return a.vol[i] / s;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) flux_kernel(const KArgs a) {
  constexpr int NV = D + 2, NF = D + 1, NQ = (D == 2) ? 2 : 4;
  const int64_t N = a.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T *__restrict__ Uf = (const T *)a.Uf;
  const T *__restrict__ fnT = (sizeof(T) == 4) ? (const T *)a.fn32 : (const T *)a.fn;
  const T *__restrict__ faT = (sizeof(T) == 4) ? (const T *)a.fa32 : (const T *)a.fa;
  const T g = (T)a.gamma;
  const uint32_t meta = a.fmeta[i];
  T Ui[NV];  // cell mean, the outside state of a transmissive face
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if constexpr (sizeof(T) == 4) {
      const float2 h = ((const float2 *)a.U32)[v * N + i];
      Ui[v] = h.x + h.y;
    } else {
      Ui[v] = a.U[v * N + i];
    }
  }
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const DevTables &tb = *a.tab;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t j = a.nbr[f * N + i];
    const int fj = (meta >> (2 * f)) & 3u;
    const bool own = (meta >> (kMetaOwnerShift + f)) & 1u;
    T n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = own ? fnT[(f * D + k) * N + i] : -fnT[(f * D + k) * N + i];
    const T area = faT[f * N + i];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T uI[NV], uO[NV], F[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uI[v] = Uf[((int64_t)(f * NQ + q) * NV + v) * N + i];
        uO[v] = (j >= 0) ? Uf[((int64_t)(fj * NQ + q) * NV + v) * N + j] : Ui[v];
      }
      if (own) hllc<D, T>(uI, uO, n, g, F);
      else hllc<D, T>(uO, uI, n, g, F);
      const double w = (double)area * tb.fw[q];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += own ? w * (double)F[v] : -w * (double)F[v];
    }
  }
  // residual and SSP-RK3 (Shu-Osher) stage update in FP64
  const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
  const double dt = a.dt[mesh];
  const double ivol = 1.0 / a.vol[i];
  double un[NV];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double u = a.U[v * N + i];
    const double upd = u - dt * acc[v] * ivol;
    double res;
    if (a.stage == 0) {
      a.Un[v * N + i] = u;
      res = upd;
    } else if (a.stage == 1) {
      res = 0.75 * a.Un[v * N + i] + 0.25 * upd;
    } else {
      res = (1.0 / 3.0) * a.Un[v * N + i] + (2.0 / 3.0) * upd;
    }
    un[v] = res;
    finite = finite && isfinite(res);
    a.U[v * N + i] = res;
    if (a.U32) {
      const float hi = (float)res;
      ((float2 *)a.U32)[v * N + i] = make_float2(hi, (float)(res - (double)hi));
    }
  }
  if (!finite) atomicOr(a.err, kErrNonFinite);
  if (a.stage == 2 && finite) atomic_min_pos(&a.dt[a.nmesh + mesh], a.cfl * local_dt<D>(a, i, un));
}

template <int D>
__global__ void dt_kernel(const KArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  double u[D + 2];
#pragma unroll
  for (int v = 0; v < D + 2; ++v) u[v] = a.U[v * a.N + i];
  const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
  atomic_min_pos(&a.dt[a.nmesh + mesh], a.cfl * local_dt<D>(a, i, u));
}

__global__ void dt_reset_kernel(double *dt, int nmesh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nmesh) dt[nmesh + i] = 1e300;
}

// src[v][c] (caller order, mesh of n cells) -> U[v][off + rank[c]] (+ FP32 shadow)
__global__ void permute_in_kernel(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                                  const double *src, double *U, float *U32) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t g = off + rank[c];
  for (int v = 0; v < nv; ++v) {
    const double x = src[v * n + c];
    U[v * N + g] = x;
    if (U32) {
      const float hi = (float)x;
      ((float2 *)U32)[v * N + g] = make_float2(hi, (float)(x - (double)hi));
    }
  }
}

__global__ void permute_out_kernel(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                                   const double *U, double *dst) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t g = off + rank[c];
  for (int v = 0; v < nv; ++v) dst[v * n + c] = U[v * N + g];
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

void launch_flux(int dim, int fp32, const KArgs &a, int block, cudaStream_t s) {
  const unsigned grid = grid_for(a.N, block);
  if (dim == 2 && fp32) flux_kernel<2, float><<<grid, block, 0, s>>>(a);
  if (dim == 2 && !fp32) flux_kernel<2, double><<<grid, block, 0, s>>>(a);
  if (dim == 3 && fp32) flux_kernel<3, float><<<grid, block, 0, s>>>(a);
  if (dim == 3 && !fp32) flux_kernel<3, double><<<grid, block, 0, s>>>(a);
}

void launch_dt(int dim, const KArgs &a, cudaStream_t s) {
  dt_reset_kernel<<<grid_for(a.nmesh, 64), 64, 0, s>>>(a.dt, a.nmesh);
  if (dim == 2) dt_kernel<2><<<grid_for(a.N, 256), 256, 0, s>>>(a);
  else dt_kernel<3><<<grid_for(a.N, 256), 256, 0, s>>>(a);
}

void launch_dt_reset(const KArgs &a, cudaStream_t s) {
  dt_reset_kernel<<<grid_for(a.nmesh, 64), 64, 0, s>>>(a.dt, a.nmesh);
}

void launch_permute_in(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                       const double *src, double *U, float *U32, cudaStream_t s) {
  permute_in_kernel<<<grid_for(n, 256), 256, 0, s>>>(nv, n, N, off, rank, src, U, U32);
}

void launch_permute_out(int nv, int64_t n, int64_t N, int64_t off, const int32_t *rank,
                        const double *U, double *dst, cudaStream_t s) {
  permute_out_kernel<<<grid_for(n, 256), 256, 0, s>>>(nv, n, N, off, rank, U, dst);
}

}  // namespace cteno
