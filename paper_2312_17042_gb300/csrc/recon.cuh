// recon.cuh -- the per-cell reconstruction kernel (templated on dimension, degree, arithmetic
// type and scheme). One thread per cell, all conserved variables of the cell in registers.
//
// Steps, per cell i (paper Sec. 2.1-2.6):
//   1. gather the stencil cell means and form U_m - U_0 (eq. 10);
//   2. a_opt = P_c (U_m - U_0) for the central stencil and a_s = P_s (U_m - U_0) for each
//      directional stencil (eq. 12 with the pseudo-inverses built by setup.cu);
//   3. p_1 = (p_opt - sum_{s>=2} lambda_s p_s) / lambda_1 with lambda from eq. 18 (eq. 17);
//   4. smoothness indicators SI = a^T O a (eq. 15), O the universal matrix of the basis;
//   5. CTENO (Alg. 1) or CTENOZ (Alg. 2) scale separation, cut-off delta_s (eqs. 22-23) and
//      the final polynomial;
//   6. its values at the face Gauss points, U_0 + sum_k a_k phi_k(xi_q) (eq. 2).
//
// Memory: the cell's pseudo-inverse record (the dominant stream) is read once with 16-byte
// loads in member-major order, interleaved with the gathers of the stencil means it multiplies;
// stencil means come from neighbouring records (L1/L2 hits after the Morton renumbering).
#pragma once

#include <algorithm>
#include <cstdint>

#include "bulk.cuh"
#include "device.h"

namespace cteno {

template <int D, int R>
struct Shape {
  static constexpr int NK = (D == 2 ? (R + 1) * (R + 2) / 2 : (R + 1) * (R + 2) * (R + 3) / 6) - 1;
  static constexpr int M = 2 * (NK + 1);
  static constexpr int NP = (D == 2) ? 2 : 6;
};

// Constant-bank copies of the universal tables of this module's degrees (filled by
// upload_recon_tables_*): the smoothness matrix O (eq. 15; upper triangle, off-diagonal doubled) and, in 2D, the face-point basis values
// phi_k at the two Gauss points of each local edge taken in local vertex order (the other edge
// orientation visits the same two symmetric points in the opposite order). Indexed with
// compile-time offsets only, so they become instruction operands.
constexpr int kLowNK = 19;  // unknowns of degree <= 3 (a cubic in 3D)
__constant__ double c_O_r2d[kLowNK * kLowNK], c_O_r3d[kLowNK * kLowNK];
__constant__ float c_O_r2f[kLowNK * kLowNK], c_O_r3f[kLowNK * kLowNK];
__constant__ double c_Phi2_r2d[3 * 2 * kLowNK], c_Phi2_r3d[3 * 2 * kLowNK];
__constant__ float c_Phi2_r2f[3 * 2 * kLowNK], c_Phi2_r3f[3 * 2 * kLowNK];

// 3D, FP32: the face rule's points in barycentric coordinates of the face's sorted vertices and
// the basis means psibar_k, for the face values of the polynomial evaluated at the point.
__constant__ float c_fbary3f[4 * 3];
__constant__ float c_psibar3_r2f[kLowNK], c_psibar3_r3f[kLowNK];

template <typename T, int R>
__device__ __forceinline__ T cO(int idx) {
  if constexpr (R == 2) {
    if constexpr (sizeof(T) == 4) return c_O_r2f[idx]; else return c_O_r2d[idx];
  } else {
    if constexpr (sizeof(T) == 4) return c_O_r3f[idx]; else return c_O_r3d[idx];
  }
}
template <typename T, int R>
__device__ __forceinline__ T cPhi2(int idx) {
  if constexpr (R == 2) {
    if constexpr (sizeof(T) == 4) return c_Phi2_r2f[idx]; else return c_Phi2_r2d[idx];
  } else {
    if constexpr (sizeof(T) == 4) return c_Phi2_r3f[idx]; else return c_Phi2_r3d[idx];
  }
}

// Host side: copy O and the 2D edge values of degree r into this module's constant banks.
inline cudaError_t upload_recon_tables(int dim, int degree, const Tables &t, cudaStream_t s) {
  double Od[kLowNK * kLowNK] = {}, Pd2[3 * 2 * kLowNK] = {};
  float Of[kLowNK * kLowNK] = {}, Pf2[3 * 2 * kLowNK] = {};
  if (t.nk > kLowNK) return cudaErrorInvalidValue;
  // O is symmetric: the kernels use the upper triangle only, with the off-diagonal entries doubled
  // (exact), a^T O a = sum_k a_k (O_kk a_k + sum_{l>k} 2 O_kl a_l)
  for (int k = 0; k < t.nk; ++k)
    for (int l = k; l < t.nk; ++l) {
      Od[k * t.nk + l] = (l == k ? 1.0 : 2.0) * t.O[k][l];
      Of[k * t.nk + l] = (float)Od[k * t.nk + l];
    }
  if (dim == 2)
    for (int f = 0; f < 3; ++f)
      for (int q = 0; q < 2; ++q)
        for (int k = 0; k < t.nk; ++k) {
          Pd2[(f * 2 + q) * t.nk + k] = t.Phi[f][0][q][k];
          Pf2[(f * 2 + q) * t.nk + k] = (float)t.Phi[f][0][q][k];
        }
  float fb[4 * 3] = {}, pb[kLowNK] = {};
  if (dim == 3) {
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < 3; ++j) fb[q * 3 + j] = (float)t.fbary[q][j];
    for (int k = 0; k < t.nk; ++k) pb[k] = (float)t.psibar[k];
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbolAsync(c_fbary3f, fb, sizeof(fb), 0, cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyToSymbolAsync(degree == 2 ? c_psibar3_r2f : c_psibar3_r3f, pb, sizeof(pb), 0,
                                   cudaMemcpyHostToDevice, s)))
    return e;
  if (degree == 2) {
    if ((e = cudaMemcpyToSymbolAsync(c_O_r2d, Od, sizeof(Od), 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_O_r2f, Of, sizeof(Of), 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_Phi2_r2d, Pd2, sizeof(Pd2), 0, cudaMemcpyHostToDevice, s))) return e;
    e = cudaMemcpyToSymbolAsync(c_Phi2_r2f, Pf2, sizeof(Pf2), 0, cudaMemcpyHostToDevice, s);
  } else {
    if ((e = cudaMemcpyToSymbolAsync(c_O_r3d, Od, sizeof(Od), 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_O_r3f, Of, sizeof(Of), 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_Phi2_r3d, Pd2, sizeof(Pd2), 0, cudaMemcpyHostToDevice, s))) return e;
    e = cudaMemcpyToSymbolAsync(c_Phi2_r3f, Pf2, sizeof(Pf2), 0, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // the host arrays above go out of scope
}

template <typename T>
__device__ __forceinline__ T pow6(T x) {
  const T x2 = x * x;
  return x2 * x2 * x2;
}
template <typename T>
__device__ __forceinline__ T pow4(T x) {
  const T x2 = x * x;
  return x2 * x2;
}

// Selection of eqs. 19-23 / Alg. 1-2 in FP64, as printed (gamma_s times lambda_s when
// lam_gamma). SI0: central; SId[f]: directional stencil of face f, used where bit f of adm is
// set. CTENOZ form 0: tau = (mean |SI_s - SI_1|)^6, gamma = 1 + tau / (SI + eps) (as printed);
// form 1: tau = mean |SI_s - SI_1|, gamma = 1 + (tau / (SI + eps))^6 (the WENO-Z arrangement).
// Returns delta bits: bit 0 central, bit 1 + f directional f.
template <int NF>
__device__ __forceinline__ uint32_t select_fp64(double SI0, const double *SId, uint32_t adm, int st,
                                                int scheme, int form, int lam_gamma, double lam1, double lams,
                                                double eps, double C_T) {
  double g0, gd[NF];
  if (scheme == 0) {
    g0 = 1.0 / pow6(SI0 + eps);
#pragma unroll
    for (int f = 0; f < NF; ++f) gd[f] = 1.0 / pow6(SId[f] + eps);
  } else {
    double tau = 0.0;
    if (st > 1) {
      double acc = 0.0;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if ((adm >> f) & 1u) acc += fabs(SId[f] - SI0);
      tau = acc / (st - 1);
      if (form == 0) tau = pow6(tau);
    }
    if (form == 0) {
      g0 = 1.0 + tau / (SI0 + eps);
#pragma unroll
      for (int f = 0; f < NF; ++f) gd[f] = 1.0 + tau / (SId[f] + eps);
    } else {
      g0 = 1.0 + pow6(tau / (SI0 + eps));
#pragma unroll
      for (int f = 0; f < NF; ++f) gd[f] = 1.0 + pow6(tau / (SId[f] + eps));
    }
  }
  if (lam_gamma) {
    g0 *= lam1;
#pragma unroll
    for (int f = 0; f < NF; ++f) gd[f] *= lams;
  }
  double sum = g0;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if ((adm >> f) & 1u) sum += gd[f];
  uint32_t bits = (g0 / sum < C_T) ? 0u : 1u;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if (((adm >> f) & 1u) && !(gd[f] / sum < C_T)) bits |= 1u << (1 + f);
  return bits;
}

// Base-2 logarithm and power with the GPU's single-instruction approximations (relative error
// about 2^-22, subnormals flushed to zero). The FP32 eps is at least the smallest normal number,
// so SI + eps is normal; a power below it contributes nothing to a decision against C_T.
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tab[k] for k in [0, N] through selects on compile-time offsets (a kernel parameter array is
// then read from the constant bank without a local copy).
template <int N, typename X>
__device__ __forceinline__ X pick(const X *tab, int k) {
  X r = tab[0];
#pragma unroll
  for (int j = 1; j <= N; ++j)
    if (k == j) r = tab[j];
  return r;
}

// The same decision in FP32 without overflow: every gamma_s is carried as its base-2 logarithm
// L_s, and chi_s = 2^(L_s - Lmax) / sum_t 2^(L_t - Lmax); chi_s < C_T is tested as
// 2^(L_s - Lmax) < C_T sum_t 2^(L_t - Lmax) (no division). inv_stm1 = 1 / (st - 1).
template <int NF>
__device__ __forceinline__ uint32_t select_fp32(float SI0, const float *SId, uint32_t adm, int st,
                                                int scheme, int form, int lam_gamma, float log2lam1,
                                                float log2lams, float inv_stm1, float eps, float C_T) {
  float L0, Ld[NF];
  if (scheme == 0) {
    L0 = -6.0f * lg2_approx(SI0 + eps);
#pragma unroll
    for (int f = 0; f < NF; ++f) Ld[f] = -6.0f * lg2_approx(SId[f] + eps);
  } else {
    float lt = -INFINITY;  // log2 of the mean |SI_s - SI_1|
    if (st > 1) {
      float acc = 0.0f;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if ((adm >> f) & 1u) acc += fabsf(SId[f] - SI0);
      lt = lg2_approx(acc * inv_stm1);
    }
    // log2(1 + 2^x), split to stay accurate for any x; x = log2 of the term added to 1:
    // form 0 tau / (SI + eps) with tau = mean^6, form 1 (mean / (SI + eps))^6
    auto l1p = [](float x) {
      return (x > 0.0f) ? x + lg2_approx(1.0f + ex2_approx(-x)) : lg2_approx(1.0f + ex2_approx(x));
    };
    if (form == 0) {
      const float lt6 = 6.0f * lt;
      L0 = l1p(lt6 - lg2_approx(SI0 + eps));
#pragma unroll
      for (int f = 0; f < NF; ++f) Ld[f] = l1p(lt6 - lg2_approx(SId[f] + eps));
    } else {
      L0 = l1p(6.0f * (lt - lg2_approx(SI0 + eps)));
#pragma unroll
      for (int f = 0; f < NF; ++f) Ld[f] = l1p(6.0f * (lt - lg2_approx(SId[f] + eps)));
    }
  }
  if (lam_gamma) {
    L0 += log2lam1;
#pragma unroll
    for (int f = 0; f < NF; ++f) Ld[f] += log2lams;
  }
  float Lmax = L0;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if ((adm >> f) & 1u) Lmax = fmaxf(Lmax, Ld[f]);
  const float e0 = ex2_approx(L0 - Lmax);
  float ed[NF], sum = e0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    ed[f] = ex2_approx(Ld[f] - Lmax);
    if ((adm >> f) & 1u) sum += ed[f];
  }
  const float cut = C_T * sum;
  uint32_t bits = (e0 < cut) ? 0u : 1u;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if (((adm >> f) & 1u) && !(ed[f] < cut)) bits |= 1u << (1 + f);
  return bits;
}

// One cell of the thread-per-cell schedule. Pci, Pdi, sti: the cell's central pseudo-inverse,
// directional operators and stencil ids, in global memory (SH = false) or in a shared-memory copy
// (SH = true); sPhi: 3D face-point basis values in shared memory.
// CWENO nonlinear weights (Sec. 2.3: the weights of eq. 14 with b = 4 on the linear coefficients
// of eq. 18): w~_s = lambda_s / (eps + SI_s)^4, normalised over the admissible stencils. FP64 as
// written; FP32 in the base-2 log domain like select_fp32 (no overflow of (eps + SI)^-4).
template <int NF>
__device__ __forceinline__ void cweno_weights(double SI0, const double *SId, uint32_t adm, double lam1,
                                              double lams, double eps, double &w0, double *wd) {
  const double g0 = lam1 / pow4(eps + SI0);
  double g[NF], sum = g0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    g[f] = ((adm >> f) & 1u) ? lams / pow4(eps + SId[f]) : 0.0;
    sum += g[f];
  }
  w0 = g0 / sum;
#pragma unroll
  for (int f = 0; f < NF; ++f) wd[f] = g[f] / sum;
}
template <int NF>
__device__ __forceinline__ void cweno_weights(float SI0, const float *SId, uint32_t adm, float log2lam1,
                                              float log2lams, float eps, float &w0, float *wd) {
  const float L0 = log2lam1 - 4.0f * lg2_approx(SI0 + eps);
  float Ld[NF], Lmax = L0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    Ld[f] = log2lams - 4.0f * lg2_approx(SId[f] + eps);
    if ((adm >> f) & 1u) Lmax = fmaxf(Lmax, Ld[f]);
  }
  const float e0 = ex2_approx(L0 - Lmax);
  float sum = e0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    wd[f] = ((adm >> f) & 1u) ? ex2_approx(Ld[f] - Lmax) : 0.0f;
    sum += wd[f];
  }
  const float inv = 1.0f / sum;
  w0 = e0 * inv;
#pragma unroll
  for (int f = 0; f < NF; ++f) wd[f] *= inv;
}

// Own cell means of cell i: FP64, or (mixed path) the FP32 pair hi + lo of every FP64 value, so
// that U_m - U_0 = (hi_m - hi_0) + (lo_m - lo_0) keeps FP64 accuracy in FP32 arithmetic.
template <int D, typename T>
__device__ __forceinline__ void cell_own(const KArgs &a, const int64_t i, T (&U0)[Lay<D>::NV],
                                         float (&L0)[Lay<D>::NV]) {
  constexpr int NV = Lay<D>::NV, NVP = Lay<D>::NVP;
  if constexpr (sizeof(T) == 4) {
    float hl[2 * NVP];
    load16<float, 2 * NVP>(a.U32 + i * 2 * NVP, hl);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      U0[v] = hl[2 * v];
      L0[v] = hl[2 * v + 1];
    }
  } else {
    double u[NVP];
    load16<double, NVP>(a.U + i * NVP, u);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      U0[v] = (T)u[v];
      L0[v] = 0.0f;
    }
  }
}

// U_j - U_0 for every variable (eq. 10), from member j's record.
template <int D, typename T>
__device__ __forceinline__ void cell_delta(const KArgs &a, const int64_t j, const T (&U0)[Lay<D>::NV],
                                           const float (&L0)[Lay<D>::NV], T *du) {
  constexpr int NV = Lay<D>::NV, NVP = Lay<D>::NVP;
  if constexpr (sizeof(T) == 4) {
    float hl[2 * NVP];
    load16<float, 2 * NVP>(a.U32 + j * 2 * NVP, hl);
#pragma unroll
    for (int v = 0; v < NV; ++v) du[v] = (T)((hl[2 * v] - (float)U0[v]) + (hl[2 * v + 1] - L0[v]));
  } else {
    double u[NVP];
    load16<double, NVP>(a.U + j * NVP, u);
#pragma unroll
    for (int v = 0; v < NV; ++v) du[v] = (T)(u[v] - (double)U0[v]);
  }
}

// The second half of the thread-per-cell schedule, from the central coefficients ao of every
// variable: the directional coefficients, p_1 (eq. 17), the smoothness indicators (eq. 15), the
// selection (eqs. 19-23, Alg. 1 / 2), the final coefficients and the values at the face Gauss
// points with the positivity guard. Pdi, sti: the cell's directional operators and stencil ids in
// global memory (SH = false) or in a shared-memory copy (SH = true).
template <int D, int R, typename T, int SCHEME, bool SH>
__device__ __forceinline__ void cell_finish(const KArgs &a, const int64_t i,
                                            T (&ao)[Shape<D, R>::NK][Lay<D>::NV], const T (&U0)[Lay<D>::NV],
                                            const float (&L0)[Lay<D>::NV], const T *__restrict__ Pdi,
                                            const int32_t *__restrict__ sti, const T *__restrict__ sPhi) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NV = L::NV, NF = L::NF, NQ = L::NQ, ND = L::ND, PDS = L::PDS;
  constexpr int NK = S::NK, NP = S::NP;
  constexpr bool F32 = sizeof(T) == 4;
  const int64_t N = a.N;
  auto delta = [&](int64_t j, T *du) { cell_delta<D, T>(a, j, U0, L0, du); };

  // directional coefficients (degree 1): members of face f are the next slots of the list
  const uint32_t info = __ldg(a.cinfo + i);
  const uint32_t adm = (info >> kInfoAdmShift) & 0xFu;
  T ad[NF][D][NV];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) ad[f][k][v] = (T)0;
  {
    int off = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int nm = (info >> (4 * f)) & 15u;
      if ((adm >> f) & 1u) {
        T pf[PDS];
        if constexpr (SH) load16<T, PDS, true>(Pdi + f * PDS, pf);
        else load16_stream<T, PDS>(Pdi + f * PDS, pf);
#pragma unroll
        for (int jj = 0; jj < ND; ++jj) {
          if (jj < nm) {
            T du[NV];
            delta(load_i1<SH>(sti + off + jj), du);
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
              for (int v = 0; v < NV; ++v) ad[f][k][v] += pf[jj * D + k] * du[v];
          }
        }
      }
      off += nm;
    }
  }

  // 3: linear coefficients of eq. 18 over the admissible stencils (lambda_1 terms from the host)
  const int stn = 1 + __popc(adm);
  T lams;
  double lamsd = 0.0;
  float log2lams = 0.0f, inv_stm1 = 0.0f;
  if constexpr (F32) {
    lams = pick<NF>(a.lams_f, stn - 1);
    log2lams = pick<NF>(a.log2_lams_f, stn - 1);
    inv_stm1 = pick<NF>(a.inv_stm1_f, stn - 1);
  } else {
    lamsd = pick<NF>(a.lams_d, stn - 1);
    lams = lamsd;
  }
  T inv_lam1;
  if constexpr (F32) inv_lam1 = a.inv_lam1_32; else inv_lam1 = a.inv_lam1;
  const float log2lam1 = a.log2_lam1;
  constexpr T INV_FACT = (D == 2) ? (T)0.5 : (T)(1.0 / 6.0);

#pragma unroll
  for (int v = 0; v < NV; ++v) {
    // p_1 (eq. 17): the directional polynomials only touch the linear coefficients
    T a1[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) a1[k] = ao[k][v];
    if (stn > 1 && a.central_split) {  // TENO keeps p_opt (Sec. 2.4)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        T s = (T)0;
#pragma unroll
        for (int f = 0; f < NF; ++f) s += ad[f][k][v];  // inadmissible stencils hold zeros
        a1[k] -= lams * s;
      }
#pragma unroll
      for (int k = 0; k < NK; ++k) a1[k] *= inv_lam1;
    }
    // 4: smoothness indicators
    T SI0 = (T)0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      T r = (T)0;
#pragma unroll
      for (int l = k; l < NK; ++l) r += cO<T, R>(k * NK + l) * a1[l];
      SI0 += a1[k] * r;
    }
    T SId[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < D; ++k) s += ad[f][k][v] * ad[f][k][v];
      SId[f] = s * INV_FACT;
    }
    // 5: selection
    uint32_t bits;
    if (a.cweno) {  // CWENO (Sec. 2.3): every stencil, with the weights of eq. 14
      T w0, wd[NF];
      if constexpr (F32) cweno_weights<NF>(SI0, SId, adm, a.log2_lam1, log2lams, a.eps32, w0, wd);
      else cweno_weights<NF>(SI0, SId, adm, a.lam1, lamsd, a.eps, w0, wd);
#pragma unroll
      for (int k = 0; k < NK; ++k) ao[k][v] = w0 * a1[k];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < D; ++k) ao[k][v] += wd[f] * ad[f][k][v];  // zero weight where inadmissible
      bits = 1u | (adm << 1);
    } else {
      if constexpr (F32) {
        bits = select_fp32<NF>(SI0, SId, adm, stn, SCHEME, a.ctenoz_form, a.lam_gamma, log2lam1, log2lams,
                               inv_stm1, a.eps32, a.C_T32);
      } else {
        bits = select_fp64<NF>(SI0, SId, adm, stn, SCHEME, a.ctenoz_form, a.lam_gamma, a.lam1, lamsd, a.eps, a.C_T);
      }
      // final coefficients, written over a_opt
      if (bits & 1u) {
#pragma unroll
        for (int k = 0; k < NK; ++k) ao[k][v] = a1[k];
      } else {
        const T w = (T)1 / (T)__popc(bits >> 1);
#pragma unroll
        for (int k = 0; k < NK; ++k) ao[k][v] = (T)0;
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if ((bits >> (1 + f)) & 1u) {
#pragma unroll
            for (int k = 0; k < D; ++k) ao[k][v] += w * ad[f][k][v];
          }
      }
      if (bits & 1u) bits = 1u;
    }
    if (a.flags) a.flags[v * N + i] = (uint8_t)bits;
  }

  // 6: face Gauss-point values, one contiguous vector per face; positivity guard (not part of
  // the paper): a non-physical face state makes the cell use its mean at all its face points
  T *__restrict__ Ufi = (T *)a.Uf + i * (int64_t)(NF * NQ * NV);
  const uint32_t perm = info >> kInfoPermShift;
  T gm1;
  if constexpr (F32) gm1 = a.gm1_32; else gm1 = a.gamma - 1.0;
  bool bad = false;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int p = (perm >> (3 * f)) & 7u;
    T fb[NQ * NV];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T val = (T)L0[v];
        if constexpr (D == 2) {
#pragma unroll
          for (int k = 0; k < NK; ++k) val += cPhi2<T, R>((f * 2 + q) * NK + k) * ao[k][v];
        } else {
          const T *ph = &sPhi[((f * NP + p) * NQ) * NK];
#pragma unroll
          for (int k = 0; k < NK; ++k) val += ph[q * NK + k] * ao[k][v];
        }
        fb[q * NV + v] = val + U0[v];
      }
      T ke = (T)0;
#pragma unroll
      for (int j = 0; j < D; ++j) ke += fb[q * NV + 1 + j] * fb[q * NV + 1 + j];
      if constexpr (F32) {  // rho > 0 and p > 0, the latter as rho E - |m|^2 / 2 > 0 (no division)
        bad = bad || !(fb[q * NV] > 0.0f) || !(fb[q * NV] * fb[q * NV + NV - 1] - 0.5f * ke > 0.0f);
      } else {
        const T pr = gm1 * (fb[q * NV + NV - 1] - (T)0.5 * ke / fb[q * NV]);
        bad = bad || !(fb[q * NV] > (T)0) || !(pr > (T)0);
      }
    }
    if constexpr (D == 2) {  // edge stored in sorted-vertex order: swap the two points
      if (p) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T t = fb[v];
          fb[v] = fb[NV + v];
          fb[NV + v] = t;
        }
      }
    }
    store16<T, NQ * NV>(Ufi + f * NQ * NV, fb);
  }
  if (a.guard_on && bad) {
    T fb[NQ * NV];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int v = 0; v < NV; ++v) fb[q * NV + v] = U0[v] + (T)L0[v];
#pragma unroll
    for (int f = 0; f < NF; ++f) store16<T, NQ * NV>(Ufi + f * NQ * NV, fb);
    atomicAdd(a.guard, 1ull);
  }

}

template <int D, int R, typename T, int SCHEME, bool SH>
__device__ __forceinline__ void recon_cell(const KArgs &a, const int64_t i, const T *__restrict__ Pci,
                                           const T *__restrict__ Pdi, const int32_t *__restrict__ sti,
                                           const T *__restrict__ sPhi) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NV = L::NV;
  constexpr int NK = S::NK, M = S::M;
  constexpr int CH = Vec16<T>::n;
  T U0[NV];
  float L0[NV];
  cell_own<D, T>(a, i, U0, L0);

  // 1-2: central coefficients a_opt = P_c (U_m - U_0), streaming the member-major record
  T ao[NK][NV];
#pragma unroll
  for (int k = 0; k < NK; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) ao[k][v] = (T)0;
  {
    T pb[CH], du[NV];
    int ids[4];
#pragma unroll
    for (int e = 0; e < M * NK; ++e) {
      const int m = e / NK, k = e % NK;
      if (e % CH == 0) {
        if constexpr (SH) load16<T, CH, true>(Pci + e, pb);
        else load16_stream<T, CH>(Pci + e, pb);
      }
      if (k == 0) {
        if (m % 4 == 0) {
          const int4 t4 = load_i4<SH>(sti + m);
          ids[0] = t4.x; ids[1] = t4.y; ids[2] = t4.z; ids[3] = t4.w;
        }
        cell_delta<D, T>(a, ids[m % 4], U0, L0, du);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) ao[k][v] += pb[e % CH] * du[v];
    }
  }
  cell_finish<D, R, T, SCHEME, SH>(a, i, ao, U0, L0, Pdi, sti, sPhi);
}

// MINB > 0: register-capped variant (at most 128 threads per block, MINB blocks per SM), which the
// autotuner weighs against the uncapped one (occupancy and wave count against spills).
template <int D, int R, typename T, int SCHEME, int MINB>
__global__ void __launch_bounds__(MINB ? 128 : 256, MINB ? MINB : 1) recon_kernel(const KArgs a) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NF = L::NF, NQ = L::NQ, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP;
  constexpr int NPHI = (D == 3) ? NF * NP * NQ * NK : 1;
  // 3D: face-point basis values for all six vertex orders of a face, staged in shared memory
  __shared__ T sPhi[NPHI];
  if constexpr (D == 3) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
    __syncthreads();
  }
  pdl_wait(a);  // the state written by the previous stage's update

  const int64_t N = a.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;

  recon_cell<D, R, T, SCHEME, false>(a, i, (const T *)a.Pc + i * (int64_t)(M * NK),
                                     (const T *)a.Pd + i * (int64_t)(NF * PDS), a.st + i * M, sPhi);

  // CFL time step bookkeeping at the first stage of a step: dt[next] -> dt[cur]
  if (a.dt_swap && i < a.nmesh) {
    a.dt[i] = a.dt[a.nmesh + i];
    a.dt[a.nmesh + i] = 1e300;
  }
}

// ---------------------------------------------------------------------------------------------
// Variable-per-lane schedule: a group of NV consecutive lanes reconstructs one cell, lane v the
// conserved variable v. The steps above are independent across variables up to the positivity
// guard, so each lane keeps only its own coefficients (K-1 central + d(d+1) directional), all
// lanes of a group read the same pseudo-inverse chunk (one broadcast request) and the gathers of a
// neighbour's record are split over the group. A warp holds floor(32 / NV) cells; spare lanes
// and lanes past the last cell work on a clamped cell and store nothing.
// ---------------------------------------------------------------------------------------------
// The selection step of the variable-per-lane schedules for one variable (or characteristic
// field) of one cell, from its central coefficients ao (K-1) and directional coefficients ad
// (KD per face; inadmissible stencils hold zeros): p_1 (eq. 17, in place of a_opt), the smoothness
// indicators (eq. 15: oc(k * NK + l) the upper triangle of the central O, off-diagonal doubled;
// sid(ad_f) a directional indicator), the selection (eqs. 19-23, Alg. 1 / 2) or the CWENO weights
// (eq. 14), and the final coefficients in ao. Returns the flags byte.
template <int NF, int NK, int KD, typename T, int SCHEME, typename OC, typename SID>
__device__ __forceinline__ uint32_t lane_select(const KArgs &a, const uint32_t adm, T (&ao)[NK],
                                                const T (&ad)[NF][KD], OC oc, SID sid) {
  constexpr bool F32 = sizeof(T) == 4;
  const int stn = 1 + __popc(adm);
  T lams;
  double lamsd = 0.0;
  float log2lams = 0.0f, inv_stm1 = 0.0f;
  if constexpr (F32) {
    lams = pick<NF>(a.lams_f, stn - 1);
    log2lams = pick<NF>(a.log2_lams_f, stn - 1);
    inv_stm1 = pick<NF>(a.inv_stm1_f, stn - 1);
  } else {
    lamsd = pick<NF>(a.lams_d, stn - 1);
    lams = lamsd;
  }
  if (stn > 1 && a.central_split) {  // TENO keeps p_opt (Sec. 2.4)
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      T s = (T)0;
#pragma unroll
      for (int f = 0; f < NF; ++f) s += ad[f][k];
      ao[k] -= lams * s;
    }
    T inv_lam1;
    if constexpr (F32) inv_lam1 = a.inv_lam1_32; else inv_lam1 = a.inv_lam1;
#pragma unroll
    for (int k = 0; k < NK; ++k) ao[k] *= inv_lam1;
  }
  T SI0 = (T)0;
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    T rr = (T)0;
#pragma unroll
    for (int l = k; l < NK; ++l) rr += oc(k * NK + l) * ao[l];
    SI0 += ao[k] * rr;
  }
  T SId[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) SId[f] = sid(ad[f]);
  uint32_t bits;
  if (a.cweno) {  // CWENO (Sec. 2.3): every stencil, with the weights of eq. 14
    T w0, wd[NF];
    if constexpr (F32) cweno_weights<NF>(SI0, SId, adm, a.log2_lam1, log2lams, a.eps32, w0, wd);
    else cweno_weights<NF>(SI0, SId, adm, a.lam1, lamsd, a.eps, w0, wd);
#pragma unroll
    for (int k = 0; k < NK; ++k) ao[k] *= w0;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < KD; ++k) ao[k] += wd[f] * ad[f][k];  // zero weight where inadmissible
    bits = 1u | (adm << 1);
  } else {
    if constexpr (F32) {
      bits = select_fp32<NF>(SI0, SId, adm, stn, SCHEME, a.ctenoz_form, a.lam_gamma, a.log2_lam1, log2lams,
                             inv_stm1, a.eps32, a.C_T32);
    } else {
      bits = select_fp64<NF>(SI0, SId, adm, stn, SCHEME, a.ctenoz_form, a.lam_gamma, a.lam1, lamsd, a.eps, a.C_T);
    }
    if (!(bits & 1u)) {  // the mean of the selected directional polynomials
      const T w = (T)1 / (T)__popc(bits >> 1);
#pragma unroll
      for (int k = 0; k < NK; ++k) ao[k] = (T)0;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if ((bits >> (1 + f)) & 1u) {
#pragma unroll
          for (int k = 0; k < KD; ++k) ao[k] += w * ad[f][k];
        }
    } else {
      bits = 1u;
    }
  }
  return bits;
}

// Positivity test of a face-point state from the group's lanes (not part of the paper): rho > 0
// and p > 0, the latter as rho E - |m|^2 / 2 > 0 on the mixed path (no division).
template <int D, typename T>
__device__ __forceinline__ bool lane_point_bad(const KArgs &a, const T val, const int base) {
  constexpr int NV = D + 2;
  const T rho = __shfl_sync(0xffffffffu, val, base);
  const T E = __shfl_sync(0xffffffffu, val, base + NV - 1);
  T ke = (T)0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const T m = __shfl_sync(0xffffffffu, val, base + 1 + j);
    ke += m * m;
  }
  if constexpr (sizeof(T) == 4) {
    return !(rho > 0.0f) || !(rho * E - 0.5f * ke > 0.0f);
  } else {
    const T pr = (T)(a.gamma - 1.0) * (E - (T)0.5 * ke / rho);
    return !(rho > (T)0) || !(pr > (T)0);
  }
}

// Eigenvectors of the Euler flux Jacobian in the unit direction n at the mean state ub (the
// characteristic decomposition of Sec. 2.2 / 3.2): row w of L and row v of R, for the fields in the
// order u_n - c, u_n (entropy), u_n (shear, one per tangent), u_n + c. With H = (E + p)/rho,
// q^2 = |u|^2, b1 = (gamma - 1)/c^2, b2 = b1 q^2/2 the columns of R are (1, u - c n, H - c u_n),
// (1, u, q^2/2), (0, t_j, u.t_j), (1, u + c n, H + c u_n), and the rows of L = R^-1 are
// (b2 + u_n/c, -b1 u - n/c, b1)/2, (1 - b2, b1 u, -b1), (-u.t_j, t_j, 0),
// (b2 - u_n/c, -b1 u + n/c, b1)/2. Tangents: (-n_y, n_x) in 2D; in 3D t_1 is the axis along which
// |n| is smallest made orthogonal to n and normalised, t_2 = n x t_1.
template <int D, typename T>
__device__ __forceinline__ void euler_eigen_rows(const T (&ub)[D + 2], const T (&n)[D], const T gm1, const int w,
                                                 T (&Lw)[D + 2], T (&Rw)[D + 2]) {
  constexpr int NV = D + 2;
  const T rho = ub[0], irho = (T)1 / rho;
  T vel[D], q2 = (T)0, un = (T)0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vel[j] = ub[1 + j] * irho;
    q2 += vel[j] * vel[j];
    un += vel[j] * n[j];
  }
  const T p = gm1 * (ub[NV - 1] - (T)0.5 * rho * q2);
  const T c2 = (gm1 + (T)1) * p * irho, c = sqrt(c2), ic = (T)1 / c;
  const T H = (ub[NV - 1] + p) * irho, b1 = gm1 / c2, b2 = (T)0.5 * b1 * q2;
  T t[D - 1][D];
  if constexpr (D == 2) {
    t[0][0] = -n[1];
    t[0][1] = n[0];
  } else {
    int ax = 0;
    if (fabs(n[1]) < fabs(n[ax])) ax = 1;
    if (fabs(n[2]) < fabs(n[ax])) ax = 2;
    const T na = (ax == 0) ? n[0] : (ax == 1) ? n[1] : n[2];
    T len = (T)0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      t[0][j] = (j == ax ? (T)1 : (T)0) - na * n[j];
      len += t[0][j] * t[0][j];
    }
    const T il = (T)1 / sqrt(len);
#pragma unroll
    for (int j = 0; j < 3; ++j) t[0][j] *= il;
    t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
    t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
    t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
  }
  T ut[D - 1];
#pragma unroll
  for (int m = 0; m < D - 1; ++m) {
    ut[m] = (T)0;
#pragma unroll
    for (int j = 0; j < D; ++j) ut[m] += vel[j] * t[m][j];
  }
  // row w of L
  if (w == 0 || w == NV - 1) {
    const T sg = (w == 0) ? (T)1 : (T)-1;
    Lw[0] = (T)0.5 * (b2 + sg * un * ic);
#pragma unroll
    for (int j = 0; j < D; ++j) Lw[1 + j] = (T)0.5 * (-b1 * vel[j] - sg * n[j] * ic);
    Lw[NV - 1] = (T)0.5 * b1;
  } else if (w == 1) {
    Lw[0] = (T)1 - b2;
#pragma unroll
    for (int j = 0; j < D; ++j) Lw[1 + j] = b1 * vel[j];
    Lw[NV - 1] = -b1;
  } else {
#pragma unroll
    for (int m = 0; m < D - 1; ++m)
      if (w == 2 + m) {
        Lw[0] = -ut[m];
#pragma unroll
        for (int j = 0; j < D; ++j) Lw[1 + j] = t[m][j];
        Lw[NV - 1] = (T)0;
      }
  }
  // row w of R (variable w, all fields)
  if (w == 0) {
    Rw[0] = (T)1;
    Rw[1] = (T)1;
#pragma unroll
    for (int m = 0; m < D - 1; ++m) Rw[2 + m] = (T)0;
    Rw[NV - 1] = (T)1;
  } else if (w == NV - 1) {
    Rw[0] = H - c * un;
    Rw[1] = (T)0.5 * q2;
#pragma unroll
    for (int m = 0; m < D - 1; ++m) Rw[2 + m] = ut[m];
    Rw[NV - 1] = H + c * un;
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (w == 1 + j) {
        Rw[0] = vel[j] - c * n[j];
        Rw[1] = vel[j];
#pragma unroll
        for (int m = 0; m < D - 1; ++m) Rw[2 + m] = t[m][j];
        Rw[NV - 1] = vel[j] + c * n[j];
      }
  }
}

// The face values of the variable-per-lane schedules after the selection, from each lane's final
// coefficients ao of variable v: U_0 + sum_k phi_k a_k at every face Gauss point (phi(f, q, k)),
// the positivity guard over the group, and the stores in the canonical point order. Conserved
// variables (the selection done by the caller) or, with a.characteristic, the characteristic
// reconstruction (CHR; a compile-time switch, so that the other schedules keep their registers):
// for each face, lane v takes field w = v of W = L U (L from the cell's mean and the face's outward
// normal), projects the conserved coefficients by shuffles (the least squares are linear in the
// data), selects, evaluates W at the face's points and transforms back, U = R W.
// Face values for lane_faces: value(f, q, a, init) = init + sum_k phi_k(x_fq) a_k at point q of
// local face f, with offset(a) subtracted from init first. PhiTab reads phi_k = psi_k - psibar_k
// from a table (offset 0; the sum in k order, from init).
template <typename F>
struct PhiTab {
  F tab;
  template <int NK, typename T>
  __device__ __forceinline__ T value(int f, int q, const T (&a)[NK], T init) const {
#pragma unroll
    for (int k = 0; k < NK; ++k) init += tab(f, q, k) * a[k];
    return init;
  }
  template <int NK, typename T>
  __device__ __forceinline__ T offset(const T (&)[NK]) const { return (T)0; }
};
template <typename F>
__device__ __forceinline__ PhiTab<F> phi_tab(F f) { return PhiTab<F>{f}; }

// Sorted position (0..2) of local vertex c + 1 (c = 0..2) on local face f of a tetrahedron, or 3
// when the face does not hold it, for each of the six orders p of the face's vertex slots (the
// lexicographic permutations, as the host tables number them): 2 bits per c, 6 bits per p.
__host__ __device__ constexpr uint64_t tet_face_positions(int f) {
  int slots[3] = {0, 0, 0}, ns = 0;
  for (int a = 0; a < 4; ++a)
    if (a != f) slots[ns++] = a;
  const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  uint64_t bits = 0;
  for (int p = 0; p < 6; ++p)
    for (int c = 0; c < 3; ++c) {
      uint64_t pos = 3;
      for (int j = 0; j < 3; ++j)
        if (slots[P[p][j]] == c + 1) pos = (uint64_t)j;
      bits |= pos << (6 * p + 2 * c);
    }
  return bits;
}
template <int F>
struct TetFacePos {
  static constexpr uint64_t bits = tet_face_positions(F);
};
// Index of the monomial x^i y^j z^l (1 <= i + j + l) in the basis order: graded, within a degree
// by the z then the y power.
__host__ __device__ constexpr int mono_index3(int i, int j, int l) {
  const int t = i + j + l;
  int k = (t + 2) * (t + 1) * t / 6 - 1;  // the monomials of degrees 1 .. t - 1
  for (int c = 0; c < l; ++c) k += t - c + 1;
  return k + j;
}

// 3D, FP32: the polynomial at the face point from the point's reference coordinates (xi_c = the
// barycentric weight of the sorted face vertex that is local vertex c + 1; local vertex 0 is the
// origin), offset sum_k psibar_k a_k. Nested Horner in x, y, z: one FMA per monomial. On face
// f >= 1 the coordinate f - 1 is zero and its monomials are skipped (exactly the value at zero).
// The same polynomial as the table, without its per-cell permutation index: no shared memory.
template <int R>
struct PhiMono3 {
  uint32_t perm;  // the cell's face orders, 3 bits per face
  template <int NK>
  __device__ __forceinline__ float value(int f, int q, const float (&a)[NK], float init) const {
    const uint64_t fb = f == 0 ? TetFacePos<0>::bits
                      : f == 1 ? TetFacePos<1>::bits
                      : f == 2 ? TetFacePos<2>::bits : TetFacePos<3>::bits;
    const int p = (int)((perm >> (3 * f)) & 7u);
    const uint32_t jp = (uint32_t)(fb >> (6 * p)) & 63u;
    const float b0 = c_fbary3f[q * 3], b1 = c_fbary3f[q * 3 + 1], b2 = c_fbary3f[q * 3 + 2];
    // a coordinate whose vertex is on the face takes one of the three weights
    auto coord = [&](uint32_t j) { return j == 0u ? b0 : j == 1u ? b1 : b2; };
    const int zc = f - 1;  // the coordinate that vanishes on this face (none for f = 0)
    const float x = zc == 0 ? 0.0f : coord(jp & 3u);
    const float y = zc == 1 ? 0.0f : coord((jp >> 2) & 3u);
    const float z = zc == 2 ? 0.0f : coord((jp >> 4) & 3u);
    const int imax = zc == 0 ? 0 : R;
    float px = 0.0f;
#pragma unroll
    for (int i = R; i >= 0; --i) {
      if (i > imax) continue;
      const int jmax = zc == 1 ? 0 : R - i;
      float qy = 0.0f;
#pragma unroll
      for (int j = R; j >= 0; --j) {
        if (j > jmax) continue;
        const int lmax = zc == 2 ? 0 : R - i - j;
        // sum_l a_ijl z^l, the constant term (i = j = l = 0) being init
        float sz = (i + j + lmax == 0) ? init : a[mono_index3(i, j, lmax)];
#pragma unroll
        for (int l = R - 1; l >= 0; --l)
          if (l < lmax) sz = fmaf(sz, z, (i + j + l == 0) ? init : a[mono_index3(i, j, l)]);
        qy = (j == jmax) ? sz : fmaf(qy, y, sz);
      }
      px = (i == imax) ? qy : fmaf(px, x, qy);
    }
    return px;
  }
  template <int NK>
  __device__ __forceinline__ float offset(const float (&a)[NK]) const {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < NK; ++k) s += (R == 2 ? c_psibar3_r2f[k] : c_psibar3_r3f[k]) * a[k];
    return s;
  }
};

template <int D, int NK, int KD, int NQ, typename T, int SCHEME, bool CHR, typename OC, typename SID,
          typename PHI>
__device__ __forceinline__ void lane_faces(const KArgs &a, const int64_t i, const bool active, const int v,
                                           const int base, T (&ao)[NK], const T (&ad)[D + 1][KD],
                                           const uint32_t info, const T U0, const float L0, OC oc, SID sid,
                                           PHI phi) {
  constexpr int NV = D + 2, NF = D + 1;
  constexpr bool F32 = sizeof(T) == 4;
  const int64_t N = a.N;
  const uint32_t adm = (info >> kInfoAdmShift) & 0xFu;
  T *__restrict__ Ufi = (T *)a.Uf + i * (int64_t)(NF * NQ * NV);
  const uint32_t perm = info >> kInfoPermShift;
  bool bad = false;
  T fv[NF][NQ];
  if constexpr (!CHR) {
    const uint32_t bits = lane_select<NF, NK, KD, T, SCHEME>(a, adm, ao, ad, oc, sid);
    if (a.flags && active) a.flags[v * N + i] = (uint8_t)bits;
    const T off = phi.offset(ao);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T val = phi.value(f, q, ao, (T)L0 - off);
        val += U0;
        fv[f][q] = val;
        // every lane takes part in the test's shuffles (no short-circuit before it)
        const bool pb = lane_point_bad<D, T>(a, val, base);
        bad = bad || pb;
      }
  } else {
    T gm1;
    if constexpr (F32) gm1 = a.gm1_32; else gm1 = (T)(a.gamma - 1.0);
    T ub[NV];
    const T mean = U0 + (T)L0;
#pragma unroll
    for (int j = 0; j < NV; ++j) ub[j] = __shfl_sync(0xffffffffu, mean, base + j);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T n[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if constexpr (F32) n[j] = __ldg(a.geo32 + (i * NF + f) * 4 + j);
        else n[j] = __ldg(a.geo + (i * NF + f) * 4 + j);
      }
      T Lw[NV], Rv[NV];
      euler_eigen_rows<D, T>(ub, n, gm1, v, Lw, Rv);
      T aw[NK], adw[NF][KD];
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        T s = (T)0;
#pragma unroll
        for (int j = 0; j < NV; ++j) s += Lw[j] * __shfl_sync(0xffffffffu, ao[k], base + j);
        aw[k] = s;
      }
#pragma unroll
      for (int g = 0; g < NF; ++g)
#pragma unroll
        for (int k = 0; k < KD; ++k) {
          T s = (T)0;
#pragma unroll
          for (int j = 0; j < NV; ++j) s += Lw[j] * __shfl_sync(0xffffffffu, ad[g][k], base + j);
          adw[g][k] = s;
        }
      T wbar = (T)0;
#pragma unroll
      for (int j = 0; j < NV; ++j) wbar += Lw[j] * ub[j];
      const uint32_t bits = lane_select<NF, NK, KD, T, SCHEME>(a, adm, aw, adw, oc, sid);
      if (a.flags && active) a.flags[(f * NV + v) * N + i] = (uint8_t)bits;
#pragma unroll
      const T off = phi.offset(aw);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const T W = phi.value(f, q, aw, wbar - off);
        T val = (T)0;
#pragma unroll
        for (int j = 0; j < NV; ++j) val += Rv[j] * __shfl_sync(0xffffffffu, W, base + j);
        fv[f][q] = val;
        const bool pb = lane_point_bad<D, T>(a, val, base);  // every lane shuffles
        bad = bad || pb;
      }
    }
  }
  if (a.guard_on && bad) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int q = 0; q < NQ; ++q) fv[f][q] = U0 + (T)L0;
    if (active && v == 0) atomicAdd(a.guard, 1ull);
  }
  if (active) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int p = (perm >> (3 * f)) & 7u;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        // 2D: an edge is stored in sorted-vertex order, the swapped orientation reverses its points
        const int qq = (D == 2 && p) ? (NQ - 1 - q) : q;
        Ufi[(f * NQ + qq) * NV + v] = fv[f][q];
      }
    }
  }
}

// The second half of the variable-per-lane schedule (degrees 2 and 3), from the central
// coefficients ao and the directional coefficients ad of variable v: selection and face values
// (lane_select, lane_faces). Every lane of the warp calls it (the guard and the characteristic
// projection exchange values by shuffles).
template <int D, int R, typename T, int SCHEME, bool CHR = false>
__device__ __forceinline__ void lane_finish(const KArgs &a, const int64_t i, const bool active, const int v,
                                            const int base, T (&ao)[Shape<D, R>::NK],
                                            const T (&ad)[Lay<D>::NF][D], const uint32_t info, const T U0,
                                            const float L0, const T *__restrict__ sPhi) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NK = S::NK, NP = S::NP, NQ = L::NQ;
  constexpr T INV_FACT = (D == 2) ? (T)0.5 : (T)(1.0 / 6.0);
  const uint32_t perm = info >> kInfoPermShift;
  auto oc = [](int idx) { return cO<T, R>(idx); };
  auto sid = [&](const T (&adf)[D]) {  // the linear block of O is |V0'| I
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < D; ++k) s += adf[k] * adf[k];
    return s * INV_FACT;
  };
  if constexpr (D == 3 && sizeof(T) == 4) {
    lane_faces<D, NK, D, NQ, T, SCHEME, CHR>(a, i, active, v, base, ao, ad, info, U0, L0, oc, sid,
                                             PhiMono3<R>{perm});
  } else {
    auto phi = [&](int f, int q, int k) -> T {
      if constexpr (D == 2) {
        return cPhi2<T, R>((f * 2 + q) * NK + k);
      } else {
        const int p = (perm >> (3 * f)) & 7u;
        return sPhi[((f * NP + p) * NQ + q) * NK + k];
      }
    };
    lane_faces<D, NK, D, NQ, T, SCHEME, CHR>(a, i, active, v, base, ao, ad, info, U0, L0, oc, sid,
                                             phi_tab(phi));
  }
}

// One cell of the variable-per-lane schedule, seen from lane v of its group (first lane base);
// every lane of the warp calls it (inactive lanes with a clamped valid cell i) because the
// positivity guard exchanges values with shuffles. Operator pointers as for recon_cell. HALO:
// sti holds the cell's uint16 local indices (members, then the cell itself) into `halo`, the
// shared-memory FP32 (hi, lo) records of its tile's distinct stencil members.
template <int D, int R, typename T, int SCHEME, bool SH, bool HALO = false, bool CHR = false>
__device__ __forceinline__ void recon_lane(const KArgs &a, const int64_t i, const bool active, const int v,
                                           const int base, const T *__restrict__ Pci,
                                           const T *__restrict__ Pdi, const void *__restrict__ sti_,
                                           const T *__restrict__ sPhi, const float *__restrict__ halo = nullptr) {
  static_assert(!HALO || (SH && sizeof(T) == 4), "gather staging: shared-memory records, mixed path");
  const int32_t *__restrict__ sti = reinterpret_cast<const int32_t *>(sti_);
  const uint16_t *__restrict__ lid = reinterpret_cast<const uint16_t *>(sti_);
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NVP = L::NVP, NF = L::NF, ND = L::ND, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M;
  constexpr int CH = Vec16<T>::n;
  constexpr bool F32 = sizeof(T) == 4;
  // own mean of variable v: FP64, or the FP32 pair (hi, lo)
  T U0;
  float L0;
  if constexpr (HALO) {
    const float2 h = reinterpret_cast<const float2 *>(halo)[(int)lid[M] * NVP + v];
    U0 = h.x;
    L0 = h.y;
  } else if constexpr (F32) {
    const float2 h = __ldg(reinterpret_cast<const float2 *>(a.U32) + i * NVP + v);
    U0 = h.x;
    L0 = h.y;
  } else {
    U0 = (T)__ldg(a.U + i * NVP + v);
    L0 = 0.0f;
  }
  auto delta = [&](int64_t j) -> T {
    if constexpr (HALO) {
      const float2 h = reinterpret_cast<const float2 *>(halo)[(int)j * NVP + v];
      return (h.x - (float)U0) + (h.y - L0);
    } else if constexpr (F32) {
      const float2 h = __ldg(reinterpret_cast<const float2 *>(a.U32) + j * NVP + v);
      return (h.x - (float)U0) + (h.y - L0);
    } else {
      return (T)(__ldg(a.U + j * NVP + v) - (double)U0);
    }
  };
  constexpr int IDV = HALO ? 8 : 4;  // ids per 16-byte load

  // central coefficients of variable v
  T ao[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) ao[k] = (T)0;
  {
    T pb[CH], du = (T)0;
    int ids[IDV];
#pragma unroll
    for (int e = 0; e < M * NK; ++e) {
      const int m = e / NK, k = e % NK;
      if (e % CH == 0) {
        if constexpr (SH) load16<T, CH, true>(Pci + e, pb);
        else load16_stream<T, CH>(Pci + e, pb);
      }
      if (k == 0) {
        if (m % IDV == 0) {
          if constexpr (HALO) {
            const uint4 w = *reinterpret_cast<const uint4 *>(lid + m);
            const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              ids[2 * t] = (int)(ww[t] & 0xFFFFu);
              ids[2 * t + 1] = (int)(ww[t] >> 16);
            }
          } else {
            const int4 t4 = load_i4<SH>(sti + m);
            ids[0] = t4.x; ids[1] = t4.y; ids[2] = t4.z; ids[3] = t4.w;
          }
        }
        du = delta(ids[m % IDV]);
      }
      ao[k] += pb[e % CH] * du;
    }
  }
  // directional coefficients of variable v
  const uint32_t info = __ldg(a.cinfo + i);
  const uint32_t adm = (info >> kInfoAdmShift) & 0xFu;
  T ad[NF][D];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < D; ++k) ad[f][k] = (T)0;
  {
    int off = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int nm = (info >> (4 * f)) & 15u;
      if ((adm >> f) & 1u) {
        T pf[PDS];
        if constexpr (SH) load16<T, PDS, true>(Pdi + f * PDS, pf);
        else load16_stream<T, PDS>(Pdi + f * PDS, pf);
#pragma unroll
        for (int jj = 0; jj < ND; ++jj) {
          if (jj < nm) {
            const T du = delta(HALO ? (int)lid[off + jj] : load_i1<SH>(sti + off + jj));
#pragma unroll
            for (int k = 0; k < D; ++k) ad[f][k] += pf[jj * D + k] * du;
          }
        }
      }
      off += nm;
    }
  }
  lane_finish<D, R, T, SCHEME, CHR>(a, i, active, v, base, ao, ad, info, U0, L0, sPhi);
}

template <int D, int R, typename T, int SCHEME, bool CHR = false>
__global__ void __launch_bounds__(256) recon_lanes_kernel(const KArgs a) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  constexpr int NV = L::NV, NF = L::NF, NQ = L::NQ, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP;
  constexpr bool TAB = D == 3 && sizeof(T) == 8;  // FP32 lanes: no face-value table
  constexpr int NPHI = TAB ? NF * NP * NQ * NK : 1;
  constexpr int CPW = 32 / NV;  // cells per warp
  __shared__ T sPhi[NPHI];
  if constexpr (TAB) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
    __syncthreads();
  }
  pdl_wait(a);
  const int lane = threadIdx.x & 31;
  const int grp = lane / NV;                // cell slot in the warp (CPW = spare lanes)
  const int v = lane - grp * NV;            // this lane's variable
  const int base = grp * NV;                // first lane of the group
  const int64_t N = a.N;
  const int64_t cell = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW + grp;
  const bool active = grp < CPW && cell < N;
  const int64_t i = active ? cell : N - 1;  // spare lanes shadow a valid cell

  recon_lane<D, R, T, SCHEME, false, false, CHR>(a, i, active, v, base, (const T *)a.Pc + i * (int64_t)(M * NK),
                                     (const T *)a.Pd + i * (int64_t)(NF * PDS), a.st + i * M, sPhi);
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }
}


// ---------------------------------------------------------------------------------------------
// Staged schedules: a persistent grid walks tiles of C consecutive cells, C the cells of one block
// of the thread-per-cell or variable-per-lane schedule. The operator records of a tile (central
// pseudo-inverses, directional operators, stencil ids) are three contiguous spans of the
// cell-major layout; one thread fetches them with three bulk copies into one of two shared-memory
// stages while the block computes on the other, so each SM keeps a whole tile of the dominant
// stream in flight instead of what its warps' outstanding loads cover.
// ---------------------------------------------------------------------------------------------
template <int D, int R, typename T>
struct StagedRecord {  // bytes per cell of each stream
  static constexpr int PC = Shape<D, R>::M * Shape<D, R>::NK * (int)sizeof(T);
  static constexpr int PD = Lay<D>::NF * Lay<D>::PDS * (int)sizeof(T);
  static constexpr int ST = Shape<D, R>::M * 4;
  static constexpr int CELL = PC + PD + ST;
  static_assert(PC % 16 == 0 && PD % 16 == 0 && ST % 16 == 0, "bulk copies need 16-byte spans");
};
constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s: far above any tile's copy time

template <int D, int R, typename T, int SCHEME, bool LANES>
__global__ void __launch_bounds__(256) recon_staged_kernel(const KArgs a) {
  using S = Shape<D, R>;
  using L = Lay<D>;
  using B = StagedRecord<D, R, T>;
  constexpr int NV = L::NV, NF = L::NF, NQ = L::NQ, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP;
  constexpr bool TAB = D == 3 && !LANES;  // FP32 lanes: no face-value table
  constexpr int NPHI = TAB ? NF * NP * NQ * NK : 1;
  constexpr int CPW = 32 / NV;
  __shared__ T sPhi[NPHI];
  __shared__ __align__(8) uint64_t bar[3];  // two stages; bar[2] only for the test hook
  extern __shared__ __align__(128) unsigned char stage_mem[];

  const int C = LANES ? (int)(blockDim.x >> 5) * CPW : (int)blockDim.x;
  const int64_t N = a.N;
  const int64_t tiles = (N + C - 1) / C;
  unsigned char *const stage0 = stage_mem, *const stage1 = stage_mem + (size_t)C * B::CELL;
  auto sPc = [&](int s) { return reinterpret_cast<T *>(s ? stage1 : stage0); };
  auto sPd = [&](int s) { return reinterpret_cast<T *>((s ? stage1 : stage0) + (size_t)C * B::PC); };
  auto sSt = [&](int s) {
    return reinterpret_cast<int32_t *>((s ? stage1 : stage0) + (size_t)C * (B::PC + B::PD));
  };
  // thread 0 only: fetch the records of `tile` into stage s
  auto issue = [&](int64_t tile, int s) {
    const int64_t c0 = tile * C;
    const uint32_t n = (uint32_t)min((int64_t)C, N - c0);
    mbar_arrive_expect_tx(&bar[s], n * (uint32_t)B::CELL);
    bulk_copy_g2s(sPc(s), (const unsigned char *)a.Pc + c0 * B::PC, n * B::PC, &bar[s]);
    bulk_copy_g2s(sPd(s), (const unsigned char *)a.Pd + c0 * B::PD, n * B::PD, &bar[s]);
    bulk_copy_g2s(sSt(s), (const unsigned char *)a.st + c0 * B::ST, n * B::ST, &bar[s]);
  };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    fence_barrier_init();
  }
  if constexpr (TAB) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if ((int64_t)blockIdx.x < tiles) issue(blockIdx.x, 0);
    if ((int64_t)blockIdx.x + gridDim.x < tiles) issue((int64_t)blockIdx.x + gridDim.x, 1);
  }
  if (a.test_wait_ns) {  // test hook: a bounded wait on a barrier that nothing completes runs out
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait(&bar[2], 0, a.test_wait_ns);
    if (__syncthreads_or(!ok)) {  // the timeout path: report, let this block's copies land, stop
      if (threadIdx.x == 0) {
        atomicOr(a.err, kErrTimeout);
        if ((int64_t)blockIdx.x < tiles) mbar_wait(&bar[0], 0, kStageWaitNs);
        if ((int64_t)blockIdx.x + gridDim.x < tiles) mbar_wait(&bar[1], 0, kStageWaitNs);
      }
      return;
    }
  }
  // the operator records do not depend on the previous kernel: their copies were issued above;
  // the states it writes (and the face states it may still read) are touched only after this
  pdl_wait(a);
  // CFL time step bookkeeping at the first stage of a step: dt[next] -> dt[cur]
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }

  int it = 0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const uint32_t parity = (it >> 1) & 1;
    const bool ok = mbar_wait(&bar[s], parity, kStageWaitNs);
    if (__syncthreads_or(!ok)) {  // the whole block stops; its copies in flight are awaited
      if (threadIdx.x == 0) {
        atomicOr(a.err, kErrTimeout);
        mbar_wait(&bar[s], parity, kStageWaitNs);
        if (tile + gridDim.x < tiles) mbar_wait(&bar[s ^ 1], ((it + 1) >> 1) & 1, kStageWaitNs);
      }
      return;
    }
    const int64_t c0 = tile * C;
    const int nvalid = (int)min((int64_t)C, N - c0);
    if constexpr (LANES) {
      const int lane = threadIdx.x & 31, grp = lane / NV;
      const int slot = (int)(threadIdx.x >> 5) * CPW + grp;
      const bool active = grp < CPW && slot < nvalid;
      const int ls = active ? slot : nvalid - 1;  // spare lanes shadow a valid cell of the tile
      recon_lane<D, R, T, SCHEME, true>(a, c0 + ls, active, lane - grp * NV, grp * NV,
                                        sPc(s) + ls * (M * NK), sPd(s) + ls * (NF * PDS),
                                        sSt(s) + ls * M, sPhi);
    } else {
      const int slot = threadIdx.x;
      if (slot < nvalid)
        recon_cell<D, R, T, SCHEME, true>(a, c0 + slot, sPc(s) + slot * (M * NK),
                                          sPd(s) + slot * (NF * PDS), sSt(s) + slot * M, sPhi);
    }
    __syncthreads();  // every thread is done with stage s
    if (threadIdx.x == 0 && tile + 2 * (int64_t)gridDim.x < tiles) {
      fence_proxy_async_shared();
      issue(tile + 2 * (int64_t)gridDim.x, s);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Gather-staged lane schedule (mixed path): as the staged lane schedule with four warps, and in
// addition the states of each tile's distinct stencil members (listed per tile on the host) are
// copied into shared memory by all threads with 16-byte asynchronous copies, one tile ahead of
// the computation; the cells' stencil ids are then 16-bit indices into that list, so every gather
// of the reconstruction is a shared-memory read and each member state crosses L2 once per tile.
// ---------------------------------------------------------------------------------------------
// ONE: one tile per block and a single stage (grid = tiles): half the shared memory, so twice the
// resident blocks hide each other's copy latency (small meshes, where a persistent block would
// see only a few tiles, and 3D degree 3, whose two stages do not fit).
template <int D, int R, int SCHEME, bool ONE>
__global__ void __launch_bounds__(kHaloWarps * 32) recon_halo_kernel(const KArgs a) {
  using T = float;
  using S = Shape<D, R>;
  using L = Lay<D>;
  using B = StagedRecord<D, R, T>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, NQ = L::NQ, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP;
  constexpr bool TAB = false;  // FP32 lanes: no face-value table
  constexpr int NPHI = TAB ? NF * NP * NQ * NK : 1;
  constexpr int CPW = 32 / NV, C = kHaloWarps * CPW;
  constexpr int MS = (M + 1 + 7) / 8 * 8;   // local ids per cell
  constexpr int HS = NVP * 2 * 4;           // bytes of one member state (FP32 pairs)
  constexpr int LI = MS * 2;                // bytes of one cell's local ids
  __shared__ T sPhi[NPHI];
  __shared__ __align__(8) uint64_t bar[3];  // two stages; bar[2] only for the test hook
  extern __shared__ __align__(128) unsigned char stage_mem[];

  const int64_t N = a.N;
  const int64_t tiles = (N + C - 1) / C;
  const int HR = a.hrec;  // words of a tile's member record
  const size_t o_pd = (size_t)C * B::PC, o_li = o_pd + (size_t)C * B::PD, o_hl = o_li + (size_t)C * LI,
               o_hs = o_hl + (size_t)HR * 4, stage_bytes = o_hs + (size_t)(HR - 4) * HS;
  auto base = [&](int s) { return stage_mem + (size_t)s * stage_bytes; };
  auto issue = [&](int64_t tile, int s) {  // thread 0: the tile's records
    const int64_t c0 = tile * C;
    const uint32_t n = (uint32_t)min((int64_t)C, N - c0);
    mbar_arrive_expect_tx(&bar[s], n * (uint32_t)(B::PC + B::PD + LI) + (uint32_t)HR * 4u);
    bulk_copy_g2s(base(s), (const unsigned char *)a.Pc + c0 * B::PC, n * B::PC, &bar[s]);
    bulk_copy_g2s(base(s) + o_pd, (const unsigned char *)a.Pd + c0 * B::PD, n * B::PD, &bar[s]);
    bulk_copy_g2s(base(s) + o_li, (const unsigned char *)a.lidx + c0 * LI, n * LI, &bar[s]);
    bulk_copy_g2s(base(s) + o_hl, a.hl + tile * HR, (uint32_t)HR * 4u, &bar[s]);
  };
  auto gather = [&](int s) {  // all threads: the tile's member states (its records have landed)
    const int32_t *hl = reinterpret_cast<const int32_t *>(base(s) + o_hl);
    const int cnt = hl[0];
    unsigned char *hs = base(s) + o_hs;
    for (int t = threadIdx.x; t < cnt * (HS / 16); t += blockDim.x) {
      const int h = t / (HS / 16), c = t - h * (HS / 16);
      cp_async16(hs + h * HS + c * 16, a.U32 + (int64_t)hl[4 + h] * (2 * NVP) + c * 4);
    }
  };
  // a timed-out wait on phase `parity` of stage s: report it, give that copy (and, with `also`,
  // the first copy into stage 1) a second bounded wait, let this thread's small copies land
  auto give_up = [&](int s, uint32_t parity, bool also) {
    if (threadIdx.x == 0) {
      atomicOr(a.err, kErrTimeout);
      mbar_wait(&bar[s], parity, kStageWaitNs);
      if (also) mbar_wait(&bar[1], 0, kStageWaitNs);
    }
    cp_async_wait<0>();
  };

  // the reconstruction of the cells of `tile` from stage s (records and member states landed)
  auto work = [&](int64_t tile, int s) {
    const int64_t c0 = tile * C;
    const int nvalid = (int)min((int64_t)C, N - c0);
    const int lane = threadIdx.x & 31, grp = lane / NV;
    const int slot = (int)(threadIdx.x >> 5) * CPW + grp;
    const bool active = grp < CPW && slot < nvalid;
    const int ls = active ? slot : nvalid - 1;  // spare lanes shadow a valid cell of the tile
    unsigned char *b = base(s);
    recon_lane<D, R, T, SCHEME, true, true>(a, c0 + ls, active, lane - grp * NV, grp * NV,
                                            reinterpret_cast<const T *>(b) + ls * (M * NK),
                                            reinterpret_cast<const T *>(b + o_pd) + ls * (NF * PDS),
                                            b + o_li + (size_t)ls * LI, sPhi,
                                            reinterpret_cast<const float *>(b + o_hs));
  };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    if (!ONE) mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    fence_barrier_init();
  }
  if constexpr (TAB) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if ((int64_t)blockIdx.x < tiles) issue(blockIdx.x, 0);
    if (!ONE && (int64_t)blockIdx.x + gridDim.x < tiles) issue((int64_t)blockIdx.x + gridDim.x, 1);
  }
  if (a.test_wait_ns) {  // test hook: a bounded wait on a barrier that nothing completes runs out
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait(&bar[2], 0, a.test_wait_ns);
    if (__syncthreads_or(!ok)) {  // the timeout path: report, let this block's copies land, stop
      if ((int64_t)blockIdx.x < tiles)
        give_up(0, 0, !ONE && (int64_t)blockIdx.x + gridDim.x < tiles);
      else if (threadIdx.x == 0)
        atomicOr(a.err, kErrTimeout);
      return;
    }
  }
  // the operator records and member lists do not depend on the previous kernel: their copies
  // were issued above; member states, face states and dt are touched only after this
  pdl_wait(a);
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }
  if constexpr (ONE) {  // grid = tiles: this block's tile only
    const bool ok = mbar_wait(&bar[0], 0, kStageWaitNs);
    if (__syncthreads_or(!ok)) {
      give_up(0, 0, false);
      return;
    }
    gather(0);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    work(blockIdx.x, 0);
    return;
  }
  // member states of the first tile
  if ((int64_t)blockIdx.x < tiles) {
    const bool ok = mbar_wait(&bar[0], 0, kStageWaitNs);
    if (__syncthreads_or(!ok)) {
      give_up(0, 0, (int64_t)blockIdx.x + gridDim.x < tiles);
      return;
    }
    gather(0);
  }
  cp_async_commit();

  int it = 0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const int64_t next = tile + gridDim.x;
    // records of the next tile, then its member states (in flight during this tile's work)
    bool ok = true;
    if (next < tiles) ok = mbar_wait(&bar[s ^ 1], ((it + 1) >> 1) & 1, kStageWaitNs);
    if (__syncthreads_or(!ok)) {
      give_up(s ^ 1, ((it + 1) >> 1) & 1, false);
      return;
    }
    if (next < tiles) gather(s ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of the current tile's states
    __syncthreads();     // everyone's
    work(tile, s);
    __syncthreads();  // stage s is free again
    if (threadIdx.x == 0 && tile + 2 * (int64_t)gridDim.x < tiles) {
      fence_proxy_async_shared();
      issue(tile + 2 * (int64_t)gridDim.x, s);
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------------
// Streamed lane schedule (mixed path): every warp is an independent pipeline over tiles of CPW
// consecutive cells (lane v of group g: variable v of cell g). The central pseudo-inverse records
// of a tile stream through a per-warp ring of NST shared-memory stages in chunks of MC members
// per cell (one bulk copy per cell and chunk, completion on the stage's mbarrier); the tile's
// directional operators and stencil ids go to one of two per-warp header buffers. Copies run NST
// chunks (and two tiles' headers) ahead of the computation, so each SM keeps tens of kilobytes of
// the dominant stream in flight while its loops stay short (few registers, little code), and no
// warp waits for another.
// ---------------------------------------------------------------------------------------------
template <int D, int R, int STAGES>
struct StreamShape {
  using S = Shape<D, R>;
  using L = Lay<D>;
  static constexpr int CPW = 32 / L::NV;                     // cells per warp
  static constexpr int MC = (S::M % 8 == 0) ? 8 : 4;          // members per chunk
  static constexpr int NCH = S::M / MC;                       // chunks per tile
  static constexpr int NST = STAGES;                          // stages of the chunk ring
  static constexpr int CHUNK_CELL = MC * S::NK * 4;           // bytes of one cell's chunk
  static constexpr int STAGE = CPW * CHUNK_CELL;
  static constexpr int HPD = CPW * L::NF * L::PDS * 4;        // header: directional operators,
  static constexpr int HST = CPW * S::M * 4;                  //   stencil ids
  static constexpr int HDR = HPD + HST;
  static constexpr int WARP_BYTES = 2 * HDR + NST * STAGE;
  static constexpr int PHI_BYTES = 16;  // FP32 face values: the polynomial at the point, no table
  static_assert(S::M % MC == 0 && CHUNK_CELL % 16 == 0 && HPD % 16 == 0 && HST % 16 == 0,
                "bulk copies need 16-byte spans");
};

template <int D, int R, int SCHEME, int STAGES>
__global__ void __launch_bounds__(512, 1) recon_stream_kernel(const KArgs a) {
  using T = float;
  using S = Shape<D, R>;
  using L = Lay<D>;
  using Q = StreamShape<D, R, STAGES>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, ND = L::ND, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP, NQ = L::NQ;
  constexpr int CPW = Q::CPW, MC = Q::MC, NCH = Q::NCH, NST = Q::NST;
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  T *const sPhi = reinterpret_cast<T *>(smem);
  unsigned char *const wbase = smem + Q::PHI_BYTES + (size_t)warp * Q::WARP_BYTES;
  uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + Q::PHI_BYTES + (size_t)W * Q::WARP_BYTES);
  uint64_t *const hbar = bars + warp * (2 + NST);  // the two header buffers
  uint64_t *const pbar = hbar + 2;                 // the NST chunk stages
  uint64_t *const tbar = bars + W * (2 + NST);     // the test hook (block)
  auto hdr = [&](int64_t it) { return wbase + (it & 1) * Q::HDR; };
  auto stage = [&](int64_t q) { return wbase + 2 * Q::HDR + (q % NST) * Q::STAGE; };

  const int64_t N = a.N;
  const int64_t tiles = (N + CPW - 1) / CPW;
  const int64_t gw = (int64_t)blockIdx.x * W + warp, TW = (int64_t)gridDim.x * W;
  auto tile_of = [&](int64_t it) { return gw + it * TW; };
  // lane 0 only: the header of tile iteration it, chunk q (tile iteration q / NCH, chunk q % NCH)
  auto issue_hdr = [&](int64_t it) {
    const int64_t t = tile_of(it);
    if (t >= tiles) return;
    const int64_t c0 = t * CPW;
    const uint32_t n = (uint32_t)min((int64_t)CPW, N - c0);
    uint64_t *bar = &hbar[it & 1];
    mbar_arrive_expect_tx(bar, n * (uint32_t)(NF * PDS * 4 + M * 4));
    bulk_copy_g2s(hdr(it), (const float *)a.Pd + c0 * (NF * PDS), n * (uint32_t)(NF * PDS * 4), bar);
    bulk_copy_g2s(hdr(it) + Q::HPD, a.st + c0 * M, n * (uint32_t)(M * 4), bar);
  };
  auto issue_chunk = [&](int64_t q) {
    const int64_t t = tile_of(q / NCH);
    if (t >= tiles) return;
    const int c = (int)(q % NCH);
    const int64_t c0 = t * CPW;
    const int n = (int)min((int64_t)CPW, N - c0);
    uint64_t *bar = &pbar[q % NST];
    mbar_arrive_expect_tx(bar, (uint32_t)(n * Q::CHUNK_CELL));
    for (int g = 0; g < n; ++g)
      bulk_copy_g2s(stage(q) + g * Q::CHUNK_CELL,
                    (const float *)a.Pc + (c0 + g) * (int64_t)(M * NK) + c * (MC * NK), Q::CHUNK_CELL, bar);
  };
  // a bounded wait of the whole warp; false (in every lane) when any lane's wait ran out
  auto wait_all = [&](uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, kStageWaitNs);
    return !__any_sync(0xffffffffu, !ok);
  };
  // timeout path: report it, let this warp's copies in flight land (bounded), then stop
  auto give_up = [&](int64_t it, int64_t q, int64_t qi) {
    if (lane == 0) {
      atomicOr(a.err, kErrTimeout);
      for (int64_t h = it; h < it + 2; ++h)
        if (tile_of(h) < tiles) mbar_wait(&hbar[h & 1], (uint32_t)((h >> 1) & 1), kStageWaitNs);
      for (int64_t c = q; c < qi; ++c)
        if (tile_of(c / NCH) < tiles) mbar_wait(&pbar[c % NST], (uint32_t)((c / NST) & 1), kStageWaitNs);
    }
    __syncwarp();
  };

  if (lane == 0) {
    for (int b = 0; b < 2 + NST; ++b) mbar_init(&hbar[b], 1);
    if (threadIdx.x == 0) mbar_init(tbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  // the operator records do not depend on the previous kernel: their copies start now
  if (lane == 0) {
    issue_hdr(0);
    issue_hdr(1);
    for (int64_t q = 0; q < NST; ++q) issue_chunk(q);
  }
  if (a.test_wait_ns) {  // test hook: a bounded wait on a barrier that nothing completes runs out
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait(tbar, 0, a.test_wait_ns);
    if (__syncthreads_or(!ok)) {
      give_up(0, 0, NST);
      return;
    }
  }
  pdl_wait(a);  // states written by the previous stage's update
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }

  const int grp = lane / NV, v = lane - grp * NV;
  int64_t q = 0, qi = NST;  // next chunk to consume / to issue
  for (int64_t it = 0; tile_of(it) < tiles; ++it) {
    const int64_t c0 = tile_of(it) * CPW;
    const int nvalid = (int)min((int64_t)CPW, N - c0);
    const bool active = grp < CPW && grp < nvalid;
    const int g = active ? grp : nvalid - 1;  // spare lanes shadow a valid cell of the tile
    const int64_t i = c0 + g;
    const float2 own = __ldg(reinterpret_cast<const float2 *>(a.U32) + i * NVP + v);
    const T U0 = own.x;
    const float L0 = own.y;
    const uint32_t info = __ldg(a.cinfo + i);
    if (!wait_all(&hbar[it & 1], (uint32_t)((it >> 1) & 1))) {
      give_up(it, q, qi);
      return;
    }
    const T *__restrict__ Pd_s = reinterpret_cast<const T *>(hdr(it)) + g * (NF * PDS);
    const int32_t *__restrict__ st_s = reinterpret_cast<const int32_t *>(hdr(it) + Q::HPD) + g * M;
    auto delta = [&](int32_t j) -> T {
      const float2 h = __ldg(reinterpret_cast<const float2 *>(a.U32) + (int64_t)j * NVP + v);
      return (h.x - U0) + (h.y - L0);
    };

    // central coefficients of variable v, chunk after chunk; the member states of chunk c + 1
    // are loaded while chunk c is multiplied
    T ao[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) ao[k] = (T)0;
    float2 nx[MC];
    auto fetch = [&](int c) {
#pragma unroll
      for (int mm = 0; mm < MC; mm += 4) {
        const int4 j4 = *reinterpret_cast<const int4 *>(st_s + c * MC + mm);
        const float2 *u = reinterpret_cast<const float2 *>(a.U32) + v;
        nx[mm] = __ldg(u + (int64_t)j4.x * NVP);
        nx[mm + 1] = __ldg(u + (int64_t)j4.y * NVP);
        nx[mm + 2] = __ldg(u + (int64_t)j4.z * NVP);
        nx[mm + 3] = __ldg(u + (int64_t)j4.w * NVP);
      }
    };
    fetch(0);
#pragma unroll 1
    for (int c = 0; c < NCH; ++c, ++q) {
      T du[MC];
#pragma unroll
      for (int mm = 0; mm < MC; ++mm) du[mm] = (nx[mm].x - U0) + (nx[mm].y - L0);
      if (c + 1 < NCH) fetch(c + 1);
      if (!wait_all(&pbar[q % NST], (uint32_t)((q / NST) & 1))) {
        give_up(it, q, qi);
        return;
      }
      const T *__restrict__ P_s = reinterpret_cast<const T *>(stage(q)) + g * (MC * NK);
      T pb[4];
#pragma unroll
      for (int e = 0; e < MC * NK; ++e) {
        if (e % 4 == 0) load16<T, 4, true>(P_s + e, pb);
        ao[e % NK] += pb[e % 4] * du[e / NK];
      }
      __syncwarp();  // every lane is done with this stage
      if (lane == 0) {
        fence_proxy_async_shared();
        issue_chunk(qi);
      }
      ++qi;
    }

    // directional coefficients (degree 1): members of face f are the next slots of the list
    const uint32_t adm = (info >> kInfoAdmShift) & 0xFu;
    T ad[NF][D];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < D; ++k) ad[f][k] = (T)0;
    {
      int off = 0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int nm = (info >> (4 * f)) & 15u;
        if ((adm >> f) & 1u) {
          T pf[PDS];
          load16<T, PDS, true>(Pd_s + f * PDS, pf);
#pragma unroll
          for (int jj = 0; jj < ND; ++jj) {
            if (jj < nm) {
              const T du = delta(st_s[off + jj]);
#pragma unroll
              for (int k = 0; k < D; ++k) ad[f][k] += pf[jj * D + k] * du;
            }
          }
        }
        off += nm;
      }
    }
    lane_finish<D, R, T, SCHEME>(a, i, active, v, grp * NV, ao, ad, info, U0, L0, sPhi);
    __syncwarp();  // every lane is done with this header
    if (lane == 0) {
      fence_proxy_async_shared();
      issue_hdr(it + 2);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Streamed thread-per-cell schedule (mixed path): every warp walks tiles of 32 consecutive cells,
// one thread per cell with all its variables, and each lane streams its own cell's central
// pseudo-inverse record through the warp's ring of NST shared-memory stages, four stencil members
// (one row of MC * NK values) at a time: each lane announces and issues the bulk copy of its row,
// lane 0 arrives on the stage's mbarrier. The arithmetic is the thread-per-cell schedule's, in the
// same order; the rows are read back with conflict-free 16-byte shared loads.
// ---------------------------------------------------------------------------------------------
template <int D, int R>
struct StreamCellShape {
  using S = Shape<D, R>;
  using L = Lay<D>;
  static constexpr int MC = 4;                                // members per chunk
  static constexpr int NCH = S::M / MC;                       // chunks per cell
  static constexpr int NST = kStreamCellStages;
  static constexpr int ROW = MC * S::NK * 4;                  // bytes of one cell's chunk
  static constexpr int STAGE = 32 * ROW;
  static constexpr int WARP_BYTES = NST * STAGE;
  static constexpr int NPHI = (D == 3) ? L::NF * S::NP * L::NQ * S::NK : 1;
  static constexpr int PHI_BYTES = (NPHI * 4 + 15) / 16 * 16;
  static_assert(S::M % MC == 0 && ROW % 16 == 0, "bulk copies need 16-byte rows");
};

template <int D, int R, int SCHEME>
__global__ void __launch_bounds__(256, 1) recon_stream_cells_kernel(const KArgs a) {
  using T = float;
  using S = Shape<D, R>;
  using L = Lay<D>;
  using Q = StreamCellShape<D, R>;
  constexpr int NV = L::NV, NF = L::NF, PDS = L::PDS, NQ = L::NQ;
  constexpr int NK = S::NK, M = S::M, NP = S::NP;
  constexpr int MC = Q::MC, NCH = Q::NCH, NST = Q::NST;
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  T *const sPhi = reinterpret_cast<T *>(smem);
  unsigned char *const wbase = smem + Q::PHI_BYTES + (size_t)warp * Q::WARP_BYTES;
  uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + Q::PHI_BYTES + (size_t)W * Q::WARP_BYTES);
  uint64_t *const pbar = bars + warp * NST;  // the NST stages of this warp
  uint64_t *const tbar = bars + W * NST;     // the test hook (block)
  auto stage = [&](int64_t q) { return wbase + (q % NST) * Q::STAGE; };

  const int64_t N = a.N;
  const int64_t tiles = (N + 31) / 32;
  const int64_t gw = (int64_t)blockIdx.x * W + warp, TW = (int64_t)gridDim.x * W;
  auto tile_of = [&](int64_t it) { return gw + it * TW; };
  // every lane: its row of chunk q (tile iteration q / NCH, members 4 (q % NCH) ..); the branch is
  // uniform across the warp
  auto issue = [&](int64_t q) {
    const int64_t t = tile_of(q / NCH);
    if (t >= tiles) return;
    const int c = (int)(q % NCH);
    const int64_t cell = t * 32 + lane;
    uint64_t *bar = &pbar[q % NST];
    if (cell < N) {
      mbar_expect_tx(bar, Q::ROW);
      bulk_copy_g2s(stage(q) + lane * Q::ROW, (const T *)a.Pc + cell * (int64_t)(M * NK) + c * (MC * NK), Q::ROW,
                    bar);
    }
    __syncwarp();  // every announcement precedes the arrival that can complete the phase
    if (lane == 0) mbar_arrive(bar);
  };
  auto wait_all = [&](uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, kStageWaitNs);
    return !__any_sync(0xffffffffu, !ok);
  };
  auto give_up = [&](int64_t q, int64_t qi) {  // report, let this warp's copies land (bounded), stop
    if (lane == 0) {
      atomicOr(a.err, kErrTimeout);
      for (int64_t c = q; c < qi; ++c)
        if (tile_of(c / NCH) < tiles) mbar_wait(&pbar[c % NST], (uint32_t)((c / NST) & 1), kStageWaitNs);
    }
    __syncwarp();
  };

  if (lane == 0) {
    for (int b = 0; b < NST; ++b) mbar_init(&pbar[b], 1);
    if (threadIdx.x == 0) mbar_init(tbar, 1);
    fence_barrier_init();
  }
  if constexpr (D == 3) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < Q::NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
  }
  __syncthreads();
  // the operator records do not depend on the previous kernel: their copies start now
  for (int64_t q = 0; q < NST; ++q) issue(q);
  if (a.test_wait_ns) {  // test hook: a bounded wait on a barrier that nothing completes runs out
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait(tbar, 0, a.test_wait_ns);
    if (__syncthreads_or(!ok)) {
      give_up(0, NST);
      return;
    }
  }
  pdl_wait(a);  // states written by the previous stage's update
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }

  int64_t q = 0, qi = NST;  // next chunk to consume / to issue
  for (int64_t it = 0; tile_of(it) < tiles; ++it) {
    const int64_t i0 = tile_of(it) * 32 + lane;
    const bool active = i0 < N;
    const int64_t i = active ? i0 : N - 1;  // lanes past the last cell shadow it and store nothing
    T U0[NV];
    float L0[NV];
    cell_own<D, T>(a, i, U0, L0);
    const int32_t *__restrict__ sti = a.st + i * M;
    T ao[NK][NV];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) ao[k][v] = (T)0;
#pragma unroll 1
    for (int c = 0; c < NCH; ++c, ++q) {
      const int4 j4 = load_i4<false>(sti + c * MC);
      T du[MC][NV];
      cell_delta<D, T>(a, j4.x, U0, L0, du[0]);
      cell_delta<D, T>(a, j4.y, U0, L0, du[1]);
      cell_delta<D, T>(a, j4.z, U0, L0, du[2]);
      cell_delta<D, T>(a, j4.w, U0, L0, du[3]);
      if (!wait_all(&pbar[q % NST], (uint32_t)((q / NST) & 1))) {
        give_up(q, qi);
        return;
      }
      const T *__restrict__ P = reinterpret_cast<const T *>(stage(q) + lane * Q::ROW);
      T pb[4];
#pragma unroll
      for (int e = 0; e < MC * NK; ++e) {
        if (e % 4 == 0) load16<T, 4, true>(P + e, pb);
#pragma unroll
        for (int v = 0; v < NV; ++v) ao[e % NK][v] += pb[e % 4] * du[e / NK][v];
      }
      fence_proxy_async_shared();  // this lane's reads of its row precede the copy that refills it
      issue(qi);
      ++qi;
    }
    if (active)
      cell_finish<D, R, T, SCHEME, false>(a, i, ao, U0, L0, (const T *)a.Pd + i * (int64_t)(NF * PDS), sti, sPhi);
  }
}

template <int D, int R, int SCHEME>
void launch_recon_stream_cells(const KArgs &a, int warps, cudaStream_t s) {
  const int threads = 32 * warps;
  const size_t smem = (size_t)recon_stream_cells_smem(D, R, warps);
  auto kern = recon_stream_cells_kernel<D, R, SCHEME>;
  static int resident[9] = {}, sms = 0;
  int &nb = resident[warps];
  if (!nb) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStreamSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    if (nb < 1) nb = 1;  // a launch that cannot fit fails loudly below
  }
  const int64_t tiles = (a.N + 31) / 32;
  const int64_t blocks = (tiles + warps - 1) / warps;
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)nb * sms);
  launch_stage_kernel(kern, grid, threads, smem, s, a);
}

template <int D, int R, int SCHEME, int STAGES>
void launch_recon_stream(const KArgs &a, int warps, cudaStream_t s) {
  using Q = StreamShape<D, R, STAGES>;
  const int threads = 32 * warps;
  const size_t smem = (size_t)recon_stream_smem(D, R, warps, STAGES);
  auto kern = recon_stream_kernel<D, R, SCHEME, STAGES>;
  static int resident[17] = {}, sms = 0;
  int &nb = resident[warps];
  if (!nb) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStreamSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    if (nb < 1) nb = 1;  // a launch that cannot fit fails loudly below
  }
  const int64_t tiles = (a.N + Q::CPW - 1) / Q::CPW;
  const int64_t blocks = (tiles + warps - 1) / warps;
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)nb * sms);
  launch_stage_kernel(kern, grid, threads, smem, s, a);
}

template <int D, int R, int SCHEME, bool ONE>
void launch_recon_halo(const KArgs &a, cudaStream_t s) {
  const int threads = kHaloWarps * 32, C = halo_tile(D);
  const size_t smem = (size_t)recon_halo_smem(D, R, a.hrec) / (ONE ? 2 : 1);
  auto kern = recon_halo_kernel<D, R, SCHEME, ONE>;
  static int resident = 0, sms = 0, for_hrec = -1;
  if (for_hrec != a.hrec) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStagedSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, threads, smem);
    if (resident < 1) resident = 1;  // a launch that cannot fit fails loudly below
    for_hrec = a.hrec;
  }
  const int64_t tiles = (a.N + C - 1) / C;
  const unsigned grid = ONE ? (unsigned)tiles : (unsigned)std::min<int64_t>(tiles, (int64_t)resident * sms);
  launch_stage_kernel(kern, grid, threads, smem, s, a);
}

// Host side: persistent launch of the staged kernel, grid = (co-resident blocks per SM) x SMs.
template <int D, int R, typename T, int SCHEME, bool LANES>
void launch_recon_staged(const KArgs &a, int threads, cudaStream_t s) {
  const int C = LANES ? (threads / 32) * (32 / (D + 2)) : threads;
  const size_t smem = (size_t)2 * C * StagedRecord<D, R, T>::CELL;
  auto kern = recon_staged_kernel<D, R, T, SCHEME, LANES>;
  static int resident[9] = {};  // per threads / 32
  static int sms = 0;
  int &nb = resident[threads / 32];
  if (!nb) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStagedSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    if (nb < 1) nb = 1;  // a launch that cannot fit fails loudly below
  }
  const int64_t tiles = (a.N + C - 1) / C;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)nb * sms);
  launch_stage_kernel(kern, grid, threads, smem, s, a);
}

}  // namespace cteno
