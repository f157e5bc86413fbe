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
//   6. its values at the face Gauss points, U_0 + sum_k a_k phi_k(xi_q) (eq. 2), written
//      structure-of-arrays for the flux kernel.
#pragma once

#include <cstdint>

#include "device.h"

namespace cteno {

template <int D, int R>
struct Shape {
  static constexpr int NV = D + 2;
  static constexpr int NF = D + 1;
  static constexpr int NQ = (D == 2) ? 2 : 4;
  static constexpr int NK = (D == 2 ? (R + 1) * (R + 2) / 2 : (R + 1) * (R + 2) * (R + 3) / 6) - 1;
  static constexpr int M = 2 * (NK + 1);
  static constexpr int ND = 2 * D;
  static constexpr int NP = (D == 2) ? 2 : 6;
};

template <typename T>
__device__ __forceinline__ T pow6(T x) {
  const T x2 = x * x;
  return x2 * x2 * x2;
}

// Selection of eqs. 19-23 / Alg. 1-2 in FP64, as printed (with lambda_s when lam_gamma).
// SI[0] central, SI[1..st-1] admissible directional. Returns delta bits (bit s).
__device__ __forceinline__ uint32_t select_fp64(const double *SI, int st, int scheme,
                                                int lam_gamma, double lam1, double lams,
                                                double eps, double C_T) {
  double g[5], sum = 0.0;
  if (scheme == 0) {
    for (int s = 0; s < st; ++s) g[s] = 1.0 / pow6(SI[s] + eps);
  } else {
    double tau = 0.0;
    if (st > 1) {
      double acc = 0.0;
      for (int s = 1; s < st; ++s) acc += fabs(SI[s] - SI[0]);
      tau = pow6(acc / (st - 1));
    }
    for (int s = 0; s < st; ++s) g[s] = 1.0 + tau / (SI[s] + eps);
  }
  if (lam_gamma)
    for (int s = 0; s < st; ++s) g[s] *= (s == 0) ? lam1 : lams;
  for (int s = 0; s < st; ++s) sum += g[s];
  uint32_t bits = 0;
  for (int s = 0; s < st; ++s)
    if (!(g[s] / sum < C_T)) bits |= 1u << s;
  return bits;
}

// The same decision in FP32 without overflow: every gamma_s is carried as its base-2 logarithm
// L_s, and chi_s = 2^(L_s - Lmax) / sum_t 2^(L_t - Lmax).
__device__ __forceinline__ uint32_t select_fp32(const float *SI, int st, int scheme,
                                                int lam_gamma, float log2lam1, float log2lams,
                                                float eps, float C_T) {
  float L[5], Lmax = -INFINITY;
  if (scheme == 0) {
    for (int s = 0; s < st; ++s) L[s] = -6.0f * log2f(SI[s] + eps);
  } else {
    float lt = -INFINITY;  // log2 tau
    if (st > 1) {
      float acc = 0.0f;
      for (int s = 1; s < st; ++s) acc += fabsf(SI[s] - SI[0]);
      lt = 6.0f * log2f(acc / (float)(st - 1));
    }
    for (int s = 0; s < st; ++s) {
      const float x = lt - log2f(SI[s] + eps);  // log2(tau / (SI + eps))
      // log2(1 + 2^x), split to stay accurate for large and small x
      L[s] = (x > 0.0f) ? x + log2f(1.0f + exp2f(-x)) : log2f(1.0f + exp2f(x));
    }
  }
  if (lam_gamma)
    for (int s = 0; s < st; ++s) L[s] += (s == 0) ? log2lam1 : log2lams;
  for (int s = 0; s < st; ++s) Lmax = fmaxf(Lmax, L[s]);
  float sum = 0.0f;
  for (int s = 0; s < st; ++s) sum += exp2f(L[s] - Lmax);
  uint32_t bits = 0;
  for (int s = 0; s < st; ++s)
    if (!(exp2f(L[s] - Lmax) / sum < C_T)) bits |= 1u << s;
  return bits;
}

template <int D, int R, typename T, int SCHEME>
__global__ void __launch_bounds__(256) recon_kernel(const KArgs a) {
  using S = Shape<D, R>;
  constexpr int NV = S::NV, NF = S::NF, NQ = S::NQ, NK = S::NK, M = S::M, ND = S::ND,
                NP = S::NP;
  constexpr int NPHI = NF * NP * NQ * NK;
  __shared__ T sPhi[NPHI];
  __shared__ T sO[NK * NK];
  {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
    for (int t = threadIdx.x; t < NK * NK; t += blockDim.x) sO[t] = (T)tb.O[t / NK][t % NK];
  }
  __syncthreads();

  const int64_t N = a.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;

  // cell means: FP64 directly, or (mixed path) the FP32 pair hi + lo of every FP64 value, so
  // that U_m - U_0 = (hi_m - hi_0) + (lo_m - lo_0) keeps FP64 accuracy in FP32 arithmetic
  const double *__restrict__ U64 = a.U;
  const float2 *__restrict__ U2 = (const float2 *)a.U32;
  const T *__restrict__ Pc = (const T *)a.Pc;
  const T *__restrict__ Pd = (const T *)a.Pd;
  const int32_t *__restrict__ st = a.st;

  T U0[NV];
  float L0[NV];  // low parts (mixed path)
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if constexpr (sizeof(T) == 4) {
      const float2 h = U2[v * N + i];
      U0[v] = (T)h.x;
      L0[v] = h.y;
    } else {
      U0[v] = (T)U64[v * N + i];
      L0[v] = 0.0f;
    }
  }
  auto delta = [&](int64_t j, T *du) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (sizeof(T) == 4) {
        const float2 h = U2[v * N + j];
        du[v] = (T)((h.x - (float)U0[v]) + (h.y - L0[v]));
      } else {
        du[v] = (T)(U64[v * N + j] - (double)U0[v]);
      }
    }
  };

  // 1-2: central coefficients a_opt = P_c (U_m - U_0)
  T ao[NK][NV];
#pragma unroll
  for (int k = 0; k < NK; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) ao[k][v] = (T)0;
#pragma unroll 4
  for (int m = 0; m < M; ++m) {
    const int64_t j = st[m * N + i];
    T du[NV];
    delta(j, du);
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const T p = Pc[((int64_t)k * M + m) * N + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) ao[k][v] += p * du[v];
    }
  }

  // directional coefficients (degree 1): members of face f are the next slots of the list
  const uint32_t info = a.cinfo[i];
  const uint32_t adm = (info >> kInfoAdmShift) & 0xFu;
  T ad[NF][D][NV];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) ad[f][k][v] = (T)0;
  int off = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nm = (info >> (4 * f)) & 15u;
    if ((adm >> f) & 1u) {
#pragma unroll
      for (int jj = 0; jj < ND; ++jj) {
        if (jj < nm) {
          const int64_t j = st[(int64_t)(off + jj) * N + i];
          T du[NV];
          delta(j, du);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const T p = Pd[((int64_t)(f * D + k) * ND + jj) * N + i];
#pragma unroll
            for (int v = 0; v < NV; ++v) ad[f][k][v] += p * du[v];
          }
        }
      }
    }
    off += nm;
  }

  // 3: linear coefficients of eq. 18 over the admissible stencils
  const int nadm = __popc(adm);
  const int stn = 1 + nadm;
  const double lam1d = 1.0 - 1.0 / a.lambda1p;
  const double lamsd = (stn > 1) ? (1.0 - lam1d) / (stn - 1) : 0.0;
  const T lam1 = (T)lam1d, lams = (T)lamsd;
  const T inv_lam1 = (T)(1.0 / lam1d);
  const float log2lam1 = (float)log2(lam1d);
  const float log2lams = (stn > 1) ? (float)log2(lamsd) : 0.0f;
  (void)lam1;

  const uint32_t perm = info >> kInfoPermShift;
  T *__restrict__ Uf = (T *)a.Uf;
  constexpr T INV_FACT = (D == 2) ? (T)0.5 : (T)(1.0 / 6.0);

#pragma unroll 1
  for (int v = 0; v < NV; ++v) {
    // p_1 (eq. 17): the directional polynomials only touch the linear coefficients
    T a1[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) a1[k] = ao[k][v];
    if (stn > 1) {
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
    T SI[1 + NF];
    {
      T s0 = (T)0;
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        T r = (T)0;
#pragma unroll
        for (int l = 0; l < NK; ++l) r += sO[k * NK + l] * a1[l];
        s0 += a1[k] * r;
      }
      SI[0] = s0;
    }
    int sidx[NF];  // admissible face of stencil slot 1 + s
    int ns = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if ((adm >> f) & 1u) {
        T s = (T)0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += ad[f][k][v] * ad[f][k][v];
        SI[1 + ns] = s * INV_FACT;
        sidx[ns] = f;
        ++ns;
      }
    }
    // 5: selection
    uint32_t bits;
    if constexpr (sizeof(T) == 8) {
      bits = select_fp64((const double *)SI, stn, SCHEME, a.lam_gamma, lam1d, lamsd, a.eps, a.C_T);
    } else {
      bits = select_fp32((const float *)SI, stn, SCHEME, a.lam_gamma, log2lam1, log2lams,
                         fmaxf((float)a.eps, 1e-40f), (float)a.C_T);
    }
    T af[NK];
    uint8_t flag;
    if (bits & 1u) {
#pragma unroll
      for (int k = 0; k < NK; ++k) af[k] = a1[k];
      flag = 1;
    } else {
#pragma unroll
      for (int k = 0; k < NK; ++k) af[k] = (T)0;
      flag = 0;
      const int nsel = __popc(bits >> 1);
      const T w = (T)1 / (T)nsel;
#pragma unroll
      for (int s = 0; s < NF; ++s) {
        if (s < ns && ((bits >> (1 + s)) & 1u)) {
          const int f = sidx[s];
          // ad[f] with a runtime f: select through an unrolled loop to stay in registers
#pragma unroll
          for (int ff = 0; ff < NF; ++ff)
            if (ff == f) {
#pragma unroll
              for (int k = 0; k < D; ++k) af[k] += w * ad[ff][k][v];
            }
          flag |= (uint8_t)(1u << (1 + f));
        }
      }
    }
    if (a.flags) a.flags[v * N + i] = flag;
    // 6: face Gauss-point values
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int p = (perm >> (3 * f)) & 7u;
      const T *ph = &sPhi[((f * NP + p) * NQ) * NK];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T val = (T)L0[v];
#pragma unroll
        for (int k = 0; k < NK; ++k) val += ph[q * NK + k] * af[k];
        val += U0[v];
        Uf[((int64_t)(f * NQ + q) * NV + v) * N + i] = val;
      }
    }
  }

  // positivity guard (not part of the paper): non-physical face state -> cell mean everywhere
  if (a.guard_on) {
    bool bad = false;
    const T gm1 = (T)(a.gamma - 1.0);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = Uf[((int64_t)(f * NQ + q) * NV + v) * N + i];
        T ke = (T)0;
#pragma unroll
        for (int j = 0; j < D; ++j) ke += u[1 + j] * u[1 + j];
        const T p = gm1 * (u[NV - 1] - (T)0.5 * ke / u[0]);
        if (!(u[0] > (T)0) || !(p > (T)0)) bad = true;
      }
    if (bad) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int v = 0; v < NV; ++v) Uf[((int64_t)(f * NQ + q) * NV + v) * N + i] = U0[v] + (T)L0[v];
      atomicAdd(a.guard, 1ull);
    }
  }

  // CFL time step bookkeeping at the first stage of a step: dt[next] -> dt[cur]
  if (a.dt_swap && i < a.nmesh) {
    a.dt[i] = a.dt[a.nmesh + i];
    a.dt[a.nmesh + i] = 1e300;
  }
}

}  // namespace cteno
