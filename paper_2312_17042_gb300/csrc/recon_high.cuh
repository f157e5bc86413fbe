// recon_high.cuh -- reconstruction of central degrees 4 to 6 in 2D (CTENO5 to CTENO7, paper Sec.
// 2.3 and Fig. 1, whose fifth-order scheme pairs the central stencil with third-order directional
// ones): central polynomials of K(r,2) - 1 = 14, 20 or 27 unknowns fitted on M = 2K(r,2) cells,
// directional polynomials of degree 2 (5 unknowns, at most 10 members each, within the central
// stencil), and n-point Gauss-Legendre edges (n = 3, 3, 4).
//
// Variable-per-lane schedule only: a group of four lanes reconstructs one cell, lane v conserved
// variable v, and keeps its own 27 + 15 coefficients at most (a thread holding all four variables
// would need four times that in registers). The steps are those of recon.cuh (eqs. 10-23,
// Alg. 1 / 2, CWENO and TENO weightings):
//   central   a_opt = P_c (U_m - U_0), the member-major record read in 16-byte aligned groups of
//             G members (G NK values a multiple of 16 bytes);
//   directional a_s = P_s (U_m - U_0) from unknown-major rows of 12 member slots (Dir<2, R>);
//   p_1 (eq. 17) subtracts lambda_s a_s from the first five (degree <= 2) coefficients;
//   SI (eq. 15) with the degree-r matrix O; a directional SI uses its top-left 5 x 5 block, the
//   same integrals of the derivatives of a quadratic;
//   face values at the edge's Gauss points, stored in sorted-vertex order (the rule is
//   symmetric, so the other orientation reverses the point order).
#pragma once

#include "recon.cuh"

namespace cteno {

template <int R>
struct HighShape {
  static_assert(R >= 4 && R <= 6, "central degrees 4 to 6");
  static constexpr int NK = (R + 1) * (R + 2) / 2 - 1;
  static constexpr int M = 2 * (NK + 1);
  static constexpr int NQ = (R + 2) / 2;                 // Gauss points per edge
  static constexpr int G = (NK % 2 == 0) ? 2 : 4;        // members per aligned group of the record
  static_assert(M % G == 0, "groups tile the stencil");
};

// Constant banks of the three degrees: O (upper triangle, off-diagonal doubled, NK x NK) and the
// basis values phi_k at the Gauss points of each local edge in local vertex order, [f][q][k].
__constant__ double c_OH4d[14 * 14], c_OH5d[20 * 20], c_OH6d[27 * 27];
__constant__ float c_OH4f[14 * 14], c_OH5f[20 * 20], c_OH6f[27 * 27];
__constant__ double c_PhiH4d[3 * 3 * 14], c_PhiH5d[3 * 3 * 20], c_PhiH6d[3 * 4 * 27];
__constant__ float c_PhiH4f[3 * 3 * 14], c_PhiH5f[3 * 3 * 20], c_PhiH6f[3 * 4 * 27];

template <typename T, int R>
__device__ __forceinline__ T cOH(int idx) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (R == 4) return c_OH4f[idx];
    else if constexpr (R == 5) return c_OH5f[idx];
    else return c_OH6f[idx];
  } else {
    if constexpr (R == 4) return c_OH4d[idx];
    else if constexpr (R == 5) return c_OH5d[idx];
    else return c_OH6d[idx];
  }
}
template <typename T, int R>
__device__ __forceinline__ T cPhiH(int idx) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (R == 4) return c_PhiH4f[idx];
    else if constexpr (R == 5) return c_PhiH5f[idx];
    else return c_PhiH6f[idx];
  } else {
    if constexpr (R == 4) return c_PhiH4d[idx];
    else if constexpr (R == 5) return c_PhiH5d[idx];
    else return c_PhiH6d[idx];
  }
}

template <typename T, typename S>
inline cudaError_t upload_symbol(const S &sym, const T *src, size_t count, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(sym, src, count * sizeof(T), 0, cudaMemcpyHostToDevice, s);
}

template <int R>
inline cudaError_t upload_high_tables(const Tables &t, cudaStream_t s) {
  constexpr int NK = HighShape<R>::NK, NQ = HighShape<R>::NQ;
  double Od[NK * NK] = {}, Pd[3 * NQ * NK] = {};
  float Of[NK * NK] = {}, Pf[3 * NQ * NK] = {};
  for (int k = 0; k < NK; ++k)
    for (int l = k; l < NK; ++l) {
      Od[k * NK + l] = (l == k ? 1.0 : 2.0) * t.O[k][l];
      Of[k * NK + l] = (float)Od[k * NK + l];
    }
  for (int f = 0; f < 3; ++f)
    for (int q = 0; q < NQ; ++q)
      for (int k = 0; k < NK; ++k) {
        Pd[(f * NQ + q) * NK + k] = t.Phi[f][0][q][k];
        Pf[(f * NQ + q) * NK + k] = (float)t.Phi[f][0][q][k];
      }
  cudaError_t e;
  if constexpr (R == 4) {
    if ((e = upload_symbol(c_OH4d, Od, NK * NK, s)) || (e = upload_symbol(c_OH4f, Of, NK * NK, s)) ||
        (e = upload_symbol(c_PhiH4d, Pd, 3 * NQ * NK, s)) || (e = upload_symbol(c_PhiH4f, Pf, 3 * NQ * NK, s)))
      return e;
  } else if constexpr (R == 5) {
    if ((e = upload_symbol(c_OH5d, Od, NK * NK, s)) || (e = upload_symbol(c_OH5f, Of, NK * NK, s)) ||
        (e = upload_symbol(c_PhiH5d, Pd, 3 * NQ * NK, s)) || (e = upload_symbol(c_PhiH5f, Pf, 3 * NQ * NK, s)))
      return e;
  } else {
    if ((e = upload_symbol(c_OH6d, Od, NK * NK, s)) || (e = upload_symbol(c_OH6f, Of, NK * NK, s)) ||
        (e = upload_symbol(c_PhiH6d, Pd, 3 * NQ * NK, s)) || (e = upload_symbol(c_PhiH6f, Pf, 3 * NQ * NK, s)))
      return e;
  }
  return cudaStreamSynchronize(s);  // the host arrays above go out of scope
}

// One block of 8-cell warps; lane v of group grp reconstructs variable v of cell 8 w + grp (the
// last cell shadows the lanes past the end and stores nothing).
template <int R, typename T, int SCHEME, bool CHR>
__device__ __forceinline__ void recon_high_body(const KArgs &a) {
  using H = HighShape<R>;
  using DR = Dir<2, R>;
  constexpr int NV = 4, NVP = 4, NF = 3, CPW = 8;
  constexpr int NK = H::NK, M = H::M, NQ = H::NQ, G = H::G;
  constexpr int KD = DR::KD, ND = DR::ND, NDP = DR::NDP, PDS = DR::PDS;
  constexpr int CH = 16 / (int)sizeof(T);
  constexpr bool F32 = sizeof(T) == 4;
  static_assert((G * NK) % CH == 0 && NDP % CH == 0 && PDS % CH == 0, "16-byte aligned records");
  pdl_wait(a);  // the state written by the previous stage's update
  const int lane = threadIdx.x & 31;
  const int grp = lane / NV, v = lane - grp * NV, base = grp * NV;
  const int64_t N = a.N;
  const int64_t cell = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW + grp;
  const bool active = cell < N;
  const int64_t i = active ? cell : N - 1;

  // own mean of variable v: FP64, or the FP32 pair (hi, lo)
  T U0;
  float L0;
  if constexpr (F32) {
    const float2 h = __ldg(reinterpret_cast<const float2 *>(a.U32) + i * NVP + v);
    U0 = h.x;
    L0 = h.y;
  } else {
    U0 = __ldg(a.U + i * NVP + v);
    L0 = 0.0f;
  }
  auto delta = [&](int64_t j) -> T {  // U_j - U_0 of variable v (eq. 10)
    if constexpr (F32) {
      const float2 h = __ldg(reinterpret_cast<const float2 *>(a.U32) + j * NVP + v);
      return (h.x - (float)U0) + (h.y - L0);
    } else {
      return __ldg(a.U + j * NVP + v) - U0;
    }
  };
  const int32_t *__restrict__ sti = a.st + i * M;

  // central coefficients a_opt = P_c (U_m - U_0), G members at a time
  const T *__restrict__ Pci = (const T *)a.Pc + i * (int64_t)(M * NK);
  T ao[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) ao[k] = (T)0;
#pragma unroll 2
  for (int m0 = 0; m0 < M; m0 += G) {
    T du[G];
#pragma unroll
    for (int g = 0; g < G; ++g) du[g] = delta(__ldg(sti + m0 + g));
#pragma unroll
    for (int c = 0; c < G * NK / CH; ++c) {
      T pb[CH];
      load16_stream<T, CH>(Pci + m0 * NK + c * CH, pb);
#pragma unroll
      for (int t = 0; t < CH; ++t) ao[(c * CH + t) % NK] += pb[t] * du[(c * CH + t) / NK];
    }
  }

  // directional coefficients (degree 2): the members of face f are the next slots of the list
  const uint32_t info = __ldg(a.cinfo + i);
  const uint32_t adm = (info >> kInfoAdmShift) & 7u;
  const T *__restrict__ Pdi = (const T *)a.Pd + i * (int64_t)(NF * PDS);
  T ad[NF][KD];
  {
    int off = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int nm = (info >> (4 * f)) & 15u;
#pragma unroll
      for (int k = 0; k < KD; ++k) ad[f][k] = (T)0;
      if ((adm >> f) & 1u) {
        T du[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) du[j] = (j < nm) ? delta(__ldg(sti + off + j)) : (T)0;
#pragma unroll
        for (int k = 0; k < KD; ++k) {
          T pk[NDP];
          load16_stream<T, NDP>(Pdi + f * PDS + k * NDP, pk);
          T s = (T)0;
#pragma unroll
          for (int j = 0; j < ND; ++j) s += pk[j] * du[j];
          ad[f][k] = s;
        }
      }
      off += nm;
    }
  }

  // p_1 (eq. 17) in place of a_opt, the smoothness indicators (eq. 15: a directional one with
  // the top-left 5 x 5 block of O), the selection or the CWENO weights, the face values
  auto oc = [](int idx) { return cOH<T, R>(idx); };
  auto sid = [](const T (&adf)[KD]) {
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      T rr = (T)0;
#pragma unroll
      for (int l = k; l < KD; ++l) rr += cOH<T, R>(k * NK + l) * adf[l];
      s += adf[k] * rr;
    }
    return s;
  };
  auto phi = [](int f, int q, int k) { return cPhiH<T, R>((f * NQ + q) * NK + k); };
  lane_faces<2, NK, KD, NQ, T, SCHEME, CHR>(a, i, active, v, base, ao, ad, info, U0, L0, oc, sid,
                                           phi_tab(phi));
  // CFL time step bookkeeping at the first stage of a step: dt[next] -> dt[cur]
  if (a.dt_swap && blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.nmesh; t += blockDim.x) {
      a.dt[t] = a.dt[a.nmesh + t];
      a.dt[a.nmesh + t] = 1e300;
    }
}

template <int R, typename T, int SCHEME, bool CHR>
__global__ void __launch_bounds__(256) recon_high_kernel(const KArgs a) {
  recon_high_body<R, T, SCHEME, CHR>(a);
}

// The FP32 body compiled for at most 64 registers per thread (launch value kHighOcc + b): 32
// resident warps per SM instead of 24-28, for a kernel that waits on its record loads and
// neighbour gathers (a few dozen bytes of spill).
template <int R, int SCHEME>
__global__ void __launch_bounds__(256, 4) recon_high_kernel_occ(const KArgs a) {
  recon_high_body<R, float, SCHEME, false>(a);
}

}  // namespace cteno
