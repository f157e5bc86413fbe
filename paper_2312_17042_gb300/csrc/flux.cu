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

// Reciprocal, quotient and square root: IEEE operations on the FP64 path; on the mixed path the
// GPU's single-instruction approximations (relative error about 2^-23, subnormal operands flushed
// to zero: densities, pressures and wave-speed differences of physical states are normal numbers).
// Both cells of a face run the same instruction sequence on the same operands, so their face
// values stay bit-identical.
template <typename T>
__device__ __forceinline__ T rcp_(T x) {
  if constexpr (sizeof(T) == 4) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else {
    return 1.0 / x;
  }
}
template <typename T>
__device__ __forceinline__ T div_(T x, T y) {
  if constexpr (sizeof(T) == 4) return x * rcp_<T>(y);
  else return x / y;
}
template <typename T>
__device__ __forceinline__ T sqrt_(T x) {
  if constexpr (sizeof(T) == 4) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else {
    return sqrt(x);
  }
}

// Finite FP64 value (exponent field not all ones), tested with integer operations.
__device__ __forceinline__ bool finite64(double x) {
  return ((__double2hiint(x) >> 20) & 0x7FF) != 0x7FF;
}

// Exact FP32 -> FP64 conversion in integer operations (the FP64 pipe of this GPU is narrow);
// subnormal FP32 values become zero, infinities and NaNs stay non-finite.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xFFu, sign = b & 0x80000000u;
  const uint32_t hi = (e == 0) ? sign : (sign | ((e == 255u ? 0x7FFu : e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3));
  const uint32_t lo = (e == 0) ? 0u : (b << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 pair (hi, lo) in integer operations: hi is x truncated to 24 significant bits and
// lo the remainder truncated to 24 bits, so |x - hi - lo| < 2^-46 |x| for 2^-126 <= |x| < 2^128.
// Smaller magnitudes give (+-0, +-0); larger ones and non-finite values an infinity in hi (the
// update reports non-finite states separately).
__device__ __forceinline__ float2 f64_split(double x) {
  const uint32_t H = (uint32_t)__double2hiint(x), L = (uint32_t)__double2loint(x);
  const uint32_t sign = H & 0x80000000u;
  const int e = (int)((H >> 20) & 0x7FFu);
  const int ef = e - 896;  // biased FP32 exponent of hi
  if (ef <= 0) return make_float2(__uint_as_float(sign), __uint_as_float(sign));
  if (ef >= 255) return make_float2(__uint_as_float(sign | 0x7F800000u), 0.0f);
  const uint32_t mhi = ((H & 0xFFFFFu) << 3) | (L >> 29);
  const float hi = __uint_as_float(sign | ((uint32_t)ef << 23) | mhi);
  const uint32_t m = L & 0x1FFFFFFFu;  // the remaining 29 bits, unit 2^(e - 1075)
  if (m == 0u) return make_float2(hi, __uint_as_float(sign));
  const int p = 31 - __clz((int)m);    // leading bit of m
  const int el = p + e - 948;          // biased FP32 exponent of lo
  if (el <= 0) return make_float2(hi, __uint_as_float(sign));
  const uint32_t ml = ((p >= 23) ? (m >> (p - 23)) : (m << (23 - p))) & 0x7FFFFFu;
  return make_float2(hi, __uint_as_float(sign | ((uint32_t)el << 23) | ml));
}

// Outside state of a reflective wall at a Gauss point (reading: the paper runs walls in Sec. 3.3
// and 3.4 without printing their treatment): the mirror image of the inside state u across the
// wall with outward unit normal n, (rho, m - 2 (m.n) n, E).
template <int D, typename T>
__device__ __forceinline__ void wall_mirror(const T *u, const T *n, T *o) {
  T mn = (T)0;
#pragma unroll
  for (int j = 0; j < D; ++j) mn += u[1 + j] * n[j];
  o[0] = u[0];
#pragma unroll
  for (int j = 0; j < D; ++j) o[1 + j] = u[1 + j] - (T)2 * mn * n[j];
  o[D + 1] = u[D + 1];
}

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
  const T iL = rcp_<T>(rL), iR = rcp_<T>(rR);
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
  const T cL = sqrt_<T>(g * pL * iL), cR = sqrt_<T>(g * pR * iR);
  const T HL = (uL[NV - 1] + pL) * iL, HR = (uR[NV - 1] + pR) * iR;
  const T Dr = sqrt_<T>(rR * iL);
  const T idn = rcp_<T>((T)1 + Dr);
  T ut2 = 0, utn = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const T ut = (vL[j] + vR[j] * Dr) * idn;
    ut2 += ut * ut;
    utn += ut * n[j];
  }
  const T Ht = (HL + HR * Dr) * idn;
  const T ct = sqrt_<T>((g - (T)1) * (Ht - (T)0.5 * ut2));
  const T SL = fmin(unL - cL, utn - ct);
  const T SR = fmax(unR + cR, utn + ct);
  const T SM = div_<T>(rR * unR * (SR - unR) - rL * unL * (SL - unL) + pL - pR,
                       rR * (SR - unR) - rL * (SL - unL));
  // The four cases, tested in the order SL > 0 (left state), SM > 0 (left star state), SR > 0
  // (right star state), else (right state), evaluated without branches (neighbouring faces of a
  // warp take different cases): the operands of side k are selected, the star correction is
  // dropped in the two supersonic cases. Each case's arithmetic is the same as written out alone.
  const bool left = (SL > (T)0) || (SM > (T)0);
  const bool sup = (SL > (T)0) || (!(SM > (T)0) && !(SR > (T)0));
  T uk[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) uk[v] = left ? uL[v] : uR[v];
  const T pk = left ? pL : pR, unk = left ? unL : unR, Sk = left ? SL : SR, rk = uk[0];
  physical_flux<D, T>(uk, n, pk, unk, F);
  const T ps = rL * (unL - SL) * (unL - SM) + pL;
  const T fct = rcp_<T>(Sk - SM), a = Sk - unk;
  T G[NV];
  G[0] = F[0] + Sk * (rk * a * fct - uk[0]);
#pragma unroll
  for (int j = 0; j < D; ++j) G[1 + j] = F[1 + j] + Sk * ((a * uk[1 + j] + (ps - pk) * n[j]) * fct - uk[1 + j]);
  G[NV - 1] = F[NV - 1] + Sk * ((a * uk[NV - 1] - pk * unk + ps * SM) * fct - uk[NV - 1]);
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = sup ? F[v] : G[v];
}

__device__ __forceinline__ int mesh_of(const KArgs &a, int64_t i) {
  int lo = 0, hi = a.nmesh - 1;
  while (lo < hi) {  // last mesh whose offset <= i
    const int mid = (lo + hi + 1) >> 1;
    if (a.mesh_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Outside state of boundary face f of cell i at NQ Gauss points (reading: the paper runs walls,
// inflow and a moving-shock boundary in Sec. 3.3 / 3.4 without printing their treatment): kind 1
// the mirror image of the inside state uI (wall_mirror); kind 2 the fixed state A; kind 3 state A
// where the moving shock line has passed the face midpoint (c_f + vs t > 0, c_f in the face's
// geometry slot 2), else B; kind 0 (transmissive) the cell mean um.
template <int D, typename T, int NQ>
__device__ __forceinline__ void boundary_state(const KArgs &a, const int64_t i, const int kind, const T *gf,
                                               const T *uI, const double *um, T *uO) {
  constexpr int NV = D + 2;
  constexpr bool F32 = sizeof(T) == 4;
  if (kind == 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) wall_mirror<D, T>(uI + q * NV, gf, uO + q * NV);
    return;
  }
  bool use_a = kind == 2;
  if (kind == 3) {
    const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
    const double t = a.time[mesh] + a.stage_c * a.dt[mesh];
    use_a = (double)gf[2] + a.shock_vs * t > 0.0;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T x;
    if (kind == 0) x = (T)um[v];
    else if constexpr (F32) x = use_a ? a.bA32[v] : a.bB32[v];
    else x = use_a ? a.bA[v] : a.bB[v];
#pragma unroll
    for (int q = 0; q < NQ; ++q) uO[q * NV + v] = x;
  }
}

// Order-preserving map of a non-negative double onto unsigned 64-bit (for an atomic minimum).
__device__ __forceinline__ void atomic_min_pos(double *addr, double v) {
  atomicMin((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Minimum of the lanes' positive values v into dt[slot] with one atomic per warp when all lanes
// of the warp target the same slot (cells of a mesh are contiguous, so a warp straddles at most a
// mesh boundary), else one per lane. Lanes with nothing to contribute pass +inf (1e300). Must be
// called by all 32 lanes of the warp.
__device__ __forceinline__ void warp_min_to(double *dt, int slot, double v) {
  const int first = __shfl_sync(0xffffffffu, slot, 0), last = __shfl_sync(0xffffffffu, slot, 31);
  if (first == last) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
      b = (x < b) ? x : b;
    }
    if ((threadIdx.x & 31) == 0 && b < (unsigned long long)__double_as_longlong(1e300))
      atomicMin((unsigned long long *)&dt[slot], b);
  } else if (v < 1e300) {
    atomic_min_pos(&dt[slot], v);
  }
}

// Local CFL step of one cell: |V_i| / sum_f |A_f| (|u_i . n_f| + c_i), in the path's arithmetic
// type (FP64 geometry for the FP64 path; FP32 values and geometry for the mixed path, where the
// step only sets the time-step size).
template <int D, typename T>
__device__ __forceinline__ double local_dt(const KArgs &a, int64_t i, const T *uu) {
  constexpr int NF = D + 1;
  constexpr bool F32 = sizeof(T) == 4;
  const T *G = F32 ? (const T *)a.geo32 : (const T *)a.geo;
  T g;
  if constexpr (F32) g = a.gamma32; else g = a.gamma;
  const T ir = rcp_<T>(uu[0]);
  T ke = 0, u[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    u[j] = uu[1 + j] * ir;
    ke += uu[1 + j] * u[j];
  }
  const T p = (g - (T)1) * (uu[D + 1] - (T)0.5 * ke);
  const T c = sqrt_<T>(g * p * ir);
  T s = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T *gf = G + (i * NF + f) * 4;
    T un = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) un += u[j] * gf[j];
    s += gf[3] * (fabs(un) + c);
  }
  if constexpr (F32) return (double)rcp_<float>(s * (float)a.vol[i]);
  else return 1.0 / (s * a.vol[i]);
}

// Error-free sum of two FP32 values (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Residual (eq. 2) and stage update in FP64, the FP32 shadow of the new state and, at the last
// stage, the cell's CFL step of the next step: the common end of the per-cell flux kernels. u64:
// the cell's current state, acc: sum_f |A_f| sum_q w_q F_q. Runge-Kutta (Sec. 2, "3rd- or
// 4th-order"): SSP-RK3 in Shu-Osher form, U1 = U^n + dt R, U2 = 3/4 U^n + 1/4 (U1 + dt R(U1)),
// U^{n+1} = 1/3 U^n + 2/3 (U2 + dt R(U2)); or the classical RK4 with its running sum in Acc:
// Acc = U^n + dt/6 k1, U = U^n + dt/2 k1; Acc += dt/3 k2, U = U^n + dt/2 k2; Acc += dt/3 k3,
// U = U^n + dt k3; U^{n+1} = Acc + dt/6 k4.
template <int D, typename T>
__device__ __forceinline__ void stage_tail(const KArgs &a, const int64_t i, const bool active,
                                           const double (&u64)[Lay<D>::NVP], const double (&acc)[Lay<D>::NV]) {
  using L = Lay<D>;
  constexpr int NV = L::NV, NVP = L::NVP;
  constexpr bool F32 = sizeof(T) == 4;
  const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
  const double dtv = a.dt[mesh] * a.vol[i];  // dt / |V_i|
  double un[NVP], res[NVP], ac[NVP];
  if (a.stage != 0) {
#pragma unroll
    for (int c = 0; c < NVP / 2; ++c) {
      const double2 x = reinterpret_cast<const double2 *>(a.Un + i * NVP)[c];
      un[2 * c] = x.x;
      un[2 * c + 1] = x.y;
    }
  }
  if (a.rk4 && a.stage != 0) {
#pragma unroll
    for (int c = 0; c < NVP / 2; ++c) {
      const double2 x = reinterpret_cast<const double2 *>(a.Acc + i * NVP)[c];
      ac[2 * c] = x.x;
      ac[2 * c + 1] = x.y;
    }
  }
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NVP; ++v) {
    if (v >= NV) {
      res[v] = 0.0;
      ac[v] = 0.0;
      continue;
    }
    if (!a.rk4) {
      const double upd = u64[v] - dtv * acc[v];
      if (a.stage == 0) res[v] = upd;
      else if (a.stage == 1) res[v] = 0.75 * un[v] + 0.25 * upd;
      else res[v] = (1.0 / 3.0) * un[v] + (2.0 / 3.0) * upd;
    } else {
      const double F = -dtv * acc[v];  // dt k_s
      if (a.stage == 0) {
        ac[v] = u64[v] + F / 6.0;
        res[v] = u64[v] + 0.5 * F;
      } else if (a.stage == 1) {
        ac[v] += F / 3.0;
        res[v] = un[v] + 0.5 * F;
      } else if (a.stage == 2) {
        ac[v] += F / 3.0;
        res[v] = un[v] + F;
      } else {
        res[v] = ac[v] + F / 6.0;
      }
    }
    finite = finite && finite64(res[v]);
  }
  if (active) {
#pragma unroll
    for (int c = 0; c < NVP / 2; ++c) {
      reinterpret_cast<double2 *>(a.U + i * NVP)[c] = make_double2(res[2 * c], res[2 * c + 1]);
      if (a.stage == 0)
        reinterpret_cast<double2 *>(a.Un + i * NVP)[c] = make_double2(u64[2 * c], u64[2 * c + 1]);
      if (a.rk4 && a.stage < 3)
        reinterpret_cast<double2 *>(a.Acc + i * NVP)[c] = make_double2(ac[2 * c], ac[2 * c + 1]);
    }
  }
  T ust[NVP];  // the new state in the path's type, for the CFL step
  if constexpr (F32) {  // FP32 (hi, lo) shadow of the new state
    float4 hl[NVP / 2];
#pragma unroll
    for (int c = 0; c < NVP / 2; ++c) {
      const float2 s0 = f64_split(res[2 * c]), s1 = f64_split(res[2 * c + 1]);
      hl[c] = make_float4(s0.x, s0.y, s1.x, s1.y);
      ust[2 * c] = s0.x;
      ust[2 * c + 1] = s1.x;
    }
    if (active) {
#pragma unroll
      for (int c = 0; c < NVP / 2; ++c) reinterpret_cast<float4 *>(a.U32 + i * 2 * NVP)[c] = hl[c];
    }
  } else {
#pragma unroll
    for (int v = 0; v < NVP; ++v) ust[v] = res[v];
  }
  if (!finite && active) atomicOr(a.err, kErrNonFinite);
  if (a.stage == a.last_stage)
    warp_min_to(a.dt, a.nmesh + mesh, (finite && active) ? a.cfl * local_dt<D, T>(a, i, ust) : 1e300);
}

template <int D, typename T, int MINB, int NQ>
__global__ void __launch_bounds__(MINB ? 128 : 256, MINB ? MINB : 1) flux_kernel(const KArgs a) {
  using L = Lay<D>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, FB = NQ * NV;
  constexpr bool F32 = sizeof(T) == 4;
  pdl_wait(a);  // face states of the reconstruction, the state of the previous stage
  const int64_t N = a.N;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // threads past the last cell shadow it and store nothing, so that every lane of the warp
  // reaches the time-step reduction
  const bool active = cell < N;
  const int64_t i = active ? cell : N - 1;
  const T *__restrict__ Uf = (const T *)a.Uf;
  const T *__restrict__ G = F32 ? (const T *)a.geo32 : (const T *)a.geo;
  T g;
  if constexpr (F32) g = a.gamma32; else g = a.gamma;
  const uint32_t meta = __ldg(a.fmeta + i);
  const int4 nb4 = __ldg(reinterpret_cast<const int4 *>(a.nbr) + i);
  const int nbv[4] = {nb4.x, nb4.y, nb4.z, nb4.w};
  // this cell's FP64 record (read before it is overwritten by this same thread)
  double u64[NVP];
#pragma unroll
  for (int c = 0; c < NVP / 2; ++c) {
    const double2 x = reinterpret_cast<const double2 *>(a.U + i * NVP)[c];
    u64[2 * c] = x.x;
    u64[2 * c + 1] = x.y;
  }
  double acc[NV];
  float acc_hi[NV], acc_lo[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    acc[v] = 0.0;
    acc_hi[v] = 0.0f;
    acc_lo[v] = 0.0f;
  }
  // faces in groups of FG: all loads of a group are issued before its arithmetic
  constexpr int FG = MINB ? 1 : ((D == 2) ? NF : 2);  // the register-capped variant: one face at a time
#pragma unroll
  for (int f0 = 0; f0 < NF; f0 += FG) {
    T gf[FG][4], uI[FG][FB], uO[FG][FB];
#pragma unroll
    for (int ff = 0; ff < FG; ++ff) {
      const int f = f0 + ff;
      if (f >= NF) break;
      const int64_t j = nbv[f];
      const int fj = (meta >> (2 * f)) & 3u;
      load16<T, 4>(G + (i * NF + f) * 4, gf[ff]);
      load16<T, FB>(Uf + (i * NF + f) * FB, uI[ff]);
      if (j >= 0) {
        load16<T, FB>(Uf + (j * NF + fj) * FB, uO[ff]);
      } else {  // boundary face: its kind's outside state
        boundary_state<D, T, NQ>(a, i, (meta >> (kMetaKindShift + 2 * f)) & 3u, gf[ff], uI[ff], u64, uO[ff]);
      }
    }
#pragma unroll
    for (int ff = 0; ff < FG; ++ff) {
      const int f = f0 + ff;
      if (f >= NF) break;
      const bool own = (meta >> (kMetaOwnerShift + f)) & 1u;
      T n[D];
#pragma unroll
      for (int k = 0; k < D; ++k) n[k] = own ? gf[ff][k] : -gf[ff][k];
      // face flux |A| sum_q w_q F_q in the path's type: both cells of the face evaluate it with
      // the same operands in the same order, so the two values are identical
      T Ff[NV];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T F[NV];
        if (own) hllc<D, T>(uI[ff] + q * NV, uO[ff] + q * NV, n, g, F);
        else hllc<D, T>(uO[ff] + q * NV, uI[ff] + q * NV, n, g, F);
        T w;
    if constexpr (F32) w = a.fw32[q]; else w = a.fw[q];
#pragma unroll
        for (int v = 0; v < NV; ++v) Ff[v] = (q == 0) ? w * F[v] : Ff[v] + w * F[v];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T x = gf[ff][3] * Ff[v];
        const T c = own ? x : -x;  // the exact negative of the other cell's value
        if constexpr (F32) {
          // exact FP32 accumulation over the faces: running (hi, lo) by TwoSum
          float s, e;
          two_sum(acc_hi[v], c, s, e);
          acc_hi[v] = s;
          acc_lo[v] += e;
        } else {
          acc[v] += c;  // FP64 accumulation over the faces
        }
      }
    }
  }
  if constexpr (F32) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = f32_to_f64(acc_hi[v]) + f32_to_f64(acc_lo[v]);
  }
  stage_tail<D, T>(a, i, active, u64, acc);
}

// Face flux of the face-based schedule: one thread per face, HLLC at the face's Gauss points in
// its owner's orientation (the same operands and order as flux_kernel's owner side), weighted and
// scaled by the area; record e holds |A| sum_q w_q F_q, padded to NFP values.
template <int D, typename T, int NQ>
__global__ void __launch_bounds__(256) face_flux_kernel(const KArgs a) {
  using L = Lay<D>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, FB = NQ * NV;
  constexpr int NFP = (NV + 3) & ~3;
  constexpr bool F32 = sizeof(T) == 4;
  pdl_wait(a);  // face states of the reconstruction
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.nfaces) return;
  const int2 codes = __ldg(reinterpret_cast<const int2 *>(a.face) + e);  // owner, neighbour side
  const int64_t i = codes.x >> 2;
  const int f = codes.x & 3;
  const T *__restrict__ Uf = (const T *)a.Uf;
  const T *__restrict__ G = F32 ? (const T *)a.geo32 : (const T *)a.geo;
  T g;
  if constexpr (F32) g = a.gamma32; else g = a.gamma;
  T gf[4], uI[FB], uO[FB];
  load16<T, 4>(G + (i * NF + f) * 4, gf);
  load16<T, FB>(Uf + (i * NF + f) * FB, uI);
  if (codes.y >= 0) {
    const int64_t j = codes.y >> 2;
    const int fj = codes.y & 3;
    load16<T, FB>(Uf + (j * NF + fj) * FB, uO);
  } else {  // boundary face: its kind's outside state
    double um[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) um[v] = a.U[i * NVP + v];
    boundary_state<D, T, NQ>(a, i, (__ldg(a.fmeta + i) >> (kMetaKindShift + 2 * f)) & 3u, gf, uI, um, uO);
  }
  T n[D];
#pragma unroll
  for (int k = 0; k < D; ++k) n[k] = gf[k];
  T Ff[NV];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T F[NV];
    hllc<D, T>(uI + q * NV, uO + q * NV, n, g, F);
    T w;
    if constexpr (F32) w = a.fw32[q]; else w = a.fw[q];
#pragma unroll
    for (int v = 0; v < NV; ++v) Ff[v] = (q == 0) ? w * F[v] : Ff[v] + w * F[v];
  }
  T out[NFP];
#pragma unroll
  for (int v = 0; v < NFP; ++v) out[v] = (v < NV) ? gf[3] * Ff[v] : (T)0;
  store16<T, NFP>((T *)a.Ff + e * NFP, out);
}

// Residual and stage update of the face-based schedule: as flux_kernel with its face fluxes read
// from face_flux_kernel's records.
template <int D, typename T, int MINB>
__global__ void __launch_bounds__(MINB ? 128 : 256, MINB ? MINB : 1) cell_update_kernel(const KArgs a) {
  using L = Lay<D>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF;
  constexpr bool F32 = sizeof(T) == 4;
  pdl_wait(a);  // the face fluxes of this stage
  const int64_t N = a.N;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // threads past the last cell shadow it and store nothing, so that every lane of the warp
  // reaches the time-step reduction
  const bool active = cell < N;
  const int64_t i = active ? cell : N - 1;
  // this cell's FP64 record (read before it is overwritten by this same thread)
  double u64[NVP];
#pragma unroll
  for (int c = 0; c < NVP / 2; ++c) {
    const double2 x = reinterpret_cast<const double2 *>(a.U + i * NVP)[c];
    u64[2 * c] = x.x;
    u64[2 * c + 1] = x.y;
  }
  double acc[NV];
  float acc_hi[NV], acc_lo[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    acc[v] = 0.0;
    acc_hi[v] = 0.0f;
    acc_lo[v] = 0.0f;
  }
  // face fluxes computed once per face (face_flux_kernel), signed for this cell, summed in face
  // order exactly as in flux_kernel
  const int4 cf4 = __ldg(reinterpret_cast<const int4 *>(a.cellface) + i);
  const int cfv[4] = {cf4.x, cf4.y, cf4.z, cf4.w};
  constexpr int NFP = (NV + 3) & ~3;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t e = cfv[f] & 0x7FFFFFFF;
    const bool neg = cfv[f] < 0;
    T x[NFP];
    load16<T, NFP>((const T *)a.Ff + e * NFP, x);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T c = neg ? -x[v] : x[v];
      if constexpr (F32) {
        float s, er;
        two_sum(acc_hi[v], c, s, er);
        acc_hi[v] = s;
        acc_lo[v] += er;
      } else {
        acc[v] += c;
      }
    }
  }
  if constexpr (F32) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = f32_to_f64(acc_hi[v]) + f32_to_f64(acc_lo[v]);
  }
  stage_tail<D, T>(a, i, active, u64, acc);
}

}  // namespace
}  // namespace cteno

#include "flux_lanes.cuh"

namespace cteno {
namespace {

// CFL step of cells [first, first + count) (all cells, or the cells of one mesh).
template <int D, typename T>
__global__ void dt_kernel(const KArgs a, int64_t first, int64_t count) {
  constexpr int NVP = Lay<D>::NVP;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = idx < count;
  const int64_t i = first + (active ? idx : count - 1);  // every lane reaches the reduction
  double u[NVP];
#pragma unroll
  for (int v = 0; v < NVP; ++v) u[v] = a.U[i * NVP + v];
  T uu[NVP];  // FP32 path: the hi part of the (hi, lo) split, as in the stage update
#pragma unroll
  for (int v = 0; v < NVP; ++v) {
    if constexpr (sizeof(T) == 4) uu[v] = f64_split(u[v]).x;
    else uu[v] = u[v];
  }
  const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
  warp_min_to(a.dt, a.nmesh + mesh, active ? a.cfl * local_dt<D, T>(a, i, uu) : 1e300);
}

__global__ void time_advance_kernel(double *time, const double *dt, int nmesh) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nmesh) time[m] += dt[m];
}

__global__ void dt_reset_kernel(double *dt, int nmesh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nmesh) dt[nmesh + i] = 1e300;
}

__global__ void dt_reset_one_kernel(double *dt, int nmesh, int mesh) { dt[nmesh + mesh] = 1e300; }

// All meshes at once: the source holds mesh after mesh, each mesh's values as [v][cell] in its
// original numbering; grank maps the concatenated original cell to its device cell.
__device__ __forceinline__ int mesh_of_offsets(const int64_t *off, int nmesh, int64_t c) {
  int lo = 0, hi = nmesh - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Set every mesh's state and compute each mesh's CFL step of it in the same pass (dt[next] must
// have been reset). src may be device memory or page-locked host memory.
template <int D, typename T>
__global__ void permute_in_all_dt_kernel(const KArgs a, const int32_t *grank, const double *src) {
  constexpr int NV = D + 2, NVP = Lay<D>::NVP;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = idx < a.N;
  const int64_t c = active ? idx : a.N - 1;  // every lane reaches the reduction
  const int k = mesh_of_offsets(a.mesh_off, a.nmesh, c);
  const int64_t off = a.mesh_off[k], n = a.mesh_off[k + 1] - off, local = c - off;
  const int64_t g = grank[c];
  double u[NVP];
  T ut[NVP];
#pragma unroll
  for (int v = 0; v < NVP; ++v) {
    u[v] = (v < NV) ? src[NV * off + v * n + local] : 0.0;
    if constexpr (sizeof(T) == 4) ut[v] = f64_split(u[v]).x;
    else ut[v] = u[v];
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < NVP / 2; ++q) {
      reinterpret_cast<double2 *>(a.U + g * NVP)[q] = make_double2(u[2 * q], u[2 * q + 1]);
      if (a.U32) {
        const float2 s0 = f64_split(u[2 * q]), s1 = f64_split(u[2 * q + 1]);
        reinterpret_cast<float4 *>(a.U32 + g * 2 * NVP)[q] = make_float4(s0.x, s0.y, s1.x, s1.y);
      }
    }
  }
  warp_min_to(a.dt, a.nmesh + k, active ? a.cfl * local_dt<D, T>(a, g, ut) : 1e300);
}

__global__ void permute_out_all_kernel(int nv, int nvp, int64_t N, int nmesh, const int64_t *mesh_off,
                                       const int32_t *grank, const double *U, double *dst) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int k = mesh_of_offsets(mesh_off, nmesh, c);
  const int64_t off = mesh_off[k], n = mesh_off[k + 1] - off, local = c - off;
  const int64_t g = grank[c];
  for (int v = 0; v < nv; ++v) dst[nv * off + v * n + local] = U[g * nvp + v];
}

// src[v][c] (caller order, mesh of n cells) -> U[off + rank[c]][v] (+ the FP32 pair)
__global__ void permute_in_kernel(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                                  const double *src, double *U, float *U32) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t g = off + rank[c];
  for (int v = 0; v < nvp; ++v) {
    const double x = (v < nv) ? src[v * n + c] : 0.0;
    U[g * nvp + v] = x;
    if (U32) {  // the same (hi, lo) split as the stage update
      const float2 s = f64_split(x);
      U32[(g * nvp + v) * 2] = s.x;
      U32[(g * nvp + v) * 2 + 1] = s.y;
    }
  }
}

__global__ void permute_out_kernel(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                                   const double *U, double *dst) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t g = off + rank[c];
  for (int v = 0; v < nv; ++v) dst[v * n + c] = U[g * nvp + v];
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

namespace {
// The flux kernels of dimension D with NQ Gauss points per face.
template <int D, int NQ>
void launch_flux_nq(int fp32, const KArgs &a, int block, cudaStream_t s) {
  if (block >= kFaceFlux) {  // face-based: HLLC once per face, then the per-cell gather and update
    const int threads = block - kFaceFlux;
    const unsigned gf = grid_for(a.nfaces, 256), gc = grid_for(a.N, threads);
    if (fp32) {
      launch_stage_kernel(face_flux_kernel<D, float, NQ>, gf, 256, 0, s, a);
      launch_stage_kernel(cell_update_kernel<D, float, 0>, gc, threads, 0, s, a);
    } else {
      launch_stage_kernel(face_flux_kernel<D, double, NQ>, gf, 256, 0, s, a);
      launch_stage_kernel(cell_update_kernel<D, double, 0>, gc, threads, 0, s, a);
    }
    return;
  }
  if (block >= kLaneSchedule) {  // face-per-lane schedule, block - kLaneSchedule threads
    const int threads = block - kLaneSchedule, cpw = 32 / (D + 1);
    const int64_t cells_per_block = (int64_t)(threads / 32) * cpw;
    const unsigned grid = (unsigned)((a.N + cells_per_block - 1) / cells_per_block);
    if (fp32) launch_stage_kernel(flux_lanes_kernel<D, float, NQ>, grid, threads, 0, s, a);
    else launch_stage_kernel(flux_lanes_kernel<D, double, NQ>, grid, threads, 0, s, a);
    return;
  }
  const bool capped = block < 0;  // register-capped variant (FP32 only)
  if (capped) block = -block;
  const unsigned grid = grid_for(a.N, block);
  if (fp32) {
    if (capped) launch_stage_kernel(flux_kernel<D, float, 8, NQ>, grid, block, 0, s, a);
    else launch_stage_kernel(flux_kernel<D, float, 0, NQ>, grid, block, 0, s, a);
  } else {
    launch_stage_kernel(flux_kernel<D, double, 0, NQ>, grid, block, 0, s, a);
  }
}
}  // namespace

void launch_flux(int dim, int nq, int fp32, const KArgs &a, int block, cudaStream_t s) {
  if (dim == 3) launch_flux_nq<3, 4>(fp32, a, block, s);
  else if (nq == 2) launch_flux_nq<2, 2>(fp32, a, block, s);
  else if (nq == 3) launch_flux_nq<2, 3>(fp32, a, block, s);
  else if (nq == 4) launch_flux_nq<2, 4>(fp32, a, block, s);
}

namespace {
void launch_dt_cells(int dim, const KArgs &a, int64_t first, int64_t count, cudaStream_t s) {
  const bool f32 = a.geo32 != nullptr;
  const unsigned g = grid_for(count, 256);
  if (dim == 2 && f32) dt_kernel<2, float><<<g, 256, 0, s>>>(a, first, count);
  if (dim == 2 && !f32) dt_kernel<2, double><<<g, 256, 0, s>>>(a, first, count);
  if (dim == 3 && f32) dt_kernel<3, float><<<g, 256, 0, s>>>(a, first, count);
  if (dim == 3 && !f32) dt_kernel<3, double><<<g, 256, 0, s>>>(a, first, count);
}
}  // namespace

void launch_dt(int dim, const KArgs &a, cudaStream_t s) {
  dt_reset_kernel<<<grid_for(a.nmesh, 64), 64, 0, s>>>(a.dt, a.nmesh);
  launch_dt_cells(dim, a, 0, a.N, s);
}

void launch_dt_mesh(int dim, const KArgs &a, int mesh, int64_t first, int64_t count, cudaStream_t s) {
  dt_reset_one_kernel<<<1, 1, 0, s>>>(a.dt, a.nmesh, mesh);
  launch_dt_cells(dim, a, first, count, s);
}

void launch_set_state_all(int dim, const KArgs &a, const int32_t *grank, const double *src, cudaStream_t s) {
  dt_reset_kernel<<<grid_for(a.nmesh, 64), 64, 0, s>>>(a.dt, a.nmesh);
  const bool f32 = a.geo32 != nullptr;
  const unsigned g = grid_for(a.N, 256);
  if (dim == 2 && f32) permute_in_all_dt_kernel<2, float><<<g, 256, 0, s>>>(a, grank, src);
  if (dim == 2 && !f32) permute_in_all_dt_kernel<2, double><<<g, 256, 0, s>>>(a, grank, src);
  if (dim == 3 && f32) permute_in_all_dt_kernel<3, float><<<g, 256, 0, s>>>(a, grank, src);
  if (dim == 3 && !f32) permute_in_all_dt_kernel<3, double><<<g, 256, 0, s>>>(a, grank, src);
}

void launch_permute_out_all(int nv, int nvp, int64_t N, int nmesh, const int64_t *mesh_off,
                            const int32_t *grank, const double *U, double *dst, cudaStream_t s) {
  permute_out_all_kernel<<<grid_for(N, 256), 256, 0, s>>>(nv, nvp, N, nmesh, mesh_off, grank, U, dst);
}

void launch_time_advance(double *time, const double *dt, int nmesh, cudaStream_t s) {
  time_advance_kernel<<<grid_for(nmesh, 64), 64, 0, s>>>(time, dt, nmesh);
}

void launch_dt_reset(const KArgs &a, cudaStream_t s) {
  dt_reset_kernel<<<grid_for(a.nmesh, 64), 64, 0, s>>>(a.dt, a.nmesh);
}

void launch_permute_in(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                       const double *src, double *U, float *U32, cudaStream_t s) {
  permute_in_kernel<<<grid_for(n, 256), 256, 0, s>>>(nv, nvp, n, off, rank, src, U, U32);
}

void launch_permute_out(int nv, int nvp, int64_t n, int64_t off, const int32_t *rank,
                        const double *U, double *dst, cudaStream_t s) {
  permute_out_kernel<<<grid_for(n, 256), 256, 0, s>>>(nv, nvp, n, off, rank, U, dst);
}

cudaError_t preload_permute_out() {
  cudaFuncAttributes attr;
  return cudaFuncGetAttributes(&attr, permute_out_kernel);
}

}  // namespace cteno
