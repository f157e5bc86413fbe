// flux_lanes.cuh -- face-per-lane schedule of the flux / update kernel (included by flux.cu after
// the HLLC, local time-step and mesh-lookup helpers).
//
// A group of NF = d+1 consecutive lanes updates one cell, lane f computing the HLLC flux through
// face f at its Gauss points. The face fluxes are exchanged by shuffles and summed in FP64 in face
// order (bitwise the same sums as the thread-per-cell kernel, so the update stays exactly
// conservative); the RK update of variable v is done by lane v mod NF.
#pragma once

namespace cteno {
namespace {

template <int D, typename T, int NQ>
__global__ void __launch_bounds__(256) flux_lanes_kernel(const KArgs a) {
  using L = Lay<D>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, FB = NQ * NV;
  constexpr int CPW = 32 / NF;
  constexpr bool F32 = sizeof(T) == 4;
  pdl_wait(a);
  const int lane = threadIdx.x & 31;
  const int grp = lane / NF;
  const int f = lane - grp * NF;  // this lane's face (spare lanes: a face index < NF as well)
  const int base = grp * NF;
  const int64_t N = a.N;
  const int64_t cell = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CPW + grp;
  const bool active = grp < CPW && cell < N;
  const int64_t i = active ? cell : N - 1;  // spare lanes shadow a valid cell, store nothing
  const T *__restrict__ Uf = (const T *)a.Uf;
  const T *__restrict__ G = F32 ? (const T *)a.geo32 : (const T *)a.geo;
  T g;
  if constexpr (F32) g = a.gamma32; else g = a.gamma;
  const uint32_t meta = __ldg(a.fmeta + i);
  const int64_t j = __ldg(a.nbr + i * 4 + f);
  const int fj = (meta >> (2 * f)) & 3u;
  const bool own = (meta >> (kMetaOwnerShift + f)) & 1u;
  T gf[4], uI[FB], uO[FB];
  load16<T, 4>(G + (i * NF + f) * 4, gf);
  load16<T, FB>(Uf + (i * NF + f) * FB, uI);
  if (j >= 0) {
    load16<T, FB>(Uf + (j * NF + fj) * FB, uO);
  } else {  // boundary face: its kind's outside state
    double um[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) um[v] = a.U[i * NVP + v];
    boundary_state<D, T, NQ>(a, i, (meta >> (kMetaKindShift + 2 * f)) & 3u, gf, uI, um, uO);
  }
  T n[D];
#pragma unroll
  for (int k = 0; k < D; ++k) n[k] = own ? gf[k] : -gf[k];
  T Ff[NV];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T F[NV];
    if (own) hllc<D, T>(uI + q * NV, uO + q * NV, n, g, F);
    else hllc<D, T>(uO + q * NV, uI + q * NV, n, g, F);
    T w;
    if constexpr (F32) w = a.fw32[q]; else w = a.fw[q];
#pragma unroll
    for (int v = 0; v < NV; ++v) Ff[v] = (q == 0) ? w * F[v] : Ff[v] + w * F[v];
  }
  T contrib[NV];  // this face's |A| F, signed for this cell
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T x = gf[3] * Ff[v];
    contrib[v] = own ? x : -x;
  }
  // residual of the variables this lane updates: FP64 sum over the faces in face order
  const int mesh = (a.nmesh > 1) ? mesh_of(a, i) : 0;
  const double dtv = a.dt[mesh] * a.vol[i];  // dt / |V_i|
  double res[NVP];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NVP; ++v) res[v] = 0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double acc = 0.0;
    float hi = 0.0f, lo = 0.0f;
    if constexpr (F32) {  // exact FP32 accumulation over the faces, as in the per-cell kernel
#pragma unroll
      for (int ff = 0; ff < NF; ++ff) {
        float s, e;
        two_sum(hi, __shfl_sync(0xffffffffu, contrib[v], base + ff), s, e);
        hi = s;
        lo += e;
      }
    } else {
#pragma unroll
      for (int ff = 0; ff < NF; ++ff) acc += (double)__shfl_sync(0xffffffffu, contrib[v], base + ff);
    }
    if (v % NF == f) {  // FP64 work only in the lane that updates variable v
      if constexpr (F32) acc = f32_to_f64(hi) + f32_to_f64(lo);
      const double u = a.U[i * NVP + v];
      double r, s4 = 0.0;
      if (!a.rk4) {  // SSP-RK3 (Shu-Osher), as stage_tail
        const double upd = u - dtv * acc;
        if (a.stage == 0) r = upd;
        else if (a.stage == 1) r = 0.75 * a.Un[i * NVP + v] + 0.25 * upd;
        else r = (1.0 / 3.0) * a.Un[i * NVP + v] + (2.0 / 3.0) * upd;
      } else {       // classical RK4 with its running sum, as stage_tail
        const double F = -dtv * acc;
        if (a.stage == 0) {
          s4 = u + F / 6.0;
          r = u + 0.5 * F;
        } else if (a.stage == 1) {
          s4 = a.Acc[i * NVP + v] + F / 3.0;
          r = a.Un[i * NVP + v] + 0.5 * F;
        } else if (a.stage == 2) {
          s4 = a.Acc[i * NVP + v] + F / 3.0;
          r = a.Un[i * NVP + v] + F;
        } else {
          r = a.Acc[i * NVP + v] + F / 6.0;
        }
      }
      res[v] = r;
      finite = finite && finite64(r);
      if (active) {
        if (a.stage == 0) a.Un[i * NVP + v] = u;
        if (a.rk4 && a.stage < 3) a.Acc[i * NVP + v] = s4;
        a.U[i * NVP + v] = r;
        if (a.U32) reinterpret_cast<float2 *>(a.U32)[i * NVP + v] = f64_split(r);
      }
    }
  }
  if (!finite && active) atomicOr(a.err, kErrNonFinite);
  if (a.stage == a.last_stage) {  // CFL step of the next step: lane 0 of the group collects the new state
    double full[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) full[v] = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) full[v] = __shfl_sync(0xffffffffu, res[v], base + (v % NF));
    bool fin = active && f == 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) fin = fin && finite64(full[v]);
    T ft[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) {
      if constexpr (F32) ft[v] = f64_split(full[v]).x;
      else ft[v] = full[v];
    }
    warp_min_to(a.dt, a.nmesh + mesh, fin ? a.cfl * local_dt<D, T>(a, i, ft) : 1e300);
  }
}

}  // namespace
}  // namespace cteno
