// recon_pair.cuh -- the streamed schedule with two lanes per cell (mixed path).
//
// As the streamed lane schedule (recon_stream_kernel: every warp streams its own tiles' operator
// records through a ring of shared-memory stages on per-warp mbarriers), but a cell is split over
// two lanes instead of d + 2: lane h of the pair holds the conserved variables h * NVL .. NVL - 1 +
// h * NVL (NVL = 3 in 3D, 2 in 2D), so a warp works on 16 cells and every operator value read from
// shared memory feeds NVL multiply-adds instead of one. The broadcast of each operator value to all
// d + 2 lanes of a cell is what bounds the one-variable-per-lane schedule (its shared-memory pipe is
// the busiest unit); here two lanes share it. The arithmetic per variable is the same as in the
// other schedules (eqs. 10-23, Alg. 1 / 2), in the same order.
#pragma once

#include "recon.cuh"

namespace cteno {

template <int D, int R, int STAGES>
struct PairShape {
  using S = Shape<D, R>;
  using L = Lay<D>;
  static constexpr int NVL = (L::NV + 1) / 2;               // variables per lane
  static constexpr int CPW = 16;                              // cells per warp
  static constexpr int MC = 4;                                // members per chunk
  static constexpr int NCH = S::M / MC;                       // chunks per tile
  static constexpr int NST = STAGES;
  static constexpr int CHUNK_CELL = MC * S::NK * 4;           // bytes of one cell's chunk
  static constexpr int STAGE = CPW * CHUNK_CELL;
  static constexpr int HPD = CPW * L::NF * L::PDS * 4;        // header: directional operators,
  static constexpr int HST = CPW * S::M * 4;                  //   stencil ids
  static constexpr int HDR = HPD + HST;
  static constexpr int WARP_BYTES = 2 * HDR + NST * STAGE;
  static constexpr int NPHI = (D == 3) ? L::NF * S::NP * L::NQ * S::NK : 1;
  static constexpr int PHI_BYTES = (NPHI * 4 + 15) / 16 * 16;
  static_assert(S::M % MC == 0 && CHUNK_CELL % 16 == 0 && HPD % 16 == 0 && HST % 16 == 0,
                "bulk copies need 16-byte spans");
};

template <int D, int R, int SCHEME, int STAGES>
__global__ void __launch_bounds__(256, 1) recon_pair_kernel(const KArgs a) {
  using T = float;
  using S = Shape<D, R>;
  using L = Lay<D>;
  using Q = PairShape<D, R, STAGES>;
  constexpr int NV = L::NV, NVP = L::NVP, NF = L::NF, ND = L::ND, PDS = L::PDS;
  constexpr int NK = S::NK, M = S::M, NP = S::NP, NQ = L::NQ;
  constexpr int NVL = Q::NVL, CPW = Q::CPW, MC = Q::MC, NCH = Q::NCH, NST = Q::NST;
  constexpr T INV_FACT = (D == 2) ? (T)0.5 : (T)(1.0 / 6.0);
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
  // lane 0 only: the header of tile iteration it; chunk q (tile iteration q / NCH, chunk q % NCH)
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
  if constexpr (D == 3) {
    const DevTables &tb = *a.tab;
    for (int t = threadIdx.x; t < Q::NPHI; t += blockDim.x) {
      const int k = t % NK, q = (t / NK) % NQ, p = (t / (NK * NQ)) % NP, f = t / (NK * NQ * NP);
      sPhi[t] = (T)tb.Phi[f][p][q][k];
    }
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

  const int grp = lane >> 1, h = lane & 1, v0 = h * NVL;  // cell slot, half, first variable
  const float2 *__restrict__ U32 = reinterpret_cast<const float2 *>(a.U32);
  int64_t q = 0, qi = NST;  // next chunk to consume / to issue
  for (int64_t it = 0; tile_of(it) < tiles; ++it) {
    const int64_t c0 = tile_of(it) * CPW;
    const int nvalid = (int)min((int64_t)CPW, N - c0);
    const bool active = grp < nvalid;
    const int g = active ? grp : nvalid - 1;  // lanes past the last cell shadow a valid cell
    const int64_t i = c0 + g;
    // this lane's variables (the second lane's last slot in 3D is the record's zero padding)
    T U0[NVL];
    float L0[NVL];
#pragma unroll
    for (int j = 0; j < NVL; ++j) {
      const float2 own = __ldg(U32 + i * NVP + v0 + j);
      U0[j] = own.x;
      L0[j] = own.y;
    }
    const uint32_t info = __ldg(a.cinfo + i);
    if (!wait_all(&hbar[it & 1], (uint32_t)((it >> 1) & 1))) {
      give_up(it, q, qi);
      return;
    }
    const T *__restrict__ Pd_s = reinterpret_cast<const T *>(hdr(it)) + g * (NF * PDS);
    const int32_t *__restrict__ st_s = reinterpret_cast<const int32_t *>(hdr(it) + Q::HPD) + g * M;

    // central coefficients of this lane's variables, chunk after chunk; the member states of
    // chunk c + 1 are loaded while chunk c is multiplied
    T ao[NVL][NK];
#pragma unroll
    for (int j = 0; j < NVL; ++j)
#pragma unroll
      for (int k = 0; k < NK; ++k) ao[j][k] = (T)0;
    float2 nx[MC][NVL];
    auto fetch = [&](int c) {
      const int4 j4 = *reinterpret_cast<const int4 *>(st_s + c * MC);
      const int ids[4] = {j4.x, j4.y, j4.z, j4.w};
#pragma unroll
      for (int mm = 0; mm < MC; ++mm)
#pragma unroll
        for (int j = 0; j < NVL; ++j) nx[mm][j] = __ldg(U32 + (int64_t)ids[mm] * NVP + v0 + j);
    };
    fetch(0);
#pragma unroll 1
    for (int c = 0; c < NCH; ++c, ++q) {
      T du[MC][NVL];
#pragma unroll
      for (int mm = 0; mm < MC; ++mm)
#pragma unroll
        for (int j = 0; j < NVL; ++j) du[mm][j] = (nx[mm][j].x - U0[j]) + (nx[mm][j].y - L0[j]);
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
#pragma unroll
        for (int j = 0; j < NVL; ++j) ao[j][e % NK] += pb[e % 4] * du[e / NK][j];
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
    T ad[NVL][NF][D];
#pragma unroll
    for (int j = 0; j < NVL; ++j)
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < D; ++k) ad[j][f][k] = (T)0;
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
              const int64_t jid = st_s[off + jj];
#pragma unroll
              for (int j = 0; j < NVL; ++j) {
                const float2 hm = __ldg(U32 + jid * NVP + v0 + j);
                const T du = (hm.x - U0[j]) + (hm.y - L0[j]);
#pragma unroll
                for (int k = 0; k < D; ++k) ad[j][f][k] += pf[jj * D + k] * du;
              }
            }
          }
        }
        off += nm;
      }
    }

    // selection per variable (eqs. 15-23), as lane_finish
    auto oc = [](int idx) { return cO<T, R>(idx); };
    auto sid = [&](const T (&adf)[D]) {  // the linear block of O is |V0'| I
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < D; ++k) s += adf[k] * adf[k];
      return s * INV_FACT;
    };
#pragma unroll
    for (int j = 0; j < NVL; ++j) {
      const uint32_t bits = lane_select<NF, NK, D, T, SCHEME>(a, adm, ao[j], ad[j], oc, sid);
      if (a.flags && active && v0 + j < NV) a.flags[(v0 + j) * N + i] = (uint8_t)bits;
    }

    // face values of this lane's variables; the pair exchanges them for the positivity guard
    T *__restrict__ Ufi = (T *)a.Uf + i * (int64_t)(NF * NQ * NV);
    const uint32_t perm = info >> kInfoPermShift;
    bool bad = false;
    T fv[NF][NQ][NVL];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int p = (perm >> (3 * f)) & 7u;
#pragma unroll
      for (int qq = 0; qq < NQ; ++qq) {
        T val[NVL];
#pragma unroll
        for (int j = 0; j < NVL; ++j) val[j] = (T)L0[j];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
          T ph;
          if constexpr (D == 2) ph = cPhi2<T, R>((f * 2 + qq) * NK + k);
          else ph = sPhi[((f * NP + p) * NQ + qq) * NK + k];
#pragma unroll
          for (int j = 0; j < NVL; ++j) val[j] += ph * ao[j][k];
        }
        T u[2 * NVL];
#pragma unroll
        for (int j = 0; j < NVL; ++j) {
          val[j] += U0[j];
          fv[f][qq][j] = val[j];
          const T other = __shfl_xor_sync(0xffffffffu, val[j], 1);
          u[j] = h ? other : val[j];
          u[NVL + j] = h ? val[j] : other;
        }
        T ke = (T)0;
#pragma unroll
        for (int jd = 0; jd < D; ++jd) ke += u[1 + jd] * u[1 + jd];
        // rho > 0 and p > 0, the latter as rho E - |m|^2 / 2 > 0 (no division)
        bad = bad || !(u[0] > 0.0f) || !(u[0] * u[NV - 1] - 0.5f * ke > 0.0f);
      }
    }
    if (a.guard_on && bad) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int j = 0; j < NVL; ++j) fv[f][qq][j] = U0[j] + (T)L0[j];
      if (active && h == 0) atomicAdd(a.guard, 1ull);
    }
    if (active) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int p = (perm >> (3 * f)) & 7u;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
          // 2D: an edge is stored in sorted-vertex order, the swapped orientation reverses its points
          const int qs = (D == 2 && p) ? (NQ - 1 - qq) : qq;
#pragma unroll
          for (int j = 0; j < NVL; ++j)
            if (v0 + j < NV) Ufi[(f * NQ + qs) * NV + v0 + j] = fv[f][qq][j];
        }
      }
    }
    __syncwarp();  // every lane is done with this header
    if (lane == 0) {
      fence_proxy_async_shared();
      issue_hdr(it + 2);
    }
  }
}

// Host side: a persistent grid of (co-resident blocks per SM) x SMs blocks of `warps` warps.
template <int D, int R, int SCHEME, int STAGES>
void launch_recon_pair(const KArgs &a, int warps, cudaStream_t s) {
  using Q = PairShape<D, R, STAGES>;
  const int threads = 32 * warps;
  const size_t smem = (size_t)recon_pair_smem(D, R, warps, STAGES);
  auto kern = recon_pair_kernel<D, R, SCHEME, STAGES>;
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
  const int64_t tiles = (a.N + Q::CPW - 1) / Q::CPW;
  const int64_t blocks = (tiles + warps - 1) / warps;
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)nb * sms);
  launch_stage_kernel(kern, grid, threads, smem, s, a);
}

}  // namespace cteno
