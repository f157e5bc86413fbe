// api.cpp -- the C ABI of include/cteno.h: context, device memory, set-up and the time loop.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "device.h"
#include "internal.h"

using namespace cteno;

struct cteno_ctx {
  cteno_params p{};
  cudaStream_t stream = nullptr;     // borrowed
  cudaStream_t capture = nullptr;    // owned, for graph capture
  int d = 0, nv = 0, nf = 0, nq = 0, nk = 0, M = 0, nd = 0;
  int nsel = 0;  // selections per cell: nv, or nf * nv (characteristic reconstruction)
  bool fp32 = false;
  std::vector<Mesh> meshes;
  bool stencils = false, built = false;
  int64_t N = 0;
  std::string err;
  Tables tab{};
  std::vector<uint32_t> h_cinfo;     // device-order cinfo after set-up (admissibility)
  // device memory
  DevTables *d_tab = nullptr;
  int64_t *d_mesh_off = nullptr;
  double *U = nullptr, *Un = nullptr;
  double *Acc = nullptr;             // RK4 running sum
  double bA[6] = {}, bB[6] = {};     // boundary states A and B (conserved)
  double shock[3] = {};              // moving shock: xs0, sy, vs
  double *time = nullptr;            // [nmesh] physical time (allocated when a moving shock exists)
  float *U32 = nullptr;
  int32_t *st = nullptr, *nbr = nullptr;
  int32_t *hl = nullptr;             // gather staging: per-tile distinct member lists (mixed path)
  uint16_t *lidx = nullptr;          //   and per-cell local indices into them
  int hrec = 0, hms = 0;
  uint32_t *cinfo = nullptr, *fmeta = nullptr;
  void *Pc = nullptr, *Pd = nullptr, *Uf = nullptr;
  uint8_t *flags = nullptr;
  double *geo = nullptr, *vol = nullptr, *dt = nullptr;
  float *geo32 = nullptr;
  int *derr = nullptr;
  unsigned long long *guard = nullptr;
  std::vector<int32_t *> d_rank;
  int32_t *d_grank = nullptr;        // device cell of each concatenated original cell (all meshes)
  int32_t *d_face = nullptr, *d_cellface = nullptr;  // face-based flux schedule
  void *Ff = nullptr;
  int64_t nfaces = 0;
  double *stage_buf = nullptr;       // staging for host <-> device state copies
  size_t stage_cap = 0;
  double *backup = nullptr;          // autotune state backup
  int recon_block = 128, flux_block = 128;
  bool record_flags = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<void *> allocations;
  int64_t member_sum = 0;            // admissible directional members over all cells
  int64_t adm_faces = 0;             // admissible directional stencils over all cells
  bool timing = false;
  int pdl = 1;                       // programmatic dependent launch of the stage kernels
  int zerocopy = 1;                  // batch-wide calls access page-locked host buffers directly
  unsigned long long test_wait_ns = 0;  // test hook of the bounded waits (0 = off)
  double *noalloc_stage = nullptr;   // device address of the allocation-free staging array
  int64_t noalloc_cap = 0;           //   and its capacity in doubles (looked up by lsq_build)
  cudaEvent_t tev[9] = {};           // event record nodes of the step graph (2 per stage + 1)
  int nst = 3;                       // Runge-Kutta stages per step (3, or 4 for RK4)
};

namespace {

int fail(cteno_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, CTENO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
cudaError_t dalloc(cteno_ctx *ctx, P **ptr, size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    ctx->allocations.push_back(p);
    *ptr = (P *)p;
  }
  return e;
}

// Kernel instantiation of the scheme: the CTENOZ measure (1) or the CTENO measure (0), which
// CWENO (weights on the same indicators) and TENO (cut-off without linear coefficients) share.
int kscheme(const cteno_ctx *ctx) { return ctx->p.scheme == CTENO_SCHEME_CTENOZ ? 1 : 0; }

KArgs make_args(cteno_ctx *ctx, int stage, int dt_swap) {
  KArgs a{};
  a.N = ctx->N;
  a.nmesh = (int)ctx->meshes.size();
  a.mesh_off = ctx->d_mesh_off;
  a.U = ctx->U;
  a.Un = ctx->Un;
  a.U32 = ctx->U32;
  a.pdl = ctx->pdl;
  a.test_wait_ns = ctx->test_wait_ns;
  a.face = ctx->d_face;
  a.cellface = ctx->d_cellface;
  a.Ff = ctx->Ff;
  a.nfaces = ctx->nfaces;
  a.st = ctx->st;
  a.hl = ctx->hl;
  a.lidx = ctx->lidx;
  a.htile = halo_tile(ctx->d);
  a.hrec = ctx->hrec;
  a.hms = ctx->hms;
  a.cinfo = ctx->cinfo;
  a.Pc = ctx->Pc;
  a.Pd = ctx->Pd;
  a.Uf = ctx->Uf;
  a.flags = ctx->record_flags ? ctx->flags : nullptr;
  a.nbr = ctx->nbr;
  a.fmeta = ctx->fmeta;
  a.geo = ctx->geo;
  a.geo32 = ctx->geo32;
  a.vol = ctx->vol;
  a.dt = ctx->dt;
  a.tab = ctx->d_tab;
  a.err = ctx->derr;
  a.guard = ctx->guard;
  a.C_T = ctx->p.C_T;
  a.lambda1p = ctx->p.lambda1p;
  a.eps = ctx->p.eps;
  a.gamma = ctx->p.gamma;
  a.cfl = ctx->p.cfl;
  a.lam_gamma = ctx->p.scheme == CTENO_SCHEME_TENO ? 0 : ctx->p.lam_gamma;  // TENO has no linear coefficients
  a.ctenoz_form = ctx->p.ctenoz_form;
  a.characteristic = ctx->p.characteristic;
  a.Acc = ctx->Acc;
  for (int v = 0; v < 6; ++v) {
    a.bA[v] = ctx->bA[v];
    a.bB[v] = ctx->bB[v];
    a.bA32[v] = (float)ctx->bA[v];
    a.bB32[v] = (float)ctx->bB[v];
  }
  a.shock_vs = ctx->shock[2];
  a.time = ctx->time;
  {  // stage time offsets: SSP-RK3 (0, 1, 1/2), RK4 (0, 1/2, 1/2, 1)
    static const double c3[3] = {0.0, 1.0, 0.5}, c4[4] = {0.0, 0.5, 0.5, 1.0};
    a.stage_c = (ctx->nst == 4) ? c4[stage] : c3[stage];
  }
  a.rk4 = ctx->nst == 4;
  a.last_stage = ctx->nst - 1;
  a.cweno = ctx->p.scheme == CTENO_SCHEME_CWENO;
  a.central_split = ctx->p.scheme != CTENO_SCHEME_TENO;
  a.guard_on = ctx->p.positivity_guard;
  a.lam1 = 1.0 - 1.0 / ctx->p.lambda1p;
  a.inv_lam1 = 1.0 / a.lam1;
  a.one_m_lam1 = 1.0 - a.lam1;
  a.log2_lam1 = (float)std::log2(a.lam1);
  a.log2_one_m_lam1 = (float)std::log2(a.one_m_lam1);
  for (int k = 0; k <= kMaxNF; ++k) {  // k = st - 1 admissible directional stencils
    a.lams_d[k] = k ? a.one_m_lam1 / k : 0.0;
    a.lams_f[k] = (float)a.lams_d[k];
    a.log2_lams_f[k] = k ? (float)std::log2(a.lams_d[k]) : 0.0f;
    a.inv_stm1_f[k] = k ? (float)(1.0 / k) : 0.0f;
  }
  for (int q = 0; q < kMaxNQ; ++q) {
    a.fw[q] = ctx->tab.fw[q];
    a.fw32[q] = (float)ctx->tab.fw[q];
  }
  a.gamma32 = (float)ctx->p.gamma;
  a.gm1_32 = (float)(ctx->p.gamma - 1.0);
  a.eps32 = std::max((float)ctx->p.eps, FLT_MIN);  // FP32 eps: at least the smallest normal number
  a.C_T32 = (float)ctx->p.C_T;
  a.inv_lam1_32 = (float)a.inv_lam1;
  a.one_m_lam1_32 = (float)a.one_m_lam1;
  a.cfl32 = (float)ctx->p.cfl;
  a.stage = stage;
  a.dt_swap = dt_swap;
  return a;
}

cudaError_t enqueue_stage(cteno_ctx *ctx, int stage, int dt_swap, cudaStream_t s) {
  const KArgs a = make_args(ctx, stage, dt_swap);
  const cudaError_t e = launch_recon(ctx->d, ctx->p.degree, ctx->fp32 ? 1 : 0, kscheme(ctx), a, ctx->recon_block, s);
  if (e != cudaSuccess) return e;
  launch_flux(ctx->d, ctx->nq, ctx->fp32 ? 1 : 0, a, ctx->flux_block, s);
  return cudaSuccess;
}

int check_built(cteno_ctx *ctx) {
  if (!ctx) return CTENO_ERR_ARG;
  if (!ctx->built) return fail(ctx, CTENO_ERR_STATE, "cteno_lsq_build has not run");
  return CTENO_OK;
}

int check_mesh(cteno_ctx *ctx, int32_t mesh_id) {
  if (mesh_id < 0 || mesh_id >= (int32_t)ctx->meshes.size())
    return fail(ctx, CTENO_ERR_ARG, "mesh_id out of range");
  return CTENO_OK;
}

int ensure_stage_buf(cteno_ctx *ctx, size_t count) {
  if (count <= ctx->stage_cap) return CTENO_OK;
  if (ctx->stage_buf) cudaFree(ctx->stage_buf);
  ctx->stage_buf = nullptr;
  ctx->stage_cap = 0;
  CK(cudaMalloc(&ctx->stage_buf, count * sizeof(double)));
  ctx->stage_cap = count;
  return CTENO_OK;
}

int device_status(cteno_ctx *ctx) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (e & kErrNonFinite) return fail(ctx, CTENO_ERR_DEVICE, "a cell state became non-finite");
  if (e & kErrRank) return fail(ctx, CTENO_ERR_RANK, "a central least-squares matrix is rank deficient");
  if (e & kErrTimeout) return fail(ctx, CTENO_ERR_DEVICE, "a bounded wait for a bulk copy timed out");
  return CTENO_OK;
}

void drop_graph(cteno_ctx *ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph_exec = nullptr;
  ctx->graph = nullptr;
}

}  // namespace

namespace cteno {

// Host read-back of one mesh's state through the staging array compiled into the library, whose
// device address cteno_lsq_build looked up (used by cteno_get_state_noalloc; allocates nothing).
int get_state_noalloc(cteno_ctx *ctx, int32_t mesh_id, double *U_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  double *const stage = ctx->noalloc_stage;
  const int64_t capacity = ctx->noalloc_cap;
  if ((rc = check_mesh(ctx, mesh_id))) return rc;
  if (!U_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  const Mesh &m = ctx->meshes[mesh_id];
  const int64_t cnt = (int64_t)ctx->nv * m.ncells;
  if (cnt > capacity)
    return fail(ctx, CTENO_ERR_ARG, "mesh state has " + std::to_string(cnt) +
                                        " values; the allocation-free staging area holds " +
                                        std::to_string(capacity));
  launch_permute_out(ctx->nv, lay_nvp(ctx->d), m.ncells, m.offset, ctx->d_rank[mesh_id], ctx->U, stage,
                     ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(U_out, stage, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return device_status(ctx);
}

}  // namespace cteno

extern "C" {

void cteno_default_params(cteno_params *p) {
  if (!p) return;
  p->dim = 2;
  p->degree = 2;
  p->scheme = CTENO_SCHEME_CTENO;
  p->precision = CTENO_FP64;
  p->lam_gamma = 1;
  p->positivity_guard = 1;
  p->ctenoz_form = 0;
  p->characteristic = 0;
  p->rk = 3;
  p->C_T = 1e-6;
  p->lambda1p = 1e15;
  p->eps = 1e-24;
  p->cfl = 0.5;
  p->gamma = 1.4;
}

int cteno_create(cteno_ctx **out, const cteno_params *p, void *cuda_stream) {
  if (!out || !p) return CTENO_ERR_ARG;
  *out = nullptr;
  if ((p->dim != 2 && p->dim != 3) || p->degree < 2 || p->degree > (p->dim == 2 ? 6 : 3) ||
      p->scheme < 0 || p->scheme > 3 || (p->precision != 0 && p->precision != 1) ||
      (p->ctenoz_form != 0 && p->ctenoz_form != 1) || (p->lam_gamma != 0 && p->lam_gamma != 1) ||
      (p->characteristic != 0 && p->characteristic != 1) || (p->rk != 3 && p->rk != 4) ||
      !(p->lambda1p > 1.0) || !(p->C_T >= 0.0 && p->C_T < 1.0) || !(p->eps >= 0.0) ||
      !(p->cfl > 0.0) || !(p->gamma > 1.0))
    return CTENO_ERR_ARG;
  cteno_ctx *ctx = new (std::nothrow) cteno_ctx();
  if (!ctx) return CTENO_ERR_NOMEM;
  ctx->p = *p;
  if (const char *e = std::getenv("CTENO_PDL")) ctx->pdl = std::atoi(e) != 0;
  if (const char *e = std::getenv("CTENO_ZEROCOPY")) ctx->zerocopy = std::atoi(e) != 0;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->d = p->dim;
  ctx->nv = p->dim + 2;
  ctx->nf = p->dim + 1;
  ctx->nq = face_points(p->dim, p->degree);
  ctx->nk = coeff_count(p->degree, p->dim) - 1;
  ctx->M = 2 * coeff_count(p->degree, p->dim);
  ctx->nd = dir_members(p->dim, p->degree);
  // the variable-per-lane schedule for degrees 4 to 6 and for the characteristic reconstruction
  if (p->degree >= 4 || p->characteristic) ctx->recon_block = kLaneSchedule + 128;
  ctx->nsel = p->characteristic ? ctx->nf * ctx->nv : ctx->nv;
  ctx->nst = p->rk;
  ctx->fp32 = (p->precision == CTENO_MIXED);
  build_tables(p->dim, p->degree, &ctx->tab);
  *out = ctx;
  return CTENO_OK;
}

int cteno_mesh_build(cteno_ctx *ctx, int64_t nverts, const double *xyz, int64_t ncells,
                     const int32_t *cell_verts, const double *period, int boundary_kind,
                     int32_t *mesh_id_out) {
  if (!ctx) return CTENO_ERR_ARG;
  if (ctx->stencils) return fail(ctx, CTENO_ERR_STATE, "meshes must be added before cteno_stencil_build");
  if (!xyz || !cell_verts || nverts <= 0 || ncells <= 0 || ncells > INT32_MAX / 2 ||
      (boundary_kind != CTENO_BOUNDARY_TRANSMISSIVE && boundary_kind != CTENO_BOUNDARY_WALL &&
       boundary_kind != CTENO_BOUNDARY_STATE_A))
    return fail(ctx, CTENO_ERR_ARG, "invalid mesh arguments");
  Mesh m;
  int rc = ingest_mesh(ctx->d, nverts, xyz, ncells, cell_verts, period, &m, &ctx->err);
  if (rc) return rc;
  if (!ctx->meshes.empty())
    for (int j = 0; j < 3; ++j)
      if (ctx->meshes[0].period[j] != m.period[j])
        return fail(ctx, CTENO_ERR_ARG, "all meshes of one context must have the same period");
  m.bkind.assign((size_t)m.ncells * (ctx->d + 1), (int8_t)boundary_kind);
  ctx->meshes.push_back(std::move(m));
  if (mesh_id_out) *mesh_id_out = (int32_t)ctx->meshes.size() - 1;
  return CTENO_OK;
}

int cteno_stencil_build(cteno_ctx *ctx) {
  if (!ctx) return CTENO_ERR_ARG;
  if (ctx->meshes.empty()) return fail(ctx, CTENO_ERR_STATE, "no mesh");
  if (ctx->stencils) return CTENO_OK;
  int64_t off = 0;
  for (auto &m : ctx->meshes) {
    int rc = build_stencils(&m, ctx->p.degree, &ctx->err);
    if (rc) return rc;
    morton_order(&m);
    m.offset = off;
    off += m.ncells;
  }
  if (off > INT32_MAX) return fail(ctx, CTENO_ERR_ARG, "more than 2^31 cells in one context");
  ctx->N = off;
  ctx->stencils = true;
  return CTENO_OK;
}

namespace {
// Gather staging lists for tiles of halo_tile(d) consecutive device cells: the distinct stencil
// members of the tile's cells and the cells themselves, ascending, in a record of hrec int32 words
// [count, 0, 0, 0, ids..., 0 padding]; per cell halo_ms(M) uint16 local indices (its stencil in
// device order, then itself). Tiles may span mesh boundaries (ids are device ids).
int build_gather_tiles(cteno_ctx *ctx, const std::vector<int32_t> &hst) {
  const int64_t N = ctx->N;
  const int M = ctx->M, C = halo_tile(ctx->d), MS = halo_ms(M);
  const int64_t ntiles = (N + C - 1) / C;
  std::vector<std::vector<int32_t>> lists(ntiles);
  std::vector<uint16_t> li((size_t)ntiles * C * MS, 0);
  int hmax = 0;
#pragma omp parallel for reduction(max : hmax) schedule(static)
  for (int64_t t = 0; t < ntiles; ++t) {
    const int64_t c0 = t * C, c1 = std::min<int64_t>(N, c0 + C);
    std::vector<int32_t> &L = lists[t];
    for (int64_t g = c0; g < c1; ++g) {
      for (int p = 0; p < M; ++p) L.push_back(hst[(size_t)g * M + p]);
      L.push_back((int32_t)g);
    }
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    auto local = [&](int32_t id) { return (uint16_t)(std::lower_bound(L.begin(), L.end(), id) - L.begin()); };
    for (int64_t g = c0; g < c1; ++g) {
      uint16_t *row = &li[(size_t)g * MS];
      for (int p = 0; p < M; ++p) row[p] = local(hst[(size_t)g * M + p]);
      row[M] = local((int32_t)g);
    }
    hmax = std::max(hmax, (int)L.size());
  }
  if (hmax > 65535) return CTENO_OK;  // not representable: the schedule stays unavailable
  const int hrec = 4 + (hmax + 3) / 4 * 4;
  std::vector<int32_t> hh((size_t)ntiles * hrec, 0);
  for (int64_t t = 0; t < ntiles; ++t) {
    int32_t *rec = &hh[(size_t)t * hrec];
    rec[0] = (int32_t)lists[t].size();
    std::copy(lists[t].begin(), lists[t].end(), rec + 4);
  }
  CK(dalloc(ctx, &ctx->hl, hh.size() * sizeof(int32_t)));
  CK(dalloc(ctx, &ctx->lidx, li.size() * sizeof(uint16_t)));
  CK(cudaMemcpyAsync(ctx->hl, hh.data(), hh.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->lidx, li.data(), li.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));  // the host arrays go out of scope
  ctx->hrec = hrec;
  ctx->hms = MS;
  return CTENO_OK;
}
}  // namespace

int cteno_lsq_build(cteno_ctx *ctx) {
  if (!ctx) return CTENO_ERR_ARG;
  if (!ctx->stencils) return fail(ctx, CTENO_ERR_STATE, "cteno_stencil_build has not run");
  if (ctx->built) return CTENO_OK;
  const int d = ctx->d, nvc = d + 1, nf = ctx->nf, M = ctx->M, nd = ctx->nd;
  const int64_t N = ctx->N;
  const int nmesh = (int)ctx->meshes.size();
  const Tables &tab = ctx->tab;
  // host arrays in device order
  std::vector<double> hX((size_t)N * nvc * d);
  std::vector<int32_t> hst((size_t)M * N), hnbr((size_t)4 * N, -1);
  std::vector<uint32_t> hinfo(N), hmeta(N);
  std::vector<int64_t> hoff(nmesh + 1);
  for (int k = 0; k < nmesh; ++k) {
    const Mesh &m = ctx->meshes[k];
    hoff[k] = m.offset;
    hoff[k + 1] = m.offset + m.ncells;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m.ncells; ++r) {
      const int64_t c = m.order[r], g = m.offset + r;
      for (int t = 0; t < nvc * d; ++t) hX[g * nvc * d + t] = m.X[c * nvc * d + t];
      // stencil: directional members face after face, then the remaining cells nearest first
      bool used[kMaxM] = {};
      int pos = 0;
      uint32_t info = 0;
      for (int f = 0; f < nf; ++f) {
        int cnt = 0;
        for (int j = 0; j < nd; ++j) {
          const int8_t p = m.dirpos[(c * nf + f) * nd + j];
          if (p < 0) continue;
          hst[(size_t)g * M + pos++] = (int32_t)(m.offset + m.rank[m.central[c * M + p]]);
          used[p] = true;
          ++cnt;
        }
        info |= (uint32_t)cnt << (4 * f);
      }
      for (int p = 0; p < M; ++p)
        if (!used[p]) hst[(size_t)g * M + pos++] = (int32_t)(m.offset + m.rank[m.central[c * M + p]]);
      // canonical Gauss-point order of each face: permutation to sorted global vertex ids
      for (int f = 0; f < nf; ++f) {
        int slots[3], ns = 0;
        for (int a = 0; a < nvc; ++a)
          if (a != f) slots[ns++] = a;
        int srt[3] = {0, 1, 2};  // face-vertex slots ordered by global vertex id
        for (int x = 1; x < d; ++x)
          for (int y = x; y > 0 && m.cv[c * nvc + slots[srt[y - 1]]] > m.cv[c * nvc + slots[srt[y]]]; --y)
            std::swap(srt[y - 1], srt[y]);
        int pidx = 0;
        for (int pp = 0; pp < tab.nperm; ++pp) {
          bool same = true;
          for (int j = 0; j < d; ++j) same = same && (tab.perm_list[pp][j] == srt[j]);
          if (same) pidx = pp;
        }
        info |= (uint32_t)pidx << (kInfoPermShift + 3 * f);
      }
      hinfo[g] = info;
      uint32_t meta = 0;
      for (int f = 0; f < nf; ++f) {
        const int32_t nb = m.nbr[c * nf + f];
        if (nb < 0) {
          hnbr[(size_t)g * 4 + f] = -1;
          meta |= 1u << (kMetaOwnerShift + f);
          const int kind = m.bkind[(size_t)c * nf + f];
          meta |= (uint32_t)kind << (kMetaKindShift + 2 * f);
        } else {
          const int64_t gn = m.offset + m.rank[nb];
          hnbr[(size_t)g * 4 + f] = (int32_t)gn;
          meta |= (uint32_t)m.nbrf[c * nf + f] << (2 * f);
          if (g < gn) meta |= 1u << (kMetaOwnerShift + f);
        }
      }
      hmeta[g] = meta;
    }
  }
  // a moving-shock boundary needs the physical time on the device
  bool shock_faces = false;
  for (int64_t g = 0; g < N && !shock_faces; ++g)
    for (int f = 0; f < nf; ++f)
      if (hnbr[(size_t)g * 4 + f] < 0 && ((hmeta[g] >> (kMetaKindShift + 2 * f)) & 3u) == CTENO_BOUNDARY_SHOCK_AB)
        shock_faces = true;
  // face list of the face-based flux schedule: owner cell-faces in (cell, face) order; every
  // cell-face refers to its face, flagged where the cell is not the owner
  std::vector<int32_t> hface, hcellface((size_t)N * 4, 0);
  for (int64_t g = 0; g < N; ++g)
    for (int f = 0; f < nf; ++f)
      if ((hmeta[g] >> (kMetaOwnerShift + f)) & 1u) {
        hcellface[(size_t)g * 4 + f] = (int32_t)(hface.size() / 2);
        const int64_t gn = hnbr[(size_t)g * 4 + f];
        hface.push_back((int32_t)(g * 4 + f));
        hface.push_back(gn < 0 ? -1 : (int32_t)(gn * 4 + ((hmeta[g] >> (2 * f)) & 3u)));
      }
  for (int64_t g = 0; g < N; ++g)
    for (int f = 0; f < nf; ++f)
      if (!((hmeta[g] >> (kMetaOwnerShift + f)) & 1u)) {
        const int64_t gn = hnbr[(size_t)g * 4 + f];
        const int fn = (hmeta[g] >> (2 * f)) & 3u;
        hcellface[(size_t)g * 4 + f] = (int32_t)(hcellface[(size_t)gn * 4 + fn] | 0x80000000u);
      }
  // every index the kernels gather with, checked once here: stencil members, face neighbours,
  // face records of the face-based flux (the gather staging lists are derived from the members)
  {
    bool ok = true;
    for (size_t k = 0; k < hst.size() && ok; ++k) ok = hst[k] >= 0 && hst[k] < N;
    for (size_t k = 0; k < hnbr.size() && ok; ++k) ok = hnbr[k] >= -1 && hnbr[k] < N;
    const int64_t nfc = (int64_t)hface.size() / 2;
    for (size_t k = 0; k < hface.size() && ok; ++k)
      ok = (k % 2 == 1 && hface[k] == -1) || (hface[k] >= 0 && hface[k] < 4 * N);
    for (int64_t g = 0; g < N && ok; ++g)
      for (int f = 0; f < nf && ok; ++f) ok = (int64_t)(hcellface[(size_t)g * 4 + f] & 0x7FFFFFFF) < nfc;
    if (!ok) return fail(ctx, CTENO_ERR_MESH, "a gathered index is out of range (inconsistent connectivity)");
  }
  // device allocations
  const size_t sT = ctx->fp32 ? sizeof(float) : sizeof(double);
  ctx->nfaces = (int64_t)hface.size() / 2;
  CK(dalloc(ctx, &ctx->d_face, sizeof(int32_t) * hface.size()));
  CK(dalloc(ctx, &ctx->d_cellface, sizeof(int32_t) * hcellface.size()));
  CK(dalloc(ctx, &ctx->Ff, sT * ((ctx->nv + 3) & ~3) * ctx->nfaces));
  CK(cudaMemcpyAsync(ctx->d_face, hface.data(), sizeof(int32_t) * hface.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cellface, hcellface.data(), sizeof(int32_t) * hcellface.size(),
                     cudaMemcpyHostToDevice, ctx->stream));
  double *dX = nullptr;
  CK(cudaMalloc(&dX, hX.size() * sizeof(double)));
  CK(dalloc(ctx, &ctx->d_tab, sizeof(DevTables)));
  CK(dalloc(ctx, &ctx->d_mesh_off, sizeof(int64_t) * (nmesh + 1)));
  const int nvp = lay_nvp(d), pds = dir_pds(d, ctx->p.degree);
  CK(dalloc(ctx, &ctx->U, sizeof(double) * nvp * N));
  CK(dalloc(ctx, &ctx->Un, sizeof(double) * nvp * N));
  if (ctx->nst == 4) CK(dalloc(ctx, &ctx->Acc, sizeof(double) * nvp * N));
  if (ctx->fp32) CK(dalloc(ctx, &ctx->U32, 2 * sizeof(float) * nvp * N));
  CK(dalloc(ctx, &ctx->st, sizeof(int32_t) * M * N));
  CK(dalloc(ctx, &ctx->nbr, sizeof(int32_t) * 4 * N));
  CK(dalloc(ctx, &ctx->cinfo, sizeof(uint32_t) * N));
  CK(dalloc(ctx, &ctx->fmeta, sizeof(uint32_t) * N));
  CK(dalloc(ctx, &ctx->Pc, sT * ctx->nk * M * N));
  CK(dalloc(ctx, &ctx->Pd, sT * nf * pds * N));
  CK(dalloc(ctx, &ctx->Uf, sT * nf * ctx->nq * ctx->nv * N));
  CK(dalloc(ctx, &ctx->geo, sizeof(double) * nf * 4 * N));
  if (ctx->fp32) CK(dalloc(ctx, &ctx->geo32, sizeof(float) * nf * 4 * N));
  CK(dalloc(ctx, &ctx->vol, sizeof(double) * N));
  CK(dalloc(ctx, &ctx->dt, sizeof(double) * 2 * nmesh));
  if (shock_faces) {
    CK(dalloc(ctx, &ctx->time, sizeof(double) * nmesh));
    CK(cudaMemsetAsync(ctx->time, 0, sizeof(double) * nmesh, ctx->stream));
  }
  CK(dalloc(ctx, &ctx->derr, sizeof(int)));
  CK(dalloc(ctx, &ctx->guard, sizeof(unsigned long long)));
  ctx->d_rank.resize(nmesh);
  std::vector<int32_t> hgrank(N);
  for (int k = 0; k < nmesh; ++k) {
    const Mesh &mk = ctx->meshes[k];
    CK(dalloc(ctx, &ctx->d_rank[k], sizeof(int32_t) * mk.ncells));
    CK(cudaMemcpyAsync(ctx->d_rank[k], mk.rank.data(), sizeof(int32_t) * mk.ncells, cudaMemcpyHostToDevice,
                       ctx->stream));
    for (int64_t c = 0; c < mk.ncells; ++c) hgrank[mk.offset + c] = (int32_t)(mk.offset + mk.rank[c]);
  }
  CK(dalloc(ctx, &ctx->d_grank, sizeof(int32_t) * N));
  CK(cudaMemcpyAsync(ctx->d_grank, hgrank.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, ctx->stream));
  DevTables dt{};
  dt.nk = tab.nk;
  dt.nq = tab.nq;
  dt.nperm = tab.nperm;
  dt.nvq = tab.nvq;
  std::memcpy(dt.ex, tab.ex, sizeof(dt.ex));
  std::memcpy(dt.psibar, tab.psibar, sizeof(dt.psibar));
  std::memcpy(dt.O, tab.O, sizeof(dt.O));
  std::memcpy(dt.Phi, tab.Phi, sizeof(dt.Phi));
  std::memcpy(dt.fw, tab.fw, sizeof(dt.fw));
  std::memcpy(dt.vq, tab.vq, sizeof(dt.vq));
  std::memcpy(dt.vw, tab.vw, sizeof(dt.vw));
  CK(cudaMemcpyAsync(ctx->d_tab, &dt, sizeof(DevTables), cudaMemcpyHostToDevice, ctx->stream));
  CK(d == 3 ? upload_recon_tables_3d(ctx->p.degree, tab, ctx->stream)
     : ctx->p.degree >= 4 ? upload_recon_tables_2d_high(ctx->p.degree, tab, ctx->stream)
                          : upload_recon_tables_2d(ctx->p.degree, tab, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_mesh_off, hoff.data(), sizeof(int64_t) * (nmesh + 1), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dX, hX.data(), hX.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->st, hst.data(), hst.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->fp32 && ctx->p.degree <= 3) {  // the gather-staged schedule exists up to degree 3
    const int rc = build_gather_tiles(ctx, hst);
    if (rc) return rc;
  }
  CK(cudaMemcpyAsync(ctx->nbr, hnbr.data(), hnbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->cinfo, hinfo.data(), hinfo.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->fmeta, hmeta.data(), hmeta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->guard, 0, sizeof(unsigned long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->U, 0, sizeof(double) * nvp * N, ctx->stream));
  if (ctx->U32) CK(cudaMemsetAsync(ctx->U32, 0, 2 * sizeof(float) * nvp * N, ctx->stream));
  SetupArgs s{};
  s.N = N;
  s.X = dX;
  s.st = ctx->st;
  s.cinfo = ctx->cinfo;
  s.nbr = ctx->nbr;
  s.fmeta = ctx->fmeta;
  for (int j = 0; j < 3; ++j) s.period[j] = 0.0;
  s.Pc = ctx->Pc;
  s.Pd = ctx->Pd;
  s.store_fp32 = ctx->fp32 ? 1 : 0;
  s.geo = ctx->geo;
  s.vol = ctx->vol;
  s.geo32 = ctx->geo32;
  s.tab = ctx->d_tab;
  s.shock_xs0 = ctx->shock[0];
  s.shock_sy = ctx->shock[1];
  s.err = ctx->derr;
  for (int j = 0; j < 3; ++j) s.period[j] = ctx->meshes[0].period[j];  // shared by all meshes
  launch_setup(d, ctx->p.degree, s, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(dX);
  int rc = device_status(ctx);
  if (rc) return rc;
  ctx->h_cinfo.resize(N);
  CK(cudaMemcpy(ctx->h_cinfo.data(), ctx->cinfo, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost));
  int64_t ms = 0, af = 0;
  for (int64_t g = 0; g < N; ++g) {
    const uint32_t info = ctx->h_cinfo[g];
    for (int f = 0; f < nf; ++f)
      if ((info >> (kInfoAdmShift + f)) & 1u) {
        ms += (info >> (4 * f)) & 15u;
        ++af;
      }
  }
  ctx->member_sum = ms;
  ctx->adm_faces = af;
  CK(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
  // the allocation-free read-back: its staging array's address on this (the context's) device,
  // and the kernel it launches, loaded now (under lazy module loading a first use would load them
  // later, and loading allocates device memory)
  CK(noalloc_stage_address(&ctx->noalloc_stage, &ctx->noalloc_cap));
  CK(preload_permute_out());
  ctx->built = true;
  return CTENO_OK;
}

int cteno_set_state(cteno_ctx *ctx, int32_t mesh_id, const double *U, int is_device) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if ((rc = check_mesh(ctx, mesh_id))) return rc;
  if (!U) return fail(ctx, CTENO_ERR_ARG, "null state");
  const Mesh &m = ctx->meshes[mesh_id];
  const size_t cnt = (size_t)ctx->nv * m.ncells;
  const double *src = U;
  if (!is_device) {
    if ((rc = ensure_stage_buf(ctx, cnt))) return rc;
    CK(cudaMemcpyAsync(ctx->stage_buf, U, cnt * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->stage_buf;
  }
  launch_permute_in(ctx->nv, lay_nvp(ctx->d), m.ncells, m.offset, ctx->d_rank[mesh_id], src, ctx->U,
                    ctx->U32, ctx->stream);
  KArgs a = make_args(ctx, 0, 0);
  launch_dt_mesh(ctx->d, a, mesh_id, m.offset, m.ncells, ctx->stream);  // this mesh's CFL step only
  CK(cudaGetLastError());
  return CTENO_OK;
}

namespace {
// Device address of page-locked host memory (the kernels then read or write it directly over
// the host link), or nullptr for pageable memory.
const void *pinned_device_address(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear: an unregistered pointer is not an error here
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace

int cteno_set_state_all(cteno_ctx *ctx, const double *U, int is_device) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!U) return fail(ctx, CTENO_ERR_ARG, "null state");
  const size_t cnt = (size_t)ctx->nv * ctx->N;
  const double *src = U;
  if (!is_device) {
    src = ctx->zerocopy ? static_cast<const double *>(pinned_device_address(U)) : nullptr;
    if (!src) {  // pageable: stage through device memory
      if ((rc = ensure_stage_buf(ctx, cnt))) return rc;
      CK(cudaMemcpyAsync(ctx->stage_buf, U, cnt * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      src = ctx->stage_buf;
    }
  }
  launch_set_state_all(ctx->d, make_args(ctx, 0, 0), ctx->d_grank, src, ctx->stream);
  CK(cudaGetLastError());
  return CTENO_OK;
}

int cteno_get_state_all(cteno_ctx *ctx, double *U_out, int is_device) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!U_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  const size_t cnt = (size_t)ctx->nv * ctx->N;
  const int nmesh = (int)ctx->meshes.size();
  if (is_device) {
    launch_permute_out_all(ctx->nv, lay_nvp(ctx->d), ctx->N, nmesh, ctx->d_mesh_off, ctx->d_grank, ctx->U,
                           U_out, ctx->stream);
    CK(cudaGetLastError());
    return CTENO_OK;
  }
  if (double *dst = ctx->zerocopy ? static_cast<double *>(const_cast<void *>(pinned_device_address(U_out)))
                                   : nullptr) {
    // page-locked output: the kernel writes it directly
    launch_permute_out_all(ctx->nv, lay_nvp(ctx->d), ctx->N, nmesh, ctx->d_mesh_off, ctx->d_grank, ctx->U, dst,
                           ctx->stream);
    CK(cudaGetLastError());
    return device_status(ctx);
  }
  if ((rc = ensure_stage_buf(ctx, cnt))) return rc;
  launch_permute_out_all(ctx->nv, lay_nvp(ctx->d), ctx->N, nmesh, ctx->d_mesh_off, ctx->d_grank, ctx->U,
                         ctx->stage_buf, ctx->stream);
  CK(cudaMemcpyAsync(U_out, ctx->stage_buf, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return device_status(ctx);
}

int cteno_rk_stage(cteno_ctx *ctx, int stage, const double *dt) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (stage < 0 || stage >= ctx->nst) return fail(ctx, CTENO_ERR_ARG, "bad stage");
  int swap = 0;
  if (dt) {
    CK(cudaMemcpyAsync(ctx->dt, dt, sizeof(double) * ctx->meshes.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (stage == 0) launch_dt_reset(make_args(ctx, 0, 0), ctx->stream);
  } else if (stage == 0) {
    swap = 1;  // the CFL step of the current state (computed by set_state or the last stage)
  }
  CK(enqueue_stage(ctx, stage, swap, ctx->stream));
  if (ctx->time && stage == ctx->nst - 1)  // the end of the step
    launch_time_advance(ctx->time, ctx->dt, (int)ctx->meshes.size(), ctx->stream);
  CK(cudaGetLastError());
  return CTENO_OK;
}

int cteno_run(cteno_ctx *ctx, int nsteps) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (nsteps < 0) return fail(ctx, CTENO_ERR_ARG, "nsteps < 0");
  if (!ctx->graph_exec) {
    CK(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
    if (ctx->timing) CK(cudaEventRecordWithFlags(ctx->tev[0], ctx->capture, cudaEventRecordExternal));
    for (int s = 0; s < ctx->nst; ++s) {
      const KArgs a = make_args(ctx, s, s == 0 ? 1 : 0);
      const cudaError_t le =
          launch_recon(ctx->d, ctx->p.degree, ctx->fp32 ? 1 : 0, kscheme(ctx), a, ctx->recon_block, ctx->capture);
      if (le != cudaSuccess) {  // end the capture before reporting
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(ctx->capture, &g);
        if (g) cudaGraphDestroy(g);
        return fail(ctx, CTENO_ERR_CUDA, std::string("reconstruction launch: ") + cudaGetErrorString(le));
      }
      if (ctx->timing) CK(cudaEventRecordWithFlags(ctx->tev[2 * s + 1], ctx->capture, cudaEventRecordExternal));
      launch_flux(ctx->d, ctx->nq, ctx->fp32 ? 1 : 0, a, ctx->flux_block, ctx->capture);
      if (ctx->timing) CK(cudaEventRecordWithFlags(ctx->tev[2 * s + 2], ctx->capture, cudaEventRecordExternal));
    }
    if (ctx->time) launch_time_advance(ctx->time, ctx->dt, (int)ctx->meshes.size(), ctx->capture);
    cudaError_t e = cudaStreamEndCapture(ctx->capture, &ctx->graph);
    if (e != cudaSuccess) return fail(ctx, CTENO_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&ctx->graph_exec, ctx->graph, 0));
  }
  for (int k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
  return CTENO_OK;
}

int cteno_get_state(cteno_ctx *ctx, int32_t mesh_id, double *U_out, int is_device) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if ((rc = check_mesh(ctx, mesh_id))) return rc;
  if (!U_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  const Mesh &m = ctx->meshes[mesh_id];
  const size_t cnt = (size_t)ctx->nv * m.ncells;
  if (is_device) {
    launch_permute_out(ctx->nv, lay_nvp(ctx->d), m.ncells, m.offset, ctx->d_rank[mesh_id], ctx->U, U_out,
                       ctx->stream);
    CK(cudaGetLastError());
    return CTENO_OK;
  }
  if ((rc = ensure_stage_buf(ctx, cnt))) return rc;
  launch_permute_out(ctx->nv, lay_nvp(ctx->d), m.ncells, m.offset, ctx->d_rank[mesh_id], ctx->U, ctx->stage_buf,
                     ctx->stream);
  CK(cudaMemcpyAsync(U_out, ctx->stage_buf, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return device_status(ctx);
}

int cteno_get_dt(cteno_ctx *ctx, double *dt_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!dt_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  CK(cudaMemcpyAsync(dt_out, ctx->dt, sizeof(double) * ctx->meshes.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CTENO_OK;
}

int cteno_record_flags(cteno_ctx *ctx, int enable) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (enable && !ctx->flags) {
    CK(dalloc(ctx, &ctx->flags, (size_t)ctx->nsel * ctx->N));
    CK(cudaMemsetAsync(ctx->flags, 0, (size_t)ctx->nsel * ctx->N, ctx->stream));
  }
  if ((bool)enable != ctx->record_flags) drop_graph(ctx);
  ctx->record_flags = enable != 0;
  return CTENO_OK;
}

int cteno_get_flags(cteno_ctx *ctx, int32_t mesh_id, uint8_t *out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if ((rc = check_mesh(ctx, mesh_id))) return rc;
  if (!out) return fail(ctx, CTENO_ERR_ARG, "null output");
  if (!ctx->flags) return fail(ctx, CTENO_ERR_STATE, "flag recording is off");
  const Mesh &m = ctx->meshes[mesh_id];
  const int64_t N = ctx->N;
  const int ns = ctx->nsel;  // one plane per selection: variable, or (face, field)
  std::vector<uint8_t> h((size_t)ns * m.ncells);
  for (int v = 0; v < ns; ++v)
    CK(cudaMemcpyAsync(h.data() + (size_t)v * m.ncells, ctx->flags + (size_t)v * N + m.offset, m.ncells,
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int64_t c = 0; c < m.ncells; ++c)
    for (int v = 0; v < ns; ++v) out[c * ns + v] = h[(size_t)v * m.ncells + m.rank[c]];
  return CTENO_OK;
}

int cteno_get_face_states(cteno_ctx *ctx, int32_t mesh_id, double *out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if ((rc = check_mesh(ctx, mesh_id))) return rc;
  if (!out) return fail(ctx, CTENO_ERR_ARG, "null output");
  const Mesh &m = ctx->meshes[mesh_id];
  const int64_t n = m.ncells;
  const int rec = ctx->nf * ctx->nq * ctx->nv;  // one cell's record [f][q][v]
  const size_t sT = ctx->fp32 ? 4 : 8;
  std::vector<unsigned char> h((size_t)rec * n * sT);
  CK(cudaMemcpyAsync(h.data(), (const char *)ctx->Uf + (size_t)m.offset * rec * sT, h.size(),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int64_t c = 0; c < n; ++c)
    for (int r = 0; r < rec; ++r) {
      const size_t idx = (size_t)m.rank[c] * rec + r;
      out[c * rec + r] = ctx->fp32 ? (double)((const float *)h.data())[idx] : ((const double *)h.data())[idx];
    }
  return CTENO_OK;
}

int cteno_get_stencil(cteno_ctx *ctx, int32_t mesh_id, int64_t cell, int32_t *central, int32_t *dir,
                      int32_t *dok) {
  if (!ctx) return CTENO_ERR_ARG;
  if (!ctx->stencils) return fail(ctx, CTENO_ERR_STATE, "cteno_stencil_build has not run");
  int rc = check_mesh(ctx, mesh_id);
  if (rc) return rc;
  const Mesh &m = ctx->meshes[mesh_id];
  if (cell < 0 || cell >= m.ncells || !central || !dir) return fail(ctx, CTENO_ERR_ARG, "bad cell");
  const int nf = ctx->nf, nd = ctx->nd, M = ctx->M;
  for (int p = 0; p < M; ++p) central[p] = m.central[cell * M + p];
  for (int f = 0; f < nf; ++f)
    for (int j = 0; j < nd; ++j) dir[f * nd + j] = m.dirpos[(cell * nf + f) * nd + j];
  if (dok) {
    if (!ctx->built) return fail(ctx, CTENO_ERR_STATE, "admissibility is known after cteno_lsq_build");
    const uint32_t info = ctx->h_cinfo[m.offset + m.rank[cell]];
    for (int f = 0; f < nf; ++f) dok[f] = (info >> (kInfoAdmShift + f)) & 1u;
  }
  return CTENO_OK;
}

int cteno_boundary_region(cteno_ctx *ctx, int32_t mesh_id, const double *lo, const double *hi, int kind) {
  if (!ctx) return CTENO_ERR_ARG;
  int rc = check_mesh(ctx, mesh_id);
  if (rc) return rc;
  if (ctx->built) return fail(ctx, CTENO_ERR_STATE, "boundary regions must be set before cteno_lsq_build");
  if (!lo || !hi || kind < CTENO_BOUNDARY_TRANSMISSIVE || kind > CTENO_BOUNDARY_SHOCK_AB ||
      (kind == CTENO_BOUNDARY_SHOCK_AB && ctx->d != 2))
    return fail(ctx, CTENO_ERR_ARG, "bad boundary region (the moving-shock kind is 2D only)");
  Mesh &m = ctx->meshes[mesh_id];
  const int d = ctx->d, nvc = d + 1, nf = d + 1;
  for (int64_t c = 0; c < m.ncells; ++c)
    for (int f = 0; f < nf; ++f) {
      if (m.nbr[c * nf + f] >= 0) continue;
      bool in = true;
      for (int k = 0; k < d; ++k) {
        double mid = 0.0;
        for (int v = 0; v < nvc; ++v)
          if (v != f) mid += m.X[(c * nvc + v) * d + k] / d;
        in = in && mid >= lo[k] && mid <= hi[k];
      }
      if (in) m.bkind[(size_t)c * nf + f] = (int8_t)kind;
    }
  return CTENO_OK;
}

int cteno_boundary_states(cteno_ctx *ctx, const double *A, const double *B, double xs0, double sy, double vs) {
  if (!ctx || !A || !B) return CTENO_ERR_ARG;
  if (ctx->built && (xs0 != ctx->shock[0] || sy != ctx->shock[1]))
    return fail(ctx, CTENO_ERR_STATE, "the shock line's position (xs0, sy) must be set before cteno_lsq_build");
  for (int v = 0; v < ctx->nv; ++v) {
    ctx->bA[v] = A[v];
    ctx->bB[v] = B[v];
  }
  ctx->shock[0] = xs0;
  ctx->shock[1] = sy;
  ctx->shock[2] = vs;
  drop_graph(ctx);
  return CTENO_OK;
}

int cteno_set_time(cteno_ctx *ctx, double t) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!ctx->time) return CTENO_OK;  // no moving-shock boundary: the time is not tracked
  std::vector<double> h(ctx->meshes.size(), t);
  CK(cudaMemcpyAsync(ctx->time, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CTENO_OK;
}

int cteno_get_time(cteno_ctx *ctx, double *t_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!t_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  if (!ctx->time) return fail(ctx, CTENO_ERR_STATE, "the time is tracked only with a moving-shock boundary");
  CK(cudaMemcpyAsync(t_out, ctx->time, sizeof(double) * ctx->meshes.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CTENO_OK;
}

int cteno_info(cteno_ctx *ctx, int32_t mesh_id, int64_t *out) {
  if (!ctx || !out) return CTENO_ERR_ARG;
  out[0] = (int64_t)ctx->meshes.size();
  int64_t tot = 0;
  for (auto &m : ctx->meshes) tot += m.ncells;
  out[1] = tot;
  out[2] = ctx->M;
  out[3] = ctx->nk;
  out[4] = ctx->nv;
  out[5] = ctx->nf;
  out[6] = ctx->nq;
  out[7] = (mesh_id >= 0 && mesh_id < (int32_t)ctx->meshes.size()) ? ctx->meshes[mesh_id].ncells : 0;
  out[8] = ctx->nd;
  out[9] = ctx->nsel;
  return CTENO_OK;
}

int cteno_sync(cteno_ctx *ctx, int64_t *guard_count) {
  int rc = check_built(ctx);
  if (rc) return rc;
  unsigned long long g = 0;
  CK(cudaMemcpyAsync(&g, ctx->guard, sizeof(g), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemsetAsync(ctx->guard, 0, sizeof(g), ctx->stream));
  rc = device_status(ctx);
  if (guard_count) *guard_count = (int64_t)g;
  return rc;
}

int cteno_set_launch(cteno_ctx *ctx, int recon_block, int flux_block) {
  if (!ctx) return CTENO_ERR_ARG;
  // positive: block size of the uncapped kernel; negative: block size of the register-capped
  // variant (mixed path only, at most 128 threads)
  auto ok = [&](int b, bool recon) {
    if (b == 0) return true;
    if (recon && ctx->p.degree >= 4) {  // degrees 4 to 6: the variable-per-lane schedule only
      if (b >= kHighOcc + 32 && b <= kHighOcc + 256 && b % 32 == 0)  // its 64-register build
        return ctx->fp32 && !ctx->p.characteristic;
      return b >= kLaneSchedule + 32 && b <= kLaneSchedule + 256 && b % 32 == 0;
    }
    // the characteristic reconstruction: the variable-per-lane schedule only
    if (recon && ctx->p.characteristic)
      return b >= kLaneSchedule + 32 && b <= kLaneSchedule + 256 && b % 32 == 0;
    if (b >= kFaceFlux)  // face-based flux schedule
      return !recon && b - kFaceFlux >= 32 && b - kFaceFlux <= 256 && b % 32 == 0;
    {
      int w = 0, st = 0;
      pair_launch(b, &w, &st);
      if (w)  // two lanes per cell: reconstruction, mixed, fits
        return recon && ctx->fp32 && recon_pair_smem(ctx->d, ctx->p.degree, w, st) <= kMaxStreamSmem;
    }
    if (b > kStreamCells && b <= kStreamCells + 8)  // streamed cells: reconstruction, mixed, fits
      return recon && ctx->fp32 &&
             recon_stream_cells_smem(ctx->d, ctx->p.degree, b - kStreamCells) <= kMaxStreamSmem;
    {
      int w = 0, st = 0;
      stream_launch(b, &w, &st);
      if (w)  // streamed lanes: reconstruction, mixed, fits
        return recon && ctx->fp32 && recon_stream_smem(ctx->d, ctx->p.degree, w, st) <= kMaxStreamSmem;
    }
    if (b == kHaloLanes || b == kHaloLanes + 1)  // gather-staged: reconstruction, mixed, lists built, fits
      return recon && ctx->fp32 && ctx->hl &&
             recon_halo_smem(ctx->d, ctx->p.degree, ctx->hrec) / (b == kHaloLanes ? 1 : 2) <= kMaxStagedSmem;
    if (b >= kStagedCells) {  // staged schedules: reconstruction, mixed path, two stages that fit
      const int t = b - (b >= kStagedLanes ? kStagedLanes : kStagedCells);
      return recon && ctx->fp32 && b < kStagedLanes + 1024 && t >= 32 && t <= 256 && t % 32 == 0 &&
             recon_staged_smem(ctx->d, ctx->p.degree, 1, b) <= kMaxStagedSmem;
    }
    if (b >= kLaneSchedule) return b - kLaneSchedule >= 32 && b - kLaneSchedule <= 256 && b % 32 == 0;
    if (b < 0) return ctx->fp32 && -b >= 32 && -b <= 128 && (-b) % 32 == 0;
    return b >= 32 && b <= 256 && b % 32 == 0;
  };
  if (!ok(recon_block, true) || !ok(flux_block, false))
    return fail(ctx, CTENO_ERR_ARG,
                "block size must be a multiple of 32 in [32, 256] (capped: [32, 128], mixed path; staged: "
                "mixed-path reconstruction whose two stages fit in shared memory)");
  if (recon_block) ctx->recon_block = recon_block;
  if (flux_block) ctx->flux_block = flux_block;
  drop_graph(ctx);
  return CTENO_OK;
}

int cteno_autotune(cteno_ctx *ctx, int32_t *best_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  const size_t cnt = (size_t)lay_nvp(ctx->d) * ctx->N;
  const size_t nm = ctx->meshes.size();
  // backup: U (FP64), the FP32 shadow and the time steps
  const size_t bytes = cnt * sizeof(double) + 2 * cnt * sizeof(float) + 2 * nm * sizeof(double);
  if (!ctx->backup) CK(cudaMalloc(&ctx->backup, bytes));
  double *bU = ctx->backup, *bdt = ctx->backup + cnt;
  float *b32 = (float *)(bdt + 2 * nm);
  auto save_restore = [&](bool save) -> cudaError_t {
    cudaError_t e;
    e = cudaMemcpyAsync(save ? bU : ctx->U, save ? ctx->U : bU, cnt * sizeof(double),
                        cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    if (ctx->U32) {
      e = cudaMemcpyAsync(save ? b32 : ctx->U32, save ? ctx->U32 : b32, 2 * cnt * sizeof(float),
                          cudaMemcpyDeviceToDevice, ctx->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(save ? bdt : ctx->dt, save ? ctx->dt : bdt, 2 * nm * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream);
  };
  CK(save_restore(true));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // candidates: uncapped kernels at 64/128/256 threads; on the mixed path also the
  // register-capped variants (8 blocks per SM) at 64/128 threads (negative values)
  std::vector<int> cand = {64, 128, 256};
  if (ctx->fp32) {
    cand.push_back(-64);
    cand.push_back(-128);
  }
  // the lane schedules (variable per lane for the reconstruction, face per lane for the flux)
  for (int b : {128, 256}) cand.push_back(kLaneSchedule + b);
  std::vector<int> rcand = cand;
  if (ctx->p.degree >= 4) rcand = {kLaneSchedule + 64, kLaneSchedule + 128, kLaneSchedule + 256};
  if (ctx->p.degree >= 4 && ctx->fp32 && !ctx->p.characteristic)
    for (int b : {64, 128, 256}) rcand.push_back(kHighOcc + b);
  // the staged schedules (mixed path) whose two stages fit
  if (ctx->fp32 && ctx->p.degree <= 3)
    for (int b : {kStagedCells + 32, kStagedCells + 64, kStagedCells + 128, kStagedLanes + 64,
                  kStagedLanes + 128, kStagedLanes + 256})
      if (recon_staged_smem(ctx->d, ctx->p.degree, 1, b) <= kMaxStagedSmem) rcand.push_back(b);
  if (ctx->fp32 && ctx->hl) {
    const long long hs = recon_halo_smem(ctx->d, ctx->p.degree, ctx->hrec);
    if (hs <= kMaxStagedSmem) rcand.push_back(kHaloLanes);
    if (hs / 2 <= kMaxStagedSmem) rcand.push_back(kHaloLanes + 1);
  }
  // the streamed lane schedule (mixed path) at the block sizes that fit
  if (ctx->fp32 && ctx->p.degree <= 3) {
    for (int w : {8, 12, 16}) {
      if (recon_stream_smem(ctx->d, ctx->p.degree, w, 3) <= kMaxStreamSmem) rcand.push_back(kStreamLanes + w);
      if (recon_stream_smem(ctx->d, ctx->p.degree, w, 2) <= kMaxStreamSmem) rcand.push_back(kStreamLanes2 + w);
    }
    for (int w : {2, 4, 6, 7, 8})
      if (recon_stream_cells_smem(ctx->d, ctx->p.degree, w) <= kMaxStreamSmem) rcand.push_back(kStreamCells + w);
    for (int w : {4, 6, 8}) {
      if (recon_pair_smem(ctx->d, ctx->p.degree, w, 2) <= kMaxStreamSmem) rcand.push_back(kPairLanes + w);
      if (recon_pair_smem(ctx->d, ctx->p.degree, w, 3) <= kMaxStreamSmem) rcand.push_back(kPairLanes3 + w);
    }
  }
  if (ctx->p.characteristic)  // the variable-per-lane schedule only
    rcand = {kLaneSchedule + 64, kLaneSchedule + 128, kLaneSchedule + 256};
  const int reps = 5;
  float best_r = 1e30f, best_f = 1e30f;
  int br = ctx->recon_block, bf = ctx->flux_block;
  const KArgs a = make_args(ctx, 1, 0);  // stage 1: reads U^n, writes U only
  for (int b : rcand) {  // the reconstruction writes only face states: no restore needed
    CK(launch_recon(ctx->d, ctx->p.degree, ctx->fp32, kscheme(ctx), a, b, ctx->stream));
    CK(cudaEventRecord(e0, ctx->stream));
    for (int r = 0; r < reps; ++r) CK(launch_recon(ctx->d, ctx->p.degree, ctx->fp32, kscheme(ctx), a, b, ctx->stream));
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_r) best_r = ms, br = b;
  }
  std::vector<int> fcand = cand;  // flux: also the face-based schedule
  for (int b : {kFaceFlux + 128, kFaceFlux + 256}) fcand.push_back(b);
  for (int b : fcand) {
    float tot = 0;
    for (int r = 0; r < reps; ++r) {
      CK(save_restore(false));
      CK(cudaEventRecord(e0, ctx->stream));
      launch_flux(ctx->d, ctx->nq, ctx->fp32, a, b, ctx->stream);
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      tot += ms;
    }
    if (tot < best_f) best_f = tot, bf = b;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(save_restore(false));
  ctx->recon_block = br;
  ctx->flux_block = bf;
  drop_graph(ctx);
  if (best_out) {
    best_out[0] = br;
    best_out[1] = bf;
  }
  return device_status(ctx);
}

int cteno_kernel_stats(cteno_ctx *ctx, double *out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!out) return fail(ctx, CTENO_ERR_ARG, "null output");
  const double N = (double)ctx->N, s = ctx->fp32 ? 4.0 : 8.0;
  const int nk = ctx->nk, M = ctx->M, nv = ctx->nv, nf = ctx->nf, nq = ctx->nq, d = ctx->d;
  const double members = (double)ctx->member_sum;
  const double nvp = lay_nvp(d), pds = dir_pds(d, ctx->p.degree);
  const double rec_u = 8.0 * nvp;  // own state record: FP32 (hi, lo) pairs or FP64 values
  // reconstruction: pseudo-inverse records (central + admissible directional faces), stencil ids,
  // cell info, own state record, face-state writes (neighbour means are re-reads of records
  // counted once as "own")
  out[0] = N * (nk * M * s + M * 4.0 + 4.0 + rec_u + nf * nq * nv * s) + ctx->adm_faces * pds * s +
           (ctx->record_flags ? N * nv : 0.0);
  // flux/update: face states (each read by both of its cells, counted once), neighbour ids,
  // face meta, face geometry, volume, U, U^n and the FP32 pair record
  out[1] = N * (nf * nq * nv * s + 16.0 + 4.0 + nf * 4 * s + 8.0 + 3 * nvp * 8.0 +
                (ctx->fp32 ? 8.0 * nvp : 0.0));
  // FLOPs: central and directional products, p_1, SI, selection (~30 per stencil), face values
  const double st = 1.0 + (N > 0 ? members / N / d : 0.0);
  // (SI = a^T O a counted in its symmetric form: nk(nk+1)/2 products and nk more per variable)
  out[2] = N * (2.0 * nk * M * nv + 2.0 * nv * (nk * (nk + 1) / 2.0 + nk) + nv * 30.0 * st +
                2.0 * nv * nf * nq * nk) +
           members * 2.0 * dir_unknowns(d, ctx->p.degree) * nv;
  // HLLC ~ 90 + 20 d operations per Gauss point, plus accumulation and the update
  out[3] = N * (nf * nq * (90.0 + 20.0 * d + 3.0 * nv) + 6.0 * nv);
  return CTENO_OK;
}

int cteno_profile_step(cteno_ctx *ctx, int nsteps, double *ms_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!ms_out || nsteps <= 0) return fail(ctx, CTENO_ERR_ARG, "bad arguments");
  const int ns = ctx->nst;
  cudaEvent_t ev[9];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  double tr = 0.0, tf = 0.0;
  for (int k = 0; k < nsteps; ++k) {
    for (int s = 0; s < ns; ++s) {
      const KArgs a = make_args(ctx, s, s == 0 ? 1 : 0);
      CK(cudaEventRecord(ev[2 * s], ctx->stream));
      CK(launch_recon(ctx->d, ctx->p.degree, ctx->fp32, kscheme(ctx), a, ctx->recon_block, ctx->stream));
      CK(cudaEventRecord(ev[2 * s + 1], ctx->stream));
      launch_flux(ctx->d, ctx->nq, ctx->fp32, a, ctx->flux_block, ctx->stream);
    }
    CK(cudaEventRecord(ev[2 * ns], ctx->stream));
    CK(cudaEventSynchronize(ev[2 * ns]));
    for (int s = 0; s < ns; ++s) {
      float a = 0, b = 0;
      CK(cudaEventElapsedTime(&a, ev[2 * s], ev[2 * s + 1]));
      CK(cudaEventElapsedTime(&b, ev[2 * s + 1], ev[2 * s + 2]));
      tr += a;
      tf += b;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  ms_out[0] = tr / nsteps;
  ms_out[1] = tf / nsteps;
  return device_status(ctx);
}

int cteno_set_timing(cteno_ctx *ctx, int enable) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (enable && !ctx->tev[0])
    for (auto &e : ctx->tev) CK(cudaEventCreate(&e));
  if ((bool)enable != ctx->timing) drop_graph(ctx);
  ctx->timing = enable != 0;
  return CTENO_OK;
}

int cteno_last_kernel_ms(cteno_ctx *ctx, double *ms_out) {
  int rc = check_built(ctx);
  if (rc) return rc;
  if (!ms_out) return fail(ctx, CTENO_ERR_ARG, "null output");
  if (!ctx->timing || !ctx->graph_exec) return fail(ctx, CTENO_ERR_STATE, "timing is off or no step has run");
  CK(cudaEventSynchronize(ctx->tev[2 * ctx->nst]));
  double r = 0.0, f = 0.0;
  for (int s = 0; s < ctx->nst; ++s) {
    float a = 0, b = 0;
    CK(cudaEventElapsedTime(&a, ctx->tev[2 * s], ctx->tev[2 * s + 1]));
    CK(cudaEventElapsedTime(&b, ctx->tev[2 * s + 1], ctx->tev[2 * s + 2]));
    r += a;
    f += b;
  }
  ms_out[0] = r;
  ms_out[1] = f;
  return CTENO_OK;
}

int cteno_test_wait_timeout(cteno_ctx *ctx, int64_t limit_ns) {
  if (!ctx) return CTENO_ERR_ARG;
  if (limit_ns < 0 || limit_ns > 1000000000LL) return fail(ctx, CTENO_ERR_ARG, "limit_ns must be in [0, 1e9]");
  ctx->test_wait_ns = (unsigned long long)limit_ns;
  drop_graph(ctx);
  return CTENO_OK;
}

const char *cteno_last_error(cteno_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void cteno_destroy(cteno_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream || ctx->built) cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  for (void *p : ctx->allocations) cudaFree(p);
  if (ctx->stage_buf) cudaFree(ctx->stage_buf);
  if (ctx->backup) cudaFree(ctx->backup);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  for (auto &e : ctx->tev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"
