// setup.cu -- FP64 set-up on the GPU: cell geometry (Sec. 2, eq. 2), basis moments of every
// stencil member in the target cell's reference space (eqs. 5, 7, 10), Householder QR of the
// least-squares matrices and the pseudo-inverses P = R^-1 Q^T diag(|V'_m|), so that the
// coefficients of eq. 12 are a = P (U_m - U_0). One thread per cell; run once per mesh set.
#include "device.h"

namespace cteno {
namespace {

template <int D>
__device__ __forceinline__ double det_rm(const double (&a)[D][D]) {
  if constexpr (D == 2) {
    return a[0][0] * a[1][1] - a[0][1] * a[1][0];
  } else {
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  }
}

template <int D>
__device__ __forceinline__ void inverse(const double (&a)[D][D], double (&inv)[D][D]) {
  const double det = det_rm<D>(a);
  if constexpr (D == 2) {
    inv[0][0] = a[1][1] / det;
    inv[0][1] = -a[0][1] / det;
    inv[1][0] = -a[1][0] / det;
    inv[1][1] = a[0][0] / det;
  } else {
    inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
    inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
    inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
  }
}

__device__ __forceinline__ double image_shift(double dx, double L) {
  return (L > 0.0) ? -L * round(dx / L) : 0.0;
}

__device__ __forceinline__ double monomial(const int *e, const double *x, int d) {
  double v = 1.0;
  for (int j = 0; j < d; ++j)
    for (int p = 0; p < e[j]; ++p) v *= x[j];
  return v;
}

// In-place Householder QR of the rows x cols matrix W (leading dimension LD). On return the
// upper triangle above the diagonal holds R, diag[] its diagonal, and column k below the diagonal
// together with vtop[k] the k-th reflector v (H_k = I - beta_k v v^T). Returns 1 when
// min |R_kk| > 1e-10 max |R_kk| (numerically full column rank).
template <int LD>
__device__ int householder(double (*W)[LD], int rows, int cols, double *diag, double *vtop,
                           double *beta) {
  for (int k = 0; k < cols; ++k) {
    double nrm2 = 0.0;
    for (int r = k; r < rows; ++r) nrm2 += W[r][k] * W[r][k];
    const double nrm = sqrt(nrm2);
    const double alpha = (W[k][k] > 0.0) ? -nrm : nrm;
    const double v0 = W[k][k] - alpha;
    double vv = v0 * v0;
    for (int r = k + 1; r < rows; ++r) vv += W[r][k] * W[r][k];
    const double b = (vv > 0.0) ? 2.0 / vv : 0.0;
    for (int c = k + 1; c < cols; ++c) {
      double s = v0 * W[k][c];
      for (int r = k + 1; r < rows; ++r) s += W[r][k] * W[r][c];
      s *= b;
      W[k][c] -= s * v0;
      for (int r = k + 1; r < rows; ++r) W[r][c] -= s * W[r][k];
    }
    diag[k] = alpha;
    vtop[k] = v0;
    beta[k] = b;
  }
  double mx = 0.0, mn = 1e300;
  for (int k = 0; k < cols; ++k) {
    mx = fmax(mx, fabs(diag[k]));
    mn = fmin(mn, fabs(diag[k]));
  }
  return (rows >= cols && mx > 0.0 && mn > 1e-10 * mx) ? 1 : 0;
}

// Column m of R^-1 Q^T (the first `cols` entries of Q^T e_m, back-substituted).
template <int LD, int MAXR>
__device__ void pinv_column(double (*W)[LD], int rows, int cols, const double *diag,
                            const double *vtop, const double *beta, int m, double *out) {
  double e[MAXR];
  for (int r = 0; r < rows; ++r) e[r] = (r == m) ? 1.0 : 0.0;
  for (int k = 0; k < cols; ++k) {
    double s = vtop[k] * e[k];
    for (int r = k + 1; r < rows; ++r) s += W[r][k] * e[r];
    s *= beta[k];
    e[k] -= s * vtop[k];
    for (int r = k + 1; r < rows; ++r) e[r] -= s * W[r][k];
  }
  for (int k = cols - 1; k >= 0; --k) {
    double s = e[k];
    for (int c = k + 1; c < cols; ++c) s -= W[k][c] * out[c];
    out[k] = s / diag[k];
  }
}

template <int D, int R>
__global__ void __launch_bounds__(128) setup_kernel(const SetupArgs a) {
  using DR = Dir<D, R>;
  constexpr int NVC = D + 1, NF = D + 1, ND = DR::ND, KD = DR::KD;
  constexpr int NK = (D == 2 ? (R + 1) * (R + 2) / 2 : (R + 1) * (R + 2) * (R + 3) / 6) - 1;
  constexpr int M = 2 * (NK + 1);
  constexpr double FACT = (D == 2) ? 2.0 : 6.0;
  const int64_t N = a.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const DevTables &T = *a.tab;

  double Xi[NVC][D];
  for (int v = 0; v < NVC; ++v)
    for (int j = 0; j < D; ++j) Xi[v][j] = a.X[(i * NVC + v) * D + j];
  double J[D][D], Ji[D][D], ci[D];
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) J[r][c] = Xi[c + 1][r] - Xi[0][r];
  inverse<D>(J, Ji);
  a.vol[i] = FACT / fabs(det_rm<D>(J));  // 1 / |V_i|
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
    for (int v = 0; v < NVC; ++v) s += Xi[v][j];
    ci[j] = s / NVC;
  }

  // faces owned by this cell: outward normal and area, written to both sides of the face
  const uint32_t meta = a.fmeta[i];
  for (int f = 0; f < NF; ++f) {
    if (!((meta >> (kMetaOwnerShift + f)) & 1u)) continue;
    int loc[3], k = 0;
    for (int v = 0; v < NVC; ++v)
      if (v != f) loc[k++] = v;
    double n[3] = {0, 0, 0}, area;
    if constexpr (D == 2) {
      const double ex = Xi[loc[1]][0] - Xi[loc[0]][0], ey = Xi[loc[1]][1] - Xi[loc[0]][1];
      n[0] = ey;
      n[1] = -ex;
      area = sqrt(ex * ex + ey * ey);
    } else {
      double u[3], w[3];
      for (int j = 0; j < 3; ++j) {
        u[j] = Xi[loc[1]][j] - Xi[loc[0]][j];
        w[j] = Xi[loc[2]][j] - Xi[loc[0]][j];
      }
      n[0] = u[1] * w[2] - u[2] * w[1];
      n[1] = u[2] * w[0] - u[0] * w[2];
      n[2] = u[0] * w[1] - u[1] * w[0];
      area = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    }
    double len = 0.0, dot = 0.0;
    for (int j = 0; j < D; ++j) {
      len += n[j] * n[j];
      dot += n[j] * (Xi[loc[0]][j] - Xi[f][j]);
    }
    len = sqrt(len);
    const double sgn = (dot > 0.0) ? 1.0 : -1.0;
    for (int j = 0; j < D; ++j) n[j] = sgn * n[j] / len;
    const int32_t nb = a.nbr[i * 4 + f];
    double gv[4] = {0.0, 0.0, 0.0, area};
    for (int j = 0; j < D; ++j) gv[j] = n[j];
    if constexpr (D == 2) {  // moving-shock boundary face: c_f = xs0 + sy y_mid - x_mid in slot 2
      if (nb < 0 && ((meta >> (kMetaKindShift + 2 * f)) & 3u) == 3u) {
        const double xm = 0.5 * (Xi[loc[0]][0] + Xi[loc[1]][0]), ym = 0.5 * (Xi[loc[0]][1] + Xi[loc[1]][1]);
        gv[2] = a.shock_xs0 + a.shock_sy * ym - xm;
      }
    }
    for (int c = 0; c < 4; ++c) {
      a.geo[(i * NF + f) * 4 + c] = gv[c];
      if (a.geo32) a.geo32[(i * NF + f) * 4 + c] = (float)gv[c];
    }
    if (nb >= 0) {  // the other side: the exact negative normal, the same area
      const int fj = (meta >> (2 * f)) & 3u;
      for (int c = 0; c < 4; ++c) {
        const double x = (c < D) ? -gv[c] : gv[c];
        a.geo[((int64_t)nb * NF + fj) * 4 + c] = x;
        if (a.geo32) a.geo32[((int64_t)nb * NF + fj) * 4 + c] = (c < D) ? -(float)gv[c] : (float)gv[c];
      }
    }
  }

  // moments A_mk = int_{V'_m} psi_k - |V'_m| psibar_k of every stencil member (eq. 10)
  double W[M][NK];
  double Vp[M];
  for (int p = 0; p < M; ++p) {
    const int64_t m = a.st[i * M + p];
    double Xm[NVC][D], cm[D];
    for (int v = 0; v < NVC; ++v)
      for (int j = 0; j < D; ++j) Xm[v][j] = a.X[(m * NVC + v) * D + j];
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
      for (int v = 0; v < NVC; ++v) s += Xm[v][j];
      cm[j] = s / NVC;
    }
    double xi[NVC][D];
    for (int v = 0; v < NVC; ++v) {
      double y[D];
      for (int j = 0; j < D; ++j) y[j] = Xm[v][j] + image_shift(cm[j] - ci[j], a.period[j]) - Xi[0][j];
      for (int r = 0; r < D; ++r) {
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += Ji[r][j] * y[j];
        xi[v][r] = s;
      }
    }
    double E[D][D];
    for (int r = 0; r < D; ++r)
      for (int c = 0; c < D; ++c) E[r][c] = xi[c + 1][r] - xi[0][r];
    const double jac = fabs(det_rm<D>(E));  // = d! |V'_m|
    Vp[p] = jac / FACT;
    for (int k = 0; k < NK; ++k) W[p][k] = -Vp[p] * T.psibar[k];
    for (int q = 0; q < T.nvq; ++q) {
      double x[3] = {0, 0, 0};
      for (int r = 0; r < D; ++r) {
        double s = xi[0][r];
        for (int c = 0; c < D; ++c) s += T.vq[q][c] * E[r][c];
        x[r] = s;
      }
      const double w = T.vw[q] * jac;
      for (int k = 0; k < NK; ++k) W[p][k] += w * monomial(T.ex[k], x, D);
    }
  }

  // directional stencils first (they read the first KD columns of A, those of the graded basis
  // functions of degree <= 1 or 2, before the QR overwrites them)
  const uint32_t info = a.cinfo[i];
  uint32_t adm = 0;
  int off = 0;
  for (int f = 0; f < NF; ++f) {
    const int nm = (info >> (4 * f)) & 15u;
    double pd[KD][ND];
    for (int k = 0; k < KD; ++k)
      for (int j = 0; j < ND; ++j) pd[k][j] = 0.0;
    if (nm >= KD) {
      double Wd[ND][KD], dg[KD], vt[KD], bt[KD];
      for (int j = 0; j < nm; ++j)
        for (int k = 0; k < KD; ++k) Wd[j][k] = W[off + j][k];
      if (householder<KD>(Wd, nm, KD, dg, vt, bt)) {
        adm |= 1u << f;
        for (int j = 0; j < nm; ++j) {
          double col[KD];
          pinv_column<KD, ND>(Wd, nm, KD, dg, vt, bt, j, col);
          for (int k = 0; k < KD; ++k) pd[k][j] = col[k] * Vp[off + j];
        }
      }
    }
    constexpr int PDS = DR::PDS;
    for (int e = 0; e < PDS; ++e) {  // see Dir: member-major (degree <= 3) or unknown-major rows
      const int j = DR::HIGH ? e % DR::NDP : e / KD, k = DR::HIGH ? e / DR::NDP : e % KD;
      const double val = (j < ND && k < KD) ? pd[k][j] : 0.0;
      const int64_t idx = (i * NF + f) * PDS + e;
      if (a.store_fp32)
        ((float *)a.Pd)[idx] = (float)val;
      else
        ((double *)a.Pd)[idx] = val;
    }
    off += nm;
  }
  a.cinfo[i] = (info & ~(0xFu << kInfoAdmShift)) | (adm << kInfoAdmShift);

  // central stencil
  double dg[NK], vt[NK], bt[NK];
  if (!householder<NK>(W, M, NK, dg, vt, bt)) atomicOr(a.err, kErrRank);
  for (int p = 0; p < M; ++p) {
    double col[NK];
    pinv_column<NK, M>(W, M, NK, dg, vt, bt, p, col);
    for (int k = 0; k < NK; ++k) {
      const int64_t idx = (i * M + p) * NK + k;
      if (a.store_fp32)
        ((float *)a.Pc)[idx] = (float)(col[k] * Vp[p]);
      else
        ((double *)a.Pc)[idx] = col[k] * Vp[p];
    }
  }
}

}  // namespace

void launch_setup(int dim, int degree, const SetupArgs &a, cudaStream_t s) {
  const int block = 128;
  const unsigned grid = (unsigned)((a.N + block - 1) / block);
  if (dim == 2 && degree == 2) setup_kernel<2, 2><<<grid, block, 0, s>>>(a);
  if (dim == 2 && degree == 3) setup_kernel<2, 3><<<grid, block, 0, s>>>(a);
  if (dim == 3 && degree == 2) setup_kernel<3, 2><<<grid, block, 0, s>>>(a);
  if (dim == 3 && degree == 3) setup_kernel<3, 3><<<grid, block, 0, s>>>(a);
  if (dim == 2 && degree == 4) setup_kernel<2, 4><<<grid, block, 0, s>>>(a);
  if (dim == 2 && degree == 5) setup_kernel<2, 5><<<grid, block, 0, s>>>(a);
  if (dim == 2 && degree == 6) setup_kernel<2, 6><<<grid, block, 0, s>>>(a);
}

}  // namespace cteno
