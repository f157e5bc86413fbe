// tables.cpp -- universal constants of the reconstruction for one (d, r), built on the host.
//
// Everything here is a property of the reference simplex V0' (Sec. 2.1, eq. 5), the same for
// every cell: the basis psi_k of eq. 7 and its means, the smoothness matrix O of eq. 15
// (SI(p) = a^T O a), the face Gauss points expressed in reference coordinates for each ordering
// of a face's vertices, and a volume rule for the moments of eq. 10.
//
// Integrals over the reference simplex use the Dirichlet formula
//   int_{V0'} xi^a eta^b zeta^c = a! b! c! / (a + b + c + d)!.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cteno {
namespace {

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// int over V0' of xi^e (e[0..d-1]).
double ref_integral(const int *e, int d) {
  int tot = 0;
  double num = 1.0;
  for (int j = 0; j < d; ++j) {
    num *= fact(e[j]);
    tot += e[j];
  }
  return num / fact(tot + d);
}

// Two-point Gauss rule on [0,1] for the weight (1-u)^a: moments mu_k = k! a! / (k+a+1)!, the
// monic orthogonal quadratic u^2 + b u + c from the two orthogonality conditions, its roots as
// nodes, and weights matching mu_0 and mu_1. Exact for polynomials of degree 3 times the weight.
void gauss_jacobi2(int a, double x[2], double w[2]) {
  double mu[4];
  for (int k = 0; k < 4; ++k) mu[k] = fact(k) * fact(a) / fact(k + a + 1);
  // [mu1 mu0; mu2 mu1] [b; c] = -[mu2; mu3]
  double det = mu[1] * mu[1] - mu[0] * mu[2];
  double b = (-mu[2] * mu[1] + mu[3] * mu[0]) / det;
  double c = (-mu[3] * mu[1] + mu[2] * mu[2]) / det;
  double disc = std::sqrt(b * b / 4.0 - c);
  x[0] = -b / 2.0 - disc;
  x[1] = -b / 2.0 + disc;
  w[1] = (mu[1] - x[0] * mu[0]) / (x[1] - x[0]);
  w[0] = mu[0] - w[1];
}

// Jacobi polynomial P_n^(al,be)(x) on [-1,1] by its three-term recurrence.
double jacobi(int n, double al, double be, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = (al + 1.0) + 0.5 * (al + be + 2.0) * (x - 1.0);
  for (int k = 2; k <= n; ++k) {
    const double s = 2.0 * k + al + be;
    const double an = 2.0 * k * (k + al + be) * (s - 2.0);
    const double bn = (s - 1.0) * (s * (s - 2.0) * x + al * al - be * be);
    const double cn = 2.0 * (k + al - 1.0) * (k + be - 1.0) * s;
    const double p2 = (bn * p1 - cn * p0) / an;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// n-point Gauss rule on [0,1] for the weight (1-u)^a (exact for polynomials of degree 2n - 1
// times the weight). Nodes: the roots of P_n^(a,0) at x = 2u - 1, bracketed by sign changes on a
// fine grid and bisected to the last bit; weights 1 / ((1 - x^2) P_n'(x)^2), with
// P_n' = (n + a + 1)/2 P_{n-1}^(a+1,1) (the Gauss-Jacobi weight formula for beta = 0, mapped to
// [0,1]). For a = 0 (Gauss-Legendre) the rule is made exactly symmetric, x_{n-1-i} = -x_i.
void gauss_jacobi(int n, int a, double *u, double *w) {
  const int S = 4093;  // odd: no grid point falls on x = 0, a root of the odd Legendre polynomials
  double x[8];
  int found = 0;
  double xl = -1.0, pl = jacobi(n, a, 0.0, xl);
  for (int s = 1; s <= S && found < n; ++s) {
    const double xr = -1.0 + 2.0 * s / S, pr = jacobi(n, a, 0.0, xr);
    if ((pl < 0.0) != (pr < 0.0)) {
      double lo = xl, hi = xr, plo = pl;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double pm = jacobi(n, a, 0.0, mid);
        if (pm == 0.0) {
          lo = hi = mid;
          break;
        }
        if ((pm < 0.0) == (plo < 0.0)) {
          lo = mid;
          plo = pm;
        } else {
          hi = mid;
        }
      }
      x[found++] = 0.5 * (lo + hi);
    }
    xl = xr;
    pl = pr;
  }
  if (a == 0) {
    for (int i = 0; i < n / 2; ++i) x[n - 1 - i] = -x[i];
    if (n % 2) x[n / 2] = 0.0;
  }
  for (int i = 0; i < n; ++i) {
    const double dp = 0.5 * (n + a + 1.0) * jacobi(n - 1, a + 1.0, 1.0, x[i]);
    u[i] = 0.5 * (1.0 + x[i]);
    w[i] = 1.0 / ((1.0 - x[i] * x[i]) * dp * dp);
  }
  if (a == 0)
    for (int i = 0; i < n / 2; ++i) w[n - 1 - i] = w[i];
}

double eval_monomial(const int *e, const double *xi, int d) {
  double v = 1.0;
  for (int j = 0; j < d; ++j)
    for (int p = 0; p < e[j]; ++p) v *= xi[j];
  return v;
}

}  // namespace

void build_tables(int dim, int degree, Tables *t) {
  *t = Tables{};
  const int d = dim, r = degree;
  t->dim = d;
  t->degree = r;
  t->nf = d + 1;
  t->nq = face_points(d, r);
  // basis exponents, graded; within a degree ordered by the zeta then eta power
  int k = 0;
  for (int tdeg = 1; tdeg <= r; ++tdeg)
    for (int c = 0; c <= (d == 3 ? tdeg : 0); ++c)
      for (int b = 0; b <= tdeg - c; ++b) {
        t->ex[k][0] = tdeg - b - c;
        t->ex[k][1] = b;
        t->ex[k][2] = c;
        ++k;
      }
  t->nk = k;
  // means over V0' (|V0'| = 1/d!)
  for (int i = 0; i < k; ++i) t->psibar[i] = ref_integral(t->ex[i], d) * fact(d);
  // O_kl = sum_{1 <= |alpha| <= r} int_{V0'} D^alpha psi_k D^alpha psi_l
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int al = 0; al < k; ++al) {  // the multi-indices 1 <= |alpha| <= r are the exponents
        const int *A = t->ex[al];
        double ci = 1.0, cj = 1.0;
        int e[3] = {0, 0, 0};
        bool zero = false;
        for (int q = 0; q < d; ++q) {
          if (A[q] > t->ex[i][q] || A[q] > t->ex[j][q]) {
            zero = true;
            break;
          }
          ci *= fact(t->ex[i][q]) / fact(t->ex[i][q] - A[q]);
          cj *= fact(t->ex[j][q]) / fact(t->ex[j][q] - A[q]);
          e[q] = t->ex[i][q] - A[q] + t->ex[j][q] - A[q];
        }
        if (!zero) s += ci * cj * ref_integral(e, d);
      }
      t->O[i][j] = s;
    }
  // volume rule: collapsed coordinates, Gauss-Jacobi in each direction (2 points up to degree 3,
  // (r + 2) / 2 points from degree 4: exact to degree 2n - 1 >= r)
  if (d == 2 && r >= 4) {
    const int n = (r + 2) / 2;
    double xa[8], wa[8], xb[8], wb[8];
    gauss_jacobi(n, 1, xa, wa);
    gauss_jacobi(n, 0, xb, wb);
    int q = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        t->vq[q][0] = xa[i];
        t->vq[q][1] = xb[j] * (1.0 - xa[i]);
        t->vw[q] = wa[i] * wb[j];
        ++q;
      }
    t->nvq = q;
  } else {
    double xa[2], wa[2], xb[2], wb[2], xc[2], wc[2];
    if (d == 2) {
      gauss_jacobi2(1, xa, wa);
      gauss_jacobi2(0, xb, wb);
      int q = 0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          t->vq[q][0] = xa[i];
          t->vq[q][1] = xb[j] * (1.0 - xa[i]);
          t->vw[q] = wa[i] * wb[j];
          ++q;
        }
      t->nvq = 4;
    } else {
      gauss_jacobi2(2, xa, wa);
      gauss_jacobi2(1, xb, wb);
      gauss_jacobi2(0, xc, wc);
      int q = 0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int l = 0; l < 2; ++l) {
            t->vq[q][0] = xa[i];
            t->vq[q][1] = xb[j] * (1.0 - xa[i]);
            t->vq[q][2] = xc[l] * (1.0 - xa[i]) * (1.0 - xb[j]);
            t->vw[q] = wa[i] * wb[j] * wc[l];
            ++q;
          }
      t->nvq = 8;
    }
  }
  // face rule in barycentric coordinates of the face's vertices, sorted by global id:
  // 2D: n-point Gauss-Legendre along the edge (symmetric: the reversed edge visits the same
  // points in the opposite order); 3D: collapsed 2x2 (Gauss-Jacobi (1-u) x Legendre)
  double (&bary)[kMaxNQ][3] = t->fbary;
  if (d == 2 && t->nq > 2) {
    double xl[8], wl[8];
    gauss_jacobi(t->nq, 0, xl, wl);
    for (int q = 0; q < t->nq; ++q) {
      bary[q][0] = 1.0 - xl[q];
      bary[q][1] = xl[q];
      t->fw[q] = wl[q];
    }
  } else {
    double xl[2], wl[2], xj[2], wj[2];
    gauss_jacobi2(0, xl, wl);
    if (d == 2) {
      for (int q = 0; q < 2; ++q) {
        bary[q][0] = 1.0 - xl[q];
        bary[q][1] = xl[q];
        t->fw[q] = wl[q];
      }
    } else {
      gauss_jacobi2(1, xj, wj);
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int q = 2 * i + j;
          bary[q][0] = (1.0 - xj[i]) * (1.0 - xl[j]);
          bary[q][1] = xj[i];
          bary[q][2] = (1.0 - xj[i]) * xl[j];
          t->fw[q] = 2.0 * wj[i] * wl[j];
        }
    }
  }
  // permutations of the d face-vertex slots, lexicographic
  {
    int np = 0;
    if (d == 2) {
      int P[2][2] = {{0, 1}, {1, 0}};
      for (auto &p : P) {
        t->perm_list[np][0] = p[0];
        t->perm_list[np][1] = p[1];
        ++np;
      }
    } else {
      int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
      for (auto &p : P) {
        for (int j = 0; j < 3; ++j) t->perm_list[np][j] = p[j];
        ++np;
      }
    }
    t->nperm = np;
  }
  for (int f = 0; f < t->nf; ++f) {
    int slots[3], ns = 0;
    for (int a = 0; a <= d; ++a)
      if (a != f) slots[ns++] = a;
    for (int p = 0; p < t->nperm; ++p)
      for (int q = 0; q < t->nq; ++q) {
        double xi[3] = {0, 0, 0};
        for (int j = 0; j < d; ++j) {
          int a = slots[t->perm_list[p][j]];  // local vertex at sorted position j
          if (a > 0) xi[a - 1] += bary[q][j];  // reference vertex a is e_{a-1}; vertex 0 at 0
        }
        for (int i = 0; i < k; ++i)
          t->Phi[f][p][q][i] = eval_monomial(t->ex[i], xi, d) - t->psibar[i];
      }
  }
}

}  // namespace cteno
