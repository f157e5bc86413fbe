/*
 * cteno_oracle.c -- plain, slow FP64 CPU oracle of the CTENO / CTENOZ finite-volume scheme
 * for the compressible Euler equations on triangle (2D) and tetrahedron (3D) meshes
 * (Ma, Chong, Feng, Zhang, Wang, Zhou, "High-order finite-volume central targeted ENO family
 * scheme for compressible flows in unstructured meshes", arXiv 2312.17042).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py load this library. The CUDA library never includes, links or calls it, and this
 * file includes nothing of the CUDA library: the two share no code.
 *
 * Every routine follows one passage of the paper, cited in its comment, in the paper's order
 * and notation. Readings where the paper is silent or garbled are marked "Reading:"; the CUDA
 * library takes the same readings, in code of its own.
 *
 * Parity pins (tests/test_oracle_*.py): quadrature exactness against the Dirichlet monomial
 * integral; least squares against numpy.linalg.lstsq; polynomial reproduction; mean
 * preservation; free-stream preservation; HLLC consistency, symmetry, exact contact
 * resolution and the exact flux of an isolated shock (Roe averages); selection invariants and
 * closed-form flip points; conservation; convergence order on the
 * smooth density wave (Table 3 of the paper); Sod exact-solution envelope; the Euler flux
 * Jacobian's eigenvectors (they diagonalise it; smooth fields and contacts; Sod exact solution);
 * reflective walls (closed-box conservation, the exact reflected-shock state); the orders of
 * the RK3 and RK4 steps in time; which faces see the fixed and the moving-shock states. Altered
 * copies of this file (misread exponents, averages, cut-off, Roe averages, RK weights) must fail
 * those pins (tests/test_oracle_mutations.py).
 * Parity unpinned: the exact stencil membership (readings of the SBC and directional-stencil
 * rules, which the paper defers to its reference [30]) is fixed only by this file, and so is the
 * direction of the characteristic decomposition (each face's normal; the paper names none).
 *
 * Build: gcc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC (oracle/build_oracle.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define MAXD 3
#define MAXK 28   /* K(6,2) = K(3,3) + 8: coefficients of a sextic in 2D, constant included (eq. 6) */
#define MAXM 56   /* M = 2K (Sec. 2.1) */
#define MAXNF 4   /* faces of a simplex */
#define MAXDIR 10 /* Reading: at most 2 (K_dir - 1) cells in a directional stencil */
#define MAXKD 5   /* unknowns of a directional polynomial: degree 1 (d of them) or, for central
                     degree >= 4 in 2D, degree 2 (5 of them) */
#define MAXNQ 4   /* face Gauss points */
#define MAXNV 5   /* conserved variables */

/* ------------------------------------------------------------------------------------------ */
/* Parameters and state                                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int dim, degree, scheme; /* 0 = CTENO (Alg. 1), 1 = CTENOZ (Alg. 2), 2 = CWENO (Sec. 2.3), 3 = TENO (Sec. 2.4) */
  int guard;               /* Reading: positivity fall-back to the cell mean */
  int lam_gamma;           /* Reading: 1 = gamma_s carries lambda_s (eq. 18), 0 = as printed */
  int ctenoz_form;         /* Reading: 0 = CTENOZ measure as printed, 1 = WENO-Z form */
  int characteristic;      /* 1: reconstruct characteristic variables, per face (Sec. 2.2, 3.2) */
  int boundary;            /* boundary faces: 0 transmissive, 1 reflective walls (Sec. 3.3, 3.4) */
  int rk;                  /* Runge-Kutta scheme (Sec. 2, "3rd- or 4th-order"): 3 SSP-RK3, 4 classical RK4 */
  double C_T, lambda1p, eps, gamma, cfl;
} orc_params;

typedef struct {
  int ready;
  int nst;                      /* cells in the central stencil (M) */
  int ids[MAXM];                /* central stencil, nearest first */
  double shift[MAXM][MAXD];     /* periodic translation of each member into this cell's frame */
  double Vp[MAXM];              /* |V'_m| */
  double *A;                    /* [M][nk]: A_mk of eq. 10 (central) */
  double *R;                    /* [nk][nk]: Householder R of A (eq. 12) */
  double *V;                    /* [M][nk]: Householder vectors of that QR (column k, rows >= k) */
  double beta[MAXK];            /*   and their factors, H_k = I - beta_k v_k v_k^T */
  int ndir[MAXNF];              /* members of each directional stencil */
  int dmem[MAXNF][MAXDIR];      /* their positions in the central list */
  int dok[MAXNF];               /* admissible? */
  double dA[MAXNF][MAXDIR][MAXKD];
  double dR[MAXNF][MAXKD][MAXKD];
  double dV[MAXNF][MAXDIR][MAXKD];
  double dbeta[MAXNF][MAXKD];
} orc_cell;

typedef struct {
  orc_params p;
  int nverts, ncells, nv, nf, nq, nk; /* nk = K-1 unknowns of the central polynomial */
  int dk, ddeg, dmax;  /* directional polynomials: unknowns, degree, members kept */
  int M;
  double period[MAXD];
  double *xyz;         /* [nverts][dim] */
  int *cv;             /* [ncells][dim+1], positively oriented */
  double *X;           /* [ncells][dim+1][dim] unwrapped, oriented vertex coordinates */
  double *vol, *cen;   /* |V_i|, centroid */
  double *Jinv;        /* [ncells][dim][dim] inverse of the reference map Jacobian */
  double *detJ;
  int *nbr, *nbrf;     /* [ncells][nf] neighbour cell / its local face; -1 = boundary */
  signed char *bkind;  /* [ncells][nf] kind of a boundary face (BND_*) */
  double bstate[2][MAXNV]; /* conserved states A and B of the fixed-state and moving-shock kinds */
  double shock[3];     /* moving shock: A where xs0 + sy y + vs t > x at the face midpoint, else B */
  double time, stage_time; /* physical time at the start of the step / of the current stage */
  double *area, *nrm;  /* [ncells][nf], [ncells][nf][dim] outward unit normal */
  double *fq;          /* [ncells][nf][nq][dim] physical face Gauss points (canonical order) */
  double fw[MAXNQ];    /* face weights (sum 1) */
  int *v2c_off, *v2c;  /* vertex -> cells */
  orc_cell **cell;
  /* exponents of the basis monomials psi_k, k = 0..nk-1, graded, linear ones first (eq. 7) */
  int ex[MAXK][MAXD];
  double psibar[MAXK]; /* mean of psi_k over the reference simplex V0' (eq. 7) */
  /* quadrature on the unit simplex: barycentric points and weights summing to 1 */
  int nqv;
  double *qlam, *qw;
  /* solution */
  double *U, *Un, *Rres, *face; /* face: [ncells][nf][nq][nv] */
  double *Acc;                  /* RK4: U^n + dt/6 (k_1 + 2 k_2 + 2 k_3) so far */
  int nsel;                     /* selections per cell: nv, or nf * nv (characteristic) */
  uint8_t *flags;               /* [ncells][nsel]: bit 0 central selected, bit 1+f directional f */
  double *SI;                   /* [ncells][nv][1+nf] smoothness indicators (debug) */
  double *chi;                  /* [ncells][nv][1+nf] chi_s of eq. 22, 0 where inadmissible (debug) */
  double *coef;                 /* [ncells][nv][nk] final polynomial coefficients (debug) */
  int *stmask;                  /* [ncells]: bit 0 central, bit 1+f admissible directional f */
  uint8_t *guarded;             /* [ncells]: the last reconstruction fell back to the mean (debug) */
  int nguard;
  int err;
} orc;

/* ------------------------------------------------------------------------------------------ */
/* Small dense helpers                                                                         */
/* ------------------------------------------------------------------------------------------ */
static double det_d(int d, const double *J) { /* J row-major d x d */
  if (d == 2) return J[0] * J[3] - J[1] * J[2];
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

/* Solve J x = b by Cramer's rule (d = 2, 3). */
static void solve_d(int d, const double *J, const double *b, double *x) {
  double D = det_d(d, J);
  for (int c = 0; c < d; ++c) {
    double T[9];
    for (int r = 0; r < d; ++r)
      for (int k = 0; k < d; ++k) T[r * d + k] = (k == c) ? b[r] : J[r * d + k];
    x[c] = det_d(d, T) / D;
  }
}

static void inv_d(int d, const double *J, double *Ji) {
  for (int c = 0; c < d; ++c) {
    double e[3] = {0, 0, 0}, x[3];
    e[c] = 1.0;
    solve_d(d, J, e, x);
    for (int r = 0; r < d; ++r) Ji[r * d + c] = x[r];
  }
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on the Legendre polynomial
 * (three-term recurrence; textbook construction). */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      pp = n * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

/* Collapsed (Duffy) product rule on the unit simplex, barycentric points, weights sum 1;
 * exact for total degree 2*n - d. */
static void simplex_rule(int d, int n, double **lam_out, double **w_out, int *np_out) {
  double g[16], gw[16];
  gauss_legendre(n, g, gw);
  for (int i = 0; i < n; ++i) {
    g[i] = 0.5 * (g[i] + 1.0);
    gw[i] *= 0.5;
  }
  int np = (d == 2) ? n * n : n * n * n;
  double *lam = (double *)malloc(sizeof(double) * np * (d + 1));
  double *w = (double *)malloc(sizeof(double) * np);
  int q = 0;
  if (d == 2) {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double u = g[a], v = g[b];
        double x = u, y = v * (1.0 - u);
        lam[q * 3 + 0] = 1.0 - x - y;
        lam[q * 3 + 1] = x;
        lam[q * 3 + 2] = y;
        w[q] = gw[a] * gw[b] * (1.0 - u) * 2.0;
        ++q;
      }
  } else {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c) {
          double u = g[a], v = g[b], s = g[c];
          double x = u, y = v * (1.0 - u), z = s * (1.0 - u) * (1.0 - v);
          lam[q * 4 + 0] = 1.0 - x - y - z;
          lam[q * 4 + 1] = x;
          lam[q * 4 + 2] = y;
          lam[q * 4 + 3] = z;
          w[q] = gw[a] * gw[b] * gw[c] * (1.0 - u) * (1.0 - u) * (1.0 - v) * 6.0;
          ++q;
        }
  }
  *lam_out = lam;
  *w_out = w;
  *np_out = np;
}

/* ------------------------------------------------------------------------------------------ */
/* Basis (eqs. 6-7)                                                                            */
/* ------------------------------------------------------------------------------------------ */
/* K(r,d) = prod_{l=1..d} (r+l) / d!  counts all monomials of degree <= r, constant included
 * (eq. 6). Reading: the unknowns are the K-1 non-constant coefficients. */
static int K_of(int r, int d) {
  double k = 1.0;
  for (int l = 1; l <= d; ++l) k *= (r + l);
  return (int)(k / factorial(d) + 0.5);
}

/* psi_k = xi, eta, zeta, xi^2, eta^2, ... : monomials of total degree 1..r, graded (eq. 7). */
static int make_exponents(int d, int r, int ex[MAXK][MAXD]) {
  int k = 0;
  for (int t = 1; t <= r; ++t)
    for (int a = t; a >= 0; --a) {
      if (d == 2) {
        ex[k][0] = a;
        ex[k][1] = t - a;
        ex[k][2] = 0;
        ++k;
      } else {
        for (int b = t - a; b >= 0; --b) {
          ex[k][0] = a;
          ex[k][1] = b;
          ex[k][2] = t - a - b;
          ++k;
        }
      }
    }
  return k;
}

static double monomial(const int *e, const double *xi, int d) {
  double v = 1.0;
  for (int j = 0; j < d; ++j)
    for (int p = 0; p < e[j]; ++p) v *= xi[j];
  return v;
}

/* D^alpha psi at xi (0 where alpha exceeds the exponent). */
static double dmonomial(const int *e, const int *al, const double *xi, int d) {
  double c = 1.0;
  int r[MAXD] = {0, 0, 0};
  for (int j = 0; j < d; ++j) {
    if (al[j] > e[j]) return 0.0;
    for (int p = 0; p < al[j]; ++p) c *= (double)(e[j] - p);
    r[j] = e[j] - al[j];
  }
  return c * monomial(r, xi, d);
}

/* ------------------------------------------------------------------------------------------ */
/* Mesh and geometry (Sec. 2, eq. 2)                                                           */
/* ------------------------------------------------------------------------------------------ */
/* Translation by a whole number of periods bringing a point at offset dx next to the origin
 * (0 in a bounded direction). */
static double image_shift(double dx, double L) { return (L > 0.0) ? -L * round(dx / L) : 0.0; }

static int build_geometry(orc *o, const double *xyz, const int *cells) {
  const int d = o->p.dim, nvc = d + 1, n = o->ncells;
  o->cv = (int *)malloc(sizeof(int) * n * nvc);
  o->X = (double *)malloc(sizeof(double) * n * nvc * d);
  o->vol = (double *)malloc(sizeof(double) * n);
  o->cen = (double *)malloc(sizeof(double) * n * d);
  o->Jinv = (double *)malloc(sizeof(double) * n * d * d);
  o->detJ = (double *)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    int v[4];
    double X[4][3];
    for (int a = 0; a < nvc; ++a) v[a] = cells[i * nvc + a];
    /* unwrap periodic images next to local vertex 0: x - L round((x - x0) / L) */
    for (int a = 0; a < nvc; ++a)
      for (int j = 0; j < d; ++j) {
        double x0 = xyz[v[0] * d + j], x = xyz[v[a] * d + j];
        X[a][j] = x + image_shift(x - x0, o->period[j]);
      }
    double J[9];
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) J[r * d + c] = X[c + 1][r] - X[0][r];
    double D = det_d(d, J);
    if (D == 0.0) return -3;
    if (D < 0.0) { /* Reading: orient positively by swapping local vertices 1 and 2 */
      int t = v[1];
      v[1] = v[2];
      v[2] = t;
      for (int j = 0; j < d; ++j) {
        double s = X[1][j];
        X[1][j] = X[2][j];
        X[2][j] = s;
      }
      for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) J[r * d + c] = X[c + 1][r] - X[0][r];
      D = det_d(d, J);
    }
    for (int a = 0; a < nvc; ++a) {
      o->cv[i * nvc + a] = v[a];
      for (int j = 0; j < d; ++j) o->X[(i * nvc + a) * d + j] = X[a][j];
    }
    o->detJ[i] = D;
    o->vol[i] = D / factorial(d);
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int a = 0; a < nvc; ++a) s += X[a][j];
      o->cen[i * d + j] = s / nvc;
    }
    inv_d(d, J, o->Jinv + i * d * d);
  }
  return 0;
}

/* Faces: local face f is opposite local vertex f; matched across cells by sorted vertex ids. */
typedef struct {
  int key[3];
  int cell, f;
} face_rec;

static int cmp_face(const void *a, const void *b) {
  const face_rec *x = (const face_rec *)a, *y = (const face_rec *)b;
  for (int j = 0; j < 3; ++j)
    if (x->key[j] != y->key[j]) return x->key[j] < y->key[j] ? -1 : 1;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->f - y->f;
}

static void sort_ints(int *a, int n) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && a[j - 1] > a[j]; --j) {
      int t = a[j];
      a[j] = a[j - 1];
      a[j - 1] = t;
    }
}

/* Face Gauss points, canonical order from the sorted global vertex ids so that both cells of a
 * face enumerate the same physical points. Reading (quadrature "suited to the polynomial
 * order", Sec. 2 after eq. 2): 2D edges use 2-point Gauss-Legendre; 3D triangles use the
 * collapsed 2x2 rule (Gauss-Jacobi with weight (1-u) in u, Gauss-Legendre in v), exact for
 * degree 3. Weights sum to 1. */
static void face_rule(int d, int nq, double t[MAXNQ][3], double *w) {
  if (d == 2 && nq == 2) {
    double g = 1.0 / sqrt(3.0);
    t[0][0] = 0.5 * (1.0 - g); /* fraction along sorted edge a->b */
    t[1][0] = 0.5 * (1.0 + g);
    w[0] = w[1] = 0.5;
  } else if (d == 2) {
    double g[MAXNQ], gw[MAXNQ];
    gauss_legendre(nq, g, gw);
    for (int q = 0; q < nq; ++q) {
      t[q][0] = 0.5 * (1.0 + g[q]); /* fraction along sorted edge a->b, ascending */
      w[q] = 0.5 * gw[q];
    }
  } else {
    /* Gauss-Jacobi, weight (1-u) on [0,1]: roots of u^2 - 0.8 u + 0.1 */
    double u[2] = {0.4 - sqrt(0.06), 0.4 + sqrt(0.06)};
    double wu2 = (1.0 / 6.0 - 0.5 * u[0]) / (u[1] - u[0]);
    double wu[2] = {0.5 - wu2, wu2};
    double g = 1.0 / sqrt(3.0);
    double v[2] = {0.5 * (1.0 - g), 0.5 * (1.0 + g)};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        int q = 2 * i + j;
        /* barycentric (lambda_a, lambda_b, lambda_c) = ((1-u)(1-v), u, (1-u) v) */
        t[q][0] = (1.0 - u[i]) * (1.0 - v[j]);
        t[q][1] = u[i];
        t[q][2] = (1.0 - u[i]) * v[j];
        w[q] = wu[i] * 0.5 * 2.0;
      }
  }
}

/* Boundary face kinds. Reading (the paper runs walls, inflow and a moving-shock top boundary in
 * Sec. 3.3 / 3.4 without printing their treatment): transmissive, the outside state is the cell
 * mean; wall, the mirror image of the reconstructed inside state; fixed state A; moving shock,
 * state A on the side of the shock line x = xs0 + sy y + vs t where x is smaller, else B, decided
 * at the face midpoint. */
enum { BND_TRANSMISSIVE = 0, BND_WALL = 1, BND_STATE_A = 2, BND_SHOCK_AB = 3 };

static int build_faces(orc *o) {
  const int d = o->p.dim, nvc = d + 1, n = o->ncells, nf = o->nf;
  face_rec *fr = (face_rec *)malloc(sizeof(face_rec) * (size_t)n * nf);
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < nf; ++f) {
      face_rec *r = &fr[i * nf + f];
      int k = 0;
      for (int a = 0; a < nvc; ++a)
        if (a != f) r->key[k++] = o->cv[i * nvc + a];
      if (d == 2) r->key[2] = -1;
      sort_ints(r->key, d);
      r->cell = i;
      r->f = f;
    }
  qsort(fr, (size_t)n * nf, sizeof(face_rec), cmp_face);
  o->nbr = (int *)malloc(sizeof(int) * n * nf);
  o->nbrf = (int *)malloc(sizeof(int) * n * nf);
  for (int k = 0; k < n * nf; ++k) o->nbr[k] = o->nbrf[k] = -1;
  for (size_t k = 0; k < (size_t)n * nf;) {
    size_t e = k + 1;
    while (e < (size_t)n * nf && memcmp(fr[e].key, fr[k].key, sizeof(int) * 3) == 0) ++e;
    if (e - k > 2) {
      free(fr);
      return -4; /* non-manifold */
    }
    if (e - k == 2) {
      o->nbr[fr[k].cell * nf + fr[k].f] = fr[k + 1].cell;
      o->nbrf[fr[k].cell * nf + fr[k].f] = fr[k + 1].f;
      o->nbr[fr[k + 1].cell * nf + fr[k + 1].f] = fr[k].cell;
      o->nbrf[fr[k + 1].cell * nf + fr[k + 1].f] = fr[k].f;
    }
    k = e;
  }
  free(fr);
  /* outward unit normals, areas, canonical Gauss points */
  double t[MAXNQ][3];
  face_rule(d, o->nq, t, o->fw);
  o->area = (double *)malloc(sizeof(double) * n * nf);
  o->nrm = (double *)malloc(sizeof(double) * n * nf * d);
  o->fq = (double *)malloc(sizeof(double) * n * nf * o->nq * d);
  for (int i = 0; i < n; ++i) {
    const double *X = o->X + (size_t)i * nvc * d;
    for (int f = 0; f < nf; ++f) {
      int loc[3], k = 0;
      for (int a = 0; a < nvc; ++a)
        if (a != f) loc[k++] = a;
      double nv_[3];
      if (d == 2) {
        double ex = X[loc[1] * 2] - X[loc[0] * 2], ey = X[loc[1] * 2 + 1] - X[loc[0] * 2 + 1];
        nv_[0] = ey;
        nv_[1] = -ex;
        o->area[i * nf + f] = sqrt(ex * ex + ey * ey);
      } else {
        double a[3], b[3];
        for (int j = 0; j < 3; ++j) {
          a[j] = X[loc[1] * 3 + j] - X[loc[0] * 3 + j];
          b[j] = X[loc[2] * 3 + j] - X[loc[0] * 3 + j];
        }
        nv_[0] = a[1] * b[2] - a[2] * b[1];
        nv_[1] = a[2] * b[0] - a[0] * b[2];
        nv_[2] = a[0] * b[1] - a[1] * b[0];
        o->area[i * nf + f] = 0.5 * sqrt(nv_[0] * nv_[0] + nv_[1] * nv_[1] + nv_[2] * nv_[2]);
      }
      double len = 0.0, dot = 0.0;
      for (int j = 0; j < d; ++j) len += nv_[j] * nv_[j];
      len = sqrt(len);
      for (int j = 0; j < d; ++j) dot += nv_[j] * (X[loc[0] * d + j] - X[f * d + j]);
      double sgn = (dot > 0.0) ? 1.0 : -1.0;
      for (int j = 0; j < d; ++j) o->nrm[(i * nf + f) * d + j] = sgn * nv_[j] / len;
      /* sorted-id order of the face vertices */
      int ord[3] = {loc[0], loc[1], d == 3 ? loc[2] : -1};
      for (int p = 1; p < d; ++p)
        for (int q2 = p; q2 > 0 && o->cv[i * nvc + ord[q2 - 1]] > o->cv[i * nvc + ord[q2]]; --q2) {
          int tt = ord[q2];
          ord[q2] = ord[q2 - 1];
          ord[q2 - 1] = tt;
        }
      for (int q = 0; q < o->nq; ++q)
        for (int j = 0; j < d; ++j) {
          double x;
          if (d == 2)
            x = (1.0 - t[q][0]) * X[ord[0] * 2 + j] + t[q][0] * X[ord[1] * 2 + j];
          else
            x = t[q][0] * X[ord[0] * 3 + j] + t[q][1] * X[ord[1] * 3 + j] +
                t[q][2] * X[ord[2] * 3 + j];
          o->fq[((size_t)(i * nf + f) * o->nq + q) * d + j] = x;
        }
    }
  }
  /* vertex -> cells */
  o->v2c_off = (int *)calloc(o->nverts + 1, sizeof(int));
  for (int k = 0; k < n * nvc; ++k) o->v2c_off[o->cv[k] + 1]++;
  for (int v = 0; v < o->nverts; ++v) o->v2c_off[v + 1] += o->v2c_off[v];
  o->v2c = (int *)malloc(sizeof(int) * n * nvc);
  int *fill = (int *)calloc(o->nverts, sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < nvc; ++a) {
      int v = o->cv[i * nvc + a];
      o->v2c[o->v2c_off[v] + fill[v]++] = i;
    }
  free(fill);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Stencils (Sec. 2.1 "SBC" central stencil of M = 2K cells; Sec. 2.3 / Fig. 1 directional)    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double dist2;
  int id;
  double sh[MAXD];
} cand;

static int cmp_cand(const void *a, const void *b) {
  const cand *x = (const cand *)a, *y = (const cand *)b;
  if (x->dist2 != y->dist2) return x->dist2 < y->dist2 ? -1 : 1;
  return x->id - y->id;
}

/* Reading of the SBC rule: gather cells layer by layer through shared vertices until at least
 * M candidates (target excluded) are known, then keep the M nearest by centroid distance in the
 * target's periodic frame, ties to the lower cell id. */
static int hset_insert(int *tab, int cap, int key) { /* 1 if newly inserted */
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(cap - 1);
  while (tab[h] != -1) {
    if (tab[h] == key) return 0;
    h = (h + 1) & (unsigned)(cap - 1);
  }
  tab[h] = key;
  return 1;
}

static int central_stencil(orc *o, int i, orc_cell *c) {
  const int d = o->p.dim, nvc = d + 1, M = o->M;
  int cap = 4096, nc = 0, hcap = 1 << 14;
  int *list = (int *)malloc(sizeof(int) * cap);
  int *seen = (int *)malloc(sizeof(int) * hcap);
  for (int k = 0; k < hcap; ++k) seen[k] = -1;
  int layer_lo = 0, layer_hi = 0;
  list[nc++] = i;
  hset_insert(seen, hcap, i);
  layer_hi = nc;
  while (nc - 1 < M) {
    int before = nc;
    for (int k = layer_lo; k < layer_hi; ++k) {
      int cc = list[k];
      for (int a = 0; a < nvc; ++a) {
        int v = o->cv[cc * nvc + a];
        for (int t = o->v2c_off[v]; t < o->v2c_off[v + 1]; ++t) {
          int m = o->v2c[t];
          if (!hset_insert(seen, hcap, m)) continue;
          if (nc == cap || nc >= hcap / 2) {
            free(list);
            free(seen);
            return -5;
          }
          list[nc++] = m;
        }
      }
    }
    if (nc == before) {
      free(list);
      free(seen);
      return -5; /* mesh too small for M */
    }
    layer_lo = layer_hi;
    layer_hi = nc;
  }
  free(seen);
  cand *cs = (cand *)malloc(sizeof(cand) * nc);
  int ncs = 0;
  for (int k = 1; k < nc; ++k) {
    int m = list[k];
    cand *q = &cs[ncs++];
    q->id = m;
    q->dist2 = 0.0;
    for (int j = 0; j < d; ++j) {
      q->sh[j] = image_shift(o->cen[m * d + j] - o->cen[i * d + j], o->period[j]);
      double w = (o->cen[m * d + j] + q->sh[j]) - o->cen[i * d + j];
      q->dist2 += w * w;
    }
  }
  qsort(cs, ncs, sizeof(cand), cmp_cand);
  c->nst = M;
  for (int k = 0; k < M; ++k) {
    c->ids[k] = cs[k].id;
    for (int j = 0; j < d; ++j) {
      c->shift[k][j] = cs[k].sh[j];
      if (o->period[j] > 0.0) {
        double dx = o->cen[cs[k].id * d + j] + cs[k].sh[j] - o->cen[i * d + j];
        if (fabs(dx) > 0.4 * o->period[j]) {
          free(cs);
          free(list);
          return -6; /* periodic mesh too coarse for the stencil */
        }
      }
    }
  }
  free(cs);
  free(list);
  return 0;
}

/* Reading of the directional ("Type 3", compact) stencils, Fig. 1 (c): one per face; a member of
 * the central stencil belongs to the stencil of face f when its centroid lies in the cone from
 * the target centroid through the vertices of face f (all cone coordinates >= 0); a centroid on a
 * shared cone boundary goes to the lowest face index; each stencil keeps its first 2d members
 * in central-list order (nearest first). Degree 1. */
static void directional_stencils(orc *o, int i, orc_cell *c) {
  const int d = o->p.dim, nvc = d + 1, nf = o->nf;
  const double *X = o->X + (size_t)i * nvc * d, *ci = o->cen + i * d;
  for (int f = 0; f < nf; ++f) c->ndir[f] = 0;
  for (int k = 0; k < c->nst; ++k) {
    int m = c->ids[k];
    double dc[3];
    for (int j = 0; j < d; ++j) dc[j] = o->cen[m * d + j] + c->shift[k][j] - ci[j];
    for (int f = 0; f < nf; ++f) {
      double Rm[9]; /* columns: rays to the face vertices */
      int col = 0;
      for (int a = 0; a < nvc; ++a) {
        if (a == f) continue;
        for (int j = 0; j < d; ++j) Rm[j * d + col] = X[a * d + j] - ci[j];
        ++col;
      }
      double beta[3];
      solve_d(d, Rm, dc, beta);
      int inside = 1;
      for (int j = 0; j < d; ++j)
        if (beta[j] < 0.0) inside = 0;
      if (inside) {
        if (c->ndir[f] < o->dmax) c->dmem[f][c->ndir[f]++] = k;
        break;
      }
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Least squares in reference space (eqs. 5, 7-12)                                             */
/* ------------------------------------------------------------------------------------------ */
/* Map the vertices of stencil member k into the target's reference space (eq. 5):
 * xi = J^-1 (x - x_v0). */
static void member_ref_vertices(orc *o, int i, const orc_cell *c, int k, double xi[4][3]) {
  const int d = o->p.dim, nvc = d + 1, m = c->ids[k];
  const double *Xm = o->X + (size_t)m * nvc * d, *X0 = o->X + (size_t)i * nvc * d;
  const double *Ji = o->Jinv + i * d * d;
  for (int a = 0; a < nvc; ++a) {
    double y[3];
    for (int j = 0; j < d; ++j) y[j] = Xm[a * d + j] + c->shift[k][j] - X0[j];
    for (int r = 0; r < d; ++r) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) s += Ji[r * d + j] * y[j];
      xi[a][r] = s;
    }
  }
}

/* A_mk = int_{V'_m} phi_k with phi_k = psi_k - mean_{V0'} psi_k (eqs. 7, 10), exact by
 * quadrature of degree >= r on the mapped simplex; also |V'_m|. */
static void moments(orc *o, double xi[4][3], int nk, double *Arow, double *Vp) {
  const int d = o->p.dim, nvc = d + 1;
  double J[9];
  for (int r = 0; r < d; ++r)
    for (int cc = 0; cc < d; ++cc) J[r * d + cc] = xi[cc + 1][r] - xi[0][r];
  double vol = fabs(det_d(d, J)) / factorial(d);
  for (int k = 0; k < nk; ++k) Arow[k] = 0.0;
  for (int q = 0; q < o->nqv; ++q) {
    double p[3] = {0, 0, 0};
    for (int a = 0; a < nvc; ++a)
      for (int j = 0; j < d; ++j) p[j] += o->qlam[q * nvc + a] * xi[a][j];
    for (int k = 0; k < nk; ++k) Arow[k] += o->qw[q] * monomial(o->ex[k], p, d);
  }
  for (int k = 0; k < nk; ++k) Arow[k] = vol * (Arow[k] - o->psibar[k]);
  *Vp = vol;
}

/* Householder QR of the m x n matrix A (Golub & Van Loan, Alg. 5.2.1), returning R (n x n)
 * and the rank test min|R_kk| > 1e-10 max|R_kk|. */
/* Householder QR of the m x n matrix A (m >= n): A = Q R with Q = H_0 H_1 ... H_{n-1},
 * H_k = I - beta_k v_k v_k^T. Stores R (n x n, upper) and the vectors v_k (column k of V, rows
 * k..m-1). Returns 1 if A has numerically full column rank (min |R_kk| > 1e-10 max |R_kk|). */
static int householder_qr(int m, int n, const double *A, int lda, double *V, int ldv, double *beta,
                          double *R, int ldr) {
  double W[MAXM][MAXK];
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < n; ++k) W[r][k] = A[r * lda + k];
  for (int k = 0; k < n; ++k) {
    for (int r = 0; r < m; ++r) V[r * ldv + k] = 0.0;
    beta[k] = 0.0;
    double nrm = 0.0;
    for (int r = k; r < m; ++r) nrm += W[r][k] * W[r][k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) continue;
    double alpha = (W[k][k] > 0.0) ? -nrm : nrm;
    double v[MAXM];
    for (int r = k; r < m; ++r) v[r] = W[r][k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int r = k; r < m; ++r) vv += v[r] * v[r];
    if (vv == 0.0) continue;
    for (int r = k; r < m; ++r) V[r * ldv + k] = v[r];
    beta[k] = 2.0 / vv;
    for (int cc = k; cc < n; ++cc) {
      double s = 0.0;
      for (int r = k; r < m; ++r) s += v[r] * W[r][cc];
      s *= beta[k];
      for (int r = k; r < m; ++r) W[r][cc] -= s * v[r];
    }
  }
  double mx = 0.0, mn = 1e300;
  for (int r = 0; r < n; ++r)
    for (int cc = 0; cc < n; ++cc) R[r * ldr + cc] = (cc >= r) ? W[r][cc] : 0.0;
  for (int r = 0; r < n; ++r) {
    double a = fabs(R[r * ldr + r]);
    if (a > mx) mx = a;
    if (a < mn) mn = a;
  }
  return (m >= n && mx > 0.0 && mn > 1e-10 * mx) ? 1 : 0;
}

/* The least-squares solution of eq. 12, a = (A^T A)^-1 A^T b, through the QR of A: y = Q^T b
 * (the reflectors applied in order), then R a = y_{0..n-1} by back substitution. */
static void lsq_solve(int m, int n, const double *V, int ldv, const double *beta, const double *R, int ldr,
                      const double *b, double *a) {
  double y[MAXM];
  for (int r = 0; r < m; ++r) y[r] = b[r];
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int r = k; r < m; ++r) s += V[r * ldv + k] * y[r];
    s *= beta[k];
    for (int r = k; r < m; ++r) y[r] -= s * V[r * ldv + k];
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = y[k];
    for (int j = k + 1; j < n; ++j) s -= R[k * ldr + j] * a[j];
    a[k] = s / R[k * ldr + k];
  }
}

static int cell_setup(orc *o, int i) {
  orc_cell *c = o->cell[i];
  if (c && c->ready) return 0;
  if (!c) {
    c = (orc_cell *)calloc(1, sizeof(orc_cell));
    o->cell[i] = c;
  }
  int rc = central_stencil(o, i, c);
  if (rc) return rc;
  directional_stencils(o, i, c);
  const int nk = o->nk;
  if (!c->A) c->A = (double *)malloc(sizeof(double) * c->nst * nk);
  if (!c->R) c->R = (double *)malloc(sizeof(double) * nk * nk);
  if (!c->V) c->V = (double *)malloc(sizeof(double) * c->nst * nk);
  for (int k = 0; k < c->nst; ++k) {
    double xi[4][3];
    member_ref_vertices(o, i, c, k, xi);
    moments(o, xi, nk, c->A + k * nk, &c->Vp[k]);
  }
  if (!householder_qr(c->nst, nk, c->A, nk, c->V, nk, c->beta, c->R, nk)) return -7;
  const int dk = o->dk;
  for (int f = 0; f < o->nf; ++f) {
    /* directional polynomial of degree 1 (or 2): its dk unknowns are the coefficients of the
     * first dk basis functions (graded), whose moments are the first dk columns of the central
     * A rows */
    for (int j = 0; j < c->ndir[f]; ++j)
      for (int k = 0; k < dk; ++k) c->dA[f][j][k] = c->A[c->dmem[f][j] * nk + k];
    c->dok[f] = (c->ndir[f] >= dk) &&
                householder_qr(c->ndir[f], dk, &c->dA[f][0][0], MAXKD, &c->dV[f][0][0], MAXKD, c->dbeta[f],
                               &c->dR[f][0][0], MAXKD);
  }
  c->ready = 1;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Reconstruction of one cell (eqs. 15-18, CTENO Alg. 1, CTENOZ Alg. 2)                        */
/* ------------------------------------------------------------------------------------------ */
/* SI = sum_{1<=|alpha|<=deg} int_{V0'} (D^alpha p)^2  (eq. 15). Reading: each multi-index is
 * counted once; integral over the reference simplex, not normalised. */
static double smoothness(orc *o, const double *a, int nterms, int deg) {
  const int d = o->p.dim, nvc = d + 1;
  const double v0 = 1.0 / factorial(d);
  double si = 0.0;
  for (int t = 0; t < o->nk; ++t) { /* alpha runs over the same exponent set, |alpha| <= deg */
    const int *al = o->ex[t];
    int na = al[0] + al[1] + al[2];
    if (na > deg) continue;
    double s = 0.0;
    for (int q = 0; q < o->nqv; ++q) {
      double xi[3] = {0, 0, 0};
      for (int aa = 1; aa < nvc; ++aa) xi[aa - 1] = o->qlam[q * nvc + aa];
      double v = 0.0;
      for (int k = 0; k < nterms; ++k) v += a[k] * dmonomial(o->ex[k], al, xi, d);
      s += o->qw[q] * v * v;
    }
    si += v0 * s;
  }
  return si;
}

static double pressure(const orc *o, const double *u) {
  const int d = o->p.dim;
  double ke = 0.0;
  for (int j = 0; j < d; ++j) ke += u[1 + j] * u[1 + j];
  return (o->p.gamma - 1.0) * (u[d + 1] - 0.5 * ke / u[0]);
}

/* Scale separation, smoothness measure and cut-off of one cell and one variable (Sec. 2.4-2.6),
 * or the nonlinear weights of CWENO (Sec. 2.2-2.3).
 * Stencil s = 0 is the central one (SI[0] = SI of p_1), s = 1 .. st-1 the admissible directional
 * ones, so st is s_t. Linear coefficients of eq. 18: lambda_1 = 1 - 1/lambda_1' and
 * lambda_s = (1 - lambda_1) / (s_t - 1).
 *   CWENO (eqs. 13-14 with the linear coefficients of eq. 18): w~_s = lambda_s / (eps + SI_s)^b,
 *     b = 4, w_s = w~_s / sum_t w~_t. chi[] receives w_s, and every stencil is kept (all bits).
 *   TENO (eqs. 19-23): gamma_s = 1 / (SI_s + eps)^6 as printed (TENO has no linear coefficients).
 *   CTENO (Alg. 1):  gamma_s = 1 / (SI_s + eps)^6.
 *   CTENOZ (Alg. 2): tau = (sum_{s>=2} |SI_s - SI_1| / (s_t - 1))^6, gamma_s = 1 + tau / (SI_s + eps).
 *     Reading (ctenoz_form = 1, not the printed form): the WENO-Z arrangement, with the power on
 *     the ratio, tau = sum_{s>=2} |SI_s - SI_1| / (s_t - 1), gamma_s = 1 + (tau / (SI_s + eps))^6.
 *   Reading (lam_gamma = 1): gamma_s is multiplied by lambda_s, the CWENO weight form of eq. 14;
 *     without it lambda_1' could not influence the selection, which Tables 1 and 3 show it does.
 * Then chi_s = gamma_s / sum_t gamma_t (eq. 22) and delta_s = 0 iff chi_s < C_T (eq. 23).
 * Writes chi[0 .. st-1] and returns the delta bits (bit s = delta of stencil s). */
static unsigned select_stencils(const orc_params *p, int st, const double *SI, double *chi) {
  const double lam1 = 1.0 - 1.0 / p->lambda1p;
  const double lams = (st > 1) ? (1.0 - lam1) / (st - 1) : 0.0;
  double gam[1 + MAXNF], sum = 0.0;
  if (p->scheme == 2) { /* CWENO: nonlinear weights, every stencil contributes */
    for (int s = 0; s < st; ++s) gam[s] = ((s == 0) ? lam1 : lams) / pow(p->eps + SI[s], 4.0);
    for (int s = 0; s < st; ++s) sum += gam[s];
    for (int s = 0; s < st; ++s) chi[s] = gam[s] / sum;
    return (1u << st) - 1u;
  }
  if (p->scheme == 0 || p->scheme == 3) {
    for (int s = 0; s < st; ++s) gam[s] = 1.0 / pow(SI[s] + p->eps, 6.0);
  } else {
    double tau = 0.0;
    if (st > 1) {
      double acc = 0.0;
      for (int s = 1; s < st; ++s) acc += fabs(SI[s] - SI[0]);
      tau = acc / (st - 1);
      if (p->ctenoz_form == 0) tau = pow(tau, 6.0);
    }
    for (int s = 0; s < st; ++s) {
      if (p->ctenoz_form == 0) gam[s] = 1.0 + tau / (SI[s] + p->eps);
      else gam[s] = 1.0 + pow(tau / (SI[s] + p->eps), 6.0);
    }
  }
  if (p->lam_gamma && p->scheme != 3)
    for (int s = 0; s < st; ++s) gam[s] *= (s == 0) ? lam1 : lams;
  for (int s = 0; s < st; ++s) sum += gam[s];
  unsigned bits = 0;
  for (int s = 0; s < st; ++s) {
    chi[s] = gam[s] / sum;                    /* eq. 22 */
    if (!(chi[s] < p->C_T)) bits |= 1u << s;  /* eq. 23 */
  }
  return bits;
}

/* Right (columns) and left (rows) eigenvectors of the Euler flux Jacobian dF(U).n/dU at the
 * conserved state u, for the unit direction n: the characteristic variables W = L U in which Sec.
 * 2.2 and Sec. 3.2 reconstruct. Fields in the order of the eigenvalues u_n - c, u_n (entropy),
 * u_n (shear: one per tangent t_j of an orthonormal frame n, t_1 .. t_{d-1}), u_n + c; with
 * H = (E + p)/rho, q^2 = |u|^2, b1 = (gamma - 1)/c^2, b2 = b1 q^2/2:
 *   r_0 = (1, u - c n, H - c u_n)           l_0 = (b2 + u_n/c, -b1 u - n/c, b1) / 2
 *   r_1 = (1, u, q^2/2)                     l_1 = (1 - b2, b1 u, -b1)
 *   r_1+j = (0, t_j, u.t_j)                 l_1+j = (-u.t_j, t_j, 0)
 *   r_d+1 = (1, u + c n, H + c u_n)         l_d+1 = (b2 - u_n/c, -b1 u + n/c, b1) / 2
 * Reading: the tangents are t = (-n_y, n_x) in 2D; in 3D t_1 is the component of the axis along
 * which |n| is smallest orthogonal to n, normalised, and t_2 = n x t_1. */
static void euler_eigen(const orc *o, const double *u, const double *n, double R[MAXNV][MAXNV],
                        double L[MAXNV][MAXNV]) {
  const int d = o->p.dim, nv = o->nv;
  const double g = o->p.gamma, rho = u[0];
  double vel[3] = {0, 0, 0}, q2 = 0.0, un = 0.0;
  for (int j = 0; j < d; ++j) {
    vel[j] = u[1 + j] / rho;
    q2 += vel[j] * vel[j];
    un += vel[j] * n[j];
  }
  const double p = pressure(o, u), c = sqrt(g * p / rho), H = (u[d + 1] + p) / rho;
  const double b1 = (g - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
  double t[2][3] = {{0, 0, 0}, {0, 0, 0}};
  if (d == 2) {
    t[0][0] = -n[1];
    t[0][1] = n[0];
  } else {
    int a = 0;
    for (int j = 1; j < 3; ++j)
      if (fabs(n[j]) < fabs(n[a])) a = j;
    double len = 0.0;
    for (int j = 0; j < 3; ++j) {
      t[0][j] = (j == a ? 1.0 : 0.0) - n[a] * n[j];
      len += t[0][j] * t[0][j];
    }
    len = sqrt(len);
    for (int j = 0; j < 3; ++j) t[0][j] /= len;
    t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
    t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
    t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
  }
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) R[a][b] = L[a][b] = 0.0;
  R[0][0] = 1.0;
  R[0][1] = 1.0;
  R[0][d + 1] = 1.0;
  for (int j = 0; j < d; ++j) {
    R[1 + j][0] = vel[j] - c * n[j];
    R[1 + j][1] = vel[j];
    R[1 + j][d + 1] = vel[j] + c * n[j];
  }
  R[d + 1][0] = H - c * un;
  R[d + 1][1] = 0.5 * q2;
  R[d + 1][d + 1] = H + c * un;
  L[0][0] = 0.5 * (b2 + un / c);
  L[1][0] = 1.0 - b2;
  L[d + 1][0] = 0.5 * (b2 - un / c);
  for (int j = 0; j < d; ++j) {
    L[0][1 + j] = 0.5 * (-b1 * vel[j] - n[j] / c);
    L[1][1 + j] = b1 * vel[j];
    L[d + 1][1 + j] = 0.5 * (-b1 * vel[j] + n[j] / c);
  }
  L[0][d + 1] = 0.5 * b1;
  L[1][d + 1] = -b1;
  L[d + 1][d + 1] = 0.5 * b1;
  for (int m = 0; m < d - 1; ++m) { /* shear fields */
    double ut = 0.0;
    for (int j = 0; j < d; ++j) ut += vel[j] * t[m][j];
    for (int j = 0; j < d; ++j) {
      R[1 + j][2 + m] = t[m][j];
      L[2 + m][1 + j] = t[m][j];
    }
    R[d + 1][2 + m] = ut;
    L[2 + m][0] = -ut;
  }
}

/* p_1, smoothness indicators, scale separation, cut-off and final polynomial (Sec. 2.3-2.6, eqs.
 * 15-23, Alg. 1 / 2, CWENO eq. 14) of one cell for one variable (or characteristic field) from its
 * central least-squares coefficients aopt and directional ones ad (admissible stencils adm[0..na));
 * debug records at selection index sel. Returns the flags byte; af receives the final
 * coefficients. */
static uint8_t weigh(orc *o, int i, int sel, int na, const int *adm, const double *aopt,
                     double ad[][MAXKD], double *af) {
  const int nf = o->nf, nk = o->nk, st = 1 + na;
  const double lam1 = 1.0 - 1.0 / o->p.lambda1p;
  const double lams = (st > 1) ? (1.0 - lam1) / (st - 1) : 0.0; /* eq. 18 */
  /* p_1 = (p_opt - sum_{s>=2} lambda_s p_s) / lambda_1  (eq. 17); the directional
   * polynomials only have the first dk coefficients, so only those receive their terms; TENO
   * keeps p_1 = p_opt */
  double a1[MAXK];
  if (st > 1 && o->p.scheme != 3) { /* TENO keeps the central polynomial itself (Sec. 2.4) */
    for (int k = 0; k < nk; ++k) {
      double s = aopt[k];
      if (k < o->dk)
        for (int t = 0; t < na; ++t) s -= lams * ad[adm[t]][k];
      a1[k] = s / lam1;
    }
  } else {
    for (int k = 0; k < nk; ++k) a1[k] = aopt[k];
  }
  /* smoothness indicators (eq. 15) of p_1 and of the directional polynomials */
  double SI[1 + MAXNF];
  SI[0] = smoothness(o, a1, nk, o->p.degree);
  for (int s = 0; s < na; ++s) SI[1 + s] = smoothness(o, ad[adm[s]], o->dk, o->ddeg);
  double *si_out = o->SI + ((size_t)i * o->nsel + sel) * (1 + nf);
  for (int s = 0; s <= nf; ++s) si_out[s] = 0.0;
  si_out[0] = SI[0];
  for (int s = 0; s < na; ++s) si_out[1 + adm[s]] = SI[1 + s];
  /* scale separation and cut-off (eqs. 19-23, Alg. 1 / Alg. 2) */
  double chi[1 + MAXNF];
  const unsigned dbits = select_stencils(&o->p, st, SI, chi);
  double *chi_out = o->chi + ((size_t)i * o->nsel + sel) * (1 + nf);
  for (int s = 0; s <= nf; ++s) chi_out[s] = 0.0;
  chi_out[0] = chi[0];
  for (int s = 0; s < na; ++s) chi_out[1 + adm[s]] = chi[1 + s];
  int delta[1 + MAXNF] = {0, 0, 0, 0, 0}, ndel = 0;
  for (int s = 0; s < st; ++s) {
    delta[s] = (dbits >> s) & 1u;
    if (s > 0) ndel += delta[s];
  }
  /* final polynomial: CWENO sum_s w_s p_s (Sec. 2.3); otherwise p_1 if delta_1, else
   * sum_{s>=2} delta_s p_s / sum delta_s (Alg. 1 / 2) */
  uint8_t fl = 0;
  if (o->p.scheme == 2) {
    for (int k = 0; k < nk; ++k) af[k] = chi[0] * a1[k];
    for (int s = 1; s < st; ++s)
      for (int k = 0; k < o->dk; ++k) af[k] += chi[s] * ad[adm[s - 1]][k];
    fl = (uint8_t)(o->stmask[i] & 0xFF);
  } else if (delta[0]) {
    for (int k = 0; k < nk; ++k) af[k] = a1[k];
    fl = 1;
  } else {
    for (int k = 0; k < nk; ++k) af[k] = 0.0;
    for (int s = 1; s < st; ++s)
      if (delta[s]) {
        for (int k = 0; k < o->dk; ++k) af[k] += ad[adm[s - 1]][k] / (double)ndel;
        fl |= (uint8_t)(1 << (1 + adm[s - 1]));
      }
  }
  o->flags[(size_t)i * o->nsel + sel] = fl;
  for (int k = 0; k < nk; ++k) o->coef[((size_t)i * o->nsel + sel) * nk + k] = af[k];
  return fl;
}

/* Value of the polynomial mean + sum_k a_k phi_k at Gauss point q of face f of cell i (eqs. 7, 2). */
static double face_value(const orc *o, int i, int f, int q, double mean, const double *af) {
  const int d = o->p.dim;
  const double *X0 = o->X + (size_t)i * (d + 1) * d, *Ji = o->Jinv + i * d * d;
  const double *x = o->fq + ((size_t)(i * o->nf + f) * o->nq + q) * d;
  double xi[3] = {0, 0, 0};
  for (int r = 0; r < d; ++r)
    for (int j = 0; j < d; ++j) xi[r] += Ji[r * d + j] * (x[j] - X0[j]);
  double val = mean;
  for (int k = 0; k < o->nk; ++k) val += af[k] * (monomial(o->ex[k], xi, d) - o->psibar[k]);
  return val;
}

static void recon_cell(orc *o, int i, const double *U) {
  const int d = o->p.dim, nv = o->nv, nf = o->nf, nq = o->nq, nk = o->nk, n = o->ncells;
  orc_cell *c = o->cell[i];
  /* admissible stencils: s = 1 central, s = 2..s_t directional */
  int adm[MAXNF], na = 0;
  for (int f = 0; f < nf; ++f)
    if (c->dok[f]) adm[na++] = f;
  int mask = 1;
  for (int s = 0; s < na; ++s) mask |= 1 << (1 + adm[s]);
  o->stmask[i] = mask;
  /* least-squares coefficients of every conserved variable (eqs. 10-12) */
  double U0[MAXNV], aopt[MAXNV][MAXK], ad[MAXNV][MAXNF][MAXKD];
  for (int v = 0; v < nv; ++v) {
    U0[v] = U[v * n + i];
    double b[MAXM];
    for (int k = 0; k < c->nst; ++k) b[k] = c->Vp[k] * (U[v * n + c->ids[k]] - U0[v]); /* eq. 10 */
    lsq_solve(c->nst, nk, c->V, nk, c->beta, c->R, nk, b, aopt[v]);   /* p_opt */
    for (int s = 0; s < na; ++s) {
      int f = adm[s];
      double bd[MAXDIR];
      for (int j = 0; j < c->ndir[f]; ++j) bd[j] = b[c->dmem[f][j]];
      lsq_solve(c->ndir[f], o->dk, &c->dV[f][0][0], MAXKD, c->dbeta[f], &c->dR[f][0][0], MAXKD, bd, ad[v][f]);
    }
  }
  double fout[MAXNF][MAXNQ][MAXNV];
  if (!o->p.characteristic) { /* conserved variables, each selected independently (Alg. 1 / 2) */
    for (int v = 0; v < nv; ++v) {
      double af[MAXK];
      weigh(o, i, v, na, adm, aopt[v], ad[v], af);
      for (int f = 0; f < nf; ++f)
        for (int q = 0; q < nq; ++q) fout[f][q][v] = face_value(o, i, f, q, U0[v], af);
    }
  } else {
    /* Reading of the characteristic reconstruction (Sec. 2.2, 3.2): for each face f, the
     * eigenvectors at the cell's mean state in the face's outward normal direction; the
     * reconstruction runs on W = L U of every stencil member, i.e. on L applied to the
     * least-squares coefficients (the least squares are linear in the data), each field selected
     * independently; the face's Gauss-point values are transformed back, U = R W. */
    for (int f = 0; f < nf; ++f) {
      double R[MAXNV][MAXNV], L[MAXNV][MAXNV];
      euler_eigen(o, U0, o->nrm + (size_t)(i * nf + f) * d, R, L);
      double W[MAXNQ][MAXNV];
      for (int w = 0; w < nv; ++w) {
        double aw[MAXK], adw[MAXNF][MAXKD], af[MAXK], Wbar = 0.0;
        for (int v = 0; v < nv; ++v) Wbar += L[w][v] * U0[v];
        for (int k = 0; k < nk; ++k) {
          aw[k] = 0.0;
          for (int v = 0; v < nv; ++v) aw[k] += L[w][v] * aopt[v][k];
        }
        for (int s = 0; s < na; ++s)
          for (int k = 0; k < o->dk; ++k) {
            adw[adm[s]][k] = 0.0;
            for (int v = 0; v < nv; ++v) adw[adm[s]][k] += L[w][v] * ad[v][adm[s]][k];
          }
        weigh(o, i, f * nv + w, na, adm, aw, adw, af);
        for (int q = 0; q < nq; ++q) W[q][w] = face_value(o, i, f, q, Wbar, af);
      }
      for (int q = 0; q < nq; ++q)
        for (int v = 0; v < nv; ++v) {
          double s = 0.0;
          for (int w = 0; w < nv; ++w) s += R[v][w] * W[q][w];
          fout[f][q][v] = s;
        }
    }
  }
  int guard_hit = 0;
  if (o->p.guard) { /* Reading: non-physical face state -> first order in this cell */
    for (int f = 0; f < nf; ++f)
      for (int q = 0; q < nq; ++q)
        if (!(fout[f][q][0] > 0.0) || !(pressure(o, fout[f][q]) > 0.0)) guard_hit = 1;
    if (guard_hit) {
      for (int f = 0; f < nf; ++f)
        for (int q = 0; q < nq; ++q)
          for (int v = 0; v < nv; ++v) fout[f][q][v] = U0[v];
    }
  }
  for (int f = 0; f < nf; ++f)
    for (int q = 0; q < nq; ++q)
      for (int v = 0; v < nv; ++v)
        o->face[(((size_t)i * nf + f) * nq + q) * nv + v] = fout[f][q][v];
  o->guarded[i] = (uint8_t)guard_hit;
  if (guard_hit) {
#pragma omp atomic
    o->nguard++;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* HLLC flux (eqs. 24-29)                                                                      */
/* ------------------------------------------------------------------------------------------ */
static void euler_flux(const orc *o, const double *u, const double *n, double *F) {
  const int d = o->p.dim;
  double rho = u[0], un = 0.0;
  for (int j = 0; j < d; ++j) un += u[1 + j] / rho * n[j];
  double p = pressure(o, u);
  F[0] = rho * un;
  for (int j = 0; j < d; ++j) F[1 + j] = u[1 + j] * un + p * n[j];
  F[d + 1] = (u[d + 1] + p) * un;
}

/* Reading of the garbled passages: F_R = F(U_R); c~^2 = (gamma-1)(H~ - |u~|^2/2) with the full
 * Roe-averaged velocity; F_R is used when S_R <= 0 (equal to F*_R at S_R = 0); the star
 * momentum is the vector form of eq. 29. */
static void hllc(const orc *o, const double *uL, const double *uR, const double *n, double *F) {
  const int d = o->p.dim, nv = o->nv;
  const double g = o->p.gamma;
  double rL = uL[0], rR = uR[0], vL[3], vR[3], unL = 0, unR = 0;
  for (int j = 0; j < d; ++j) {
    vL[j] = uL[1 + j] / rL;
    vR[j] = uR[1 + j] / rR;
    unL += vL[j] * n[j];
    unR += vR[j] * n[j];
  }
  double pL = pressure(o, uL), pR = pressure(o, uR);
  double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
  double HL = (uL[d + 1] + pL) / rL, HR = (uR[d + 1] + pR) / rR;
  double D = sqrt(rR / rL); /* eq. 26 */
  double ut[3], ut2 = 0.0, utn = 0.0;
  for (int j = 0; j < d; ++j) {
    ut[j] = (vL[j] + vR[j] * D) / (1.0 + D);
    ut2 += ut[j] * ut[j];
    utn += ut[j] * n[j];
  }
  double Ht = (HL + HR * D) / (1.0 + D);
  double ct = sqrt((g - 1.0) * (Ht - 0.5 * ut2));
  double SL = fmin(unL - cL, utn - ct), SR = fmax(unR + cR, utn + ct); /* eq. 25 */
  double SM = (rR * unR * (SR - unR) - rL * unL * (SL - unL) + pL - pR) /
              (rR * (SR - unR) - rL * (SL - unL)); /* eq. 28 */
  double ps = rL * (unL - SL) * (unL - SM) + pL;
  double FL[MAXNV], FR[MAXNV];
  euler_flux(o, uL, n, FL);
  euler_flux(o, uR, n, FR);
  if (SL > 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FL[v];
  } else if (SM > 0.0) { /* S_L <= 0 < S_M */
    double f = 1.0 / (SL - SM), us[MAXNV];
    us[0] = rL * (SL - unL) * f;
    for (int j = 0; j < d; ++j) us[1 + j] = ((SL - unL) * uL[1 + j] + (ps - pL) * n[j]) * f;
    us[d + 1] = ((SL - unL) * uL[d + 1] - pL * unL + ps * SM) * f;
    for (int v = 0; v < nv; ++v) F[v] = FL[v] + SL * (us[v] - uL[v]);
  } else if (SR > 0.0) { /* S_M <= 0 < S_R */
    double f = 1.0 / (SR - SM), us[MAXNV];
    us[0] = rR * (SR - unR) * f;
    for (int j = 0; j < d; ++j) us[1 + j] = ((SR - unR) * uR[1 + j] + (ps - pR) * n[j]) * f;
    us[d + 1] = ((SR - unR) * uR[d + 1] - pR * unR + ps * SM) * f;
    for (int v = 0; v < nv; ++v) F[v] = FR[v] + SR * (us[v] - uR[v]);
  } else {
    for (int v = 0; v < nv; ++v) F[v] = FR[v];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Residual (eq. 2), time step, SSP-RK3                                                        */
/* ------------------------------------------------------------------------------------------ */
/* dU_i/dt = -(1/|V_i|) sum_faces sum_q F(U_L, U_R) w_q |A|  (eq. 2). Reading: on a transmissive
 * boundary face the outside state is the cell mean, U_R = U_i (zeroth-order extrapolation); on a
 * reflective wall it is the mirror image of the reconstructed inside state, U_R = (rho, m - 2 (m.n) n,
 * E) at each Gauss point (zero normal velocity at the wall, same density and pressure); the
 * reconstructed U_L stays the inside state. */
static void residual_cell(orc *o, int i, double *Rout) {
  const int d = o->p.dim, nv = o->nv, nf = o->nf, nq = o->nq;
  double acc[MAXNV] = {0, 0, 0, 0, 0};
  for (int f = 0; f < nf; ++f) {
    int j = o->nbr[i * nf + f], fj = o->nbrf[i * nf + f];
    const double *n = o->nrm + (size_t)(i * nf + f) * d;
    for (int q = 0; q < nq; ++q) {
      const double *uL = o->face + (((size_t)i * nf + f) * nq + q) * nv;
      double ub[MAXNV];
      const int kind = (j >= 0) ? -1 : o->bkind[i * nf + f];
      if (kind == BND_WALL) {
        double mn = 0.0;
        for (int k = 0; k < d; ++k) mn += uL[1 + k] * n[k];
        ub[0] = uL[0];
        for (int k = 0; k < d; ++k) ub[1 + k] = uL[1 + k] - 2.0 * mn * n[k];
        ub[d + 1] = uL[d + 1];
      } else if (kind == BND_STATE_A || kind == BND_SHOCK_AB) {
        int use_a = 1;
        if (kind == BND_SHOCK_AB) {
          double mid[3] = {0, 0, 0};
          const double *X = o->X + (size_t)i * (d + 1) * d;
          for (int a = 0; a <= d; ++a)
            if (a != f)
              for (int k = 0; k < d; ++k) mid[k] += X[a * d + k] / d;
          use_a = o->shock[0] + o->shock[1] * mid[1] + o->shock[2] * o->stage_time > mid[0];
        }
        for (int v = 0; v < nv; ++v) ub[v] = o->bstate[use_a ? 0 : 1][v];
      } else {
        for (int v = 0; v < nv; ++v) ub[v] = o->U[v * o->ncells + i];
      }
      const double *uR = (j >= 0) ? o->face + (((size_t)j * nf + fj) * nq + q) * nv : ub;
      double F[MAXNV];
      hllc(o, uL, uR, n, F);
      for (int v = 0; v < nv; ++v) acc[v] += o->fw[q] * o->area[i * nf + f] * F[v];
    }
  }
  for (int v = 0; v < nv; ++v) Rout[v] = -acc[v] / o->vol[i];
}

static void residual_all(orc *o, const double *U) {
  const int n = o->ncells, nv = o->nv;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) recon_cell(o, i, U);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double r[MAXNV];
    residual_cell(o, i, r);
    for (int v = 0; v < nv; ++v) o->Rres[v * n + i] = r[v];
  }
}

/* Reading (time step not given in the paper): dt = CFL min_i |V_i| / sum_f |A_f| (|u_i.n_f| + c_i)
 * from the cell means at the start of the step. */
double orc_dt(orc *o) {
  const int d = o->p.dim, n = o->ncells, nf = o->nf;
  double best = 1e300;
  for (int i = 0; i < n; ++i) {
    double u[MAXNV];
    for (int v = 0; v < o->nv; ++v) u[v] = o->U[v * n + i];
    double p = pressure(o, u), c = sqrt(o->p.gamma * p / u[0]), s = 0.0;
    for (int f = 0; f < nf; ++f) {
      double un = 0.0;
      for (int j = 0; j < d; ++j) un += u[1 + j] / u[0] * o->nrm[(i * nf + f) * d + j];
      s += o->area[i * nf + f] * (fabs(un) + c);
    }
    double dt = o->vol[i] / s;
    if (dt < best) best = dt;
  }
  return o->p.cfl * best;
}

/* The paper's explicit Runge-Kutta step ("3rd- or 4th-order", Sec. 2). rk = 3: third-order SSP
 * Runge-Kutta in Shu-Osher form, U1 = U^n + dt R(U^n), U2 = 3/4 U^n + 1/4 (U1 + dt R(U1)),
 * U^{n+1} = 1/3 U^n + 2/3 (U2 + dt R(U2)). rk = 4: the classical four-stage method, k_s = R(U_s),
 * U_1 = U^n, U_2 = U^n + dt/2 k_1, U_3 = U^n + dt/2 k_2, U_4 = U^n + dt k_3,
 * U^{n+1} = U^n + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4) (accumulated stage by stage in Acc). */
void orc_stage(orc *o, int stage, double dt) {
  const int n = o->ncells, nv = o->nv;
  /* the stage's time, for the time-dependent boundary: t^n + c_s dt with c = (0, 1, 1/2) for
   * SSP-RK3 and (0, 1/2, 1/2, 1) for RK4 */
  static const double c3[3] = {0.0, 1.0, 0.5}, c4[4] = {0.0, 0.5, 0.5, 1.0};
  o->stage_time = o->time + (o->p.rk == 4 ? c4[stage] : c3[stage]) * dt;
  if (stage == 0) memcpy(o->Un, o->U, sizeof(double) * nv * n);
  residual_all(o, o->U);
  if (o->p.rk == 4) {
    for (int k = 0; k < nv * n; ++k) {
      const double dk = dt * o->Rres[k];
      if (stage == 0) {
        o->Acc[k] = o->Un[k] + dk / 6.0;
        o->U[k] = o->Un[k] + 0.5 * dk;
      } else if (stage == 1) {
        o->Acc[k] += dk / 3.0;
        o->U[k] = o->Un[k] + 0.5 * dk;
      } else if (stage == 2) {
        o->Acc[k] += dk / 3.0;
        o->U[k] = o->Un[k] + dk;
      } else {
        o->U[k] = o->Acc[k] + dk / 6.0;
      }
    }
    return;
  }
  static const double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < nv * n; ++k)
    o->U[k] = a[stage] * o->Un[k] + b[stage] * (o->U[k] + dt * o->Rres[k]);
}

double orc_step(orc *o, double dt) {
  if (!(dt > 0.0)) dt = orc_dt(o);
  for (int s = 0; s < (o->p.rk == 4 ? 4 : 3); ++s) orc_stage(o, s, dt);
  o->time += dt;
  return dt;
}

/* Sets the time of the next step (and of a residual evaluated outside a step). */
void orc_set_time(orc *o, double t) { o->time = o->stage_time = t; }
double orc_get_time(const orc *o) { return o->time; }

/* Every boundary face whose midpoint lies in the box [lo, hi] (inclusive) becomes of the given
 * kind (later calls override earlier ones). */
void orc_boundary_region(orc *o, const double *lo, const double *hi, int kind) {
  const int d = o->p.dim, nf = o->nf;
  for (int i = 0; i < o->ncells; ++i)
    for (int f = 0; f < nf; ++f) {
      if (o->nbr[i * nf + f] >= 0) continue;
      const double *X = o->X + (size_t)i * (d + 1) * d;
      int in = 1;
      for (int k = 0; k < d; ++k) {
        double m = 0.0;
        for (int a = 0; a <= d; ++a)
          if (a != f) m += X[a * d + k] / d;
        in = in && m >= lo[k] && m <= hi[k];
      }
      if (in) o->bkind[i * nf + f] = (signed char)kind;
    }
}

/* States A and B (conserved) and the moving shock x = xs0 + sy y + vs t of the fixed-state kinds. */
void orc_boundary_states(orc *o, const double *A, const double *B, double xs0, double sy, double vs) {
  for (int v = 0; v < o->nv; ++v) {
    o->bstate[0][v] = A[v];
    o->bstate[1][v] = B[v];
  }
  o->shock[0] = xs0;
  o->shock[1] = sy;
  o->shock[2] = vs;
}

/* ------------------------------------------------------------------------------------------ */
/* Construction and accessors (ctypes interface)                                               */
/* ------------------------------------------------------------------------------------------ */
orc *orc_create(int dim, int degree, int scheme, int lam_gamma, int ctenoz_form, int characteristic,
                int boundary, int rk, double C_T, double lambda1p, double eps, double gamma, double cfl, int guard, int nverts,
                const double *xyz, int ncells, const int *cells, const double *period, int *err) {
  *err = 0;
  if ((dim != 2 && dim != 3) || degree < 1 || degree > (dim == 2 ? 6 : 3) || (boundary != 0 && boundary != 1) ||
      (rk != 3 && rk != 4)) {
    *err = -1;
    return NULL;
  }
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->p.dim = dim;
  o->p.degree = degree;
  o->p.scheme = scheme;
  o->p.C_T = C_T;
  o->p.lambda1p = lambda1p;
  o->p.eps = eps;
  o->p.gamma = gamma;
  o->p.cfl = cfl;
  o->p.guard = guard;
  o->p.lam_gamma = lam_gamma;
  o->p.ctenoz_form = ctenoz_form;
  o->p.characteristic = characteristic;
  o->p.boundary = boundary;
  o->p.rk = rk;
  o->nverts = nverts;
  o->ncells = ncells;
  o->nv = dim + 2;
  o->nf = dim + 1;
  o->nsel = characteristic ? o->nf * o->nv : o->nv;
  /* Reading ("a Gauss rule suited to the polynomial order", Sec. 2): edges carry
   * ceil((r + 1) / 2) Gauss-Legendre points, exact for the degree-r face polynomials */
  o->nq = (dim == 2) ? (degree + 2) / 2 : 4;
  if (dim == 2 && o->nq < 2) o->nq = 2;
  /* Reading (Fig. 1: third-order directional stencils beside a fifth-order central one):
   * directional polynomials of degree 1, or 2 when the central degree is 4 or more; each
   * directional stencil keeps up to twice as many cells as its polynomial has unknowns */
  o->ddeg = (degree >= 4) ? 2 : 1;
  o->dk = K_of(o->ddeg, dim) - 1;
  o->dmax = 2 * o->dk;
  o->nk = make_exponents(dim, degree, o->ex);
  o->M = 2 * K_of(degree, dim);
  for (int j = 0; j < dim; ++j) o->period[j] = period ? period[j] : 0.0;
  /* volume rule with r+1 points per direction: exact to degree 2(r+1)-d, which covers the
   * moments (degree r) and the smoothness integrands (degree 2r-2) for d <= 3 */
  simplex_rule(dim, degree + 1, &o->qlam, &o->qw, &o->nqv);
  for (int k = 0; k < o->nk; ++k) { /* mean of psi_k over V0' */
    double s = 0.0;
    for (int q = 0; q < o->nqv; ++q) {
      double xi[3] = {0, 0, 0};
      for (int a = 1; a <= dim; ++a) xi[a - 1] = o->qlam[q * (dim + 1) + a];
      s += o->qw[q] * monomial(o->ex[k], xi, dim);
    }
    o->psibar[k] = s;
  }
  int rc = build_geometry(o, xyz, cells);
  if (!rc) rc = build_faces(o);
  if (rc) {
    *err = rc;
    return o;
  }
  const size_t n = ncells;
  o->cell = (orc_cell **)calloc(n, sizeof(orc_cell *));
  o->U = (double *)calloc(n * o->nv, sizeof(double));
  o->Un = (double *)calloc(n * o->nv, sizeof(double));
  o->Acc = (double *)calloc(n * o->nv, sizeof(double));
  o->bkind = (signed char *)malloc(n * o->nf);
  for (size_t k = 0; k < n * (size_t)o->nf; ++k) o->bkind[k] = (signed char)(boundary == 1 ? BND_WALL : BND_TRANSMISSIVE);
  o->Rres = (double *)calloc(n * o->nv, sizeof(double));
  o->face = (double *)calloc(n * o->nf * o->nq * o->nv, sizeof(double));
  o->flags = (uint8_t *)calloc(n * o->nsel, 1);
  o->SI = (double *)calloc(n * o->nsel * (1 + o->nf), sizeof(double));
  o->chi = (double *)calloc(n * o->nsel * (1 + o->nf), sizeof(double));
  o->stmask = (int *)calloc(n, sizeof(int));
  o->guarded = (uint8_t *)calloc(n, 1);
  o->coef = (double *)calloc(n * o->nsel * o->nk, sizeof(double));
  return o;
}

/* Stencils + least-squares set-up for every cell (parallel over cells). */
int orc_setup_all(orc *o) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < o->ncells; ++i) {
    int rc = cell_setup(o, i);
    if (rc) {
#pragma omp critical
      bad = rc;
    }
  }
  return bad;
}

/* Set-up of a subset of cells only (for sampled checks on large meshes); parallel over the
 * distinct cells of the list. */
int orc_setup_cells(orc *o, int count, const int *ids) {
  uint8_t *want = (uint8_t *)calloc(o->ncells, 1);
  for (int k = 0; k < count; ++k) want[ids[k]] = 1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < o->ncells; ++i) {
    if (!want[i]) continue;
    int rc = cell_setup(o, i);
    if (rc) {
#pragma omp critical
      bad = rc;
    }
  }
  free(want);
  return bad;
}

void orc_destroy(orc *o) {
  if (!o) return;
  if (o->cell) {
    for (int i = 0; i < o->ncells; ++i)
      if (o->cell[i]) {
        free(o->cell[i]->A);
        free(o->cell[i]->R);
        free(o->cell[i]->V);
        free(o->cell[i]);
      }
    free(o->cell);
  }
  free(o->cv); free(o->X); free(o->vol); free(o->cen); free(o->Jinv); free(o->detJ);
  free(o->nbr); free(o->nbrf); free(o->area); free(o->nrm); free(o->fq);
  free(o->v2c_off); free(o->v2c); free(o->qlam); free(o->qw);
  free(o->U); free(o->Un); free(o->Acc); free(o->bkind); free(o->Rres); free(o->face); free(o->flags); free(o->SI); free(o->chi);
  free(o->stmask);
  free(o->guarded);
  free(o->coef);
  free(o);
}

void orc_set_state(orc *o, const double *U) { memcpy(o->U, U, sizeof(double) * o->nv * o->ncells); }
void orc_get_state(const orc *o, double *U) { memcpy(U, o->U, sizeof(double) * o->nv * o->ncells); }

/* Residual of the current state for every cell (all cells must be set up). */
void orc_residual(orc *o, double *R) {
  residual_all(o, o->U);
  memcpy(R, o->Rres, sizeof(double) * o->nv * o->ncells);
}

/* Residual of a subset of cells: reconstructs the subset and its face neighbours (which must be
 * set up, see orc_setup_cells), then evaluates eq. 2 for the subset. R_out: [count][nv]. */
int orc_residual_cells(orc *o, int count, const int *ids, double *R_out) {
  for (int k = 0; k < count; ++k) {
    int i = ids[k], rc = cell_setup(o, i);
    for (int f = 0; f < o->nf && !rc; ++f) {
      int j = o->nbr[i * o->nf + f];
      if (j >= 0) rc = cell_setup(o, j);
    }
    if (rc) return rc;
    recon_cell(o, i, o->U);
    for (int f = 0; f < o->nf; ++f) {
      int j = o->nbr[i * o->nf + f];
      if (j >= 0) recon_cell(o, j, o->U);
    }
    residual_cell(o, i, R_out + (size_t)k * o->nv);
  }
  return 0;
}

/* Residual of a subset of cells, reconstructing each cell of the subset and of its face
 * neighbours once (parallel over cells). Cells must be set up (orc_setup_cells), their face
 * neighbours included. R_out: [count][nv]. */
int orc_residual_subset(orc *o, int count, const int *ids, double *R_out) {
  const int nf = o->nf;
  uint8_t *need = (uint8_t *)calloc(o->ncells, 1);
  for (int k = 0; k < count; ++k) {
    need[ids[k]] = 1;
    for (int f = 0; f < nf; ++f) {
      int j = o->nbr[ids[k] * nf + f];
      if (j >= 0) need[j] = 1;
    }
  }
  int nn = 0;
  for (int i = 0; i < o->ncells; ++i) nn += need[i];
  int *list = (int *)malloc(sizeof(int) * (nn ? nn : 1));
  nn = 0;
  for (int i = 0; i < o->ncells; ++i)
    if (need[i]) list[nn++] = i;
  free(need);
  int bad = 0;
  for (int k = 0; k < nn; ++k)
    if (!o->cell[list[k]] || !o->cell[list[k]]->ready) bad = -8;
  if (!bad) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int k = 0; k < nn; ++k) recon_cell(o, list[k], o->U);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < count; ++k) residual_cell(o, ids[k], R_out + (size_t)k * o->nv);
  }
  free(list);
  return bad;
}

/* Reconstruct a subset of cells (face states, flags and SI are then readable for them). */
int orc_reconstruct_cells(orc *o, int count, const int *ids) {
  for (int k = 0; k < count; ++k) {
    int rc = cell_setup(o, ids[k]);
    if (rc) return rc;
    recon_cell(o, ids[k], o->U);
  }
  return 0;
}

int orc_info(const orc *o, int *out) {
  out[0] = o->nv; out[1] = o->nf; out[2] = o->nq; out[3] = o->nk; out[4] = o->M;
  out[5] = o->err; out[6] = o->nguard; out[7] = o->dmax;
  return 0;
}

void orc_get_geometry(const orc *o, double *vol, double *cen, int *cv, double *area, double *nrm,
                      int *nbr, int *nbrf) {
  const size_t n = o->ncells;
  const int d = o->p.dim, nf = o->nf;
  if (vol) memcpy(vol, o->vol, sizeof(double) * n);
  if (cen) memcpy(cen, o->cen, sizeof(double) * n * d);
  if (cv) memcpy(cv, o->cv, sizeof(int) * n * (d + 1));
  if (area) memcpy(area, o->area, sizeof(double) * n * nf);
  if (nrm) memcpy(nrm, o->nrm, sizeof(double) * n * nf * d);
  if (nbr) memcpy(nbr, o->nbr, sizeof(int) * n * nf);
  if (nbrf) memcpy(nbrf, o->nbrf, sizeof(int) * n * nf);
}

void orc_get_face_points(const orc *o, double *fq, double *fw) {
  if (fq) memcpy(fq, o->fq, sizeof(double) * o->ncells * o->nf * o->nq * o->p.dim);
  if (fw) memcpy(fw, o->fw, sizeof(double) * o->nq);
}

/* Stencil of cell i: central ids [M], directional member positions [nf][dmax] (-1 padded),
 * admissibility [nf]. Cell i must be set up. */
void orc_get_stencil(const orc *o, int i, int *central, int *dir, int *dok) {
  const orc_cell *c = o->cell[i];
  for (int k = 0; k < o->M; ++k) central[k] = c->ids[k];
  for (int f = 0; f < o->nf; ++f) {
    for (int j = 0; j < o->dmax; ++j) dir[f * o->dmax + j] = (j < c->ndir[f]) ? c->dmem[f][j] : -1;
    dok[f] = c->dok[f];
  }
}

/* Least-squares matrices of cell i: A [M][nk] (eq. 10) and |V'_m| [M]. */
void orc_get_lsq(const orc *o, int i, double *A, double *Vp) {
  const orc_cell *c = o->cell[i];
  for (int k = 0; k < c->nst; ++k) {
    for (int j = 0; j < o->nk; ++j) A[k * o->nk + j] = c->A[k * o->nk + j];
    Vp[k] = c->Vp[k];
  }
}

/* Central least-squares coefficients of cell i for a given vector of member values
 * (b_m = |V'_m| (Um - U0), eq. 12). */
void orc_lsq_apply(const orc *o, int i, const double *Um, double U0, double *a) {
  const orc_cell *c = o->cell[i];
  double b[MAXM];
  for (int k = 0; k < c->nst; ++k) b[k] = c->Vp[k] * (Um[k] - U0);
  lsq_solve(c->nst, o->nk, c->V, o->nk, c->beta, c->R, o->nk, b, a);
}

void orc_get_face_states(const orc *o, double *out) {
  memcpy(out, o->face, sizeof(double) * o->ncells * o->nf * o->nq * o->nv);
}
/* Debug records per cell and selection: [ncells][nsel] with nsel = nv, or nf * nv (face-major)
 * for the characteristic reconstruction. */
void orc_get_flags(const orc *o, uint8_t *out) { memcpy(out, o->flags, (size_t)o->ncells * o->nsel); }
void orc_get_si(const orc *o, double *out) {
  memcpy(out, o->SI, sizeof(double) * o->ncells * o->nsel * (1 + o->nf));
}
void orc_get_chi(const orc *o, double *out) {
  memcpy(out, o->chi, sizeof(double) * o->ncells * o->nsel * (1 + o->nf));
}
void orc_get_coeffs(const orc *o, double *out) {
  memcpy(out, o->coef, sizeof(double) * o->ncells * o->nsel * o->nk);
}
/* Eigenvectors of the Euler flux Jacobian in direction n at the conserved state u (row-major
 * [nv][nv]), as the characteristic reconstruction uses them. */
void orc_eigen(const orc *o, const double *u, const double *n, double *R, double *L) {
  double Rm[MAXNV][MAXNV], Lm[MAXNV][MAXNV];
  euler_eigen(o, u, n, Rm, Lm);
  for (int a = 0; a < o->nv; ++a)
    for (int b = 0; b < o->nv; ++b) {
      R[a * o->nv + b] = Rm[a][b];
      L[a * o->nv + b] = Lm[a][b];
    }
}
/* Reference map of cell i: oriented vertex coordinates [(d+1)][d] (unwrapped) and J^-1. */
void orc_get_refmap(const orc *o, int i, double *X, double *Jinv) {
  const int d = o->p.dim;
  memcpy(X, o->X + (size_t)i * (d + 1) * d, sizeof(double) * (d + 1) * d);
  memcpy(Jinv, o->Jinv + (size_t)i * d * d, sizeof(double) * d * d);
}
void orc_get_stmask(const orc *o, int *out) { memcpy(out, o->stmask, sizeof(int) * o->ncells); }
void orc_get_guarded(const orc *o, uint8_t *out) { memcpy(out, o->guarded, (size_t)o->ncells); }
void orc_get_exponents(const orc *o, int *ex) {
  for (int k = 0; k < o->nk; ++k)
    for (int j = 0; j < 3; ++j) ex[k * 3 + j] = o->ex[k][j];
}
double orc_psibar(const orc *o, int k) { return o->psibar[k]; }

/* Exposed pieces for the pin tests. */
/* The selection of one cell and variable from given indicators (see select_stencils): SI[st],
 * chi_out[st]; returns the delta bits. */
unsigned orc_select(int scheme, int ctenoz_form, int lam_gamma, double C_T, double lambda1p, double eps,
                    int st, const double *SI, double *chi_out) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.scheme = scheme;
  p.ctenoz_form = ctenoz_form;
  p.lam_gamma = lam_gamma;
  p.C_T = C_T;
  p.lambda1p = lambda1p;
  p.eps = eps;
  return select_stencils(&p, st, SI, chi_out);
}
void orc_hllc(const orc *o, const double *uL, const double *uR, const double *n, double *F) {
  hllc(o, uL, uR, n, F);
}
void orc_euler_flux(const orc *o, const double *u, const double *n, double *F) {
  euler_flux(o, u, n, F);
}
double orc_smoothness(orc *o, const double *a, int nterms, int deg) {
  return smoothness(o, a, nterms, deg);
}
/* Integral over the simplex with vertices xi [(d+1)][d] of monomial k, by the oracle's rule. */
double orc_simplex_monomial(orc *o, const double *xi, int k) {
  const int d = o->p.dim, nvc = d + 1;
  double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) J[r * d + c] = xi[(c + 1) * d + r] - xi[r];
  double vol = fabs(det_d(d, J)) / factorial(d), s = 0.0;
  for (int q = 0; q < o->nqv; ++q) {
    double p[3] = {0, 0, 0};
    for (int a = 0; a < nvc; ++a)
      for (int j = 0; j < d; ++j) p[j] += o->qlam[q * nvc + a] * xi[a * d + j];
    s += o->qw[q] * monomial(o->ex[k], p, d);
  }
  return vol * s;
}
int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
