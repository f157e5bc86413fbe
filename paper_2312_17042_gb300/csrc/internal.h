// internal.h -- shared declarations of the CTENO library (host C++ and CUDA translation units).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cteno.h"

namespace cteno {

constexpr int kMaxDim = 3;
constexpr int kMaxNK = 27;   // K(6,2) - 1 unknown coefficients of a sextic in 2D (cubic in 3D: 19)
constexpr int kMaxM = 56;    // M = 2K(6,2)
constexpr int kMaxNF = 4;    // faces of a tetrahedron
constexpr int kMaxNQ = 4;    // Gauss points per face (3D; 2D degree 6)
constexpr int kMaxNV = 5;    // conserved variables in 3D
constexpr int kMaxDir = 10;  // members of a directional stencil (2d; 10 for the quadratic ones)
constexpr int kMaxPerm = 6;  // orderings of a face's vertices
constexpr int kMaxVQ = 16;   // points of the volume rule (4 x 4 in 2D at degree 6)

// K(r,d) of eq. 6: number of monomials of degree <= r in d variables, constant included.
inline int coeff_count(int r, int d) {
  int num = 1, den = 1;
  for (int l = 1; l <= d; ++l) {
    num *= (r + l);
    den *= l;
  }
  return num / den;
}

// Directional stencils (Sec. 2.3, Fig. 1): degree 1 for central degrees up to 3, degree 2 (2D)
// for central degrees 4 to 6; at most twice as many members as unknowns.
inline int dir_degree(int r) { return r >= 4 ? 2 : 1; }
inline int dir_unknowns(int d, int r) { return coeff_count(dir_degree(r), d) - 1; }
inline int dir_members(int d, int r) { return 2 * dir_unknowns(d, r); }
// Gauss points per face: 2D edges n-point Gauss-Legendre with n = max(2, (r+2)/2) (exact to
// degree r + 1); 3D faces the collapsed 2 x 2 rule.
inline int face_points(int d, int r) { return d == 3 ? 4 : (r + 2) / 2 > 2 ? (r + 2) / 2 : 2; }

// Universal constants of one (d, r): basis exponents, basis means, smoothness matrix, face
// Gauss-point basis values and volume/face quadrature rules. Built once on the host (tables.cpp)
// and copied to the device as one flat block.
struct Tables {
  int dim = 0, degree = 0, nk = 0, nf = 0, nq = 0, nperm = 0;
  int ex[kMaxNK][3] = {};               // exponents of psi_k (graded, linear first)
  double psibar[kMaxNK] = {};           // mean of psi_k over the reference simplex
  double O[kMaxNK][kMaxNK] = {};        // SI(p) = a^T O a for a polynomial of degree r
  // phi_k at face Gauss point q of local face f when the face's sorted vertex order is
  // permutation p of its local vertices
  double Phi[kMaxNF][kMaxPerm][kMaxNQ][kMaxNK] = {};
  double fw[kMaxNQ] = {};               // face weights, sum 1
  double fbary[kMaxNQ][3] = {};         // face points, barycentric in the sorted face vertices
  // collapsed Gauss-Jacobi rule on the unit reference simplex, exact to degree max(3, r)
  int nvq = 0;
  double vq[kMaxVQ][3] = {};            // reference coordinates
  double vw[kMaxVQ] = {};               // weights, sum |V0'| = 1/d!
  int perm_list[kMaxPerm][3] = {};      // permutations of the face's vertex slots
};

void build_tables(int dim, int degree, Tables *t);

// One mesh as ingested on the host.
struct Mesh {
  int dim = 0;
  int64_t nverts = 0, ncells = 0, offset = 0;  // offset: first global (device) cell index
  double period[3] = {0, 0, 0};
  std::vector<int8_t> bkind;     // [ncells][nf] kind of each boundary face (CTENO_BOUNDARY_*)
  std::vector<double> xyz;       // [nverts][dim]
  std::vector<int32_t> cv;       // [ncells][dim+1], positively oriented
  std::vector<double> X;         // [ncells][dim+1][dim] unwrapped oriented vertex coordinates
  std::vector<double> cen;       // [ncells][dim]
  std::vector<int32_t> nbr;      // [ncells][nf] neighbour (original id) or -1
  std::vector<int8_t> nbrf;      // [ncells][nf] neighbour's local face
  std::vector<int64_t> v2c_off;  // vertex -> cells (CSR)
  std::vector<int32_t> v2c;
  // stencils, original numbering
  std::vector<int32_t> central;  // [ncells][M], nearest first
  std::vector<int8_t> dirpos;    // [ncells][nf][dir_members], positions in `central`, -1 padded
  std::vector<int32_t> order;    // Morton order: new index -> original id
  std::vector<int32_t> rank;     // original id -> new index
};

int ingest_mesh(int dim, int64_t nverts, const double *xyz, int64_t ncells, const int32_t *cv,
                const double *period, Mesh *m, std::string *err);
int build_stencils(Mesh *m, int degree, std::string *err);
void morton_order(Mesh *m);

// Device-side arguments shared by the kernels. All arrays are in the renumbered (device) order
// and structure-of-arrays: element e of cell c lives at base[e * N + c].
struct DevMesh {
  int64_t N = 0;            // total cells
  int nmesh = 0;
  const int64_t *mesh_off = nullptr;  // [nmesh + 1]
  int dim = 0, degree = 0, nk = 0, M = 0, nf = 0, nq = 0, nv = 0;
};

// Kernel launchers (setup.cu, recon.cu, flux.cu).
struct Device;  // defined in device.h
}  // namespace cteno
