// mesh.cpp -- host ingestion of a triangle / tetrahedron mesh (Sec. 2, eq. 2), the central and
// directional stencils (Sec. 2.1, Sec. 2.3 / Fig. 1) and the locality renumbering.
//
// Conventions shared with every other implementation of these readings (they decide integer
// results, so they are fixed exactly):
//   * a periodic cell is unwrapped next to its local vertex 0: x - L round((x - x0) / L);
//   * a cell with negative Jacobian determinant swaps its local vertices 1 and 2;
//   * the centroid is (X_0 + ... + X_d) / (d + 1) over the oriented vertices, in that order;
//   * a stencil member m of target i is moved by s = -L round((c_m - c_i) / L) and its offset is
//     ((c_m + s) - c_i), its squared distance the sum of the squared offset components;
//   * the central stencil is the M nearest cells (ties to the lower id) among the vertex-adjacency
//     layers around the target, taken until they hold at least M cells;
//   * a member belongs to the directional stencil of local face f when its offset has
//     non-negative coordinates along the rays from c_i to the vertices of face f (Cramer's rule),
//     the first such face in local order owning it; a directional stencil keeps its first 2d
//     members in nearest-first order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace cteno {
namespace {

inline double image_shift(double dx, double L) { return (L > 0.0) ? -L * std::round(dx / L) : 0.0; }

inline double det2(double a00, double a01, double a10, double a11) { return a00 * a11 - a01 * a10; }

// determinant of a row-major 2x2 or 3x3 matrix
inline double detn(int d, const double *a) {
  if (d == 2) return det2(a[0], a[1], a[2], a[3]);
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}

struct FaceKey {
  int32_t v[3];
  int32_t cell;
  int8_t f;
};

}  // namespace

int ingest_mesh(int dim, int64_t nverts, const double *xyz, int64_t ncells, const int32_t *cvin,
                const double *period, Mesh *m, std::string *err) {
  const int d = dim, nvc = d + 1, nf = d + 1;
  m->dim = d;
  m->nverts = nverts;
  m->ncells = ncells;
  for (int j = 0; j < 3; ++j) m->period[j] = (period && j < d && period[j] > 0.0) ? period[j] : 0.0;
  m->xyz.assign(xyz, xyz + nverts * d);
  m->cv.resize(ncells * nvc);
  m->X.resize(ncells * nvc * d);
  m->cen.resize(ncells * d);
  for (int64_t c = 0; c < ncells; ++c) {
    int32_t v[4];
    double X[4][3];
    for (int a = 0; a < nvc; ++a) {
      v[a] = cvin[c * nvc + a];
      if (v[a] < 0 || v[a] >= nverts) {
        *err = "cell " + std::to_string(c) + " has a vertex id out of range";
        return CTENO_ERR_MESH;
      }
    }
    for (int a = 0; a < nvc; ++a)
      for (int j = 0; j < d; ++j) {
        double x = xyz[(int64_t)v[a] * d + j], x0 = xyz[(int64_t)v[0] * d + j];
        X[a][j] = x + image_shift(x - x0, m->period[j]);
      }
    double J[9];
    for (int r = 0; r < d; ++r)
      for (int k = 0; k < d; ++k) J[r * d + k] = X[k + 1][r] - X[0][r];
    double D = detn(d, J);
    if (!(D != 0.0) || !std::isfinite(D)) {
      *err = "cell " + std::to_string(c) + " is degenerate";
      return CTENO_ERR_MESH;
    }
    if (D < 0.0) {
      std::swap(v[1], v[2]);
      for (int j = 0; j < d; ++j) std::swap(X[1][j], X[2][j]);
    }
    for (int a = 0; a < nvc; ++a) {
      m->cv[c * nvc + a] = v[a];
      for (int j = 0; j < d; ++j) m->X[(c * nvc + a) * d + j] = X[a][j];
    }
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int a = 0; a < nvc; ++a) s += X[a][j];
      m->cen[c * d + j] = s / nvc;
    }
  }
  // face matching by sorted vertex ids
  std::vector<FaceKey> keys(ncells * nf);
  for (int64_t c = 0; c < ncells; ++c)
    for (int f = 0; f < nf; ++f) {
      FaceKey &k = keys[c * nf + f];
      int n = 0;
      for (int a = 0; a < nvc; ++a)
        if (a != f) k.v[n++] = m->cv[c * nvc + a];
      if (d == 2) k.v[2] = -1;
      std::sort(k.v, k.v + d);
      k.cell = (int32_t)c;
      k.f = (int8_t)f;
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey &a, const FaceKey &b) {
    if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
    if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
    if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
    return a.cell < b.cell;
  });
  m->nbr.assign(ncells * nf, -1);
  m->nbrf.assign(ncells * nf, -1);
  for (size_t s = 0; s < keys.size();) {
    size_t e = s + 1;
    while (e < keys.size() && keys[e].v[0] == keys[s].v[0] && keys[e].v[1] == keys[s].v[1] &&
           keys[e].v[2] == keys[s].v[2])
      ++e;
    if (e - s > 2) {
      *err = "a face is shared by more than two cells";
      return CTENO_ERR_MESH;
    }
    if (e - s == 2) {
      const FaceKey &a = keys[s], &b = keys[s + 1];
      if (a.cell == b.cell) {
        *err = "a cell is its own neighbour (periodic box too small)";
        return CTENO_ERR_MESH;
      }
      m->nbr[(int64_t)a.cell * nf + a.f] = b.cell;
      m->nbrf[(int64_t)a.cell * nf + a.f] = b.f;
      m->nbr[(int64_t)b.cell * nf + b.f] = a.cell;
      m->nbrf[(int64_t)b.cell * nf + b.f] = a.f;
    }
    s = e;
  }
  // vertex -> cells
  m->v2c_off.assign(nverts + 1, 0);
  for (int64_t k = 0; k < ncells * nvc; ++k) m->v2c_off[m->cv[k] + 1]++;
  for (int64_t v = 0; v < nverts; ++v) m->v2c_off[v + 1] += m->v2c_off[v];
  m->v2c.resize(ncells * nvc);
  std::vector<int64_t> fill(m->v2c_off.begin(), m->v2c_off.end() - 1);
  for (int64_t c = 0; c < ncells; ++c)
    for (int a = 0; a < nvc; ++a) m->v2c[fill[m->cv[c * nvc + a]]++] = (int32_t)c;
  return CTENO_OK;
}

namespace {

// Small open-addressing set of cell ids for one stencil search.
struct IdSet {
  std::vector<int32_t> slot;
  explicit IdSet(int cap) : slot(cap, -1) {}
  void clear() { std::fill(slot.begin(), slot.end(), -1); }
  bool insert(int32_t id) {  // true if new
    const uint32_t mask = (uint32_t)slot.size() - 1;
    uint32_t h = ((uint32_t)id * 0x9E3779B1u) & mask;
    for (;;) {
      if (slot[h] == id) return false;
      if (slot[h] < 0) {
        slot[h] = id;
        return true;
      }
      h = (h + 1) & mask;
    }
  }
};

struct Cand {
  double dist2;
  int32_t id;
};

}  // namespace

int build_stencils(Mesh *m, int degree, std::string *err) {
  const int d = m->dim, nvc = d + 1, nf = d + 1, nd = dir_members(d, degree);
  const int M = 2 * coeff_count(degree, d);
  const int64_t n = m->ncells;
  m->central.assign(n * M, -1);
  m->dirpos.assign(n * nf * nd, -1);
  int status = CTENO_OK;
  std::string msg;
#pragma omp parallel
  {
    IdSet seen(2048);
    std::vector<int32_t> list;
    std::vector<Cand> cand;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      if (status != CTENO_OK) continue;
      seen.clear();
      list.clear();
      list.push_back((int32_t)i);
      seen.insert((int32_t)i);
      size_t lo = 0, hi = 1;
      bool fail = false;
      while ((int)list.size() - 1 < M) {
        for (size_t k = lo; k < hi; ++k) {
          const int32_t c = list[k];
          for (int a = 0; a < nvc; ++a) {
            const int32_t v = m->cv[(int64_t)c * nvc + a];
            for (int64_t t = m->v2c_off[v]; t < m->v2c_off[v + 1]; ++t)
              if (seen.insert(m->v2c[t])) list.push_back(m->v2c[t]);
          }
        }
        if (list.size() == hi || list.size() > 1000) {
          fail = true;
          break;
        }
        lo = hi;
        hi = list.size();
      }
      if (fail) {
#pragma omp critical
        {
          status = CTENO_ERR_STENCIL;
          msg = "cell " + std::to_string(i) + " cannot gather M = " + std::to_string(M) +
                " stencil cells (mesh too small)";
        }
        continue;
      }
      const double *ci = &m->cen[i * d];
      cand.clear();
      for (size_t k = 1; k < list.size(); ++k) {
        const int32_t c = list[k];
        double s2 = 0.0;
        for (int j = 0; j < d; ++j) {
          double sh = image_shift(m->cen[(int64_t)c * d + j] - ci[j], m->period[j]);
          double w = (m->cen[(int64_t)c * d + j] + sh) - ci[j];
          s2 += w * w;
        }
        cand.push_back({s2, c});
      }
      std::partial_sort(cand.begin(), cand.begin() + M, cand.end(), [](const Cand &a, const Cand &b) {
        return a.dist2 < b.dist2 || (a.dist2 == b.dist2 && a.id < b.id);
      });
      int32_t *cen_list = &m->central[i * M];
      int count[kMaxNF] = {0, 0, 0, 0};
      const double *Xi = &m->X[i * nvc * d];
      for (int p = 0; p < M; ++p) {
        const int32_t c = cand[p].id;
        cen_list[p] = c;
        double off[3];
        for (int j = 0; j < d; ++j) {
          double sh = image_shift(m->cen[(int64_t)c * d + j] - ci[j], m->period[j]);
          off[j] = (m->cen[(int64_t)c * d + j] + sh) - ci[j];
          if (m->period[j] > 0.0 && std::fabs(off[j]) > 0.4 * m->period[j]) fail = true;
        }
        for (int f = 0; f < nf; ++f) {
          double R[9];  // rows: coordinates; columns: rays to the vertices of face f
          int col = 0;
          for (int a = 0; a < nvc; ++a) {
            if (a == f) continue;
            for (int j = 0; j < d; ++j) R[j * d + col] = Xi[a * d + j] - ci[j];
            ++col;
          }
          const double D = detn(d, R);
          bool inside = true;
          for (int cc = 0; cc < d && inside; ++cc) {
            double T[9];
            for (int j = 0; j < d; ++j)
              for (int k = 0; k < d; ++k) T[j * d + k] = (k == cc) ? off[j] : R[j * d + k];
            if (detn(d, T) / D < 0.0) inside = false;
          }
          if (inside) {
            if (count[f] < nd) m->dirpos[(i * nf + f) * nd + count[f]++] = (int8_t)p;
            break;
          }
        }
      }
      if (fail) {
#pragma omp critical
        {
          status = CTENO_ERR_STENCIL;
          msg = "the stencil of cell " + std::to_string(i) +
                " spans more than 0.4 of a periodic box length";
        }
      }
    }
  }
  if (status != CTENO_OK) *err = msg;
  return status;
}

// Morton (Z-order) renumbering of the cells of one mesh by their centroids, so that stencil
// gathers of neighbouring threads touch nearby memory.
void morton_order(Mesh *m) {
  const int d = m->dim;
  const int64_t n = m->ncells;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t c = 0; c < n; ++c)
    for (int j = 0; j < d; ++j) {
      lo[j] = std::min(lo[j], m->cen[c * d + j]);
      hi[j] = std::max(hi[j], m->cen[c * d + j]);
    }
  const int bits = (d == 2) ? 31 : 21;
  const double scale = (double)((1u << bits) - 1);
  std::vector<std::pair<uint64_t, int32_t>> key(n);
  for (int64_t c = 0; c < n; ++c) {
    uint64_t q[3] = {0, 0, 0};
    for (int j = 0; j < d; ++j) {
      double t = (hi[j] > lo[j]) ? (m->cen[c * d + j] - lo[j]) / (hi[j] - lo[j]) : 0.0;
      q[j] = (uint64_t)(t * scale);
    }
    uint64_t k = 0;
    for (int b = bits - 1; b >= 0; --b)
      for (int j = d - 1; j >= 0; --j) k = (k << 1) | ((q[j] >> b) & 1u);
    key[c] = {k, (int32_t)c};
  }
  std::sort(key.begin(), key.end());
  m->order.resize(n);
  m->rank.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    m->order[k] = key[k].second;
    m->rank[key[k].second] = (int32_t)k;
  }
}

}  // namespace cteno
