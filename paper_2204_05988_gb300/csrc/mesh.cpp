// Nested uniformly refined simplicial meshes and P1 transfer operators
// (Sect. 2: V_1 subset V_2 subset ... by uniform refinement; Sect. 4.2: the
// embedding E of a coarse level into the next finer one).
//
// Refinement: 1D bisection, 2D red refinement through the edge midpoints,
// 3D regular refinement after Bey (eight children: four corner tetrahedra and
// the inner octahedron split along the diagonal between the midpoints of
// edges 02 and 13; a Kuhn tetrahedron with its vertices in lattice-path order
// gives the Kuhn tetrahedra of the halved lattice, so a Kuhn coarse mesh stays
// a Kuhn lattice on every level).  Vertex order on every level:
// lexicographic by coordinates, last axis slowest.  Periodic axes identify
// the upper-bound vertex with the lower-bound one.  E_{l+1<-l} evaluates a level-l P1 function at the level
// l+1 vertices: 1 at a kept vertex, 1/2 + 1/2 at an edge midpoint.
#include <algorithm>
#include <cmath>
#include <array>
#include <cstring>
#include <map>
#include <unordered_map>

#include "internal.h"

namespace sgdg {

namespace {

struct RawMesh {
  int d = 0;
  std::vector<double> coords;               // nv * d
  std::vector<int> cells;                   // nc * (d+1)
  std::vector<std::pair<int, int>> parent;  // per vertex: (a, b) in the coarser raw mesh
  int nv() const { return (int)coords.size() / d; }
  int nc() const { return (int)cells.size() / (d + 1); }
};

RawMesh refine(const RawMesh& c) {
  RawMesh f;
  f.d = c.d;
  f.coords = c.coords;
  const int nv = c.nv();
  f.parent.resize(nv);
  for (int i = 0; i < nv; ++i) f.parent[i] = {i, i};
  std::unordered_map<uint64_t, int> mid;
  mid.reserve((size_t)c.nc() * 3);
  auto midpoint = [&](int a, int b) {
    int lo = std::min(a, b), hi = std::max(a, b);
    uint64_t key = ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
    auto it = mid.find(key);
    if (it != mid.end()) return it->second;
    int id = (int)(f.coords.size() / f.d);
    for (int k = 0; k < f.d; ++k)
      f.coords.push_back(0.5 * (c.coords[(size_t)a * f.d + k] + c.coords[(size_t)b * f.d + k]));
    f.parent.push_back({lo, hi});
    mid.emplace(key, id);
    return id;
  };
  const int d1 = c.d + 1;
  f.cells.reserve((size_t)c.nc() * d1 * (c.d == 1 ? 2 : c.d == 2 ? 4 : 8));
  for (int e = 0; e < c.nc(); ++e) {
    const int* v = &c.cells[(size_t)e * d1];
    if (c.d == 1) {
      int m = midpoint(v[0], v[1]);
      int ch[4] = {v[0], m, m, v[1]};
      f.cells.insert(f.cells.end(), ch, ch + 4);
    } else if (c.d == 2) {
      int a = v[0], b = v[1], cc = v[2];
      int mab = midpoint(a, b), mbc = midpoint(b, cc), mca = midpoint(cc, a);
      int ch[12] = {a, mab, mca, mab, b, mbc, mca, mbc, cc, mab, mbc, mca};
      f.cells.insert(f.cells.end(), ch, ch + 12);
    } else {
      // children in Bey's order, vertices of each child in its own path order
      const int x0 = v[0], x1 = v[1], x2 = v[2], x3 = v[3];
      const int m01 = midpoint(x0, x1), m02 = midpoint(x0, x2), m03 = midpoint(x0, x3);
      const int m12 = midpoint(x1, x2), m13 = midpoint(x1, x3), m23 = midpoint(x2, x3);
      const int ch[32] = {x0,  m01, m02, m03,  m01, x1,  m12, m13,  m02, m12, x2,  m23,  m03, m13, m23, x3,
                          m01, m02, m03, m13,  m01, m02, m12, m13,  m02, m03, m13, m23,  m02, m12, m13, m23};
      f.cells.insert(f.cells.end(), ch, ch + 32);
    }
  }
  return f;
}

struct CoordKey {
  std::array<double, 3> x{};
  bool operator<(const CoordKey& o) const {
    // lexicographic, last axis slowest
    for (int k = 2; k >= 0; --k) {
      if (x[k] < o.x[k]) return true;
      if (x[k] > o.x[k]) return false;
    }
    return false;
  }
};

// Canonical numbering of one raw level.  raw2can maps raw vertices (slaves
// included) to canonical master ids.
void canonical(const RawMesh& r, const sgdg_mesh& m, MeshLevel& lv, std::vector<int>& raw2can) {
  const int d = r.d, nv = r.nv();
  std::vector<CoordKey> wrapped(nv), own(nv);
  for (int i = 0; i < nv; ++i) {
    for (int k = 0; k < d; ++k) {
      double x = r.coords[(size_t)i * d + k];
      own[i].x[k] = x;
      wrapped[i].x[k] = (m.periodic && m.periodic[k] && x == m.hi[k]) ? m.lo[k] : x;
    }
  }
  // masters: vertices that are their own wrap image
  std::vector<int> masters;
  std::map<CoordKey, int> master_of;
  for (int i = 0; i < nv; ++i) {
    bool same = true;
    for (int k = 0; k < d; ++k) same = same && (own[i].x[k] == wrapped[i].x[k]);
    if (same) { masters.push_back(i); master_of[own[i]] = i; }
  }
  std::sort(masters.begin(), masters.end(), [&](int a, int b) { return own[a] < own[b]; });
  std::vector<int> can_of_raw_master(nv, -1);
  for (size_t c = 0; c < masters.size(); ++c) can_of_raw_master[masters[c]] = (int)c;
  raw2can.assign(nv, -1);
  for (int i = 0; i < nv; ++i) raw2can[i] = can_of_raw_master[master_of.at(wrapped[i])];
  lv.n = (int)masters.size();
  lv.coords.resize((size_t)lv.n * d);
  for (int c = 0; c < lv.n; ++c)
    for (int k = 0; k < d; ++k) lv.coords[(size_t)c * d + k] = own[masters[c]].x[k];
  const int d1 = d + 1, nc = r.nc();
  lv.cells.resize((size_t)nc * d1);
  lv.cell_coords.resize((size_t)nc * d1 * d);
  for (int e = 0; e < nc; ++e)
    for (int a = 0; a < d1; ++a) {
      int rv = r.cells[(size_t)e * d1 + a];
      lv.cells[(size_t)e * d1 + a] = raw2can[rv];
      for (int k = 0; k < d; ++k) lv.cell_coords[((size_t)e * d1 + a) * d + k] = r.coords[(size_t)rv * d + k];
    }
  // boundary faces, not on a periodic side.  d <= 2: faces of exactly one
  // cell (sorted vertex ids packed into one 64-bit key).  d = 3: the faces
  // whose vertices all lie on one side of the box - on a box domain exactly
  // the faces of one cell, found without a face table (a Kuhn mesh at level 7
  // has 5 10^7 cell faces)
  auto add_face = [&](const int* f) {
    for (int ax = 0; ax < d; ++ax)
      for (int side = -1; side <= 1; side += 2) {
        double bound = side < 0 ? m.lo[ax] : m.hi[ax];
        bool on = true;
        for (int a = 0; a < d; ++a) on = on && (r.coords[(size_t)f[a] * d + ax] == bound);
        if (!on || (m.periodic && m.periodic[ax])) continue;
        for (int a = 0; a < d; ++a) {
          lv.bfaces.push_back(raw2can[f[a]]);
          for (int k = 0; k < d; ++k) lv.bface_coords.push_back(r.coords[(size_t)f[a] * d + k]);
        }
        lv.bface_axis.push_back(ax);
        lv.bface_side.push_back(side);
      }
  };
  if (d == 3) {
    for (int e = 0; e < nc; ++e)
      for (int drop = 0; drop < d1; ++drop) {
        int f[3], k = 0;
        for (int a = 0; a < d1; ++a)
          if (a != drop) f[k++] = r.cells[(size_t)e * d1 + a];
        std::sort(f, f + 3);
        add_face(f);
      }
  } else {
    std::unordered_map<uint64_t, int> count;
    count.reserve((size_t)nc * d1);
    auto face_key = [&](int e, int drop) {
      int f[2] = {0, 0}, k = 0;
      for (int a = 0; a < d1; ++a)
        if (a != drop) f[k++] = r.cells[(size_t)e * d1 + a];
      if (k == 2 && f[0] > f[1]) std::swap(f[0], f[1]);
      return k == 1 ? (uint64_t)(uint32_t)f[0] : (((uint64_t)(uint32_t)f[0] << 32) | (uint32_t)f[1]);
    };
    for (int e = 0; e < nc; ++e)
      for (int drop = 0; drop < d1; ++drop) count[face_key(e, drop)]++;
    std::vector<uint64_t> once;
    for (auto& kv : count)
      if (kv.second == 1) once.push_back(kv.first);
    std::sort(once.begin(), once.end());
    for (uint64_t key : once) {
      int f[2];
      if (d == 1) f[0] = (int)key;
      else { f[0] = (int)(key >> 32); f[1] = (int)(key & 0xffffffffu); }
      add_face(f);
    }
  }
  // P1 adjacency pattern
  std::vector<std::vector<int>> adj(lv.n);
  for (int e = 0; e < nc; ++e)
    for (int a = 0; a < d1; ++a)
      for (int b = 0; b < d1; ++b) adj[lv.cells[(size_t)e * d1 + a]].push_back(lv.cells[(size_t)e * d1 + b]);
  Csr& P = lv.pattern;
  P.nrows = P.ncols = lv.n;
  P.rowptr.assign(lv.n + 1, 0);
  for (int i = 0; i < lv.n; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
    P.rowptr[i + 1] = P.rowptr[i] + (int)adj[i].size();
  }
  P.col.reserve(P.rowptr[lv.n]);
  for (int i = 0; i < lv.n; ++i) P.col.insert(P.col.end(), adj[i].begin(), adj[i].end());
}

Csr transpose(const Csr& A) {
  Csr T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.rowptr.assign(T.nrows + 1, 0);
  for (int c : A.col) T.rowptr[c + 1]++;
  for (int i = 0; i < T.nrows; ++i) T.rowptr[i + 1] += T.rowptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.col.size());
  std::vector<int> pos(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int i = 0; i < A.nrows; ++i)
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      int q = pos[A.col[p]]++;
      T.col[q] = i;
      T.val[q] = A.val[p];
    }
  return T;
}

}  // namespace

Status validate_mesh(const sgdg_mesh& m) {
  if (m.dim < 1 || m.dim > 3) return {SGDG_EINVAL, "mesh dim must be 1, 2 or 3"};
  if (m.n_vertices <= 0 || m.n_cells <= 0 || !m.coords || !m.cells || !m.lo || !m.hi)
    return {SGDG_EINVAL, "empty or incomplete mesh"};
  const int d = m.dim, k = d + 1;
  double box = 1.0, ext = 0.0;
  for (int a = 0; a < d; ++a) {
    if (!std::isfinite(m.lo[a]) || !std::isfinite(m.hi[a]) || !(m.lo[a] < m.hi[a]))
      return {SGDG_EINVAL, "mesh box: lo < hi (finite) on every axis"};
    box *= m.hi[a] - m.lo[a];
    ext = std::max(ext, m.hi[a] - m.lo[a]);
  }
  const double tol = 1e-12 * ext;
  auto X = [&](int v, int a) { return m.coords[(size_t)v * d + a]; };
  for (int v = 0; v < m.n_vertices; ++v)
    for (int a = 0; a < d; ++a)
      if (!std::isfinite(X(v, a)) || X(v, a) < m.lo[a] - tol || X(v, a) > m.hi[a] + tol)
        return {SGDG_EINVAL, "mesh vertex outside its box"};
  {
    std::vector<std::vector<double>> pts(m.n_vertices, std::vector<double>(d));
    for (int v = 0; v < m.n_vertices; ++v)
      for (int a = 0; a < d; ++a) pts[v][a] = X(v, a);
    std::sort(pts.begin(), pts.end());
    for (int v = 1; v < m.n_vertices; ++v)
      if (pts[v] == pts[v - 1]) return {SGDG_EINVAL, "two mesh vertices share their coordinates"};
  }
  // cells: indices in range, positive volume; the volumes tile the box
  double vol_sum = 0.0, fact = d == 1 ? 1.0 : d == 2 ? 2.0 : 6.0;
  std::map<std::vector<int>, int> faces;   // sorted face vertices -> cells holding it
  for (int c = 0; c < m.n_cells; ++c) {
    const int* cv = m.cells + (size_t)c * k;
    for (int i = 0; i < k; ++i)
      if (cv[i] < 0 || cv[i] >= m.n_vertices) return {SGDG_EINVAL, "cell vertex index out of range"};
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 1; i < k; ++i)
      for (int a = 0; a < d; ++a) J[a][i - 1] = X(cv[i], a) - X(cv[0], a);
    const double det = d == 1 ? J[0][0]
                     : d == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                     : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double vol = std::fabs(det) / fact;
    if (!(vol > 1e-12 * box)) return {SGDG_EINVAL, "degenerate mesh cell (zero volume)"};
    vol_sum += vol;
    for (int drop = 0; drop < k; ++drop) {
      std::vector<int> f;
      for (int i = 0; i < k; ++i)
        if (i != drop) f.push_back(cv[i]);
      std::sort(f.begin(), f.end());
      faces[f]++;
    }
  }
  if (std::fabs(vol_sum - box) > 1e-10 * box)
    return {SGDG_EINVAL, "mesh cells do not tile the box (overlap or hole)"};
  // conformity: a face lies in at most two cells, and a face of one cell lies
  // on a side of the box
  for (const auto& fc : faces) {
    if (fc.second > 2) return {SGDG_EINVAL, "a mesh face is shared by more than two cells"};
    if (fc.second == 2) continue;
    bool on_side = false;
    for (int a = 0; a < d && !on_side; ++a)
      for (double bound : {m.lo[a], m.hi[a]}) {
        bool all = true;
        for (int v : fc.first) all = all && std::fabs(X(v, a) - bound) <= tol;
        on_side = on_side || all;
      }
    if (!on_side) return {SGDG_EINVAL, "a boundary face of the mesh is not on a side of its box"};
  }
  // periodic axes: the vertices on the two opposite sides match
  for (int a = 0; a < d; ++a) {
    if (!m.periodic || !m.periodic[a]) continue;
    std::vector<std::vector<double>> side[2];
    for (int v = 0; v < m.n_vertices; ++v)
      for (int sd = 0; sd < 2; ++sd)
        if (std::fabs(X(v, a) - (sd ? m.hi[a] : m.lo[a])) <= tol) {
          std::vector<double> y;
          for (int b = 0; b < d; ++b)
            if (b != a) y.push_back(X(v, b));
          side[sd].push_back(y);
        }
    std::sort(side[0].begin(), side[0].end());
    std::sort(side[1].begin(), side[1].end());
    if (side[0] != side[1]) return {SGDG_EINVAL, "periodic axis: the vertices of the two sides do not match"};
  }
  return {};
}

Status build_hierarchy(const sgdg_mesh& m, int L, Hierarchy& h) {
  Status st;
  if (m.dim < 1 || m.dim > 3) return {SGDG_EINVAL, "mesh dim must be 1, 2 or 3"};
  if (m.n_vertices <= 0 || m.n_cells <= 0 || !m.coords || !m.cells || !m.lo || !m.hi)
    return {SGDG_EINVAL, "empty or incomplete mesh"};
  h.d = m.dim;
  h.L = L;
  RawMesh raw;
  raw.d = m.dim;
  raw.coords.assign(m.coords, m.coords + (size_t)m.n_vertices * m.dim);
  raw.cells.assign(m.cells, m.cells + (size_t)m.n_cells * (m.dim + 1));
  for (int v : raw.cells)
    if (v < 0 || v >= m.n_vertices) return {SGDG_EINVAL, "cell vertex index out of range"};
  raw.parent.resize(m.n_vertices);
  for (int i = 0; i < m.n_vertices; ++i) raw.parent[i] = {i, i};
  h.lev.assign(L + 1, MeshLevel());
  std::vector<int> r2c_prev, r2c;
  for (int l = 0; l <= L; ++l) {
    if (l > 0) raw = refine(raw);
    canonical(raw, m, h.lev[l], r2c);
    if (l > 0) {
      // E_{l <- l-1}
      const int nf = h.lev[l].n, nc = h.lev[l - 1].n;
      Csr E;
      E.nrows = nf;
      E.ncols = nc;
      std::vector<std::vector<std::pair<int, double>>> rows(nf);
      std::vector<char> done(nf, 0);
      std::vector<int> inj(nc, -1);
      for (int rv = 0; rv < raw.nv(); ++rv) {
        int i = r2c[rv];
        auto pr = raw.parent[rv];
        if (pr.first == pr.second) inj[r2c_prev[pr.first]] = r2c[rv];
        if (done[i]) continue;
        done[i] = 1;
        if (pr.first == pr.second) {
          rows[i].push_back({r2c_prev[pr.first], 1.0});
        } else {
          int a = r2c_prev[pr.first], b = r2c_prev[pr.second];
          if (a == b) rows[i].push_back({a, 1.0});
          else {
            rows[i].push_back({std::min(a, b), 0.5});
            rows[i].push_back({std::max(a, b), 0.5});
          }
        }
      }
      E.rowptr.assign(nf + 1, 0);
      for (int i = 0; i < nf; ++i) {
        if (!done[i]) return {SGDG_EINVAL, "refinement left a vertex without parents"};
        E.rowptr[i + 1] = E.rowptr[i] + (int)rows[i].size();
        for (auto& pv : rows[i]) { E.col.push_back(pv.first); E.val.push_back(pv.second); }
      }
      for (int k : inj)
        if (k < 0) return {SGDG_EINVAL, "injection map incomplete"};
      h.Rt.push_back(transpose(E));
      h.E.push_back(std::move(E));
      h.inj.push_back(std::move(inj));
    }
    r2c_prev = r2c;
  }
  return st;
}

}  // namespace sgdg
