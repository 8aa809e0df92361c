// Host-side macro mesh of the spherical shell (Sec. 2.2) and the canonical
// node layout of its refinement levels (Sec. 2.3).
//
// Macro mesh: the 12 vertices of the icosahedron (cyclic permutations of
// (0, +-1, +-g), g the golden ratio) on the unit sphere; `tang` 1:4 splits of
// every surface triangle with edge midpoints projected to the sphere; `layers`
// uniform radial layers between r1 and r2; every prism cut into the three
// tetrahedra {b0 b1 b2 t2}, {b0 b1 t1 t2}, {b0 t0 t1 t2} (surface ids
// s0 < s1 < s2, bottom b, top t), which cuts each quadrilateral from the
// bottom of its lower id to the top of its higher id and so conforms.
//
// This file is compiled with floating-point contraction disabled so that the
// same positions come out on every host architecture.
#include "mesh.h"

#include <algorithm>
#include <cmath>
#include <set>
#include <stdexcept>

#include "common.h"

namespace hhg {

namespace {

using V3 = std::array<double, 3>;

V3 unit(const V3& x) {
  const double n = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  return {x[0] / n, x[1] / n, x[2] / n};
}

void icosahedron(std::vector<V3>& xs, std::vector<std::array<int, 3>>& tris) {
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  const double raw[12][3] = {{0, -1, -g}, {0, -1, g}, {0, 1, -g}, {0, 1, g},
                             {-1, -g, 0}, {-1, g, 0}, {1, -g, 0}, {1, g, 0},
                             {-g, 0, -1}, {-g, 0, 1}, {g, 0, -1}, {g, 0, 1}};
  auto d2 = [&](int a, int b) {
    double s = 0;
    for (int c = 0; c < 3; ++c) s += (raw[a][c] - raw[b][c]) * (raw[a][c] - raw[b][c]);
    return s;
  };
  tris.clear();
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b)
      for (int c = b + 1; c < 12; ++c)
        if (std::fabs(d2(a, b) - 4) < 1e-9 && std::fabs(d2(a, c) - 4) < 1e-9 && std::fabs(d2(b, c) - 4) < 1e-9)
          tris.push_back({a, b, c});
  xs.clear();
  for (auto& r : raw) xs.push_back(unit({r[0], r[1], r[2]}));
}

void refine_sphere(std::vector<V3>& xs, std::vector<std::array<int, 3>>& tris) {
  std::set<std::array<int, 2>> eset;
  for (auto& t : tris) {
    eset.insert({t[0], t[1]});
    eset.insert({t[0], t[2]});
    eset.insert({t[1], t[2]});
  }
  std::map<std::array<int, 2>, int> eid;
  const int n0 = (int)xs.size();
  int m = 0;
  std::vector<V3> mids;
  for (auto& e : eset) {
    eid[e] = n0 + m++;
    const V3& a = xs[e[0]];
    const V3& b = xs[e[1]];
    mids.push_back(unit({a[0] + b[0], a[1] + b[1], a[2] + b[2]}));
  }
  for (auto& x : mids) xs.push_back(x);
  std::vector<std::array<int, 3>> out;
  for (auto& t : tris) {
    const int a = t[0], b = t[1], c = t[2];
    const int ab = eid[{a, b}], ac = eid[{a, c}], bc = eid[{b, c}];
    std::array<int, 3> ch[4] = {{a, ab, ac}, {ab, b, bc}, {ac, bc, c}, {ab, bc, ac}};
    for (auto& x : ch) {
      std::sort(x.begin(), x.end());
      out.push_back(x);
    }
  }
  std::sort(out.begin(), out.end());
  tris = out;
}

}  // namespace

MacroMesh build_shell(double r1, double r2, int tang, int layers) {
  return build_shells({{r1, r2}}, tang, layers);
}

// Several shells as one macro mesh of disjoint components: shell s gets the
// vertex ids after those of shells 0..s-1, so its vertices, edges, faces and
// cells follow theirs in every primitive class.
MacroMesh build_shells(const std::vector<std::pair<double, double>>& radii_in, int tang, int layers) {
  MacroMesh m;
  m.r1 = radii_in.front().first;
  m.r2 = radii_in.front().second;
  m.tang = tang;
  m.layers = layers;
  std::vector<V3> xs;
  std::vector<std::array<int, 3>> tris;
  icosahedron(xs, tris);
  for (int t = 0; t < tang; ++t) refine_sphere(xs, tris);
  const int nS = (int)xs.size();
  m.nS = nS;
  for (const auto& rr : radii_in) {
    const double r1 = rr.first, r2 = rr.second;
    const int vo = (int)m.vx.size();
    std::vector<double> radii(layers + 1);
    for (int l = 0; l <= layers; ++l) radii[l] = r1 + (r2 - r1) * l / layers;
    for (int l = 0; l <= layers; ++l)
      for (int s = 0; s < nS; ++s) {
        m.vx.push_back({radii[l] * xs[s][0], radii[l] * xs[s][1], radii[l] * xs[s][2]});
        m.vr.push_back(radii[l]);
        m.vlayer.push_back(l);
      }
    for (int l = 0; l < layers; ++l)
      for (auto& t : tris) {
        const int b0 = vo + l * nS + t[0], b1 = vo + l * nS + t[1], b2 = vo + l * nS + t[2];
        const int t0 = b0 + nS, t1 = b1 + nS, t2 = b2 + nS;
        std::array<int, 4> cs[3] = {{b0, b1, b2, t2}, {b0, b1, t1, t2}, {b0, t0, t1, t2}};
        for (auto& c : cs) {
          std::sort(c.begin(), c.end());
          m.cells.push_back(c);
        }
      }
  }
  std::set<std::array<int, 2>> es;
  std::set<std::array<int, 3>> fs;
  for (auto& c : m.cells) {
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        es.insert({c[a], c[b]});
        for (int d = b + 1; d < 4; ++d) fs.insert({c[a], c[b], c[d]});
      }
  }
  m.edges.assign(es.begin(), es.end());
  m.faces.assign(fs.begin(), fs.end());
  for (int e = 0; e < m.nE(); ++e) m.edge_id[m.edges[e]] = e;
  for (int f = 0; f < m.nF(); ++f) m.face_id[m.faces[f]] = f;
  for (auto& c : m.cells) {
    m.cell_edges.push_back({m.edge_id[{c[0], c[1]}], m.edge_id[{c[0], c[2]}], m.edge_id[{c[0], c[3]}],
                            m.edge_id[{c[1], c[2]}], m.edge_id[{c[1], c[3]}], m.edge_id[{c[2], c[3]}]});
    m.cell_faces.push_back({m.face_id[{c[0], c[1], c[2]}], m.face_id[{c[0], c[1], c[3]}],
                            m.face_id[{c[0], c[2], c[3]}], m.face_id[{c[1], c[2], c[3]}]});
  }
  for (auto& f : m.faces)
    m.face_edges.push_back({m.edge_id[{f[0], f[1]}], m.edge_id[{f[0], f[2]}], m.edge_id[{f[1], f[2]}]});
  return m;
}

LevelLayout make_layout(const MacroMesh& m, int N) {
  LevelLayout L;
  L.N = N;
  L.nV = m.nV();
  L.nE = m.nE();
  L.nF = m.nF();
  L.nC = m.nC();
  L.n_int = n_cell_interior(N);
  L.n_face = n_face_interior(N);
  L.n_full = n_cell_full(N);
  L.off_E = L.nV;
  L.off_F = L.off_E + L.nE * (N - 1);
  L.off_C = L.off_F + L.nF * L.n_face;
  L.n_total = L.off_C + L.nC * L.n_int;
  return L;
}

int64_t node_index(const MacroMesh& m, const LevelLayout& lay, int d, const int* g, const int* lam, int cell) {
  int sg[4], sl[4], n = 0;
  for (int a = 0; a < d; ++a)
    if (lam[a] > 0) {
      sg[n] = g[a];
      sl[n] = lam[a];
      ++n;
    }
  const int N = lay.N;
  switch (n) {
    case 1:
      return sg[0];
    case 2: {
      auto it = m.edge_id.find({sg[0], sg[1]});
      if (it == m.edge_id.end()) throw std::runtime_error("node_index: not an edge");
      return lay.off_E + (int64_t)it->second * (N - 1) + (sl[1] - 1);
    }
    case 3: {
      auto it = m.face_id.find({sg[0], sg[1], sg[2]});
      if (it == m.face_id.end()) throw std::runtime_error("node_index: not a face");
      return lay.off_F + (int64_t)it->second * lay.n_face + lin_face(sl[1], sl[2], N);
    }
    case 4:
      return lay.off_C + (int64_t)cell * lay.n_int + lin_interior(sl[1], sl[2], sl[3], N);
  }
  throw std::runtime_error("node_index: empty support");
}

int64_t cell_node_index(const MacroMesh& m, const LevelLayout& lay, int c, int i, int j, int k) {
  const int N = lay.N;
  const int lam[4] = {N - i - j - k, i, j, k};
  int mask = 0;
  for (int a = 0; a < 4; ++a)
    if (lam[a] > 0) mask |= 1 << a;
  const auto& C = m.cells[c];
  const auto& E = m.cell_edges[c];
  const auto& F = m.cell_faces[c];
  switch (mask) {
    case 1: return C[0];
    case 2: return C[1];
    case 4: return C[2];
    case 8: return C[3];
    case 3: return lay.off_E + (int64_t)E[0] * (N - 1) + (lam[1] - 1);
    case 5: return lay.off_E + (int64_t)E[1] * (N - 1) + (lam[2] - 1);
    case 9: return lay.off_E + (int64_t)E[2] * (N - 1) + (lam[3] - 1);
    case 6: return lay.off_E + (int64_t)E[3] * (N - 1) + (lam[2] - 1);
    case 10: return lay.off_E + (int64_t)E[4] * (N - 1) + (lam[3] - 1);
    case 12: return lay.off_E + (int64_t)E[5] * (N - 1) + (lam[3] - 1);
    case 7: return lay.off_F + (int64_t)F[0] * lay.n_face + lin_face(lam[1], lam[2], N);
    case 11: return lay.off_F + (int64_t)F[1] * lay.n_face + lin_face(lam[1], lam[3], N);
    case 13: return lay.off_F + (int64_t)F[2] * lay.n_face + lin_face(lam[2], lam[3], N);
    case 14: return lay.off_F + (int64_t)F[3] * lay.n_face + lin_face(lam[2], lam[3], N);
    case 15: return lay.off_C + (int64_t)c * lay.n_int + lin_interior(i, j, k, N);
  }
  throw std::runtime_error("cell_node_index: point outside the cell");
}

bool node_dirichlet(const MacroMesh& m, const LevelLayout& lay, int64_t idx) {
  if (idx < lay.off_E) return m.vertex_dirichlet((int)idx);
  if (idx < lay.off_F) return m.edge_dirichlet((int)((idx - lay.off_E) / (lay.N - 1)));
  if (idx < lay.off_C) return m.face_dirichlet((int)((idx - lay.off_F) / lay.n_face));
  return false;
}

void blend_point(const MacroMesh& m, int d, const int* g, const int* lam, int N, double out[3]) {
  double xh[3] = {0, 0, 0}, rho = 0;
  for (int a = 0; a < d; ++a) {
    const double l = (double)lam[a];
    for (int c = 0; c < 3; ++c) xh[c] = xh[c] + l * m.vx[g[a]][c];
    rho = rho + l * m.vr[g[a]];
  }
  for (int c = 0; c < 3; ++c) xh[c] = xh[c] / N;
  if (!m.blend) {  // unprojected shell: Phi = Id
    for (int c = 0; c < 3; ++c) out[c] = xh[c];
    return;
  }
  rho = rho / N;
  const double nrm = std::sqrt(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
  for (int c = 0; c < 3; ++c) out[c] = rho * xh[c] / nrm;
}

void level_coords(const MacroMesh& m, const LevelLayout& lay, double* xyz) {
  const int N = lay.N;
  for (int v = 0; v < m.nV(); ++v)
    for (int c = 0; c < 3; ++c) xyz[3 * v + c] = m.vx[v][c];
  for (int e = 0; e < m.nE(); ++e)
    for (int p = 1; p < N; ++p) {
      const int lam[2] = {N - p, p};
      blend_point(m, 2, m.edges[e].data(), lam, N, xyz + 3 * (lay.off_E + (int64_t)e * (N - 1) + p - 1));
    }
  for (int f = 0; f < m.nF(); ++f)
    for (int q = 1; q < N - 1; ++q)
      for (int p = 1; p < N - q; ++p) {
        const int lam[3] = {N - p - q, p, q};
        blend_point(m, 3, m.faces[f].data(), lam, N,
                    xyz + 3 * (lay.off_F + (int64_t)f * lay.n_face + lin_face(p, q, N)));
      }
  for (int c = 0; c < m.nC(); ++c) {
    int64_t o = lay.off_C + (int64_t)c * lay.n_int;
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N - k; ++j)
        for (int i = 1; i < N - j - k; ++i) {
          const int lam[4] = {N - i - j - k, i, j, k};
          blend_point(m, 4, m.cells[c].data(), lam, N, xyz + 3 * (o++));
        }
  }
}

}  // namespace hhg
