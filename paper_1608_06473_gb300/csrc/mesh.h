// Host-side macro mesh of the spherical shell and per-level index maps.
//
// Sec. 2.2: an unstructured tetrahedral macro mesh T_{-2} of the shell is
// refined regularly; the refined nodes are moved by the blending map Phi.
// Sec. 2.3: nodes are grouped into vertex, edge, face and volume primitives.
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace hhg {

struct MacroMesh {
  double r1 = 0, r2 = 0;
  bool blend = true;                             // false: nodes stay on the polyhedral macro mesh (Phi = Id)
  int tang = 0, layers = 1;
  int nS = 0;                                    // surface vertices
  std::vector<std::array<double, 3>> vx;         // macro vertex positions
  std::vector<double> vr;                        // radius of each vertex's layer
  std::vector<int> vlayer;
  std::vector<std::array<int, 4>> cells;         // ascending global ids
  std::vector<std::array<int, 2>> edges;         // sorted pairs
  std::vector<std::array<int, 3>> faces;         // sorted triples
  std::map<std::array<int, 2>, int> edge_id;
  std::map<std::array<int, 3>, int> face_id;
  std::vector<std::array<int, 6>> cell_edges;    // local pairs 01 02 03 12 13 23
  std::vector<std::array<int, 4>> cell_faces;    // local triples 012 013 023 123
  std::vector<std::array<int, 3>> face_edges;    // local pairs 01 02 12 of a face

  int nV() const { return (int)vx.size(); }
  int nE() const { return (int)edges.size(); }
  int nF() const { return (int)faces.size(); }
  int nC() const { return (int)cells.size(); }

  bool vertex_dirichlet(int v) const { return vlayer[v] == 0 || vlayer[v] == layers; }
  bool edge_dirichlet(int e) const {
    const auto& E = edges[e];
    return vlayer[E[0]] == vlayer[E[1]] && vertex_dirichlet(E[0]);
  }
  bool face_dirichlet(int f) const {
    const auto& F = faces[f];
    return vlayer[F[0]] == vlayer[F[1]] && vlayer[F[1]] == vlayer[F[2]] && vertex_dirichlet(F[0]);
  }
};

MacroMesh build_shell(double r1, double r2, int tang, int layers);
MacroMesh build_shells(const std::vector<std::pair<double, double>>& radii, int tang, int layers);

// Canonical layout of the nodes of one level (N intervals per macro edge).
struct LevelLayout {
  int N = 0;
  int64_t nV = 0, nE = 0, nF = 0, nC = 0;
  int64_t off_E = 0, off_F = 0, off_C = 0, n_total = 0;
  int64_t n_int = 0, n_face = 0, n_full = 0;
};

LevelLayout make_layout(const MacroMesh& m, int N);

// Canonical index of a point given by integer barycentric weights lam[0..d-1]
// (summing to N) over the ascending global vertex ids g[0..d-1]; `cell` is
// needed when all four weights of a cell point are positive.
int64_t node_index(const MacroMesh& m, const LevelLayout& lay, int d, const int* g, const int* lam,
                   int cell);

// Same for a cell-local point (i, j, k) of cell c, using the cell's cached
// edge and face ids.
int64_t cell_node_index(const MacroMesh& m, const LevelLayout& lay, int c, int i, int j, int k);

// Dirichlet flag of a canonical node.
bool node_dirichlet(const MacroMesh& m, const LevelLayout& lay, int64_t idx);

// Mapped position Phi(x) of the point with weights lam over vertices g.
void blend_point(const MacroMesh& m, int d, const int* g, const int* lam, int N, double out[3]);

// Mapped positions of all nodes of a level (canonical order).
void level_coords(const MacroMesh& m, const LevelLayout& lay, double* xyz);

}  // namespace hhg
