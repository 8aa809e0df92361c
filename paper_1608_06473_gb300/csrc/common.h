// Shared index arithmetic, direction tables and error plumbing of libhhg.
//
// Macro-cell indexing (Sec. 2.3): a point of a macro cell refined into N
// intervals per edge is (i, j, k) with i, j, k >= 0 and i + j + k <= N; its
// barycentric weights are (N - i - j - k, i, j, k) over the cell's vertices
// in ascending global id.  Interior points (i, j, k >= 1, i + j + k <= N - 1)
// form the volume primitive; their count is n_l of Eq. 2.5.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/hhg.h"

#define HD __host__ __device__ __forceinline__

namespace hhg {

// ---------------------------------------------------------------------------
// Counting and linear positions inside one macro cell / face
// ---------------------------------------------------------------------------

// Points (a, b, c) >= 0 with a + b + c <= n.
HD int64_t tet_points(int64_t n) { return (n + 1) * (n + 2) * (n + 3) / 6; }

// Position of (i, j, k) in the full cell (all i + j + k <= N), i fastest.
HD int64_t lin_full(int i, int j, int k, int N) {
  const int64_t m = N - k;
  return tet_points(N) - tet_points(N - k) + (int64_t)j * (m + 1) - (int64_t)j * (j - 1) / 2 + i;
}

// Position of an interior (i, j, k) among the cell's interior points.
HD int64_t lin_interior(int i, int j, int k, int N) { return lin_full(i - 1, j - 1, k - 1, N - 4); }

// Position of a face-interior point (p, q) (p, q >= 1, p + q <= N - 1), p fastest.
HD int64_t lin_face(int p, int q, int N) {
  return (int64_t)(q - 1) * (N - 1) - (int64_t)q * (q - 1) / 2 + (p - 1);
}

HD int64_t n_cell_interior(int N) { return (int64_t)(N - 1) * (N - 2) * (N - 3) / 6; }
HD int64_t n_face_interior(int N) { return (int64_t)(N - 1) * (N - 2) / 2; }
HD int64_t n_cell_full(int N) { return tet_points(N); }

HD bool is_interior(int i, int j, int k, int N) {
  return i >= 1 && j >= 1 && k >= 1 && i + j + k <= N - 1;
}

// ---------------------------------------------------------------------------
// The 15 stencil directions (Sec. 2.3): first letter bottom / middle / top
// plane (k - 1, k, k + 1), then the direction inside the plane; mc = centre.
// ---------------------------------------------------------------------------
enum Dir { ME = 0, MW, MN, MS, MNW, MSE, TC, TW, TS, TSE, BC, BE, BN, BNW, MC, NDIR };

HD int dir_di(int w) { const int t[15] = {1, -1, 0, 0, -1, 1, 0, -1, 0, 1, 0, 1, 0, -1, 0}; return t[w]; }
HD int dir_dj(int w) { const int t[15] = {0, 0, 1, -1, 1, -1, 0, 0, -1, -1, 0, 0, 1, 1, 0}; return t[w]; }
HD int dir_dk(int w) { const int t[15] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1, 0}; return t[w]; }

// Direction index of an (i, j, k) offset, -1 if it is not a stencil edge.
inline int dir_of(int di, int dj, int dk) {
  for (int w = 0; w < 15; ++w)
    if (dir_di(w) == di && dir_dj(w) == dj && dir_dk(w) == dk) return w;
  return -1;
}

// The 24 tetrahedra of the refined mesh that meet at a node, each as the
// three direction indices of its other vertices (filled by kuhn_star()).
struct Star { int8_t t[24][3]; };
void kuhn_star(Star* s);

// Counts kernel launches (diagnostics).
void count_launch(int n = 1);

// ---------------------------------------------------------------------------
// Status plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

struct Error {
  hhg_status st;
  std::string msg;
};

}  // namespace hhg

#define HHG_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::hhg::Error{HHG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};   \
  } while (0)

#define HHG_CHECK(cond, status, msg)                     \
  do {                                                   \
    if (!(cond)) throw ::hhg::Error{(status), (msg)};    \
  } while (0)
