// Host numerics for the setup: the least-squares pseudo-inverse of the LSQP
// sampling matrix (Sec. 3.2) and the derivation of the 24-tetrahedra star.
#include "linalg.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>

#include "common.h"

namespace hhg {

// A (m x n, row-major, m >= n, full column rank) = Q1 R by Householder
// reflections; returns A+ = R^{-1} Q1^T (n x m, row-major), the matrix that
// maps sample values b to the least-squares coefficients argmin ||A z - b||.
// DGELS, which the paper uses (Sec. 4.2.2), solves the same problem by the
// same QR factorisation.
std::vector<double> lsq_pinv(const std::vector<double>& A_in, int m, int n) {
  if (m < n) throw std::runtime_error("lsq_pinv: fewer samples than coefficients");
  std::vector<double> A = A_in;            // overwritten by R (upper part) and reflectors
  std::vector<std::vector<double>> V(n);   // Householder vectors
  for (int c = 0; c < n; ++c) {
    double nrm = 0;
    for (int r = c; r < m; ++r) nrm += A[(size_t)r * n + c] * A[(size_t)r * n + c];
    nrm = std::sqrt(nrm);
    if (nrm == 0) throw std::runtime_error("lsq_pinv: rank deficient sampling matrix");
    const double a0 = A[(size_t)c * n + c];
    const double alpha = a0 > 0 ? -nrm : nrm;
    std::vector<double> v(m - c);
    for (int r = c; r < m; ++r) v[r - c] = A[(size_t)r * n + c];
    v[0] -= alpha;
    double vn = 0;
    for (double x : v) vn += x * x;
    for (int cc = c; cc < n; ++cc) {  // A <- (I - 2 v v^T / v^T v) A
      double d = 0;
      for (int r = c; r < m; ++r) d += v[r - c] * A[(size_t)r * n + cc];
      const double s = 2 * d / vn;
      for (int r = c; r < m; ++r) A[(size_t)r * n + cc] -= s * v[r - c];
    }
    for (double& x : v) x /= std::sqrt(vn);  // unit reflector
    V[c] = v;
  }
  // Q1 = H_0 H_1 ... H_{n-1} [I_n; 0]
  std::vector<double> Q((size_t)m * n, 0.0);
  for (int c = 0; c < n; ++c) Q[(size_t)c * n + c] = 1.0;
  for (int c = n - 1; c >= 0; --c) {
    const auto& v = V[c];
    for (int cc = 0; cc < n; ++cc) {
      double d = 0;
      for (int r = c; r < m; ++r) d += v[r - c] * Q[(size_t)r * n + cc];
      for (int r = c; r < m; ++r) Q[(size_t)r * n + cc] -= 2 * d * v[r - c];
    }
  }
  // A+ = R^{-1} Q1^T: back substitution for every sample column
  std::vector<double> P((size_t)n * m);
  for (int r = 0; r < m; ++r) {
    for (int i = n - 1; i >= 0; --i) {
      double s = Q[(size_t)r * n + i];
      for (int k = i + 1; k < n; ++k) s -= A[(size_t)i * n + k] * P[(size_t)k * m + r];
      P[(size_t)i * m + r] = s / A[(size_t)i * n + i];
    }
  }
  return P;
}

void kuhn_star(Star* s) {
  // Freudenthal-Kuhn simplices in (alpha, beta, gamma) = (i+j+k, j+k, k):
  // x0, x0 + e_s1, x0 + e_s1 + e_s2, x0 + (1,1,1) for every permutation s of
  // the three axes; keep the 24 that contain the origin.
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int n = 0;
  for (int sx = 0; sx < 2; ++sx)
    for (int sy = 0; sy < 2; ++sy)
      for (int sz = 0; sz < 2; ++sz)
        for (auto& p : perms) {
          std::array<std::array<int, 3>, 4> v;
          v[0] = {-sx, -sy, -sz};
          v[1] = v[0];
          v[1][p[0]] += 1;
          v[2] = v[1];
          v[2][p[1]] += 1;
          v[3] = {v[0][0] + 1, v[0][1] + 1, v[0][2] + 1};
          int at = -1;
          for (int a = 0; a < 4; ++a)
            if (v[a][0] == 0 && v[a][1] == 0 && v[a][2] == 0) at = a;
          if (at < 0) continue;
          int m = 0;
          for (int a = 0; a < 4; ++a) {
            if (a == at) continue;
            const int di = v[a][0] - v[a][1], dj = v[a][1] - v[a][2], dk = v[a][2];
            const int w = dir_of(di, dj, dk);
            if (w < 0) throw std::runtime_error("kuhn_star: edge outside the 14 directions");
            s->t[n][m++] = (int8_t)w;
          }
          ++n;
        }
  if (n != 24) throw std::runtime_error("kuhn_star: expected 24 tetrahedra");
}

}  // namespace hhg
