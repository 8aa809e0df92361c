// Device helpers shared by the kernels: the blending map, on-the-fly element
// matrices (IFEM), value loads across the cell boundary, block reductions.
#pragma once

#include <cstdint>

#include "common.h"
#include "shell.h"

namespace hhg {

// The 24 tetrahedra around a node of the regular refinement, as direction
// triples (DIRS order of common.h).  They are the Freudenthal-Kuhn simplices
// x0, x0 + e_s1, x0 + e_s1 + e_s2, x0 + (1,1,1) in (alpha, beta, gamma) =
// (i + j + k, j + k, k) that contain the node; kuhn_star() derives the same
// table on the host and setup checks the two agree.
HD constexpr int star(int t, int a) {
  switch (t * 3 + a) {
    case 0: return 0; case 1: return 2; case 2: return 6;
    case 3: return 0; case 4: return 9; case 5: return 6;
    case 6: return 4; case 7: return 2; case 8: return 6;
    case 9: return 4; case 10: return 7; case 11: return 6;
    case 12: return 8; case 13: return 9; case 14: return 6;
    case 15: return 8; case 16: return 7; case 17: return 6;
    case 18: return 12; case 19: return 0; case 20: return 2;
    case 21: return 12; case 22: return 4; case 23: return 2;
    case 24: return 5; case 25: return 0; case 26: return 9;
    case 27: return 5; case 28: return 8; case 29: return 9;
    case 30: return 11; case 31: return 12; case 32: return 0;
    case 33: return 11; case 34: return 5; case 35: return 0;
    case 36: return 1; case 37: return 4; case 38: return 7;
    case 39: return 1; case 40: return 8; case 41: return 7;
    case 42: return 13; case 43: return 12; case 44: return 4;
    case 45: return 13; case 46: return 1; case 47: return 4;
    case 48: return 3; case 49: return 5; case 50: return 8;
    case 51: return 3; case 52: return 1; case 53: return 8;
    case 54: return 10; case 55: return 11; case 56: return 12;
    case 57: return 10; case 58: return 11; case 59: return 5;
    case 60: return 10; case 61: return 13; case 62: return 12;
    case 63: return 10; case 64: return 13; case 65: return 1;
    case 66: return 10; case 67: return 3; case 68: return 5;
    case 69: return 10; case 70: return 3; case 71: return 1;
  }
  return -1;
}

// Stencil direction offsets (DIRS order of common.h).
HD constexpr int DI(int w) {
  return w == 0 || w == 5 || w == 9 || w == 11 ? 1 : (w == 1 || w == 4 || w == 7 || w == 13 ? -1 : 0);
}
HD constexpr int DJ(int w) {
  return w == 2 || w == 4 || w == 12 || w == 13 ? 1 : (w == 3 || w == 5 || w == 8 || w == 9 ? -1 : 0);
}
HD constexpr int DK(int w) { return (w >= 6 && w <= 9) ? 1 : ((w >= 10 && w <= 13) ? -1 : 0); }

// Phi applied to the cell-local point (i, j, k) (Sec. 2.2), or the identity
// for an unprojected shell (the CONS operator on the polyhedral domain, Sec.
// 4.1; flagged by negative radii in the cell's geometry): the affine point
// sum_a lam_a v_a / N moved along its ray to radius sum_a lam_a r_a / N.
// Terms are accumulated in ascending vertex id, so a point shared by several
// cells gets the same position from each of them.
__device__ __forceinline__ void mapped_point(const CellGeom& g, int i, int j, int k, int N, double X[3]) {
  const double lam[4] = {(double)(N - i - j - k), (double)i, (double)j, (double)k};
  double x0 = 0, x1 = 0, x2 = 0, rho = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    x0 = fma(lam[a], g.x[a][0], x0);
    x1 = fma(lam[a], g.x[a][1], x1);
    x2 = fma(lam[a], g.x[a][2], x2);
    rho = fma(lam[a], g.r[a], rho);
  }
  // X = (rho / N) x / |x| with x, rho the unscaled sums (1/N is exact); a
  // cell of an unprojected shell (radii stored negative) keeps the affine
  // point x / N
  const double s = g.r[0] < 0.0 ? 1.0 / (double)N : (rho / (double)N) / sqrt(fma(x0, x0, fma(x1, x1, x2 * x2)));
  X[0] = s * x0;
  X[1] = s * x1;
  X[2] = s * x2;
}

// Row of node x in the element matrix of the tetrahedron (x, x+ea, x+eb, x+ec)
// (edge vectors from x): K_xa = (c0 . ca) / (6 |det|) with ca = eb x ec etc.
// and c0 = -(ca + cb + cc) (cofactors of the edge matrix), K_xx = c0.c0/(6|det|).
__device__ __forceinline__ void tet_row(const double ea[3], const double eb[3], const double ec[3],
                                        double& ka, double& kb, double& kc, double& kx) {
  const double ca0 = eb[1] * ec[2] - eb[2] * ec[1], ca1 = eb[2] * ec[0] - eb[0] * ec[2],
               ca2 = eb[0] * ec[1] - eb[1] * ec[0];
  const double cb0 = ec[1] * ea[2] - ec[2] * ea[1], cb1 = ec[2] * ea[0] - ec[0] * ea[2],
               cb2 = ec[0] * ea[1] - ec[1] * ea[0];
  const double cc0 = ea[1] * eb[2] - ea[2] * eb[1], cc1 = ea[2] * eb[0] - ea[0] * eb[2],
               cc2 = ea[0] * eb[1] - ea[1] * eb[0];
  const double det = ea[0] * ca0 + ea[1] * ca1 + ea[2] * ca2;
  const double inv = 1.0 / (6.0 * fabs(det));
  const double c00 = -(ca0 + cb0 + cc0), c01 = -(ca1 + cb1 + cc1), c02 = -(ca2 + cb2 + cc2);
  ka = (c00 * ca0 + c01 * ca1 + c02 * ca2) * inv;
  kb = (c00 * cb0 + c01 * cb1 + c02 * cb2) * inv;
  kc = (c00 * cc0 + c01 * cc1 + c02 * cc2) * inv;
  kx = (c00 * c00 + c01 * c01 + c02 * c02) * inv;
}

// Exact stencil of an interior node (IFEM, Sec. 4.2.1): the mapped positions
// of the node and its 14 neighbours, the 24 element-matrix rows summed per
// direction, centre by the row-sum property (the 1343-flop variant of
// Table 4.2).
__device__ __forceinline__ void ifem_stencil(const CellGeom& g, int N, int i, int j, int k, double s[15]) {
  double X[3];
  mapped_point(g, i, j, k, N, X);
  double e[14][3];
#pragma unroll
  for (int w = 0; w < 14; ++w) {
    double Y[3];
    mapped_point(g, i + DI(w), j + DJ(w), k + DK(w), N, Y);
    e[w][0] = Y[0] - X[0];
    e[w][1] = Y[1] - X[1];
    e[w][2] = Y[2] - X[2];
    s[w] = 0.0;
  }
#pragma unroll
  for (int t = 0; t < 24; ++t) {
    double ka, kb, kc, kx;
    tet_row(e[star(t, 0)], e[star(t, 1)], e[star(t, 2)], ka, kb, kc, kx);
    s[star(t, 0)] += ka;
    s[star(t, 1)] += kb;
    s[star(t, 2)] += kc;
  }
  double c = 0.0;
#pragma unroll
  for (int w = 0; w < 14; ++w) c -= s[w];
  s[MC] = c;
}

// Value of level vector v at cell-local point (i, j, k) of cell c: interior
// points from the canonical vector, boundary points from the cell's halo.
template <class T>
__device__ __forceinline__ T load_pt(const LevelView<T>& lv, const T* __restrict__ v, int c, int i, int j, int k) {
  if (is_interior(i, j, k, lv.N))
    return v[lv.off_C + (int64_t)c * lv.n_int + lin_interior(i, j, k, lv.N)];
  return lv.ghost[(int64_t)c * lv.n_full + lin_full(i, j, k, lv.N)];
}

// 32-bit position of an interior point among the cell's interior points
// (same value as lin_interior; fits int32 for N <= 1024).
__device__ __forceinline__ int lin_interior32(int i, int j, int k, int N) {
  const int M = N - 4, a = i - 1, b = j - 1, c = k - 1, m = M - c;
  auto tet = [](int n) { return (n + 1) * (n + 2) * (n + 3) / 6; };
  return tet(M) - tet(M - c) + b * (m + 1) - b * (b - 1) / 2 + a;
}

// True when all 14 neighbours of interior point (i, j, k) are interior too.
__device__ __forceinline__ bool deep_interior(int i, int j, int k, int N) {
  return i >= 2 && j >= 2 && k >= 2 && i + j + k <= N - 2;
}

// Offsets (in interior positions) of the 14 neighbours of a deep-interior
// point, DIRS order: with L = N-1-j-k the length of line (j, k) and
// T(m) = m(m+1)/2 the size of an interior plane, tc = T(N-2-k) - j + 1 and
// bc = -T(N-1-k) + j - 1; the others follow by +-1 and +-L.
__device__ __forceinline__ void neighbour_offsets(int j, int k, int N, int off[14]) {
  const int L = N - 1 - j - k;
  const int m1 = N - 2 - k, m0 = N - 1 - k;
  const int tc = m1 * (m1 + 1) / 2 - j + 1;
  const int bc = -(m0 * (m0 + 1) / 2) + j - 1;
  off[ME] = 1;
  off[MW] = -1;
  off[MN] = L;
  off[MS] = -(L + 1);
  off[MNW] = L - 1;
  off[MSE] = -L;
  off[TC] = tc;
  off[TW] = tc - 1;
  off[TS] = tc - L;
  off[TSE] = tc - L + 1;
  off[BC] = bc;
  off[BE] = bc + 1;
  off[BN] = bc + L + 1;
  off[BNW] = bc + L;
}

// Sum over a block (blockDim.x a multiple of 32, at most 1024); result valid
// in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? part[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// ---- FP32 surrogate: per-plane polynomials in (i, j) ----------------------

// Index of A_{a,b,d} (coefficient of i^a j^b k^d) in the storage order
// for a = 0..Q, for d = 0..Q-a, for b = 0..Q-a-d.
template <int Q>
__host__ __device__ constexpr int coef_index(int a, int b, int d) {
  int t = 0;
  for (int aa = 0; aa < a; ++aa) t += (Q - aa + 1) * (Q - aa + 2) / 2;
  for (int dd = 0; dd < d; ++dd) t += Q - a - dd + 1;
  return t + b;
}
// Per plane and direction: D_{a,b}(k) = sum_d A_{a,b,d} k^d, stored for
// a = 0..Q, b = 0..Q-a; (Q+1)(Q+2)/2 values.
template <int Q>
__host__ __device__ constexpr int plane_index(int a, int b) {
  int t = 0;
  for (int aa = 0; aa < a; ++aa) t += Q - aa + 1;
  return t + b;
}

template <class T, int Q>
__device__ __forceinline__ void plane_coeffs(const T* A, T k, T* P) {
#pragma unroll
  for (int a = 0; a <= Q; ++a)
#pragma unroll
    for (int b = 0; b <= Q - a; ++b) {
      T v = A[coef_index<Q>(a, b, Q - a - b)];
#pragma unroll
      for (int d = Q - a - b - 1; d >= 0; --d) v = fma(v, k, A[coef_index<Q>(a, b, d)]);
      P[plane_index<Q>(a, b)] = v;
    }
}

template <class T, int Q>
__device__ __forceinline__ T eval_plane(const T* P, T i, T j) {
  T s = 0;
#pragma unroll
  for (int a = Q; a >= 0; --a) {
    T c = P[plane_index<Q>(a, Q - a)];
#pragma unroll
    for (int b = Q - a - 1; b >= 0; --b) c = fma(c, j, P[plane_index<Q>(a, b)]);
    s = (a == Q) ? c : fma(s, i, c);
  }
  return s;
}

// Per-plane coefficients of one direction padded to a multiple of 4 floats
// (128-bit shared-memory loads).
template <int Q>
__host__ __device__ constexpr int np_pad() { return ((Q + 1) * (Q + 2) / 2 + 3) / 4 * 4; }

// Per-plane coefficients of the FP32 surrogate, paired by direction for
// packed FP32 arithmetic: pair m holds directions 2m and 2m + 1 (the centre,
// 14, is paired with zeros), NPP2 float2 per pair (a multiple of 16 bytes).
template <int Q>
__host__ __device__ constexpr int npp2() { return ((Q + 1) * (Q + 2) / 2 + 1) / 2 * 2; }
constexpr int NPAIR = 8;

// Two directions' polynomials in (i, j) at once (packed FP32 FMA).
template <int Q>
__device__ __forceinline__ float2 eval_plane2(const float2* P, float2 I, float2 J) {
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int a = Q; a >= 0; --a) {
    float2 c = P[plane_index<Q>(a, Q - a)];
#pragma unroll
    for (int b = Q - a - 1; b >= 0; --b) c = __ffma2_rn(c, J, P[plane_index<Q>(a, b)]);
    s = (a == Q) ? c : __ffma2_rn(s, I, c);
  }
  return s;
}

}  // namespace hhg
