// Line-wise evaluation of the FP64 surrogate weights (Sec. 3.4, Eq. 5.4):
// along a line (j, k) of a macro cell each direction's polynomial is a
// polynomial of degree q in i, so its values at i0, i0 + h, i0 + 2h, .. follow
// from a difference table by additions.  The table holds integers (the plane
// coefficients scaled by 2^E and rounded at fit time), and all arithmetic is
// exact modulo 2^64, so every value equals the direct (Horner) evaluation of
// the same integer polynomial.  Shared by the per-colour run kernel (cell.cu)
// and the cell-resident sweep (resident.cu).
#pragma once

#include <cstdint>

#include "arith.cuh"
#include "device.cuh"

namespace hhg {

// int64 per direction and plane in the FP64 plane table: the (Q+1)(Q+2)/2
// coefficients of the polynomial in (i, j), rounded up to an even count.
template <int Q>
constexpr int NPP64 = ((Q + 1) * (Q + 2) / 2 + 1) / 2 * 2;

// Offset (in interior positions) of neighbour w of a deep-interior point of
// line (j, k), for a direction known only at run time: the closed forms of
// neighbour_offsets with L = N - 1 - j - k and its plane offsets tc, bc.
__device__ __forceinline__ int neighbour_offset(int w, int L, int tc, int bc) {
  const int di = DI(w), dj = DJ(w), dk = DK(w);
  if (dk == 0) return di + (dj == 1 ? L : (dj == -1 ? -(L + 1) : 0));
  if (dk == 1) return tc + di + (dj == -1 ? -L : 0);
  return bc + di + (dj == 1 ? L + 1 : 0);
}

// Difference table of one direction's polynomial along line j from i0 with
// step h: the line coefficients A_a(j) (Horner in j, as eval_plane_i64),
// the values at i0, i0 + h, .., i0 + Q h (Horner in i), then D[m] = the m-th
// forward difference at i0.  All integer arithmetic is exact modulo 2^64, so
// after s steps D[0] is the same integer as eval_plane_i64 at i0 + s h.
template <int Q>
__device__ __forceinline__ void run_start(const long long* P, unsigned i0, unsigned j, unsigned h, long long D[Q + 1]) {
  long long r[NPP64<Q>];
#pragma unroll
  for (int t = 0; t < NPP64<Q> / 2; ++t) {
    const longlong2 x = reinterpret_cast<const longlong2*>(P)[t];
    r[2 * t] = x.x;
    r[2 * t + 1] = x.y;
  }
  long long A[Q + 1];
#pragma unroll
  for (int a = 0; a <= Q; ++a) {
    long long c = r[plane_index<Q>(a, Q - a)];
#pragma unroll
    for (int b = Q - a - 1; b >= 0; --b) c = mad_i64_u32(c, j, r[plane_index<Q>(a, b)]);
    A[a] = c;
  }
#pragma unroll
  for (int s = 0; s <= Q; ++s) {
    const unsigned x = i0 + (unsigned)s * h;
    long long v = A[Q];
#pragma unroll
    for (int a = Q - 1; a >= 0; --a) v = mad_i64_u32(v, x, A[a]);
    D[s] = v;
  }
#pragma unroll
  for (int m = 1; m <= Q; ++m)
#pragma unroll
    for (int s = Q; s >= m; --s) D[s] = (long long)((unsigned long long)D[s] - (unsigned long long)D[s - 1]);
}

// One step along the line: D[0] becomes the value at the next point.
template <int Q>
__device__ __forceinline__ void run_step(long long D[Q + 1]) {
#pragma unroll
  for (int m = 0; m < Q; ++m) D[m] = (long long)((unsigned long long)D[m] + (unsigned long long)D[m + 1]);
}

}  // namespace hhg
