// Load vector of the accuracy study (Sec. 4): b_I = V_I f_I for every
// unknown, with V_I = sum of |T| / 4 over the fine tetrahedra T containing
// node I (the vertex quadrature rule on each tetrahedron; V_I is the row sum
// of the P1 mass matrix) on the blended (or, for an unprojected shell,
// straight) fine mesh; 0 at Dirichlet nodes.
#include "device.cuh"
#include "kernels.h"

namespace hhg {
namespace {

unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// |det(ea, eb, ec)| = 6 |T| for the tetrahedron spanned by three edge vectors.
__device__ __forceinline__ double det6(const double ea[3], const double eb[3], const double ec[3]) {
  const double c0 = eb[1] * ec[2] - eb[2] * ec[1], c1 = eb[2] * ec[0] - eb[0] * ec[2], c2 = eb[0] * ec[1] - eb[1] * ec[0];
  return fabs(ea[0] * c0 + ea[1] * c1 + ea[2] * c2);
}

// Sum of |T| / 4 over the star tetrahedra of cell-local point (i, j, k) that
// lie in the closed cell (all 24 for an interior point).
__device__ double star_volume(const CellGeom& g, int N, int i, int j, int k) {
  double X[3];
  mapped_point(g, i, j, k, N, X);
  double e[14][3];
  bool in[14];
  for (int w = 0; w < 14; ++w) {
    const int a = i + DI(w), b = j + DJ(w), d = k + DK(w);
    in[w] = a >= 0 && b >= 0 && d >= 0 && a + b + d <= N;
    if (in[w]) {
      double Y[3];
      mapped_point(g, a, b, d, N, Y);
      e[w][0] = Y[0] - X[0];
      e[w][1] = Y[1] - X[1];
      e[w][2] = Y[2] - X[2];
    }
  }
  double v = 0.0;
  for (int t = 0; t < 24; ++t) {
    const int wa = star(t, 0), wb = star(t, 1), wc = star(t, 2);
    if (in[wa] && in[wb] && in[wc]) v += det6(e[wa], e[wb], e[wc]);
  }
  return v / 24.0;
}

__global__ void load_cell_kernel(LevelView<double> lv, const double* __restrict__ f, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)lv.nC * lv.n_int) return;
  const int c = (int)(t / lv.n_int);
  const uint32_t p = lv.int_ijk[t - (int64_t)c * lv.n_int];
  const int64_t r = lv.off_C + t;
  b[r] = star_volume(lv.geom[c], lv.N, unpack_i(p), unpack_j(p), unpack_k(p)) * f[r];
}

__global__ void load_low_kernel(LevelView<double> lv, const int64_t* __restrict__ inc_ptr,
                                const int* __restrict__ inc_cb, const double* __restrict__ f, double* __restrict__ b) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= lv.off_C) return;
  double v = 0.0;
  for (int64_t q = inc_ptr[r]; q < inc_ptr[r + 1]; ++q) {
    const int cb = inc_cb[q];
    const int c = cb / lv.n_bnd;
    const uint32_t p = lv.bnd_ijk[cb - c * lv.n_bnd];
    v += star_volume(lv.geom[c], lv.N, unpack_i(p), unpack_j(p), unpack_k(p));
  }
  b[r] = v * f[r];  // Dirichlet nodes have no incidence: 0
}

}  // namespace

void launch_load_vector(const LevelView<double>& lv, const int64_t* inc_ptr, const int* inc_cb, const double* f,
                        double* b, cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * lv.n_int;
  if (n) load_cell_kernel<<<grid_for(n, 128), 128, 0, st>>>(lv, f, b);
  if (lv.off_C) load_low_kernel<<<grid_for(lv.off_C, 64), 64, 0, st>>>(lv, inc_ptr, inc_cb, f, b);
  HHG_CUDA(cudaGetLastError());
  count_launch((n ? 1 : 0) + (lv.off_C ? 1 : 0));
}

}  // namespace hhg
