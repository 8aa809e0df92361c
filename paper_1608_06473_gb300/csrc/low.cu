// Kernels for the lower primitives (macro vertices, edges and faces), the
// halo copies, the grid transfers, reductions and the coarse-solver vectors.
//
// Lower-primitive nodes keep their exact stencils (Sec. 3.4: only volume
// primitive stencils are replaced).  They are assembled once per level at
// setup from the element matrices of every adjacent macro cell (the same
// values the paper reassembles on the fly, Sec. 2.3) and stored as sliced
// ELL rows over canonical columns.  Their O(2^{2l}) nodes (Sec. 2.3) are a
// small share of the work.
#include <algorithm>

#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace hhg {

namespace {

constexpr int LOW_THREADS = 256;
constexpr int LOW_MAX_COLS = 96;

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Halo: copy the owner value of every boundary point of every cell into the
// cell's halo array (0 at Dirichlet points).  Stands where the paper's HHG
// exchanges ghost layers between primitives (Sec. 4; Sec. 6).
// Right-hand side blockIdx.y.
template <class T>
__global__ void halo_kernel(LevelView<T> lv, const T* __restrict__ u) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)lv.nC * lv.n_bnd) return;
  const int c = (int)(t / lv.n_bnd), b = (int)(t % lv.n_bnd);
  const uint32_t p = lv.bnd_ijk[b];
  const int src = lv.halo_src[t];
  const int64_t rb = blockIdx.y;
  lv.ghost[rb * lv.gstride + (int64_t)c * lv.n_full + lin_full(unpack_i(p), unpack_j(p), unpack_k(p), lv.N)] =
      src >= 0 ? u[rb * lv.vstride + src] : T(0);
}

// Off-diagonal part of the lower row stored at position p.
template <class T>
__device__ __forceinline__ T low_row_offdiag(const LevelView<T>& lv, int64_t p, const T* __restrict__ u) {
  const int64_t s = p >> 5, lane = p & 31;
  const int64_t beg = lv.sell_ptr[s], width = (lv.sell_ptr[s + 1] - beg) >> 5;
  T acc = 0;
  for (int64_t kk = 0; kk < width; ++kk) {
    const int64_t e = beg + kk * 32 + lane;
    const int col = lv.sell_col[e];
    if (col >= 0) acc = fma(lv.sell_val[e], u[col], acc);
  }
  return acc;
}

// Right-hand side blockIdx.y.
template <class T, Mode MODE>
__global__ void __launch_bounds__(LOW_THREADS) low_kernel(LevelView<T> lv, const T* __restrict__ u, T* __restrict__ out,
                                                        const T* __restrict__ f, double* partial) {
  const int64_t rb = blockIdx.y;
  u += rb * lv.vstride;
  out += rb * lv.vstride;
  if (MODE == RESIDUAL) {
    f += rb * lv.vstride;
    partial += rb * lv.pstride;
  }
  double nrm = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < lv.off_C; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = lv.low_perm[p];
    const T d = lv.low_diag[r];
    T y = 0;
    if (d != T(0)) y = fma(d, u[r], low_row_offdiag(lv, p, u));
    if (MODE == APPLY) {
      out[r] = y;
    } else {
      const T res = (d != T(0)) ? f[r] - y : T(0);
      out[r] = res;
      nrm += (double)res * (double)res;
    }
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
  }
}

// One lower-primitive colour step: new values of every listed node from the
// values at the start of the step (Eq. 5.1), written to tmp.
template <class T>
__global__ void low_step_kernel(LevelView<T> lv, int pbeg, int n, const T* __restrict__ u, const T* __restrict__ f,
                                T* __restrict__ tmp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t rb = blockIdx.y;
  u += rb * lv.vstride;
  f += rb * lv.vstride;
  tmp += rb * lv.tstride;
  const int r = lv.low_perm[pbeg + t];
  tmp[t] = (f[r] - low_row_offdiag(lv, pbeg + t, u)) / lv.low_diag[r];
}

template <class T>
__global__ void scatter_kernel(const int* __restrict__ list, int n, const T* __restrict__ tmp, T* __restrict__ u,
                               int64_t tstride, int64_t vstride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) u[blockIdx.y * vstride + list[t]] = tmp[blockIdx.y * tstride + t];
}

template <class T>
__global__ void zero_list_kernel(const int* __restrict__ list, int n, T* __restrict__ v, int64_t vstride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) v[blockIdx.y * vstride + list[t]] = T(0);
}

// Parity of a fine point -> the coarse-edge direction it is the midpoint of
// (in (i, j, k)); (0,0,0) for points of the coarse lattice.
__device__ __forceinline__ void midpoint_dir(int I, int J, int K, int& di, int& dj, int& dk) {
  const int pi = I & 1, pj = J & 1, pk = K & 1;
  di = dj = dk = 0;
  if (pi && pj && pk) { di = 1; dj = -1; dk = 1; }
  else if (pi && pj) { di = -1; dj = 1; }
  else if (pj && pk) { dj = -1; dk = 1; }
  else if (pi && pk) { di = -1; dk = 1; }
  else if (pi) di = 1;
  else if (pj) dj = 1;
  else if (pk) dk = 1;
}

// u_f += P e_c on fine cell-interior points: coarse points are injected, the
// midpoint of a coarse edge takes the mean of its two ends.
template <class T>
__global__ void prolong_cell_kernel(LevelView<T> fine, LevelView<T> coarse, const T* __restrict__ ec, T* __restrict__ uf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)fine.nC * fine.n_int) return;
  const int64_t rb = blockIdx.y;
  ec += rb * coarse.vstride;
  uf += rb * fine.vstride;
  coarse.ghost += rb * coarse.gstride;
  const int c = (int)(t / fine.n_int);
  const uint32_t p = fine.int_ijk[t % fine.n_int];
  const int I = unpack_i(p), J = unpack_j(p), K = unpack_k(p);
  int di, dj, dk;
  midpoint_dir(I, J, K, di, dj, dk);
  T v;
  if (di == 0 && dj == 0 && dk == 0) {
    v = load_pt(coarse, ec, c, I >> 1, J >> 1, K >> 1);
  } else {
    const T a = load_pt(coarse, ec, c, (I + di) >> 1, (J + dj) >> 1, (K + dk) >> 1);
    const T b = load_pt(coarse, ec, c, (I - di) >> 1, (J - dj) >> 1, (K - dk) >> 1);
    v = T(0.5) * (a + b);
  }
  uf[fine.off_C + t] += v;
}

template <class T>
__global__ void prolong_low_kernel(LevelView<T> fine, const int* __restrict__ par, const T* __restrict__ ec,
                                   T* __restrict__ uf, int64_t cstride) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= fine.off_C) return;
  ec += blockIdx.y * cstride;
  uf += blockIdx.y * fine.vstride;
  if (fine.low_diag[r] == T(0)) return;
  const int a = par[2 * r], b = par[2 * r + 1];
  const T va = a >= 0 ? ec[a] : T(0);
  T v;
  if (a == b) v = va;
  else v = T(0.5) * (va + (b >= 0 ? ec[b] : T(0)));
  uf[r] += v;
}

// r_c = P^T r_f on coarse cell-interior points: the coincident fine point
// plus half of each of its 14 fine neighbours (all fine-interior).
template <class T>
__global__ void restrict_cell_kernel(LevelView<T> fine, LevelView<T> coarse, const T* __restrict__ rf, T* __restrict__ rc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)coarse.nC * coarse.n_int) return;
  rf += blockIdx.y * fine.vstride;
  rc += blockIdx.y * coarse.vstride;
  const int c = (int)(t / coarse.n_int);
  const uint32_t p = coarse.int_ijk[t % coarse.n_int];
  const int I = 2 * unpack_i(p), J = 2 * unpack_j(p), K = 2 * unpack_k(p);
  const int64_t base = fine.off_C + (int64_t)c * fine.n_int;
  T s = 0;
#pragma unroll
  for (int w = 0; w < 14; ++w) s += rf[base + lin_interior(I + DI(w), J + DJ(w), K + DK(w), fine.N)];
  rc[coarse.off_C + t] = fma(T(0.5), s, rf[base + lin_interior(I, J, K, fine.N)]);
}

// Coarse lower points: the fine point at the same place plus half of each of
// its fine neighbours (the columns of its fine row).
template <class T>
__global__ void restrict_low_kernel(LevelView<T> fine, LevelView<T> coarse, const int* __restrict__ clf,
                                    const T* __restrict__ rf, T* __restrict__ rc) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= coarse.off_C) return;
  rf += blockIdx.y * fine.vstride;
  rc += blockIdx.y * coarse.vstride;
  const int fi = clf[r];
  if (fi < 0) { rc[r] = T(0); return; }
  const int64_t pf = fine.low_pos[fi];
  const int64_t s = pf >> 5, lane = pf & 31;
  const int64_t beg = fine.sell_ptr[s], width = (fine.sell_ptr[s + 1] - beg) >> 5;
  T acc = 0;
  for (int64_t kk = 0; kk < width; ++kk) {
    const int col = fine.sell_col[beg + kk * 32 + lane];
    if (col >= 0) acc += rf[col];
  }
  rc[r] = fma(T(0.5), acc, rf[fi]);
}

// One block per right-hand side: out[b] = sum of its n partials.
__global__ void sum_kernel(const double* __restrict__ partial, int n, int pstride, double* out) {
  partial += (int64_t)blockIdx.x * pstride;
  double v = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) v += partial[t];
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// Partial sums of ||a_b - b_b||^2 per block and right-hand side (grid y).
__global__ void diff_norm_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                 double* partial, int pstride) {
  const int64_t rb = blockIdx.y;
  a += rb * n;
  b += rb * n;
  double v = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double d = a[t] - b[t];
    v = fma(d, d, v);
  }
  v = block_sum(v);
  if (threadIdx.x == 0) partial[rb * pstride + blockIdx.x] = v;
}

template <class T>
__global__ void copy_cast_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (T)src[t];
}

__global__ void widen_kernel(const float* __restrict__ src, double* __restrict__ dst, int64_t n, int add) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = add ? dst[t] + (double)src[t] : (double)src[t];
}

// Canonical index of the neighbour of a cell's boundary point, or -1 when it
// is a Dirichlet point (dropped from the rows: Dirichlet values are 0).
__device__ __forceinline__ int64_t nb_index(const LevelView<double>& lv, int c, int i, int j, int k) {
  if (is_interior(i, j, k, lv.N)) return lv.off_C + (int64_t)c * lv.n_int + lin_interior(i, j, k, lv.N);
  const int slot = lv.bnd_slot[lin_full(i, j, k, lv.N)];
  return lv.halo_src[(int64_t)c * lv.n_bnd + slot];
}

// Row of one lower node: the element-matrix rows of every tetrahedron of
// every adjacent macro cell that contains the node, merged per canonical
// column (fixed cell order, so the sums are deterministic).
__global__ void low_assemble_kernel(LevelView<double> lv, int pass, const int64_t* __restrict__ inc_ptr,
                                    const int* __restrict__ inc_cb, int* row_len, const int64_t* sell_ptr, int* sell_col,
                                    double* sell_val, double* diag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= lv.off_C) return;
  const int64_t beg = inc_ptr[r], end = inc_ptr[r + 1];
  int cols[LOW_MAX_COLS];
  double vals[LOW_MAX_COLS];
  int n = 0;
  double dsum = 0.0;
  bool overflow = false;
  for (int64_t q = beg; q < end; ++q) {
    const int cb = inc_cb[q];
    const int c = cb / lv.n_bnd, b = cb % lv.n_bnd;
    const uint32_t p = lv.bnd_ijk[b];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const CellGeom& g = lv.geom[c];
    double X[3];
    mapped_point(g, i, j, k, lv.N, X);
    double e[14][3];
    bool in[14];
    for (int w = 0; w < 14; ++w) {
      const int a = i + DI(w), bb = j + DJ(w), d = k + DK(w);
      in[w] = a >= 0 && bb >= 0 && d >= 0 && a + bb + d <= lv.N;
      if (in[w]) {
        double Y[3];
        mapped_point(g, a, bb, d, lv.N, Y);
        e[w][0] = Y[0] - X[0];
        e[w][1] = Y[1] - X[1];
        e[w][2] = Y[2] - X[2];
      }
    }
    double s[14];
    bool used[14];
    for (int w = 0; w < 14; ++w) { s[w] = 0.0; used[w] = false; }
    for (int t = 0; t < 24; ++t) {
      const int wa = star(t, 0), wb = star(t, 1), wc = star(t, 2);
      if (!(in[wa] && in[wb] && in[wc])) continue;
      double ka, kb, kc, kx;
      tet_row(e[wa], e[wb], e[wc], ka, kb, kc, kx);
      s[wa] += ka; s[wb] += kb; s[wc] += kc;
      used[wa] = used[wb] = used[wc] = true;
      dsum += kx;
    }
    for (int w = 0; w < 14; ++w) {
      if (!used[w]) continue;
      const int64_t col = nb_index(lv, c, i + DI(w), j + DJ(w), k + DK(w));
      if (col < 0) continue;
      int m = 0;
      while (m < n && cols[m] != (int)col) ++m;
      if (m == n) {
        if (n == LOW_MAX_COLS) { overflow = true; continue; }
        cols[n] = (int)col;
        vals[n] = 0.0;
        ++n;
      }
      vals[m] += s[w];
    }
  }
  if (pass == 0) {
    row_len[r] = overflow ? -1 : n;
    return;
  }
  diag[r] = dsum;
  const int64_t pr = lv.low_pos[r];
  const int64_t sl = pr >> 5, lane = pr & 31;
  const int64_t sb = sell_ptr[sl], width = (sell_ptr[sl + 1] - sb) >> 5;
  for (int64_t kk = 0; kk < width; ++kk) {
    const int64_t e = sb + kk * 32 + lane;
    if (kk < n) { sell_col[e] = cols[kk]; sell_val[e] = vals[kk]; }
    else { sell_col[e] = -1; sell_val[e] = 0.0; }
  }
}

}  // namespace

int low_blocks(int64_t rows) {
  const int64_t b = (rows + LOW_THREADS - 1) / LOW_THREADS;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

template <class T>
void launch_halo(const LevelView<T>& lv, const T* u, cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * lv.n_bnd;
  halo_kernel<T><<<dim3(grid_for(n, 256), lv.nrhs), 256, 0, st>>>(lv, u);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <class T>
void launch_low(const LevelView<T>& lv, Mode mode, const T* u, T* out, const T* f, double* partial, int nblk,
                cudaStream_t st) {
  const dim3 g(nblk, lv.nrhs);
  if (mode == APPLY) low_kernel<T, APPLY><<<g, LOW_THREADS, 0, st>>>(lv, u, out, f, partial);
  else low_kernel<T, RESIDUAL><<<g, LOW_THREADS, 0, st>>>(lv, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <class T>
void launch_low_step(const LevelView<T>& lv, int pbeg, int n, T* u, const T* f, T* tmp, cudaStream_t st) {
  if (n == 0) return;
  const dim3 g(grid_for(n, 256), lv.nrhs);
  low_step_kernel<T><<<g, 256, 0, st>>>(lv, pbeg, n, u, f, tmp);
  scatter_kernel<T><<<g, 256, 0, st>>>(lv.low_perm + pbeg, n, tmp, u, lv.tstride, lv.vstride);
  HHG_CUDA(cudaGetLastError());
  count_launch(2);
}

template <class T>
void launch_zero_list(const int* list, int n, T* v, int nrhs, int64_t vstride, cudaStream_t st) {
  if (n == 0) return;
  zero_list_kernel<T><<<dim3(grid_for(n, 256), nrhs), 256, 0, st>>>(list, n, v, vstride);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <class T>
void launch_prolong_add(const LevelView<T>& fine, const LevelView<T>& coarse, const int* low_par, const T* ec, T* uf,
                        cudaStream_t st) {
  const int64_t n = (int64_t)fine.nC * fine.n_int;
  if (n) prolong_cell_kernel<T><<<dim3(grid_for(n, 256), fine.nrhs), 256, 0, st>>>(fine, coarse, ec, uf);
  prolong_low_kernel<T><<<dim3(grid_for(fine.off_C, 256), fine.nrhs), 256, 0, st>>>(fine, low_par, ec, uf,
                                                                                    coarse.vstride);
  HHG_CUDA(cudaGetLastError());
  count_launch(n ? 2 : 1);
}

template <class T>
void launch_restrict(const LevelView<T>& fine, const LevelView<T>& coarse, const int* clf, const T* rf, T* rc,
                     cudaStream_t st) {
  const int64_t n = (int64_t)coarse.nC * coarse.n_int;
  if (n) restrict_cell_kernel<T><<<dim3(grid_for(n, 256), fine.nrhs), 256, 0, st>>>(fine, coarse, rf, rc);
  restrict_low_kernel<T><<<dim3(grid_for(coarse.off_C, 256), fine.nrhs), 256, 0, st>>>(fine, coarse, clf, rf, rc);
  HHG_CUDA(cudaGetLastError());
  count_launch(n ? 2 : 1);
}

void launch_diff_norm(const double* a, const double* b, int64_t n, int nrhs, double* partial, int pstride,
                      double* out, cudaStream_t st) {
  const int nblk = std::min(pstride, 1024);
  diff_norm_kernel<<<dim3(nblk, nrhs), 256, 0, st>>>(a, b, n, partial, pstride);
  HHG_CUDA(cudaGetLastError());
  count_launch();
  launch_sum(partial, nblk, nrhs, pstride, out, st);
}

void launch_sum(const double* partial, int n, int nrhs, int pstride, double* out, cudaStream_t st) {
  sum_kernel<<<nrhs, 1024, 0, st>>>(partial, n, pstride, out);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <class T>
void launch_copy_cast(const double* src, T* dst, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  copy_cast_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(src, dst, n);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

void launch_widen(const float* src, double* dst, int64_t n, bool add, cudaStream_t st) {
  if (n == 0) return;
  widen_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, add ? 1 : 0);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

void launch_low_assemble(const LevelView<double>& lv, int pass, const int64_t* inc_ptr, const int* inc_cb,
                         int* row_len, int64_t* sell_ptr, int* sell_col, double* sell_val, double* diag,
                         cudaStream_t st) {
  low_assemble_kernel<<<grid_for(lv.off_C, 64), 64, 0, st>>>(lv, pass, inc_ptr, inc_cb, row_len, sell_ptr, sell_col,
                                                             sell_val, diag);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

#define INST(T)                                                                                                   \
  template void launch_halo<T>(const LevelView<T>&, const T*, cudaStream_t);                                      \
  template void launch_low<T>(const LevelView<T>&, Mode, const T*, T*, const T*, double*, int, cudaStream_t);    \
  template void launch_low_step<T>(const LevelView<T>&, int, int, T*, const T*, T*, cudaStream_t);               \
  template void launch_zero_list<T>(const int*, int, T*, int, int64_t, cudaStream_t);                             \
  template void launch_prolong_add<T>(const LevelView<T>&, const LevelView<T>&, const int*, const T*, T*,         \
                                      cudaStream_t);                                                              \
  template void launch_restrict<T>(const LevelView<T>&, const LevelView<T>&, const int*, const T*, T*,            \
                                   cudaStream_t);                                                                 \
  template void launch_copy_cast<T>(const double*, T*, int64_t, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace hhg
