// Coarsest-level solver: Jacobi-preconditioned conjugate gradients on the
// exact operator of the N = 4 level, pre-assembled once at setup.
//
// The paper uses its Gauss-Seidel smoother as coarse solver (Sec. 4); here the
// coarsest system is solved to a tight tolerance instead, so that the cycle
// does not depend on that choice.  At N = 4 every macro cell has one interior
// node, whose exact stencil (the 24 element matrices around it, Sec. 2.3) is
// assembled once; the vertex, edge and face rows are the level's
// pre-assembled lower-primitive rows.  One iteration is three kernels; each
// kernel's blocks re-sum the previous kernel's per-block partials in a fixed
// order, so no separate reduction launch is needed and the result is
// deterministic.  Several right-hand sides are solved together (grid y =
// right-hand side; vectors n_total apart, partials 3 CG_BLOCKS apart, one
// scalar of each kind per right-hand side).
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace hhg {

namespace {

// (A p)_r for the pre-assembled coarse operator.
__device__ __forceinline__ double coarse_row(const CoarseOp& A, int64_t r, const double* __restrict__ p) {
  if (r < A.off_C) {
    const double d = A.low_diag[r];
    if (d == 0.0) return 0.0;
    const int64_t pr = A.low_pos[r];
    const int64_t s = pr >> 5, lane = pr & 31;
    const int64_t beg = A.sell_ptr[s], width = (A.sell_ptr[s + 1] - beg) >> 5;
    double acc = d * p[r];
    for (int64_t kk = 0; kk < width; ++kk) {
      const int col = A.sell_col[beg + kk * 32 + lane];
      if (col >= 0) acc = fma(A.sell_val[beg + kk * 32 + lane], p[col], acc);
    }
    return acc;
  }
  const int c = (int)(r - A.off_C);
  double acc = A.int_diag[c] * p[r];
#pragma unroll
  for (int w = 0; w < 14; ++w) {
    const int col = A.int_col[w * A.nC + c];
    if (col >= 0) acc = fma(A.int_val[w * A.nC + c], p[col], acc);
  }
  return acc;
}

// Sum of the CG_BLOCKS partials of the previous kernel, same order in every block.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part) {
  __shared__ double tot;
  double v = 0.0;
  for (int t = threadIdx.x; t < CG_BLOCKS; t += blockDim.x) v += part[t];
  v = block_sum(v);
  if (threadIdx.x == 0) tot = v;
  __syncthreads();
  return tot;
}

__global__ void coarse_interior_kernel(LevelView<double> lv, int* __restrict__ col, double* __restrict__ val,
                                       double* __restrict__ diag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= lv.nC) return;
  double s[15];
  ifem_stencil(lv.geom[c], lv.N, 1, 1, 1, s);
  for (int w = 0; w < 14; ++w) {
    const int i = 1 + DI(w), j = 1 + DJ(w), k = 1 + DK(w);
    const int slot = lv.bnd_slot[lin_full(i, j, k, lv.N)];
    col[w * lv.nC + c] = lv.halo_src[(int64_t)c * lv.n_bnd + slot];
    val[w * lv.nC + c] = s[w];
  }
  diag[c] = s[MC];
}

__global__ void coarse_dinv_kernel(CoarseOp A, double* __restrict__ dinv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.n_total) return;
  const double d = r < A.off_C ? A.low_diag[r] : A.int_diag[r - A.off_C];
  dinv[r] = d != 0.0 ? 1.0 / d : 0.0;
}

// Offsets of right-hand side blockIdx.y.
#define CG_RHS(vec) vec += (int64_t)blockIdx.y * A.n_total
#define CG_PART(ptr) ptr += (int64_t)blockIdx.y * 3 * CG_BLOCKS

// x = 0, r = f (0 on Dirichlet rows), z = D^-1 r, p = z; partials of r.z, r.r
__global__ void cg_init_kernel(CoarseOp A, const double* __restrict__ f, double* x, double* r, double* z, double* p,
                               double* part_rz, double* part_rr) {
  CG_RHS(f); CG_RHS(x); CG_RHS(r); CG_RHS(z); CG_RHS(p); CG_PART(part_rz); CG_PART(part_rr);
  double rz = 0.0, rr = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n_total; t += (int64_t)gridDim.x * blockDim.x) {
    const double di = A.dinv[t];
    const double rv = di != 0.0 ? f[t] : 0.0;
    const double zv = rv * di;
    x[t] = 0.0;
    r[t] = rv;
    z[t] = zv;
    p[t] = zv;
    rz = fma(rv, zv, rz);
    rr = fma(rv, rv, rr);
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) part_rz[blockIdx.x] = rz;
  rr = block_sum(rr);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = rr;
}

// Fixed-count (graph-captured) iterations skip a right-hand side once its
// residual has converged: rr_cur <= 1e-26 ff (ff = r0.r0); rr_cur == nullptr
// disables the test (host-driven iterations).
__device__ __forceinline__ bool cg_converged(const double* rr_cur, const double* ff) {
  return rr_cur != nullptr && rr_cur[blockIdx.y] <= 1e-26 * ff[blockIdx.y];
}

// q = A p; partials of p.q
__global__ void cg_spmv_kernel(CoarseOp A, const double* __restrict__ p, double* __restrict__ q, double* part_pq,
                               const double* rr_cur, const double* ff) {
  if (cg_converged(rr_cur, ff)) return;
  CG_RHS(p); CG_RHS(q); CG_PART(part_pq);
  double pq = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n_total; t += (int64_t)gridDim.x * blockDim.x) {
    const double qv = coarse_row(A, t, p);
    q[t] = qv;
    pq = fma(p[t], qv, pq);
  }
  pq = block_sum(pq);
  if (threadIdx.x == 0) part_pq[blockIdx.x] = pq;
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = D^-1 r; partials of r.z, r.r
__global__ void cg_update_kernel(CoarseOp A, double* x, double* r, double* z, const double* __restrict__ p,
                                 const double* __restrict__ q, const double* __restrict__ part_pq,
                                 const double* __restrict__ rz_cur, double* part_rz, double* part_rr,
                                 const double* rr_cur, const double* ff) {
  if (cg_converged(rr_cur, ff)) return;
  CG_RHS(x); CG_RHS(r); CG_RHS(z); CG_RHS(p); CG_RHS(q); CG_PART(part_pq); CG_PART(part_rz); CG_PART(part_rr);
  rz_cur += blockIdx.y;
  const double pq = sum_partials(part_pq);
  const double alpha = pq != 0.0 ? *rz_cur / pq : 0.0;
  double rz = 0.0, rr = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n_total; t += (int64_t)gridDim.x * blockDim.x) {
    x[t] = fma(alpha, p[t], x[t]);
    const double rv = fma(-alpha, q[t], r[t]);
    const double zv = rv * A.dinv[t];
    r[t] = rv;
    z[t] = zv;
    rz = fma(rv, zv, rz);
    rr = fma(rv, rv, rr);
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) part_rz[blockIdx.x] = rz;
  rr = block_sum(rr);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = rr;
}

// beta = rz_new / rz_cur; p = z + beta p; rz_next = rz_new, rr_out = r.r
__global__ void cg_dir_kernel(CoarseOp A, double* p, const double* __restrict__ z, const double* __restrict__ part_rz,
                              const double* __restrict__ part_rr, const double* __restrict__ rz_cur, double* rz_next,
                              double* rr_out, const double* rr_cur, const double* ff) {
  if (cg_converged(rr_cur, ff)) {  // carry the scalars to the next iteration's buffers
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      rz_next[blockIdx.y] = rz_cur[blockIdx.y];
      rr_out[blockIdx.y] = rr_cur[blockIdx.y];
    }
    return;
  }
  CG_RHS(p); CG_RHS(z); CG_PART(part_rz); CG_PART(part_rr);
  rz_cur += blockIdx.y;
  rz_next += blockIdx.y;
  rr_out += blockIdx.y;
  const double rz_new = sum_partials(part_rz);
  const double o = *rz_cur;
  const double beta = o != 0.0 ? rz_new / o : 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n_total; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = fma(beta, p[t], z[t]);
  if (blockIdx.x == 0) {
    const double rr = sum_partials(part_rr);
    if (threadIdx.x == 0) {
      *rz_next = rz_new;
      *rr_out = rr;
    }
  }
}

// rz_out = sum of part_rz, rr_out = sum of part_rr (after cg_init)
// one block per right-hand side
__global__ void cg_sums_kernel(const double* __restrict__ part_rz, const double* __restrict__ part_rr, double* rz_out,
                               double* rr_out) {
  part_rz += (int64_t)blockIdx.x * 3 * CG_BLOCKS;
  part_rr += (int64_t)blockIdx.x * 3 * CG_BLOCKS;
  const double a = sum_partials(part_rz);
  const double b = sum_partials(part_rr);
  if (threadIdx.x == 0) {
    rz_out[blockIdx.x] = a;
    rr_out[blockIdx.x] = b;
  }
}

// Sets *flag when some right-hand side has not converged.
__global__ void cg_check_kernel(const double* rr, const double* ff, int nrhs, int* flag) {
  for (int b = threadIdx.x; b < nrhs; b += blockDim.x)
    if (!(rr[b] <= 1e-26 * ff[b])) atomicExch(flag, 1);
}

#undef CG_RHS
#undef CG_PART

}  // namespace

void launch_coarse_setup(const LevelView<double>& lv, CoarseOp& A, int* col, double* val, double* diag, double* dinv,
                         cudaStream_t st) {
  coarse_interior_kernel<<<(lv.nC + 127) / 128, 128, 0, st>>>(lv, col, val, diag);
  A.int_col = col;
  A.int_val = val;
  A.int_diag = diag;
  coarse_dinv_kernel<<<(unsigned)((A.n_total + 255) / 256), 256, 0, st>>>(A, dinv);
  A.dinv = dinv;
  HHG_CUDA(cudaGetLastError());
  count_launch(2);
}

void launch_cg_init(const CoarseOp& A, const double* f, double* x, double* r, double* z, double* p, double* part,
                    double* rz_out, double* rr_out, int nrhs, cudaStream_t st) {
  cg_init_kernel<<<dim3(CG_BLOCKS, nrhs), 256, 0, st>>>(A, f, x, r, z, p, part, part + CG_BLOCKS);
  cg_sums_kernel<<<nrhs, 256, 0, st>>>(part, part + CG_BLOCKS, rz_out, rr_out);
  HHG_CUDA(cudaGetLastError());
  count_launch(2);
}

void launch_cg_iteration(const CoarseOp& A, double* x, double* r, double* z, double* p, double* q, double* part,
                         const double* rz_cur, double* rz_next, double* rr_out, int nrhs, cudaStream_t st,
                         const double* rr_cur, const double* ff) {
  double* part_pq = part;
  double* part_rz = part + CG_BLOCKS;
  double* part_rr = part + 2 * CG_BLOCKS;
  const dim3 g(CG_BLOCKS, nrhs);
  cg_spmv_kernel<<<g, 256, 0, st>>>(A, p, q, part_pq, rr_cur, ff);
  cg_update_kernel<<<g, 256, 0, st>>>(A, x, r, z, p, q, part_pq, rz_cur, part_rz, part_rr, rr_cur, ff);
  cg_dir_kernel<<<g, 256, 0, st>>>(A, p, z, part_rz, part_rr, rz_cur, rz_next, rr_out, rr_cur, ff);
  HHG_CUDA(cudaGetLastError());
  count_launch(3);
}

}  // namespace hhg

namespace hhg {
void launch_cg_check(const double* rr, const double* ff, int nrhs, int* flag, cudaStream_t st) {
  cg_check_kernel<<<1, 64, 0, st>>>(rr, ff, nrhs, flag);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}
}  // namespace hhg
