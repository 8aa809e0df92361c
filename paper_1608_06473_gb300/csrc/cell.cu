// Cell-interior kernels: the volume primitives, which hold all but
// O(2^{2l}) of the nodes (Sec. 2.3).
//
// One CTA per macro cell walks the planes k = 1 .. N-3 of the cell.  For the
// surrogate (LSQP, Sec. 3.4), the 3-variate polynomial of every direction is
// reduced once per line (j, k) to a polynomial in i -- the line-wise
// evaluation the paper builds on (Sec. 3.4; Eq. 5.4) -- and kept in shared
// memory; each node then needs q multiply-adds per weight.  For IFEM
// (Sec. 4.2.1) every node assembles its 15 weights from the 24 element
// matrices around it.
//
// The smoother (Eq. 5.1) runs the four colours (i + 2j + 3k) mod 4 of the
// cell in one launch: in step s the CTA updates colour c on plane s + 1 - c,
// c = 0..3, in that order, with a barrier after each colour.  Every update of
// colour c then sees all colour < c updates of its neighbours (planes k - 1,
// k, k + 1) and none of colour > c, exactly as four separate colour sweeps.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace hhg {

namespace {

constexpr int CELL_THREADS = 128;

// Coefficients of the polynomial in i along line (j, k): c_a(j, k) =
// sum_{b,d} A_{a,b,d} j^b k^d.  Storage order of A (per direction):
// for a = 0..Q, for d = 0..Q-a, for b = 0..Q-a-d.
template <class T, int Q>
__device__ __forceinline__ void line_coeffs(const T* A, T j, T k, T* out) {
  int t = 0;
#pragma unroll
  for (int a = 0; a <= Q; ++a) {
    T inner[Q + 1];
#pragma unroll
    for (int d = 0; d <= Q - a; ++d) {
      const int n = Q - a - d + 1;
      T v = A[t + n - 1];
#pragma unroll
      for (int b = n - 2; b >= 0; --b) v = fma(v, j, A[t + b]);
      inner[d] = v;
      t += n;
    }
    T ca = inner[Q - a];
#pragma unroll
    for (int d = Q - a - 1; d >= 0; --d) ca = fma(ca, k, inner[d]);
    out[a] = ca;
  }
}

template <class T, int Q>
__device__ __forceinline__ T eval_line(const T* cl, T i) {
  T v = cl[Q];
#pragma unroll
  for (int a = Q - 1; a >= 0; --a) v = fma(v, i, cl[a]);
  return v;
}

// Stencil application at one interior node from its 15 weights.
template <class T, Mode MODE>
__device__ __forceinline__ void node_update(const LevelView<T>& lv, int c, int i, int j, int k, const T* sw,
                                            T* u, T* out, const T* f, double& nrm) {
  const int64_t I = lv.off_C + (int64_t)c * lv.n_int + lin_interior(i, j, k, lv.N);
  if (MODE == SMOOTH) {
    T acc = f[I];
#pragma unroll
    for (int w = 0; w < 14; ++w) acc = fma(-sw[w], load_pt(lv, (const T*)u, c, i + DI(w), j + DJ(w), k + DK(w)), acc);
    u[I] = acc / sw[MC];
  } else if (MODE == APPLY) {
    T acc = sw[MC] * u[I];
#pragma unroll
    for (int w = 0; w < 14; ++w) acc = fma(sw[w], load_pt(lv, (const T*)u, c, i + DI(w), j + DJ(w), k + DK(w)), acc);
    out[I] = acc;
  } else {
    T acc = fma(-sw[MC], u[I], f[I]);
#pragma unroll
    for (int w = 0; w < 14; ++w) acc = fma(-sw[w], load_pt(lv, (const T*)u, c, i + DI(w), j + DJ(w), k + DK(w)), acc);
    out[I] = acc;
    nrm += (double)acc * (double)acc;
  }
}

template <class T, int Q, Mode MODE>
__global__ void __launch_bounds__(CELL_THREADS) lsqp_cell_kernel(LevelView<T> lv, T* u, T* out, const T* f,
                                                                  double* partial) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NSLOT = (MODE == SMOOTH) ? 4 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);   // [15][MQ]
  T* ring = sA + 15 * MQ;                   // [NSLOT][NL][15][Q+1]
  const int c = blockIdx.x;
  const int N = lv.N;
  const int NL = N - 3;
  for (int t = threadIdx.x; t < 15 * MQ; t += blockDim.x) sA[t] = lv.coef[(int64_t)c * 15 * MQ + t];
  __syncthreads();
  double nrm = 0.0;

  auto prologue = [&](int k) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    for (int jj = threadIdx.x; jj < N - 2 - k; jj += blockDim.x) {
      T* dst = ring + ((slot * NL + jj) * 15) * (Q + 1);
#pragma unroll 1
      for (int w = 0; w < 15; ++w) line_coeffs<T, Q>(sA + w * MQ, (T)(jj + 1), (T)k, dst + w * (Q + 1));
    }
  };
  auto process = [&](int k, int beg, int end) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    for (int t = beg + threadIdx.x; t < end; t += blockDim.x) {
      const uint32_t p = lv.plane_nodes[t];
      const int i = unpack_i(p), j = unpack_j(p);
      const T* cl = ring + ((slot * NL + (j - 1)) * 15) * (Q + 1);
      T sw[15];
#pragma unroll
      for (int w = 0; w < 15; ++w) sw[w] = eval_line<T, Q>(cl + w * (Q + 1), (T)i);
      node_update<T, MODE>(lv, c, i, j, k, sw, u, out, f, nrm);
    }
  };

  if (MODE == SMOOTH) {
    for (int s = 0; s <= N - 1; ++s) {
      if (s + 1 <= N - 3) prologue(s + 1);
      __syncthreads();
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        const int k = s + 1 - cc;
        if (k >= 1 && k <= N - 3) process(k, lv.plane_off[k * 4 + cc], lv.plane_off[k * 4 + cc + 1]);
        __syncthreads();
      }
    }
  } else {
    for (int k = 1; k <= N - 3; ++k) {
      prologue(k);
      __syncthreads();
      process(k, lv.plane_off[k * 4], lv.plane_off[k * 4 + 4]);
      __syncthreads();
    }
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// FP64 surrogate kernel with the weights evaluated in exact 64-bit integer
// arithmetic.  GB300 issues FP64 at a small fraction of its FP32/INT32 rate,
// and evaluating the 15 line polynomials is half of the FP64 work of an
// update.  Here the line coefficients are scaled by 2^E (E per cell, chosen
// so that every partial sum stays below 2^62) and rounded to integers once
// per line; per node the polynomial is evaluated by integer Horner (exact) and
// converted to FP64 once per weight.  The weights equal the FP64 ones to the
// rounding of the conversion; the factor 2^-E is applied once per node.
__device__ __forceinline__ long long horner_i64(const long long* C, int i, int Q) {
  long long v = C[Q];
  for (int a = Q - 1; a >= 0; --a) v = v * (long long)i + C[a];
  return v;
}

template <int Q, Mode MODE, int THREADS>
__global__ void __launch_bounds__(THREADS) lsqp_cell_kernel_iw(LevelView<double> lv, double* u, double* out,
                                                                const double* f, double* partial) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NSLOT = (MODE == SMOOTH) ? 4 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sA = reinterpret_cast<double*>(smem_raw);          // [15][MQ]
  long long* ring = reinterpret_cast<long long*>(sA + 15 * MQ);  // [NSLOT][NL][15][Q+1]
  __shared__ double s_bound[THREADS / 32];
  const int c = blockIdx.x;
  const int N = lv.N;
  const int NL = N - 3;
  for (int t = threadIdx.x; t < 15 * MQ; t += blockDim.x) sA[t] = lv.coef[(int64_t)c * 15 * MQ + t];
  __syncthreads();
  // B = max_w sum_t |A_wt| N^deg(t) bounds |c_a(j,k)| i^a for every line and node
  double bnd = 0.0;
  if (threadIdx.x < 15) {
    int t = 0;
    for (int a = 0; a <= Q; ++a)
      for (int d = 0; d <= Q - a; ++d)
        for (int b = 0; b <= Q - a - d; ++b, ++t)
          bnd += fabs(sA[threadIdx.x * MQ + t]) * ldexp(1.0, (a + b + d) * (31 - __clz(N)));  // N = 2^L
  }
  for (int o = 16; o > 0; o >>= 1) bnd = fmax(bnd, __shfl_down_sync(0xffffffffu, bnd, o));
  if ((threadIdx.x & 31) == 0) s_bound[threadIdx.x >> 5] = bnd;
  __syncthreads();
  double B = 0.0;
  for (int w = 0; w < THREADS / 32; ++w) B = fmax(B, s_bound[w]);
  const int ex = ilogb(B > 0.0 ? B : 1.0) + 1;  // B < 2^ex
  const int E = 60 - ex;          // B 2^E < 2^60: |C2 i^2 + C1 i + C0| < 3 * 2^60
  const double scale = ldexp(1.0, E), inv_scale = ldexp(1.0, -E);
  double nrm = 0.0;

  auto prologue = [&](int k) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    for (int jj = threadIdx.x; jj < N - 2 - k; jj += blockDim.x) {
      long long* dst = ring + ((slot * NL + jj) * 15) * (Q + 1);
#pragma unroll 1
      for (int w = 0; w < 15; ++w) {
        double cl[Q + 1];
        line_coeffs<double, Q>(sA + w * MQ, (double)(jj + 1), (double)k, cl);
#pragma unroll
        for (int a = 0; a <= Q; ++a) dst[w * (Q + 1) + a] = __double2ll_rn(cl[a] * scale);
      }
    }
  };
  auto process = [&](int k, int beg, int end) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    for (int t = beg + threadIdx.x; t < end; t += blockDim.x) {
      const uint32_t p = lv.plane_nodes[t];
      const int i = unpack_i(p), j = unpack_j(p);
      const long long* cl = ring + ((slot * NL + (j - 1)) * 15) * (Q + 1);
      double sw[15];
#pragma unroll
      for (int w = 0; w < 15; ++w) sw[w] = (double)horner_i64(cl + w * (Q + 1), i, Q);
      const int64_t I = lv.off_C + (int64_t)c * lv.n_int + lin_interior(i, j, k, N);
      if (MODE == SMOOTH) {
        double acc = f[I] * scale;
#pragma unroll
        for (int w = 0; w < 14; ++w) acc = fma(-sw[w], load_pt(lv, (const double*)u, c, i + DI(w), j + DJ(w), k + DK(w)), acc);
        u[I] = acc / sw[MC];
      } else {
        double acc = sw[MC] * u[I];
#pragma unroll
        for (int w = 0; w < 14; ++w) acc = fma(sw[w], load_pt(lv, (const double*)u, c, i + DI(w), j + DJ(w), k + DK(w)), acc);
        if (MODE == APPLY) {
          out[I] = acc * inv_scale;
        } else {
          const double r = fma(-inv_scale, acc, f[I]);
          out[I] = r;
          nrm += r * r;
        }
      }
    }
  };

  if (MODE == SMOOTH) {
    for (int s = 0; s <= N - 1; ++s) {
      if (s + 1 <= N - 3) prologue(s + 1);
      __syncthreads();
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        const int k = s + 1 - cc;
        if (k >= 1 && k <= N - 3) process(k, lv.plane_off[k * 4 + cc], lv.plane_off[k * 4 + cc + 1]);
        __syncthreads();
      }
    }
  } else {
    for (int k = 1; k <= N - 3; ++k) {
      prologue(k);
      __syncthreads();
      process(k, lv.plane_off[k * 4], lv.plane_off[k * 4 + 4]);
      __syncthreads();
    }
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

template <class T, Mode MODE>
__global__ void __launch_bounds__(CELL_THREADS) ifem_cell_kernel(LevelView<T> lv, T* u, T* out, const T* f,
                                                                  double* partial) {
  __shared__ CellGeom g;
  const int c = blockIdx.x;
  const int N = lv.N;
  if (threadIdx.x < 16) reinterpret_cast<double*>(&g)[threadIdx.x] = reinterpret_cast<const double*>(&lv.geom[c])[threadIdx.x];
  __syncthreads();
  double nrm = 0.0;
  auto process = [&](int k, int beg, int end) {
    for (int t = beg + threadIdx.x; t < end; t += blockDim.x) {
      const uint32_t p = lv.plane_nodes[t];
      const int i = unpack_i(p), j = unpack_j(p);
      double s[15];
      ifem_stencil(g, N, i, j, k, s);
      T sw[15];
#pragma unroll
      for (int w = 0; w < 15; ++w) sw[w] = (T)s[w];
      node_update<T, MODE>(lv, c, i, j, k, sw, u, out, f, nrm);
    }
  };
  if (MODE == SMOOTH) {
    for (int s = 0; s <= N - 1; ++s) {
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        const int k = s + 1 - cc;
        if (k >= 1 && k <= N - 3) process(k, lv.plane_off[k * 4 + cc], lv.plane_off[k * 4 + cc + 1]);
        __syncthreads();
      }
    }
  } else {
    for (int k = 1; k <= N - 3; ++k) process(k, lv.plane_off[k * 4], lv.plane_off[k * 4 + 4]);
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

template <class T, int Q, Mode MODE>
void launch_lsqp(const LevelView<T>& lv, T* u, T* out, const T* f, double* partial, cudaStream_t st) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NSLOT = (MODE == SMOOTH) ? 4 : 1;
  const size_t smem = sizeof(T) * (15 * MQ + (size_t)NSLOT * (lv.N - 3) * 15 * (Q + 1));
  if constexpr (sizeof(T) == 8) {
    auto k2 = lsqp_cell_kernel_iw<Q, MODE, 256>;
    if (smem > 48 * 1024) HHG_CUDA(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k2<<<lv.nC, 256, smem, st>>>(lv, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  auto kern = lsqp_cell_kernel<T, Q, MODE>;
  if (smem > 48 * 1024) HHG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<lv.nC, CELL_THREADS, smem, st>>>(lv, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <class T, Mode MODE>
void dispatch_q(const LevelView<T>& lv, T* u, T* out, const T* f, double* partial, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_lsqp<T, 1, MODE>(lv, u, out, f, partial, st); break;
    case 2: launch_lsqp<T, 2, MODE>(lv, u, out, f, partial, st); break;
    case 3: launch_lsqp<T, 3, MODE>(lv, u, out, f, partial, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}

__global__ void sample_kernel(LevelView<double> lv, const uint32_t* __restrict__ pts, int n_pts,
                              double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)lv.nC * n_pts) return;
  const int c = (int)(t / n_pts);
  const uint32_t p = pts[t % n_pts];
  double s[15];
  ifem_stencil(lv.geom[c], lv.N, unpack_i(p), unpack_j(p), unpack_k(p), s);
#pragma unroll
  for (int w = 0; w < 14; ++w) b[t * 14 + w] = s[w];
}

__global__ void fit_coef_kernel(int nC, int mq, int n_pts, const double* __restrict__ aplus,
                                const double* __restrict__ scale, const double* __restrict__ b,
                                double* __restrict__ coef, float* __restrict__ coef32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nC * mq) return;
  const int c = (int)(t / mq), m = (int)(t % mq);
  double acc[14];
#pragma unroll
  for (int w = 0; w < 14; ++w) acc[w] = 0.0;
  const double* bc = b + (int64_t)c * n_pts * 14;
  const double* ap = aplus + (int64_t)m * n_pts;
  for (int p = 0; p < n_pts; ++p) {
    const double a = ap[p];
#pragma unroll
    for (int w = 0; w < 14; ++w) acc[w] = fma(a, bc[p * 14 + w], acc[w]);
  }
  double centre = 0.0;
  double* out = coef + (int64_t)c * 15 * mq;
#pragma unroll
  for (int w = 0; w < 14; ++w) {
    const double v = acc[w] * scale[m];
    out[w * mq + m] = v;
    centre -= v;
  }
  out[14 * mq + m] = centre;
  if (coef32) {
    float* o32 = coef32 + (int64_t)c * 15 * mq;
#pragma unroll
    for (int w = 0; w < 15; ++w) o32[w * mq + m] = (float)out[w * mq + m];
  }
}

}  // namespace

template <class T>
void launch_cell(const LevelView<T>& lv, int op, Mode mode, T* u, T* out, const T* f, double* partial,
                 cudaStream_t st) {
  if (lv.N < 4 || lv.n_int == 0) return;
  if (op == HHG_OP_LSQP && lv.q > 0) {
    switch (mode) {
      case APPLY: dispatch_q<T, APPLY>(lv, u, out, f, partial, st); break;
      case RESIDUAL: dispatch_q<T, RESIDUAL>(lv, u, out, f, partial, st); break;
      case SMOOTH: dispatch_q<T, SMOOTH>(lv, u, out, f, partial, st); break;
    }
    return;
  }
  switch (mode) {
    case APPLY: ifem_cell_kernel<T, APPLY><<<lv.nC, CELL_THREADS, 0, st>>>(lv, u, out, f, partial); break;
    case RESIDUAL: ifem_cell_kernel<T, RESIDUAL><<<lv.nC, CELL_THREADS, 0, st>>>(lv, u, out, f, partial); break;
    case SMOOTH: ifem_cell_kernel<T, SMOOTH><<<lv.nC, CELL_THREADS, 0, st>>>(lv, u, out, f, partial); break;
  }
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template void launch_cell<double>(const LevelView<double>&, int, Mode, double*, double*, const double*, double*,
                                  cudaStream_t);
template void launch_cell<float>(const LevelView<float>&, int, Mode, float*, float*, const float*, double*,
                                 cudaStream_t);

void launch_sample(const LevelView<double>& lv, const uint32_t* pts, int n_pts, double* b, cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * n_pts;
  if (n == 0) return;
  sample_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(lv, pts, n_pts, b);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

void launch_fit_coef(int nC, int mq, int n_pts, const double* aplus, const double* scale, const double* b,
                     double* coef, float* coef32, cudaStream_t st) {
  const int64_t n = (int64_t)nC * mq;
  fit_coef_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(nC, mq, n_pts, aplus, scale, b, coef, coef32);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

}  // namespace hhg
