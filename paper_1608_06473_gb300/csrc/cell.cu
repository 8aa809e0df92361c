// Cell-interior kernels: the volume primitives, which hold all but
// O(2^{2l}) of the nodes (Sec. 2.3).
//
// Surrogate (LSQP, Sec. 3.4).  For a fixed line (j, k) each of the 15
// 3-variate polynomials is a polynomial of degree q in i -- the line-wise
// evaluation the paper builds on (Sec. 3.4; Eq. 5.4).  Two designs, one per
// precision, because GB300 issues FP64 at a small fraction of its FP32 and
// INT32 rate:
//
//  * FP64: per plane k each direction's polynomial is reduced to a
//    polynomial in (i, j) at fit time and stored as integers scaled by 2^E
//    (E per cell, chosen so every partial sum stays below 2^61): 15 m
//    numbers per plane with m = (q+1)(q+2)/2, 44 KB per cell at q = 2,
//    N = 64.  A CTA stages its cell's table in shared memory, and every node
//    evaluates its weights exactly by integer Horner in j and i, converts
//    them on the integer pipe, and forms the reciprocal of its centre weight
//    on the integer pipe too; the FP64 pipe carries only the 14 stencil
//    products and one multiply.  Kernels are thread-per-node with one CTA per
//    macro cell and no barriers after the staging; the smoother is one
//    launch per colour.
//  * FP32: per plane k each direction's polynomial is reduced to a
//    polynomial in (i, j) at fit time (FP32 table) and evaluated per node
//    from shared memory, thread per node, one launch per colour.  The
//    smoother may instead run as a one-launch sweep per cell: the plane
//    wavefront of wave.cu or the shared-memory staged sweep of stage.cu; a
//    tuner times the candidates per level and picks one (lv.smooth_cfg).
//
// IFEM (Sec. 4.2.1): every node assembles its 15 weights from the 24 element
// matrices around it (thread per node, one launch per colour).
//
// Batched right-hand sides: persistent kernels (grid-stride over cells) that
// form a node's weights once and apply them to every vector.
//
// Neighbour addressing: nodes whose 14 neighbours are all interior use
// closed-form 32-bit offsets within the cell's block of the canonical
// vector; nodes next to the cell boundary read boundary neighbours from the
// cell's halo copy.
#include <algorithm>

#include <cuda_runtime.h>

#include "arith.cuh"
#include "device.cuh"
#include "kernels.h"
#include "runs.cuh"

namespace hhg {

namespace {

constexpr int NODE_THREADS = 256;  // thread-per-node kernels
// FP64 surrogate kernel: 512 threads x 2 CTAs per SM (64 registers a thread,
// 32 warps) measured 10% faster than 256 x 3 (80 registers) on GB300: the
// kernel waits on memory, more warps hide it.
constexpr int NODE64_THREADS = 512;
// FP32 surrogate kernel: 512 threads x 2 CTAs per SM measured 4% (N = 64) and
// 14% (N = 128) faster than 256 x 4 on GB300.
constexpr int NODE32_THREADS = 512;

// Stencil application at one interior node.  wt(w) returns weight w (the
// centre is w = MC), possibly scaled by 2^E; `scale` = 2^E, `inv_scale` =
// 2^-E (1 when unscaled).  Deep-interior nodes read their neighbours through
// closed-form offsets, the others through the interior / halo lookup.
template <class T, Mode MODE, class WT>
__device__ __forceinline__ void node_update(const LevelView<T>& lv, int c, int i, int j, int k, WT wt, T* u, T* out,
                                            const T* f, double& nrm, T scale, T inv_scale) {
  const int64_t base = lv.off_C + (int64_t)c * lv.n_int;
  const int lin = lin_interior32(i, j, k, lv.N);
  const int64_t I = base + lin;
  auto body = [&](auto nb) {
    if (MODE == SMOOTH) {
      T a0 = f[I] * scale, a1 = 0;
#pragma unroll
      for (int w = 0; w < 14; w += 2) {
        a0 = fma(-wt(w), nb(w), a0);
        a1 = fma(-wt(w + 1), nb(w + 1), a1);
      }
      u[I] = (a0 + a1) / wt(MC);
    } else {
      T a0 = wt(MC) * u[I], a1 = 0;
#pragma unroll
      for (int w = 0; w < 14; w += 2) {
        a0 = fma(wt(w), nb(w), a0);
        a1 = fma(wt(w + 1), nb(w + 1), a1);
      }
      const T y = a0 + a1;
      if (MODE == APPLY) {
        out[I] = y * inv_scale;
      } else {
        const T r = fma(-inv_scale, y, f[I]);
        out[I] = r;
        nrm += (double)r * (double)r;
      }
    }
  };
  if (deep_interior(i, j, k, lv.N)) {
    int off[14];
    neighbour_offsets(j, k, lv.N, off);
    const T* p = u + I;
    body([&](int w) -> T { return p[off[w]]; });
  } else {
    body([&](int w) -> T { return load_pt(lv, (const T*)u, c, i + DI(w), j + DJ(w), k + DK(w)); });
  }
}

// ---------------------------------------------------------------------------
// Batched right-hand sides: a node's 15 weights (and, for the smoother, the
// reciprocal of its centre weight) are formed once and applied to all
// lv.nrhs vectors.  Residual norms accumulate per thread and right-hand side
// in shared memory (s_nrm[b blockDim + thread]) and are summed per cell.
// ---------------------------------------------------------------------------
template <class T, Mode MODE>
__device__ __forceinline__ void node_apply_all(const LevelView<T>& lv, int c, int i, int j, int k, const T (&w)[15],
                                               T rc, T* u, T* out, const T* f, double* s_nrm) {
  const int64_t cb = lv.off_C + (int64_t)c * lv.n_int;
  const int64_t I = cb + lin_interior32(i, j, k, lv.N);
  const bool deep = deep_interior(i, j, k, lv.N);
  int off[14];
  if (deep) neighbour_offsets(j, k, lv.N, off);
  for (int b = 0; b < lv.nrhs; ++b) {
    T* ub = u + (int64_t)b * lv.vstride;
    const T* gb = lv.ghost + (int64_t)b * lv.gstride;
    auto nb = [&](int v) -> T {
      if (deep) return ub[I + off[v]];
      const int i2 = i + DI(v), j2 = j + DJ(v), k2 = k + DK(v);
      if (is_interior(i2, j2, k2, lv.N)) return ub[cb + lin_interior32(i2, j2, k2, lv.N)];
      return gb[(int64_t)c * lv.n_full + lin_full(i2, j2, k2, lv.N)];
    };
    if (MODE == SMOOTH) {
      T acc = f[(int64_t)b * lv.vstride + I];
#pragma unroll
      for (int v = 0; v < 14; ++v) acc = fma(-w[v], nb(v), acc);
      ub[I] = acc * rc;
    } else {
      T y = w[MC] * ub[I];
#pragma unroll
      for (int v = 0; v < 14; ++v) y = fma(w[v], nb(v), y);
      if (MODE == APPLY) {
        out[(int64_t)b * lv.vstride + I] = y;
      } else {
        const T r = f[(int64_t)b * lv.vstride + I] - y;
        out[(int64_t)b * lv.vstride + I] = r;
        double& acc = s_nrm[b * blockDim.x + threadIdx.x];
        acc = fma((double)r, (double)r, acc);
      }
    }
  }
}

// Per-right-hand-side sums of the shared-memory norm accumulators of cell c.
__device__ __forceinline__ void batch_norms_out(const double* s_nrm, int nrhs, int pstride, int c, double* partial) {
  for (int b = 0; b < nrhs; ++b) {
    const double tot = block_sum(s_nrm[b * blockDim.x + threadIdx.x]);
    if (threadIdx.x == 0) partial[(int64_t)b * pstride + c] = tot;
  }
}

// ---------------------------------------------------------------------------
// FP64 surrogate: integer plane table at fit time, staged per cell in shared
// memory; thread-per-node application
// ---------------------------------------------------------------------------


// E per cell: B = max_w sum_t |A_wt| N^deg(t) bounds every partial sum of
// the nested Horner evaluation (in j, then in i) of any direction's
// polynomial at any node, so with B 2^E < 2^60 every partial sum of the
// integer evaluation stays below 2^61 (the rounded plane coefficients add at
// most (q + 1)(q + 2) N^q / 4).
template <int Q>
__global__ void lsqp_scale_kernel(const double* __restrict__ coef, int nC, int N, int* __restrict__ cell_e) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nC) return;
  const int L = 31 - __clz(N);
  double B = 0.0;
  for (int w = 0; w < 15; ++w) {
    double s = 0.0;
    int t = 0;
    for (int a = 0; a <= Q; ++a)
      for (int d = 0; d <= Q - a; ++d)
        for (int b = 0; b <= Q - a - d; ++b, ++t)
          s += fabs(coef[((int64_t)c * 15 + w) * MQ + t]) * ldexp(1.0, (a + b + d) * L);
    B = fmax(B, s);
  }
  cell_e[c] = 60 - (ilogb(B > 0.0 ? B : 1.0) + 1);
}

// Plane table: for cell c, plane k and direction w, D_ab(k) = sum_d A_abd k^d
// (FP64) times 2^E, rounded to int64, NPP64 values per direction.
template <int Q>
__global__ void lsqp_plane64_kernel(const double* __restrict__ coef, const int* __restrict__ cell_e, int nC, int N,
                                    long long* __restrict__ table) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  const int np = N - 3;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nC * np * 15) return;
  const int w = (int)(t % 15);
  const int64_t cp = t / 15;
  const int c = (int)(cp / np), k = (int)(cp % np) + 1;
  double P[NP];
  plane_coeffs<double, Q>(coef + ((int64_t)c * 15 + w) * MQ, (double)k, P);
  const double sc = ldexp(1.0, cell_e[c]);
  long long* dst = table + t * NPP64<Q>;
#pragma unroll
  for (int a = 0; a < NPP64<Q>; ++a) dst[a] = a < NP ? __double2ll_rn(P[a] * sc) : 0ll;
}

// The polynomial of one direction in (i, j) evaluated exactly in integer
// arithmetic: Horner in j for each power of i, then Horner in i (the same
// nesting as eval_plane).  P: NPP64 int64 in shared memory.
template <int Q>
__device__ __forceinline__ long long eval_plane_i64(const long long* P, unsigned i, unsigned j) {
  long long r[NPP64<Q>];
#pragma unroll
  for (int h = 0; h < NPP64<Q> / 2; ++h) {
    const longlong2 x = reinterpret_cast<const longlong2*>(P)[h];
    r[2 * h] = x.x;
    r[2 * h + 1] = x.y;
  }
  long long s = 0;
#pragma unroll
  for (int a = Q; a >= 0; --a) {
    long long c = r[plane_index<Q>(a, Q - a)];
#pragma unroll
    for (int b = Q - a - 1; b >= 0; --b) c = mad_i64_u32(c, j, r[plane_index<Q>(a, b)]);
    s = (a == Q) ? c : mad_i64_u32(s, i, c);
  }
  return s;
}

// Cell c's plane table into shared memory (16-byte loads).
template <int Q>
__device__ __forceinline__ void load_plane64(const LevelView<double>& lv, int c, long long* s_tab) {
  const int n2 = (lv.N - 3) * 15 * NPP64<Q> / 2;
  const longlong2* src = reinterpret_cast<const longlong2*>(lv.plane64 + (int64_t)c * 2 * n2);
  longlong2* dst = reinterpret_cast<longlong2*>(s_tab);
  for (int t = threadIdx.x; t < n2; t += blockDim.x) dst[t] = __ldg(src + t);
}

// One interior node of the FP64 surrogate.  P: the node's plane in shared
// memory (15 directions x NPP64 int64, scaled by 2^E).  Every weight is
// evaluated exactly on the integer pipe and converted with the scale undone
// (i64_to_f64_scaled); the smoother's divide by the centre weight is a
// product with its reciprocal, also formed on the integer pipe
// (rcp_i64_scaled).  The FP64 pipe carries only the 14 products and that
// one multiply (15 operations per update).
template <int Q, Mode MODE, class NB>
__device__ __forceinline__ void lsqp64_node(const long long* P, unsigned i, unsigned j, int E, NB nb, int64_t I,
                                            double* u, double* out, const double* f, double& nrm) {
  auto wt = [&](int w) { return i64_to_f64_scaled(eval_plane_i64<Q>(P + w * NPP64<Q>, i, j), E); };
  if (MODE == SMOOTH) {
    double acc = f[I];
#pragma unroll
    for (int w = 0; w < 14; ++w) acc = fma(-wt(w), nb(w), acc);
    u[I] = acc * rcp_i64_scaled(eval_plane_i64<Q>(P + MC * NPP64<Q>, i, j), E);
  } else {
    double y = wt(MC) * u[I];
#pragma unroll
    for (int w = 0; w < 14; ++w) y = fma(wt(w), nb(w), y);
    if (MODE == APPLY) {
      out[I] = y;
    } else {
      const double r = f[I] - y;
      out[I] = r;
      nrm = fma(r, r, nrm);
    }
  }
}

template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE64_THREADS, 2) lsqp_node_kernel(LevelView<double> lv, const uint32_t* __restrict__ list,
                                                                  int n_list, double* u, double* out, const double* f,
                                                                  double* partial) {
  extern __shared__ __align__(16) long long s_tab64[];   // [N - 3][15][NPP64]
  const int c = blockIdx.x;
  const int N = lv.N;
  load_plane64<Q>(lv, c, s_tab64);
  const int E = lv.cell_e[c];
  const int64_t base = lv.off_C + (int64_t)c * lv.n_int;
  __syncthreads();
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const long long* P = s_tab64 + (k - 1) * 15 * NPP64<Q>;
    const int64_t I = base + lin_interior32(i, j, k, N);
    if (deep_interior(i, j, k, N)) {
      int off[14];
      neighbour_offsets(j, k, N, off);
      const double* pu = u + I;
      lsqp64_node<Q, MODE>(P, (unsigned)i, (unsigned)j, E, [&](int w) { return pu[off[w]]; }, I, u, out, f, nrm);
    } else {
      lsqp64_node<Q, MODE>(P, (unsigned)i, (unsigned)j, E,
                           [&](int w) { return load_pt(lv, (const double*)u, c, i + DI(w), j + DJ(w), k + DK(w)); },
                           I, u, out, f, nrm);
    }
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// FP64 surrogate for all lv.nrhs right-hand sides at once, persistent over
// cells (grid-stride loop): per cell the plane table is staged once, per
// node the 15 weights and the centre reciprocal are formed once.
template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 2) lsqp_node_batch_kernel(LevelView<double> lv,
                                                                          const uint32_t* __restrict__ list, int n_list,
                                                                          double* u, double* out, const double* f,
                                                                          double* partial) {
  extern __shared__ __align__(16) long long s_tab64[];   // [N - 3][15][NPP64], then [nrhs][blockDim] doubles
  const int N = lv.N;
  double* s_nrm = reinterpret_cast<double*>(s_tab64 + (N - 3) * 15 * NPP64<Q>);
  for (int c = blockIdx.x; c < lv.nC; c += gridDim.x) {
    __syncthreads();
    load_plane64<Q>(lv, c, s_tab64);
    if (MODE == RESIDUAL)
      for (int b = 0; b < lv.nrhs; ++b) s_nrm[b * blockDim.x + threadIdx.x] = 0.0;
    const int E = lv.cell_e[c];
    __syncthreads();
    for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
      const uint32_t p = list[t];
      const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
      const long long* P = s_tab64 + (k - 1) * 15 * NPP64<Q>;
      double w[15];
#pragma unroll
      for (int v = 0; v < 15; ++v) w[v] = i64_to_f64_scaled(eval_plane_i64<Q>(P + v * NPP64<Q>, i, j), E);
      const double rc = MODE == SMOOTH ? rcp_i64_scaled(eval_plane_i64<Q>(P + MC * NPP64<Q>, i, j), E) : 0.0;
      node_apply_all<double, MODE>(lv, c, i, j, k, w, rc, u, out, f, s_nrm);
    }
    if (MODE == RESIDUAL) batch_norms_out(s_nrm, lv.nrhs, lv.pstride, c, partial);
  }
}

// ---------------------------------------------------------------------------
// FP64 surrogate along runs of a line: forward differences in exact integer
// arithmetic (Sec. 3.4, Eq. 5.4)
// ---------------------------------------------------------------------------

// 256 threads x 3 CTAs per SM: 80 registers a thread without spills (512 x 2
// caps them at 64 and spills).
constexpr int RUN64_THREADS = 256;

// One run of `cnt` points i0, i0 + h, .. of line (j, k) of cell c.  The
// weights are the same integers as in the per-node kernel, reached by
// additions instead of multiplies (Q additions per weight and point after a
// start of Q (Q + 1) / 2 + Q (Q + 1) multiply-adds per weight and run),
// converted and inverted on the integer pipe as there, and applied in the
// same order, so every result is bitwise that of lsqp_node_kernel.  The
// direction loop is outermost so only the run's accumulators and one
// difference table are live.
template <int Q, Mode MODE, bool DEEP>
__device__ __forceinline__ void lsqp64_run(const LevelView<double>& lv, const long long* P, int c, int E, int i0,
                                           int j, int k, int cnt, int h, int64_t I0, double* u, double* out,
                                           const double* f, double& nrm) {
  const int N = lv.N;
  const int L = N - 1 - j - k, m1 = N - 2 - k, m0 = N - 1 - k;
  const int tc = m1 * (m1 + 1) / 2 - j + 1, bc = -(m0 * (m0 + 1) / 2) + j - 1;
  double acc[RUN64];
  long long D[Q + 1];
  if (MODE == SMOOTH) {
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) acc[s] = f[I0 + s * h];
  } else {
    run_start<Q>(P + MC * NPP64<Q>, (unsigned)i0, (unsigned)j, (unsigned)h, D);
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        acc[s] = i64_to_f64_scaled(D[0], E) * u[I0 + s * h];
        run_step<Q>(D);
      }
  }
#pragma unroll 1
  for (int w = 0; w < 14; ++w) {
    run_start<Q>(P + w * NPP64<Q>, (unsigned)i0, (unsigned)j, (unsigned)h, D);
    const int off = neighbour_offset(w, L, tc, bc);
    const int di = DI(w), dj = DJ(w), dk = DK(w);
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        const double nb =
            DEEP ? u[I0 + s * h + off] : load_pt(lv, (const double*)u, c, i0 + s * h + di, j + dj, k + dk);
        const double wt = i64_to_f64_scaled(D[0], E);
        acc[s] = MODE == SMOOTH ? fma(-wt, nb, acc[s]) : fma(wt, nb, acc[s]);
        run_step<Q>(D);
      }
  }
  if (MODE == SMOOTH) {
    run_start<Q>(P + MC * NPP64<Q>, (unsigned)i0, (unsigned)j, (unsigned)h, D);
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        u[I0 + s * h] = acc[s] * rcp_i64_scaled(D[0], E);
        run_step<Q>(D);
      }
  } else {
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        if (MODE == APPLY) {
          out[I0 + s * h] = acc[s];
        } else {
          const double r = f[I0 + s * h] - acc[s];
          out[I0 + s * h] = r;
          nrm = fma(r, r, nrm);
        }
      }
  }
}

// FP64 surrogate over a run list (one colour with h = 4, or all interior
// points with h = 1): one CTA per macro cell, its plane table staged in
// shared memory, a thread per run.
template <int Q, Mode MODE>
__global__ void __launch_bounds__(RUN64_THREADS, 3) lsqp_run64_kernel(LevelView<double> lv,
                                                                      const uint2* __restrict__ items, int n_items,
                                                                      int h, double* u, double* out, const double* f,
                                                                      double* partial) {
  extern __shared__ __align__(16) long long s_tab64[];   // [N - 3][15][NPP64]
  const int c = blockIdx.x;
  const int N = lv.N;
  load_plane64<Q>(lv, c, s_tab64);
  const int E = lv.cell_e[c];
  const int64_t base = lv.off_C + (int64_t)c * lv.n_int;
  __syncthreads();
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_items; t += blockDim.x) {
    const uint2 it = items[t];
    const int i0 = unpack_i(it.x), j = unpack_j(it.x), k = unpack_k(it.x);
    const int cnt = (int)(it.y & 0xffu);
    const long long* P = s_tab64 + (k - 1) * 15 * NPP64<Q>;
    const int64_t I0 = base + lin_interior32(i0, j, k, N);
    if (it.y & 0x100u)
      lsqp64_run<Q, MODE, true>(lv, P, c, E, i0, j, k, cnt, h, I0, u, out, f, nrm);
    else
      lsqp64_run<Q, MODE, false>(lv, P, c, E, i0, j, k, cnt, h, I0, u, out, f, nrm);
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// ---------------------------------------------------------------------------
// FP32 surrogate: per-plane polynomials in (i, j), thread per node
// ---------------------------------------------------------------------------

// FP32 per-plane table (fit time): for every cell, plane k = 1..N-3 and
// direction, the (Q+1)(Q+2)/2 coefficients of the polynomial in (i, j),
// formed in FP64 from the fitted coefficients and rounded once to FP32.
template <int Q>
__global__ void lsqp_plane_table_kernel(const double* __restrict__ coef, int nC, int N, float* __restrict__ table) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  const int np = N - 3;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nC * np * 15) return;
  const int w = (int)(t % 15);
  const int64_t cp = t / 15;
  const int c = (int)(cp / np), k = (int)(cp % np) + 1;
  double P[NP];
  plane_coeffs<double, Q>(coef + ((int64_t)c * 15 + w) * MQ, (double)k, P);
  float* dst = table + t * NP;
#pragma unroll
  for (int a = 0; a < NP; ++a) dst[a] = (float)P[a];
}

template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE32_THREADS, 2) lsqp_node32_kernel(LevelView<float> lv,
                                                                     const uint32_t* __restrict__ list, int n_list,
                                                                     float* u, float* out, const float* f,
                                                                     double* partial) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NPP = np_pad<Q>();
  extern __shared__ __align__(16) float s_tab[];   // [N - 3][15][NPP]
  const int c = blockIdx.x;
  const int np = lv.N - 3;
  const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
  for (int t = threadIdx.x; t < np * 15 * NPP; t += blockDim.x) {
    const int e = t % NPP, pw = t / NPP;
    s_tab[t] = e < NP ? tab[pw * NP + e] : 0.0f;
  }
  __syncthreads();
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const float* P = s_tab + (k - 1) * 15 * NPP;
    const float ti = (float)i, tj = (float)j;
    auto wt = [&](int w) -> float {
      float Pw[NPP];
#pragma unroll
      for (int v = 0; v < NPP; v += 4) {
        const float4 q4 = *reinterpret_cast<const float4*>(P + w * NPP + v);
        Pw[v] = q4.x;
        Pw[v + 1] = q4.y;
        Pw[v + 2] = q4.z;
        Pw[v + 3] = q4.w;
      }
      return eval_plane<float, Q>(Pw, ti, tj);
    };
    node_update<float, MODE>(lv, c, i, j, k, wt, u, out, f, nrm, 1.0f, 1.0f);
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// The same update with two nodes per thread in flight: both nodes' list
// entries, neighbours and f are loaded before either is computed, so their
// memory latencies overlap (same arithmetic per node as lsqp_node32_kernel).
template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 4) lsqp_node32_x2_kernel(LevelView<float> lv,
                                                                        const uint32_t* __restrict__ list, int n_list,
                                                                        float* u, float* out, const float* f,
                                                                        double* partial) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NPP = np_pad<Q>();
  extern __shared__ __align__(16) float s_tab[];   // [N - 3][15][NPP]
  const int c = blockIdx.x;
  const int N = lv.N, np = N - 3;
  const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
  for (int t = threadIdx.x; t < np * 15 * NPP; t += blockDim.x) {
    const int e = t % NPP, pw = t / NPP;
    s_tab[t] = e < NP ? tab[pw * NP + e] : 0.0f;
  }
  __syncthreads();
  const int64_t base = lv.off_C + (int64_t)c * lv.n_int;
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += 2 * blockDim.x) {
    float nbv[2][14], fv[2], uc[2];
    int ii[2], jj[2], kk[2];
    int64_t I[2];
    bool ok[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int th = t + h * (int)blockDim.x;
      ok[h] = th < n_list;
      const uint32_t p = list[ok[h] ? th : t];
      ii[h] = unpack_i(p);
      jj[h] = unpack_j(p);
      kk[h] = unpack_k(p);
      I[h] = base + lin_interior32(ii[h], jj[h], kk[h], N);
      if (deep_interior(ii[h], jj[h], kk[h], N)) {
        int off[14];
        neighbour_offsets(jj[h], kk[h], N, off);
#pragma unroll
        for (int w = 0; w < 14; ++w) nbv[h][w] = u[I[h] + off[w]];
      } else {
#pragma unroll
        for (int w = 0; w < 14; ++w)
          nbv[h][w] = load_pt(lv, (const float*)u, c, ii[h] + DI(w), jj[h] + DJ(w), kk[h] + DK(w));
      }
      fv[h] = MODE != APPLY ? f[I[h]] : 0.0f;
      uc[h] = MODE != SMOOTH ? u[I[h]] : 0.0f;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!ok[h]) continue;
      const float* P = s_tab + (kk[h] - 1) * 15 * NPP;
      const float ti = (float)ii[h], tj = (float)jj[h];
      auto wt = [&](int w) -> float {
        float Pw[NPP];
#pragma unroll
        for (int v = 0; v < NPP; v += 4) {
          const float4 q4 = *reinterpret_cast<const float4*>(P + w * NPP + v);
          Pw[v] = q4.x;
          Pw[v + 1] = q4.y;
          Pw[v + 2] = q4.z;
          Pw[v + 3] = q4.w;
        }
        return eval_plane<float, Q>(Pw, ti, tj);
      };
      if (MODE == SMOOTH) {
        float a0 = fv[h], a1 = 0.0f;
#pragma unroll
        for (int w = 0; w < 14; w += 2) {
          a0 = fmaf(-wt(w), nbv[h][w], a0);
          a1 = fmaf(-wt(w + 1), nbv[h][w + 1], a1);
        }
        u[I[h]] = (a0 + a1) / wt(MC);
      } else {
        float a0 = wt(MC) * uc[h], a1 = 0.0f;
#pragma unroll
        for (int w = 0; w < 14; w += 2) {
          a0 = fmaf(wt(w), nbv[h][w], a0);
          a1 = fmaf(wt(w + 1), nbv[h][w + 1], a1);
        }
        const float y = a0 + a1;
        if (MODE == APPLY) {
          out[I[h]] = y;
        } else {
          const float r = fmaf(-1.0f, y, fv[h]);
          out[I[h]] = r;
          nrm += (double)r * (double)r;
        }
      }
    }
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// ---------------------------------------------------------------------------
// FP32 surrogate smoother over chunked colour lists: a thread takes up to
// CHUNK32 deep-interior points i0, i0 + 4, .. of one line (j, k) of the
// colour, so the index arithmetic (position, the 14 neighbour offsets of the
// line) and each direction pair's line coefficients C_a(j) are formed once
// per chunk; per point the weights are a Horner step in i (packed FP32 FMA).
// The same operations in the same order as eval_plane2, so the same FP32
// weights as the one-point kernels.  Points next to the cell boundary are
// single items.  blockIdx.x = (cell - c0) * splits + part: a cell's items are
// shared by `splits` CTAs.
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(NODE_THREADS, 4) lsqp_chunk32_smooth(LevelView<float> lv,
                                                                      const uint32_t* __restrict__ items,
                                                                      int n_deep, int n, int c0, int splits,
                                                                      float* u, const float* f) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NP2 = npp2<Q>();
  extern __shared__ __align__(16) float2 s_tab2[];   // [N - 3][NPAIR][NP2]
  const int N = lv.N, np = N - 3;
  const int c = c0 + blockIdx.x / splits, part = blockIdx.x % splits;
  {
    const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
    float* d = reinterpret_cast<float*>(s_tab2);
    for (int t = threadIdx.x; t < np * NPAIR * NP2 * 2; t += blockDim.x) {
      const int h = t & 1, e = (t >> 1) % NP2, m = ((t >> 1) / NP2) % NPAIR, k = (t >> 1) / (NP2 * NPAIR);
      const int w = 2 * m + h;
      d[t] = (e < NP && w < 15) ? tab[((int64_t)k * 15 + w) * NP + e] : 0.0f;
    }
  }
  __syncthreads();
  float* uc = u + lv.off_C + (int64_t)c * lv.n_int;
  const float* fc = f + lv.off_C + (int64_t)c * lv.n_int;
  const int t0 = (int)((int64_t)n * part / splits), t1 = (int)((int64_t)n * (part + 1) / splits);
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const uint32_t p = items[t];
    const int i0 = (int)(p & 1023u), j = (int)((p >> 10) & 1023u), k = (int)((p >> 20) & 1023u);
    const float2* P = s_tab2 + (k - 1) * NPAIR * NP2;
    const float2 Jv = make_float2((float)j, (float)j);
    const int lin0 = lin_interior32(i0, j, k, N);
    if (t < n_deep) {
      const int cnt = (int)(p >> 30) + 1;
      int off[14];
      neighbour_offsets(j, k, N, off);
      float2 acc[CHUNK32];
#pragma unroll
      for (int q = 0; q < CHUNK32; ++q) acc[q] = make_float2(0.0f, 0.0f);
      float2 C[Q + 1];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
#pragma unroll
        for (int a = 0; a <= Q; ++a) {
          float2 ca = P[m * NP2 + plane_index<Q>(a, Q - a)];
#pragma unroll
          for (int b = Q - a - 1; b >= 0; --b) ca = __ffma2_rn(ca, Jv, P[m * NP2 + plane_index<Q>(a, b)]);
          C[a] = ca;
        }
#pragma unroll
        for (int q = 0; q < CHUNK32; ++q) {
          if (q < cnt) {
            const float fi = (float)(i0 + 4 * q);
            const float2 Iv = make_float2(fi, fi);
            float2 w2 = C[Q];
#pragma unroll
            for (int a = Q - 1; a >= 0; --a) w2 = __ffma2_rn(w2, Iv, C[a]);
            if (m < 7) {
              const int x = lin0 + 4 * q;
              acc[q] = __ffma2_rn(w2, make_float2(uc[x + off[2 * m]], uc[x + off[2 * m + 1]]), acc[q]);
            } else {
              const int x = lin0 + 4 * q;
              uc[x] = div_nr32(fc[x] - acc[q].x - acc[q].y, w2.x);
            }
          }
        }
      }
    } else {
      const float2 Iv = make_float2((float)i0, (float)i0);
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        const float a = load_pt(lv, (const float*)u, c, i0 + DI(2 * m), j + DJ(2 * m), k + DK(2 * m));
        const float b = load_pt(lv, (const float*)u, c, i0 + DI(2 * m + 1), j + DJ(2 * m + 1), k + DK(2 * m + 1));
        acc = __ffma2_rn(eval_plane2<Q>(P + m * NP2, Iv, Jv), make_float2(a, b), acc);
      }
      const float wc = eval_plane2<Q>(P + 7 * NP2, Iv, Jv).x;
      uc[lin0] = div_nr32(fc[lin0] - acc.x - acc.y, wc);
    }
  }
}

// FP32 surrogate for all lv.nrhs right-hand sides at once, persistent over
// cells: per cell the per-plane table is staged once, per node the 15
// weights (5 FMA each from the table) and the centre reciprocal are formed
// once and applied to every vector.
template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 2) lsqp_node32_batch_kernel(LevelView<float> lv,
                                                                            const uint32_t* __restrict__ list,
                                                                            int n_list, float* u, float* out,
                                                                            const float* f, double* partial) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NPP = np_pad<Q>();
  extern __shared__ __align__(16) float s_tab[];   // [N - 3][15][NPP], then [nrhs][blockDim] doubles
  const int np = lv.N - 3;
  double* s_nrm = reinterpret_cast<double*>(s_tab + np * 15 * NPP);
  for (int c = blockIdx.x; c < lv.nC; c += gridDim.x) {
    __syncthreads();
    const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
    for (int t = threadIdx.x; t < np * 15 * NPP; t += blockDim.x) {
      const int e = t % NPP, pw = t / NPP;
      s_tab[t] = e < NP ? tab[pw * NP + e] : 0.0f;
    }
    if (MODE == RESIDUAL)
      for (int b = 0; b < lv.nrhs; ++b) s_nrm[b * blockDim.x + threadIdx.x] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
      const uint32_t p = list[t];
      const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
      const float* P = s_tab + (k - 1) * 15 * NPP;
      float w[15];
#pragma unroll
      for (int v = 0; v < 15; ++v) w[v] = eval_plane<float, Q>(P + v * NPP, (float)i, (float)j);
      const float rc = MODE == SMOOTH ? 1.0f / w[MC] : 0.0f;
      node_apply_all<float, MODE>(lv, c, i, j, k, w, rc, u, out, f, s_nrm);
    }
    if (MODE == RESIDUAL) batch_norms_out(s_nrm, lv.nrhs, lv.pstride, c, partial);
  }
}

// ---------------------------------------------------------------------------
// IFEM: exact stencils assembled on the fly, thread per node
// ---------------------------------------------------------------------------

template <class T, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS) ifem_node_kernel(LevelView<T> lv, const uint32_t* __restrict__ list,
                                                                  int n_list, T* u, T* out, const T* f,
                                                                  double* partial) {
  __shared__ CellGeom g;
  const int c = blockIdx.x;
  if (threadIdx.x < 16)
    reinterpret_cast<double*>(&g)[threadIdx.x] = reinterpret_cast<const double*>(&lv.geom[c])[threadIdx.x];
  __syncthreads();
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    double s[15];
    ifem_stencil(g, lv.N, i, j, k, s);
    auto wt = [&](int w) -> T { return (T)s[w]; };
    node_update<T, MODE>(lv, c, i, j, k, wt, u, out, f, nrm, T(1), T(1));
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// IFEM for all lv.nrhs right-hand sides at once, persistent over cells: one
// stencil assembly per node, applied to every vector.
template <class T, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS) ifem_node_batch_kernel(LevelView<T> lv, const uint32_t* __restrict__ list,
                                                                        int n_list, T* u, T* out, const T* f,
                                                                        double* partial) {
  __shared__ CellGeom g;
  extern __shared__ __align__(16) double s_nrm_ifem[];   // [nrhs][blockDim]
  for (int c = blockIdx.x; c < lv.nC; c += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < 16)
      reinterpret_cast<double*>(&g)[threadIdx.x] = reinterpret_cast<const double*>(&lv.geom[c])[threadIdx.x];
    if (MODE == RESIDUAL)
      for (int b = 0; b < lv.nrhs; ++b) s_nrm_ifem[b * blockDim.x + threadIdx.x] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
      const uint32_t p = list[t];
      const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
      double s[15];
      ifem_stencil(g, lv.N, i, j, k, s);
      T w[15];
#pragma unroll
      for (int v = 0; v < 15; ++v) w[v] = (T)s[v];
      const T rc = MODE == SMOOTH ? (T)(1.0 / s[MC]) : T(0);
      node_apply_all<T, MODE>(lv, c, i, j, k, w, rc, u, out, f, s_nrm_ifem);
    }
    if (MODE == RESIDUAL) batch_norms_out(s_nrm_ifem, lv.nrhs, lv.pstride, c, partial);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// Largest dynamic shared memory a batched launch plans for (the device
// allows 227 KB per CTA; the rest is left to static shared memory).
constexpr size_t SMEM_BATCH_MAX = 220 * 1024;

// Grid of a persistent kernel: as many CTAs as are resident at once, at most nC.
int persistent_grid(const void* kern, int threads, size_t smem, int nC) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    HHG_CUDA(cudaGetDevice(&dev));
    HHG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  int per = 0;
  HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem));
  return std::max(1, std::min(nC, sms * std::max(per, 1)));
}

// A batched cell kernel over all lv.nrhs right-hand sides.  In RESIDUAL mode
// the per-thread norm accumulators (nrhs x NODE_THREADS doubles) follow the
// table in shared memory, so right-hand sides go in chunks that fit.
template <class T, Mode MODE, class K>
void launch_batch(K kern, const LevelView<T>& lv, size_t table_bytes, const uint32_t* list, int n, T* u, T* out,
                  const T* f, double* partial, cudaStream_t st) {
  const size_t per_rhs = MODE == RESIDUAL ? sizeof(double) * NODE_THREADS : 0;
  HHG_CHECK(table_bytes + per_rhs <= SMEM_BATCH_MAX, HHG_EINVAL, "batched cell kernel: table exceeds shared memory");
  const int chunk = per_rhs ? (int)std::min<size_t>(lv.nrhs, (SMEM_BATCH_MAX - table_bytes) / per_rhs) : lv.nrhs;
  for (int b0 = 0; b0 < lv.nrhs; b0 += chunk) {
    LevelView<T> sub = lv;
    sub.nrhs = std::min(chunk, lv.nrhs - b0);
    sub.ghost = lv.ghost + (int64_t)b0 * lv.gstride;
    const int64_t vo = (int64_t)b0 * lv.vstride;
    const size_t smem = table_bytes + per_rhs * sub.nrhs;
    ensure_smem_limit((const void*)kern, smem);
    const int grid = persistent_grid((const void*)kern, NODE_THREADS, smem, lv.nC);
    kern<<<grid, NODE_THREADS, smem, st>>>(sub, list, n, u + vo, out ? out + vo : nullptr, f ? f + vo : nullptr,
                                           partial ? partial + (int64_t)b0 * lv.pstride : nullptr);
    HHG_CUDA(cudaGetLastError());
    count_launch();
  }
}

template <int Q, Mode MODE>
void launch_node64(const LevelView<double>& lv, const uint32_t* list, int n, double* u, double* out, const double* f,
                   double* partial, cudaStream_t st) {
  HHG_CHECK(lv.plane64 != nullptr, HHG_ENOTFIT, "FP64 surrogate plane table missing");
  const size_t table = sizeof(long long) * (size_t)(lv.N - 3) * 15 * NPP64<Q>;
  if (lv.nrhs == 1) {
    auto kern = lsqp_node_kernel<Q, MODE>;
    ensure_smem_limit((const void*)kern, table);
    kern<<<lv.nC, NODE64_THREADS, table, st>>>(lv, list, n, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  launch_batch<double, MODE>(lsqp_node_batch_kernel<Q, MODE>, lv, table, list, n, u, out, f, partial, st);
}

// Run-list segment g (colour g = 0..3 with stride 4, or 4 = all interior
// points with stride 1) through the FP64 run kernel (single right-hand side).
template <int Q, Mode MODE>
void launch_run64(const LevelView<double>& lv, int g, double* u, double* out, const double* f, double* partial,
                  cudaStream_t st) {
  HHG_CHECK(lv.plane64 != nullptr, HHG_ENOTFIT, "FP64 surrogate plane table missing");
  const size_t table = sizeof(long long) * (size_t)(lv.N - 3) * 15 * NPP64<Q>;
  auto kern = lsqp_run64_kernel<Q, MODE>;
  ensure_smem_limit((const void*)kern, table);
  kern<<<lv.nC, RUN64_THREADS, table, st>>>(lv, lv.run_nodes + lv.run_off[g], lv.run_off[g + 1] - lv.run_off[g],
                                            g < 4 ? 4 : 1, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <int Q>
void lsqp64(const LevelView<double>& lv, Mode mode, double* u, double* out, const double* f, double* partial,
            cudaStream_t st) {
  if (mode == SMOOTH && lv.fp64_kernel == FP64_RESIDENT && resident_supported(lv)) {
    launch_resident_sweep<double>(lv, u, f, st);
    return;
  }
  if (lv.nrhs == 1 && lv.fp64_kernel != FP64_NODES) {
    switch (mode) {
      case APPLY: launch_run64<Q, APPLY>(lv, 4, u, out, f, partial, st); break;
      case RESIDUAL: launch_run64<Q, RESIDUAL>(lv, 4, u, out, f, partial, st); break;
      case SMOOTH:
        for (int cc = 0; cc < 4; ++cc) launch_run64<Q, SMOOTH>(lv, cc, u, out, f, partial, st);
        break;
    }
    return;
  }
  switch (mode) {
    case APPLY: launch_node64<Q, APPLY>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case RESIDUAL: launch_node64<Q, RESIDUAL>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case SMOOTH:
      for (int cc = 0; cc < 4; ++cc)
        launch_node64<Q, SMOOTH>(lv, lv.colour_nodes + lv.colour_off[cc], lv.colour_off[cc + 1] - lv.colour_off[cc],
                                 u, out, f, partial, st);
      break;
  }
}

template <int Q, Mode MODE>
void launch_node32(const LevelView<float>& lv, const uint32_t* list, int n, float* u, float* out, const float* f,
                   double* partial, cudaStream_t st) {
  HHG_CHECK(lv.plane32 != nullptr, HHG_ENOTFIT, "FP32 surrogate plane table missing");
  const size_t smem = sizeof(float) * (size_t)(lv.N - 3) * 15 * np_pad<Q>();
  if (lv.nrhs == 1) {
    auto kern = lv.smooth_cfg == -2 ? lsqp_node32_x2_kernel<Q, MODE> : lsqp_node32_kernel<Q, MODE>;
    ensure_smem_limit((const void*)kern, smem);
    kern<<<lv.nC, lv.smooth_cfg == -2 ? NODE_THREADS : NODE32_THREADS, smem, st>>>(lv, list, n, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  launch_batch<float, MODE>(lsqp_node32_batch_kernel<Q, MODE>, lv, smem, list, n, u, out, f, partial, st);
}

// The chunked FP32 smoother over one colour for cells [c0, c0 + nc), each
// cell's items shared by `splits` CTAs.
template <int Q>
void launch_chunk32(const LevelView<float>& lv, int cc, int c0, int nc, int splits, float* u, const float* f,
                    cudaStream_t st) {
  const size_t smem = sizeof(float2) * (size_t)(lv.N - 3) * NPAIR * npp2<Q>();
  auto kern = lsqp_chunk32_smooth<Q>;
  ensure_smem_limit((const void*)kern, smem);
  const int beg = lv.chunk_off[cc];
  kern<<<nc * splits, NODE_THREADS, smem, st>>>(lv, lv.chunk_nodes + beg, lv.chunk_mid[cc] - beg,
                                                lv.chunk_off[cc + 1] - beg, c0, splits, u, f);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

// One sweep of the four colours by the chunked kernel, each colour one
// launch over all cells.
template <int Q>
void chunk32_sweep(const LevelView<float>& lv, float* u, const float* f, cudaStream_t st) {
  for (int cc = 0; cc < 4; ++cc) launch_chunk32<Q>(lv, cc, 0, lv.nC, 1, u, f, st);
}

template <int Q>
void lsqp32(const LevelView<float>& lv, Mode mode, float* u, float* out, const float* f, double* partial,
            cudaStream_t st) {
  switch (mode) {
    case APPLY: launch_node32<Q, APPLY>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case RESIDUAL: launch_node32<Q, RESIDUAL>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case SMOOTH:
      for (int cc = 0; cc < 4; ++cc)
        launch_node32<Q, SMOOTH>(lv, lv.colour_nodes + lv.colour_off[cc], lv.colour_off[cc + 1] - lv.colour_off[cc],
                                 u, out, f, partial, st);
      break;
  }
}

template <class T, Mode MODE>
void launch_ifem(const LevelView<T>& lv, const uint32_t* list, int n, T* u, T* out, const T* f, double* partial,
                 cudaStream_t st) {
  if (lv.nrhs == 1) {
    ifem_node_kernel<T, MODE><<<lv.nC, NODE_THREADS, 0, st>>>(lv, list, n, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  launch_batch<T, MODE>(ifem_node_batch_kernel<T, MODE>, lv, 0, list, n, u, out, f, partial, st);
}

template <class T>
void ifem_all(const LevelView<T>& lv, Mode mode, T* u, T* out, const T* f, double* partial, cudaStream_t st) {
  switch (mode) {
    case APPLY: launch_ifem<T, APPLY>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case RESIDUAL: launch_ifem<T, RESIDUAL>(lv, lv.all_nodes, (int)lv.n_int, u, out, f, partial, st); break;
    case SMOOTH:
      for (int cc = 0; cc < 4; ++cc)
        launch_ifem<T, SMOOTH>(lv, lv.colour_nodes + lv.colour_off[cc], lv.colour_off[cc + 1] - lv.colour_off[cc], u,
                               out, f, partial, st);
      break;
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

bool chunk32_supported(const LevelView<float>& lv) {
  if (lv.q < 1 || lv.q > 3 || lv.N < 8 || lv.plane32 == nullptr || lv.chunk_nodes == nullptr) return false;
  static int optin = 0;
  if (optin == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
  }
  const int np2 = lv.q == 1 ? npp2<1>() : (lv.q == 2 ? npp2<2>() : npp2<3>());
  return sizeof(float2) * (size_t)(lv.N - 3) * NPAIR * np2 <= (size_t)optin;
}

template <>
void launch_cell<double>(const LevelView<double>& lv, int op, Mode mode, double* u, double* out, const double* f,
                         double* partial, cudaStream_t st) {
  if (lv.N < 4 || lv.n_int == 0) return;
  if (op == HHG_OP_LSQP && lv.q > 0) {
    switch (lv.q) {
      case 1: lsqp64<1>(lv, mode, u, out, f, partial, st); break;
      case 2: lsqp64<2>(lv, mode, u, out, f, partial, st); break;
      case 3: lsqp64<3>(lv, mode, u, out, f, partial, st); break;
      default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
    }
    return;
  }
  ifem_all<double>(lv, mode, u, out, f, partial, st);
}

template <>
void launch_cell<float>(const LevelView<float>& lv, int op, Mode mode, float* u, float* out, const float* f,
                        double* partial, cudaStream_t st) {
  if (lv.N < 4 || lv.n_int == 0) return;
  if (op == HHG_OP_LSQP && lv.q > 0) {
    // the staged sweep holds one vector's planes; batches take the batched
    // per-colour kernel, which forms every node's weights once for all of them
    if (mode == SMOOTH && lv.nrhs == 1 && lv.smooth_cfg >= 0 && smooth32_supported(lv, u, lv.smooth_cfg)) {
      const int cfg = lv.smooth_cfg;
      if (cfg < STAGE32_CONFIGS) {
        launch_stage32_smooth(lv, u, f, cfg, st);
      } else if (cfg < STAGE32_CONFIGS + WAVE32_CONFIGS) {
        launch_wave32_smooth(lv, u, f, cfg - STAGE32_CONFIGS, st);
      } else if (cfg < STAGE32_CONFIGS + WAVE32_CONFIGS + CHUNK32_CONFIGS) {
        switch (lv.q) {
          case 1: chunk32_sweep<1>(lv, u, f, st); break;
          case 2: chunk32_sweep<2>(lv, u, f, st); break;
          default: chunk32_sweep<3>(lv, u, f, st); break;
        }
      } else {
        launch_resident_sweep<float>(lv, u, f, st);
      }
      return;
    }
    switch (lv.q) {
      case 1: lsqp32<1>(lv, mode, u, out, f, partial, st); break;
      case 2: lsqp32<2>(lv, mode, u, out, f, partial, st); break;
      case 3: lsqp32<3>(lv, mode, u, out, f, partial, st); break;
      default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
    }
    return;
  }
  ifem_all<float>(lv, mode, u, out, f, partial, st);
}

void launch_plane64_table(const LevelView<double>& lv, int q, const double* coef, int* cell_e, long long* table,
                          cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * (lv.N - 3) * 15;
  const unsigned gs = (unsigned)((lv.nC + 127) / 128), gl = (unsigned)((n + 127) / 128);
  switch (q) {
    case 1:
      lsqp_scale_kernel<1><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_plane64_kernel<1><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
      break;
    case 2:
      lsqp_scale_kernel<2><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_plane64_kernel<2><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
      break;
    case 3:
      lsqp_scale_kernel<3><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_plane64_kernel<3><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
      break;
    default:
      throw Error{HHG_EINVAL, "q must be 1, 2 or 3"};
  }
  HHG_CUDA(cudaGetLastError());
  count_launch(2);
}

void launch_plane_table(const LevelView<double>& lv, int q, const double* coef, float* table, cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * (lv.N - 3) * 15;
  const unsigned g = (unsigned)((n + 127) / 128);
  switch (q) {
    case 1: lsqp_plane_table_kernel<1><<<g, 128, 0, st>>>(coef, lv.nC, lv.N, table); break;
    case 2: lsqp_plane_table_kernel<2><<<g, 128, 0, st>>>(coef, lv.nC, lv.N, table); break;
    case 3: lsqp_plane_table_kernel<3><<<g, 128, 0, st>>>(coef, lv.nC, lv.N, table); break;
    default: throw Error{HHG_EINVAL, "q must be 1, 2 or 3"};
  }
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

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
