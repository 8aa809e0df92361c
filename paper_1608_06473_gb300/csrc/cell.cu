// Cell-interior kernels: the volume primitives, which hold all but
// O(2^{2l}) of the nodes (Sec. 2.3).
//
// Surrogate (LSQP, Sec. 3.4).  For a fixed line (j, k) each of the 15
// 3-variate polynomials is a polynomial of degree q in i -- the line-wise
// evaluation the paper builds on (Sec. 3.4; Eq. 5.4).  Two designs, one per
// precision, because GB300 issues FP64 at a small fraction of its FP32 and
// INT32 rate:
//
//  * FP64: the line polynomials of every cell are computed once per fit
//    (lsqp_line_table_kernel) as integers scaled by 2^E (E per cell, chosen so
//    every partial sum stays below 2^62) and kept in HBM.  Per node the
//    polynomial is evaluated exactly by integer Horner and converted to FP64
//    once per weight; the FP64 pipe then only carries the conversions, the 14
//    stencil products and the divide.  Kernels are thread-per-node with one
//    CTA per macro cell and no barriers; the smoother is one launch per colour.
//  * FP32: one CTA per cell walks its planes; per plane k each direction's
//    polynomial is reduced to a polynomial in (i, j) in shared memory and
//    evaluated per node (FP32 arithmetic is cheap, HBM traffic is the
//    bound), and the four colours run in one launch as a plane wavefront:
//    in step s colour c is updated on plane s + 1 - c, c = 0..3, with a
//    barrier after each colour, so every update sees all lower-colour updates
//    of planes k - 1, k, k + 1 and none of the higher ones -- exactly four
//    colour sweeps in one pass over the cell.
//
// IFEM (Sec. 4.2.1): every node assembles its 15 weights from the 24 element
// matrices around it (thread per node, one launch per colour).
//
// Neighbour addressing: nodes whose 14 neighbours are all interior use
// closed-form 32-bit offsets within the cell's block of the canonical
// vector; nodes next to the cell boundary read boundary neighbours from the
// cell's halo copy.
#include <cstdlib>

#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace hhg {

namespace {

constexpr int WAVE_THREADS = 256;  // FP32 wavefront kernel
constexpr int NODE_THREADS = 256;  // thread-per-node kernels

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
// FP64 surrogate: line table at fit time, thread-per-node application
// ---------------------------------------------------------------------------

// E per cell: B = max_w sum_t |A_wt| N^deg(t) bounds |c_a(j,k)| i^a on every
// line and node, so with B 2^E < 2^60 every Horner partial sum of
// C_q i^q + .. + C_0 stays below (q + 1) 2^60 <= 2^62.
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

template <int Q>
__global__ void lsqp_line_table_kernel(const double* __restrict__ coef, const int* __restrict__ cell_e, int nC, int N,
                                       long long* __restrict__ table) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  const int nl = (int)n_cell_lines(N);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nC * nl) return;
  const int c = (int)(t / nl), line = (int)(t % nl);
  int k = 1, j = line + 1;
  while (j > N - 2 - k) {
    j -= N - 2 - k;
    ++k;
  }
  const double sc = ldexp(1.0, cell_e[c]);
  long long* dst = table + t * line_rec(Q);
  for (int w = 0; w < 15; ++w) {
    double cl[Q + 1];
    line_coeffs<double, Q>(coef + ((int64_t)c * 15 + w) * MQ, (double)j, (double)k, cl);
#pragma unroll
    for (int a = 0; a <= Q; ++a) dst[w * (Q + 1) + a] = __double2ll_rn(cl[a] * sc);
  }
  for (int r = 15 * (Q + 1); r < line_rec(Q); ++r) dst[r] = 0;
}

template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 3) lsqp_node_kernel(LevelView<double> lv, const uint32_t* __restrict__ list,
                                                                  int n_list, double* u, double* out, const double* f,
                                                                  double* partial) {
  const int c = blockIdx.x;
  const int N = lv.N;
  const int E = lv.cell_e[c];
  const double scale = ldexp(1.0, E), inv_scale = ldexp(1.0, -E);
  const long long* tab = lv.line64 + (int64_t)c * lv.n_lines * line_rec(Q);
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const long long* C = tab + (int64_t)line_id(j, k, N) * line_rec(Q);
    auto wt = [&](int w) -> double {
      long long v = C[w * (Q + 1) + Q];
#pragma unroll
      for (int a = Q - 1; a >= 0; --a) v = v * (long long)i + C[w * (Q + 1) + a];
      return (double)v;
    };
    node_update<double, MODE>(lv, c, i, j, k, wt, u, out, f, nrm, scale, inv_scale);
  }
  if (MODE == RESIDUAL) {
    const double tot = block_sum(nrm);
    if (threadIdx.x == 0) partial[c] = tot;
  }
}

// ---------------------------------------------------------------------------
// FP32 surrogate: plane wavefront, per-plane polynomials in (i, j)
// ---------------------------------------------------------------------------

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

template <class T, int Q, Mode MODE>
__global__ void __launch_bounds__(WAVE_THREADS, 2) lsqp_wave_kernel(LevelView<T> lv, T* u, T* out, const T* f,
                                                                 double* partial) {
  constexpr int MQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  constexpr int NP = (Q + 1) * (Q + 2) / 2;       // per-plane values per direction
  constexpr int NSLOT = (MODE == SMOOTH) ? 4 : 1;
  __shared__ T sA[15 * MQ];
  __shared__ T ring[NSLOT][15 * NP];
  const int c = blockIdx.x;
  const int N = lv.N;
  for (int t = threadIdx.x; t < 15 * MQ; t += blockDim.x) sA[t] = lv.coef[(int64_t)c * 15 * MQ + t];
  __syncthreads();
  double nrm = 0.0;

  auto prologue = [&](int k) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    if (threadIdx.x < 15) plane_coeffs<T, Q>(sA + threadIdx.x * MQ, (T)k, &ring[slot][threadIdx.x * NP]);
  };
  auto process = [&](int k, int beg, int end) {
    const int slot = (NSLOT == 4) ? (k & 3) : 0;
    for (int t = beg + threadIdx.x; t < end; t += blockDim.x) {
      const uint32_t p = lv.plane_nodes[t];
      const int i = unpack_i(p), j = unpack_j(p);
      const T* P = ring[slot];
      const T ti = (T)i, tj = (T)j;
      auto wt = [&](int w) -> T { return eval_plane<T, Q>(P + w * NP, ti, tj); };
      node_update<T, MODE>(lv, c, i, j, k, wt, u, out, f, nrm, T(1), T(1));
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

// Per-plane coefficients of one direction padded to a multiple of 4 floats
// (128-bit shared-memory loads).
template <int Q>
__host__ __device__ constexpr int np_pad() { return ((Q + 1) * (Q + 2) / 2 + 3) / 4 * 4; }

template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 4) lsqp_node32_kernel(LevelView<float> lv,
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

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <class T, int Q, Mode MODE>
void launch_wave(const LevelView<T>& lv, T* u, T* out, const T* f, double* partial, cudaStream_t st) {
  lsqp_wave_kernel<T, Q, MODE><<<lv.nC, WAVE_THREADS, 0, st>>>(lv, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <int Q, Mode MODE>
void launch_node64(const LevelView<double>& lv, const uint32_t* list, int n, double* u, double* out, const double* f,
                   double* partial, cudaStream_t st) {
  HHG_CHECK(lv.line64 != nullptr, HHG_ENOTFIT, "FP64 surrogate line table missing");
  lsqp_node_kernel<Q, MODE><<<lv.nC, NODE_THREADS, 0, st>>>(lv, list, n, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <int Q>
void lsqp64(const LevelView<double>& lv, Mode mode, double* u, double* out, const double* f, double* partial,
            cudaStream_t st) {
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
  auto kern = lsqp_node32_kernel<Q, MODE>;
  if (smem > 48 * 1024) HHG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<lv.nC, NODE_THREADS, smem, st>>>(lv, list, n, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
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
void dispatch_wave(const LevelView<T>& lv, T* u, T* out, const T* f, double* partial, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_wave<T, 1, MODE>(lv, u, out, f, partial, st); break;
    case 2: launch_wave<T, 2, MODE>(lv, u, out, f, partial, st); break;
    case 3: launch_wave<T, 3, MODE>(lv, u, out, f, partial, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}

template <class T, Mode MODE>
void launch_ifem(const LevelView<T>& lv, const uint32_t* list, int n, T* u, T* out, const T* f, double* partial,
                 cudaStream_t st) {
  ifem_node_kernel<T, MODE><<<lv.nC, NODE_THREADS, 0, st>>>(lv, list, n, u, out, f, partial);
  HHG_CUDA(cudaGetLastError());
  count_launch();
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
  static const bool wave = getenv("HHG_F32_WAVE") != nullptr;
  if (op == HHG_OP_LSQP && lv.q > 0 && !wave) {
    switch (lv.q) {
      case 1: lsqp32<1>(lv, mode, u, out, f, partial, st); break;
      case 2: lsqp32<2>(lv, mode, u, out, f, partial, st); break;
      case 3: lsqp32<3>(lv, mode, u, out, f, partial, st); break;
      default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
    }
    return;
  }
  if (op == HHG_OP_LSQP && lv.q > 0) {
    switch (mode) {
      case APPLY: dispatch_wave<float, APPLY>(lv, u, out, f, partial, st); break;
      case RESIDUAL: dispatch_wave<float, RESIDUAL>(lv, u, out, f, partial, st); break;
      case SMOOTH: dispatch_wave<float, SMOOTH>(lv, u, out, f, partial, st); break;
    }
    return;
  }
  ifem_all<float>(lv, mode, u, out, f, partial, st);
}

void launch_line_table(const LevelView<double>& lv, int q, const double* coef, int* cell_e, long long* table,
                       cudaStream_t st) {
  const int64_t n = (int64_t)lv.nC * n_cell_lines(lv.N);
  const unsigned gs = (unsigned)((lv.nC + 127) / 128), gl = (unsigned)((n + 127) / 128);
  switch (q) {
    case 1:
      lsqp_scale_kernel<1><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_line_table_kernel<1><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
      break;
    case 2:
      lsqp_scale_kernel<2><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_line_table_kernel<2><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
      break;
    case 3:
      lsqp_scale_kernel<3><<<gs, 128, 0, st>>>(coef, lv.nC, lv.N, cell_e);
      lsqp_line_table_kernel<3><<<gl, 128, 0, st>>>(coef, cell_e, lv.nC, lv.N, table);
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
