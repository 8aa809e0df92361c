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
//    on the integer pipe; the FP64 pipe carries only the 14 stencil products,
//    the scaling and a Newton-Raphson divide.  Kernels are thread-per-node
//    with one CTA per macro cell and no barriers; the smoother is one launch
//    per colour.
//  * FP32: per plane k each direction's polynomial is reduced to a
//    polynomial in (i, j) at fit time (FP32 table) and evaluated per node
//    from shared memory, thread per node, one launch per colour.  The
//    smoother may instead run as the shared-memory staged one-launch sweep
//    of stage.cu; a tuner times both per level and picks (lv.smooth_cfg).
//
// IFEM (Sec. 4.2.1): every node assembles its 15 weights from the 24 element
// matrices around it (thread per node, one launch per colour).
//
// Neighbour addressing: nodes whose 14 neighbours are all interior use
// closed-form 32-bit offsets within the cell's block of the canonical
// vector; nodes next to the cell boundary read boundary neighbours from the
// cell's halo copy.
#include <algorithm>

#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

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

// Right-hand sides per batched launch: the weights of a node are evaluated
// once and applied to RB vectors.
constexpr int RB = 4;

// The update of node (i, j, k) of cell c for right-hand sides b0 .. b0+G-1
// (G <= RB) with its 15 weights w[] already evaluated.  CHAIN: one FMA chain
// in direction order and the Newton-Raphson divide (the FP64 surrogate
// kernel's arithmetic); otherwise node_update's two-accumulator form.
template <class T, Mode MODE, bool CHAIN, class W>
__device__ __forceinline__ void node_update_batch(const LevelView<T>& lv, int c, int i, int j, int k, const W* w,
                                                  T* u, T* out, const T* f, double (&nrm)[RB], int b0, int G,
                                                  T scale, T inv_scale);

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

// v * i + c (mod 2^64) for a 32-bit multiplier i >= 0: the low word times i
// widened to 64 bits plus c, then the high word times i added to the top
// half (two integer multiply-adds instead of a full 64 x 64 product).
__device__ __forceinline__ long long mad_i64_u32(long long v, unsigned i, long long c) {
  const unsigned long long vu = (unsigned long long)v;
  unsigned long long r = (unsigned long long)(unsigned)vu * i + (unsigned long long)c;
  r += (unsigned long long)((unsigned)(vu >> 32) * i) << 32;
  return (long long)r;
}

// Line polynomial C_Q i^Q + ... + C_0 in exact integer arithmetic (Horner).
template <int Q>
__device__ __forceinline__ long long horner_i64(const long long* C, unsigned i) {
  long long v = C[Q];
#pragma unroll
  for (int a = Q - 1; a >= 0; --a) v = mad_i64_u32(v, i, C[a]);
  return v;
}

// int64 -> FP64 on the integer pipe (GB300 issues FP64 conversions on its
// narrow FP64 pipe): magnitude, leading-zero count, normalising shift, and
// the biased exponent added to the top bits, where the leading one of the
// shifted magnitude carries into the exponent field.  The mantissa is
// truncated toward zero (relative error below 2^-52); 0 maps to +0.
__device__ __forceinline__ double i64_to_f64(long long v) {
  const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  unsigned long long m;
  asm("shl.b64 %0, %1, %2;" : "=l"(m) : "l"(a), "r"(lz));  // PTX clamps a shift of 64 to 0
  const unsigned long long bits = ((unsigned long long)(1085 - lz) << 52) + (m >> 11);
  return a ? __longlong_as_double((long long)(bits | sign)) : 0.0;
}

// n / d for normal d: the hardware reciprocal estimate refined by two
// Newton-Raphson steps x <- x + x (1 - d x) (each squares the relative error),
// the last one folded into the product: n x (1 + e) with e = 1 - d x.  The
// result is within a few ulp of the correctly rounded quotient, at 5 FP64
// operations instead of the longer IEEE division sequence.
__device__ __forceinline__ double div_nr(double n, double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  const double t = n * x;
  return fma(t, e, t);
}

// One interior node of the FP64 surrogate.  C is the line record of (j, k):
// 15 polynomials in i of degree Q, Q + 1 int64 each, scaled by 2^E.  Weights
// are formed in pairs (w, w + 1) from 16-byte loads (the pair starts at an
// even int64 offset) and converted on the integer pipe; the FP64 pipe
// carries only the 14 products, the scaling and the divide.
template <int Q, Mode MODE, class NB>
__device__ __forceinline__ void lsqp64_node(const long long* __restrict__ C, unsigned i, NB nb, int64_t I, double* u,
                                            double* out, const double* f, double& nrm, double scale,
                                            double inv_scale) {
  auto pair = [&](int w, double& a, double& b) {
    long long r[2 * (Q + 1)];
    const longlong2* p2 = reinterpret_cast<const longlong2*>(C + w * (Q + 1));
#pragma unroll
    for (int h = 0; h < Q + 1; ++h) {
      const longlong2 x = __ldg(p2 + h);
      r[2 * h] = x.x;
      r[2 * h + 1] = x.y;
    }
    a = i64_to_f64(horner_i64<Q>(r, i));
    b = i64_to_f64(horner_i64<Q>(r + Q + 1, i));
  };
  auto centre = [&]() {
    long long r[Q + 2];
    const longlong2* p2 = reinterpret_cast<const longlong2*>(C + MC * (Q + 1));
#pragma unroll
    for (int h = 0; h < (Q + 2) / 2; ++h) {
      const longlong2 x = __ldg(p2 + h);
      r[2 * h] = x.x;
      r[2 * h + 1] = x.y;
    }
    return i64_to_f64(horner_i64<Q>(r, i));
  };
  if (MODE == SMOOTH) {
    double acc = f[I] * scale;
#pragma unroll
    for (int w = 0; w < 14; w += 2) {
      double a, b;
      pair(w, a, b);
      acc = fma(-a, nb(w), acc);
      acc = fma(-b, nb(w + 1), acc);
    }
    u[I] = div_nr(acc, centre());
  } else {
    double y = centre() * u[I];
#pragma unroll
    for (int w = 0; w < 14; w += 2) {
      double a, b;
      pair(w, a, b);
      y = fma(a, nb(w), y);
      y = fma(b, nb(w + 1), y);
    }
    if (MODE == APPLY) {
      out[I] = y * inv_scale;
    } else {
      const double r = fma(-inv_scale, y, f[I]);
      out[I] = r;
      nrm = fma(r, r, nrm);
    }
  }
}

template <class T, Mode MODE, bool CHAIN, class W>
__device__ __forceinline__ void node_update_batch(const LevelView<T>& lv, int c, int i, int j, int k, const W* w,
                                                  T* u, T* out, const T* f, double (&nrm)[RB], int b0, int G,
                                                  T scale, T inv_scale) {
  const int64_t I = lv.off_C + (int64_t)c * lv.n_int + lin_interior32(i, j, k, lv.N);
  const bool deep = deep_interior(i, j, k, lv.N);
  int off[14];
  if (deep) neighbour_offsets(j, k, lv.N, off);
#pragma unroll
  for (int g = 0; g < RB; ++g) {
    if (g >= G) break;
    const int64_t b = b0 + g;
    T* ub = u + b * lv.vstride;
    const T* gb = lv.ghost + b * lv.gstride;
    auto nb = [&](int v) -> T {
      if (deep) return ub[I + off[v]];
      const int i2 = i + DI(v), j2 = j + DJ(v), k2 = k + DK(v);
      if (is_interior(i2, j2, k2, lv.N)) return ub[lv.off_C + (int64_t)c * lv.n_int + lin_interior32(i2, j2, k2, lv.N)];
      return gb[(int64_t)c * lv.n_full + lin_full(i2, j2, k2, lv.N)];
    };
    if (MODE == SMOOTH) {
      const T fb = f[b * lv.vstride + I];
      if (CHAIN) {
        T acc = fb * scale;
#pragma unroll
        for (int v = 0; v < 14; ++v) acc = fma(-(T)w[v], nb(v), acc);
        ub[I] = (T)div_nr((double)acc, (double)w[MC]);
      } else {
        T a0 = fb * scale, a1 = 0;
#pragma unroll
        for (int v = 0; v < 14; v += 2) {
          a0 = fma(-(T)w[v], nb(v), a0);
          a1 = fma(-(T)w[v + 1], nb(v + 1), a1);
        }
        ub[I] = (a0 + a1) / (T)w[MC];
      }
    } else {
      T y;
      if (CHAIN) {
        y = (T)w[MC] * ub[I];
#pragma unroll
        for (int v = 0; v < 14; ++v) y = fma((T)w[v], nb(v), y);
      } else {
        T a0 = (T)w[MC] * ub[I], a1 = 0;
#pragma unroll
        for (int v = 0; v < 14; v += 2) {
          a0 = fma((T)w[v], nb(v), a0);
          a1 = fma((T)w[v + 1], nb(v + 1), a1);
        }
        y = a0 + a1;
      }
      if (MODE == APPLY) {
        out[b * lv.vstride + I] = y * inv_scale;
      } else {
        const T r = fma(-inv_scale, y, f[b * lv.vstride + I]);
        out[b * lv.vstride + I] = r;
        nrm[g] = CHAIN ? fma((double)r, (double)r, nrm[g]) : nrm[g] + (double)r * (double)r;
      }
    }
  }
}

// Per-right-hand-side block sums of a batched residual into partial.
__device__ __forceinline__ void batch_partials(const double (&nrm)[RB], int b0, int G, int pstride, int c,
                                               double* partial) {
#pragma unroll
  for (int g = 0; g < RB; ++g) {
    if (g >= G) break;
    const double tot = block_sum(nrm[g]);
    if (threadIdx.x == 0) partial[(int64_t)(b0 + g) * pstride + c] = tot;
  }
}

// FP64 surrogate for RB right-hand sides at once: the 15 weights of a node
// are formed once (integer pipe) and applied to every vector of the group.
template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 2) lsqp_node_batch_kernel(LevelView<double> lv,
                                                                          const uint32_t* __restrict__ list, int n_list,
                                                                          double* u, double* out, const double* f,
                                                                          double* partial, int b0, int G) {
  const int c = blockIdx.x;
  const int N = lv.N;
  const int E = lv.cell_e[c];
  const double scale = ldexp(1.0, E), inv_scale = ldexp(1.0, -E);
  const long long* tab = lv.line64 + (int64_t)c * lv.n_lines * line_rec(Q);
  double nrm[RB] = {};
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const long long* C = tab + (int64_t)line_id(j, k, N) * line_rec(Q);
    double w[15];
#pragma unroll
    for (int v = 0; v < 15; ++v) w[v] = i64_to_f64(horner_i64<Q>(C + v * (Q + 1), (unsigned)i));
    node_update_batch<double, MODE, true>(lv, c, i, j, k, w, u, out, f, nrm, b0, G, scale, inv_scale);
  }
  if (MODE == RESIDUAL) batch_partials(nrm, b0, G, lv.pstride, c, partial);
}

template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE64_THREADS, 2) lsqp_node_kernel(LevelView<double> lv, const uint32_t* __restrict__ list,
                                                                  int n_list, double* u, double* out, const double* f,
                                                                  double* partial) {
  const int c = blockIdx.x;
  const int N = lv.N;
  const int E = lv.cell_e[c];
  const double scale = ldexp(1.0, E), inv_scale = ldexp(1.0, -E);
  const long long* tab = lv.line64 + (int64_t)c * lv.n_lines * line_rec(Q);
  const int64_t base = lv.off_C + (int64_t)c * lv.n_int;
  double nrm = 0.0;
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const long long* C = tab + (int64_t)line_id(j, k, N) * line_rec(Q);
    const int64_t I = base + lin_interior32(i, j, k, N);
    if (deep_interior(i, j, k, N)) {
      int off[14];
      neighbour_offsets(j, k, N, off);
      const double* pu = u + I;
      lsqp64_node<Q, MODE>(C, (unsigned)i, [&](int w) { return pu[off[w]]; }, I, u, out, f, nrm, scale, inv_scale);
    } else {
      lsqp64_node<Q, MODE>(C, (unsigned)i,
                           [&](int w) { return load_pt(lv, (const double*)u, c, i + DI(w), j + DJ(w), k + DK(w)); },
                           I, u, out, f, nrm, scale, inv_scale);
    }
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

// FP32 surrogate for RB right-hand sides at once (weights evaluated once per
// node from the per-plane table in shared memory).
template <int Q, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS, 2) lsqp_node32_batch_kernel(LevelView<float> lv,
                                                                            const uint32_t* __restrict__ list,
                                                                            int n_list, float* u, float* out,
                                                                            const float* f, double* partial, int b0,
                                                                            int G) {
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
  double nrm[RB] = {};
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    const float* P = s_tab + (k - 1) * 15 * NPP;
    float w[15];
#pragma unroll
    for (int v = 0; v < 15; ++v) w[v] = eval_plane<float, Q>(P + v * NPP, (float)i, (float)j);
    node_update_batch<float, MODE, false>(lv, c, i, j, k, w, u, out, f, nrm, b0, G, 1.0f, 1.0f);
  }
  if (MODE == RESIDUAL) batch_partials(nrm, b0, G, lv.pstride, c, partial);
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

// IFEM for RB right-hand sides at once (one stencil assembly per node).
template <class T, Mode MODE>
__global__ void __launch_bounds__(NODE_THREADS) ifem_node_batch_kernel(LevelView<T> lv, const uint32_t* __restrict__ list,
                                                                        int n_list, T* u, T* out, const T* f,
                                                                        double* partial, int b0, int G) {
  __shared__ CellGeom g;
  const int c = blockIdx.x;
  if (threadIdx.x < 16)
    reinterpret_cast<double*>(&g)[threadIdx.x] = reinterpret_cast<const double*>(&lv.geom[c])[threadIdx.x];
  __syncthreads();
  double nrm[RB] = {};
  for (int t = threadIdx.x; t < n_list; t += blockDim.x) {
    const uint32_t p = list[t];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    double s[15];
    ifem_stencil(g, lv.N, i, j, k, s);
    node_update_batch<T, MODE, false>(lv, c, i, j, k, s, u, out, f, nrm, b0, G, T(1), T(1));
  }
  if (MODE == RESIDUAL) batch_partials(nrm, b0, G, lv.pstride, c, partial);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <int Q, Mode MODE>
void launch_node64(const LevelView<double>& lv, const uint32_t* list, int n, double* u, double* out, const double* f,
                   double* partial, cudaStream_t st) {
  HHG_CHECK(lv.line64 != nullptr, HHG_ENOTFIT, "FP64 surrogate line table missing");
  if (lv.nrhs == 1) {
    lsqp_node_kernel<Q, MODE><<<lv.nC, NODE64_THREADS, 0, st>>>(lv, list, n, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  for (int b0 = 0; b0 < lv.nrhs; b0 += RB) {
    lsqp_node_batch_kernel<Q, MODE><<<lv.nC, NODE_THREADS, 0, st>>>(lv, list, n, u, out, f, partial, b0,
                                                                    std::min(RB, lv.nrhs - b0));
    HHG_CUDA(cudaGetLastError());
    count_launch();
  }
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
  if (lv.nrhs == 1) {
    auto kern = lv.smooth_cfg == -2 ? lsqp_node32_x2_kernel<Q, MODE> : lsqp_node32_kernel<Q, MODE>;
    ensure_smem_limit((const void*)kern, smem);
    kern<<<lv.nC, lv.smooth_cfg == -2 ? NODE_THREADS : NODE32_THREADS, smem, st>>>(lv, list, n, u, out, f, partial);
    HHG_CUDA(cudaGetLastError());
    count_launch();
    return;
  }
  auto kern = lsqp_node32_batch_kernel<Q, MODE>;
  ensure_smem_limit((const void*)kern, smem);
  for (int b0 = 0; b0 < lv.nrhs; b0 += RB) {
    kern<<<lv.nC, NODE_THREADS, smem, st>>>(lv, list, n, u, out, f, partial, b0, std::min(RB, lv.nrhs - b0));
    HHG_CUDA(cudaGetLastError());
    count_launch();
  }
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
  for (int b0 = 0; b0 < lv.nrhs; b0 += RB) {
    ifem_node_batch_kernel<T, MODE><<<lv.nC, NODE_THREADS, 0, st>>>(lv, list, n, u, out, f, partial, b0,
                                                                    std::min(RB, lv.nrhs - b0));
    HHG_CUDA(cudaGetLastError());
    count_launch();
  }
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
  if (op == HHG_OP_LSQP && lv.q > 0) {
    if (mode == SMOOTH && lv.smooth_cfg >= 0 && stage32_supported(lv, u, lv.smooth_cfg) &&
        (lv.nrhs == 1 || (lv.vstride % 4) == 0)) {
      // one launch per right-hand side (the plane ring holds one vector)
      for (int b = 0; b < lv.nrhs; ++b) {
        LevelView<float> one = lv;
        one.nrhs = 1;
        one.ghost = lv.ghost + b * lv.gstride;
        launch_stage32_smooth(one, u + b * lv.vstride, f + b * lv.vstride, lv.smooth_cfg, st);
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
