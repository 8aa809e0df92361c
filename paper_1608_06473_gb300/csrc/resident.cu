// Cell-resident multicolour sweep of the surrogate smoother (Sec. 3.4,
// Eq. 5.1): the four colour steps (i + 2j + 3k) mod 4 = 0..3 of every macro
// cell's interior in one launch, with the cell's interior values held in the
// shared memory of one thread-block cluster for the whole sweep.
//
// The interior points of a cell are one contiguous block of the canonical
// vector, plane after plane (k), so the cluster splits it into CS slabs of
// whole planes with near-equal point counts, one per CTA.  Each CTA brings
// its slab in with one bulk (TMA) copy (plus at most a few plain loads at
// the unaligned ends), stages its planes' surrogate table, and then runs the
// four colour steps on shared memory: neighbours on planes k - 1 and k + 1
// that belong to the adjacent slab are read from that CTA's shared memory
// (distributed shared memory of the cluster), neighbours on the cell
// boundary from the cell's halo copy, f from global memory.  A cluster
// barrier separates the colour steps, so a colour-c update sees colours < c
// of this sweep and colours >= c of the last one on all three planes, which
// are the values the four per-colour launches give.  The slab goes back to
// HBM once at the end: every interior u is read and written once per sweep
// and f read once, the 12 (FP32) or 24 (FP64) bytes per update of the
// paper's memory model.
//
// Work inside a colour step is the run list of the colour (up to RUN64
// points of a line, stride 4).  Weights: FP64 by exact integer forward
// differences along the run (runs.cuh), FP32 by Horner from the per-plane
// table at every point; both in the same operations and order as the
// per-colour kernels (cell.cu), so the results are bitwise theirs.
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "arith.cuh"
#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"
#include "runs.cuh"

namespace cg = cooperative_groups;

namespace hhg {

namespace {

// Interior points of plane k (k = 1 .. N - 3) and the position of the first
// of them in the cell's block (lin_interior(1, 1, k)).
__host__ __device__ inline int64_t plane_start(int N, int k) {
  auto tet = [](int64_t n) { return (n + 1) * (n + 2) * (n + 3) / 6; };
  return tet(N - 4) - tet(N - 4 - (k - 1));
}

// Planes [k0, k1) of slab r of CS: k0 is the first plane whose start is at
// or beyond r n_int / CS (planes 1 .. N - 3 hold points; plane N - 2 starts
// at n_int).
__host__ __device__ inline void slab_planes(int N, int CS, int r, int& k0, int& k1) {
  const int64_t n_int = plane_start(N, N - 2);
  auto first = [&](int rr) {
    if (rr >= CS) return N - 2;
    const int64_t target = n_int * rr / CS;
    int k = 1;
    while (k < N - 2 && plane_start(N, k) < target) ++k;
    return k;
  };
  k0 = first(r);
  k1 = first(r + 1);
}

template <class T>
struct Tab;   // per-plane surrogate table staged in shared memory
template <>
struct Tab<double> {
  using E = long long;
  template <int Q>
  static constexpr int per_dir() { return NPP64<Q>; }
};
template <>
struct Tab<float> {
  using E = float;
  template <int Q>
  static constexpr int per_dir() { return np_pad<Q>(); }
};

// Elements of T per 16 bytes.
template <class T>
constexpr int VEC = 16 / (int)sizeof(T);

// Shared-memory bytes of slab r: values (with up to VEC - 1 of alignment
// shift and rounding), the slab planes' table, and the mbarrier.
template <class T, int Q>
__host__ __device__ inline size_t slab_smem(int N, int k0, int k1) {
  const int64_t n = plane_start(N, k1) - plane_start(N, k0);
  const size_t vals = (size_t)((n + 2 * VEC<T> + VEC<T> - 1) / VEC<T> * VEC<T>) * sizeof(T);
  const size_t tab = sizeof(typename Tab<T>::E) * (size_t)(k1 - k0) * 15 * Tab<T>::template per_dir<Q>();
  return vals + tab + 16;
}

template <class T>
constexpr int RES_THREADS = sizeof(T) == 8 ? 512 : 768;

// Where the values of one slab live: a (generic) pointer to its shared
// memory and the shift that maps a cell position p to p + delta there.
template <class T>
struct SlabRef {
  T* s;
  int64_t delta;
  __device__ T at(int64_t p) const { return s[p + delta]; }
};

// Value of interior point (i2, j2, k2), or of a boundary point from the
// cell's halo copy, for a point of plane k (neighbours lie on k - 1 .. k + 1;
// lo / hi hold planes k - 1 / k + 1, mid plane k).
template <class T>
__device__ __forceinline__ T nb_value(const LevelView<T>& lv, const T* ghost_c, SlabRef<T> lo, SlabRef<T> mid,
                                      SlabRef<T> hi, int k, int i2, int j2, int k2) {
  const int N = lv.N;
  if (!is_interior(i2, j2, k2, N)) return ghost_c[lin_full(i2, j2, k2, N)];
  const int64_t p = lin_interior32(i2, j2, k2, N);
  const T* s = k2 < k ? lo.s : (k2 > k ? hi.s : mid.s);
  const int64_t d = k2 < k ? lo.delta : (k2 > k ? hi.delta : mid.delta);
  return s[p + d];
}

// The slab holding plane k + dk (dk = -1, 0, 1), selected by value.
template <class T>
__device__ __forceinline__ SlabRef<T> pick(int dk, SlabRef<T> lo, SlabRef<T> mid, SlabRef<T> hi) {
  return SlabRef<T>{dk < 0 ? lo.s : (dk > 0 ? hi.s : mid.s), dk < 0 ? lo.delta : (dk > 0 ? hi.delta : mid.delta)};
}

// One run of the FP64 surrogate on shared-memory values (the arithmetic of
// lsqp64_run in SMOOTH mode).
template <int Q, bool DEEP>
__device__ __forceinline__ void run64_resident(const LevelView<double>& lv, const long long* P, int E, int i0, int j,
                                               int k, int cnt, SlabRef<double> lo, SlabRef<double> mid,
                                               SlabRef<double> hi, const double* ghost_c, const double* f_c) {
  const int N = lv.N;
  const int L = N - 1 - j - k, m1 = N - 2 - k, m0 = N - 1 - k;
  const int tc = m1 * (m1 + 1) / 2 - j + 1, bc = -(m0 * (m0 + 1) / 2) + j - 1;
  const int64_t p0 = lin_interior32(i0, j, k, N);
  double acc[RUN64];
  long long D[Q + 1];
#pragma unroll
  for (int s = 0; s < RUN64; ++s)
    if (s < cnt) acc[s] = f_c[p0 + 4 * s];
#pragma unroll 1
  for (int w = 0; w < 14; ++w) {
    run_start<Q>(P + w * NPP64<Q>, (unsigned)i0, (unsigned)j, 4u, D);
    const int off = neighbour_offset(w, L, tc, bc);
    const int di = DI(w), dj = DJ(w), dk = DK(w);
    const SlabRef<double> sr = pick(dk, lo, mid, hi);
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        const double nb = DEEP ? sr.at(p0 + 4 * s + off)
                               : nb_value(lv, ghost_c, lo, mid, hi, k, i0 + 4 * s + di, j + dj, k + dk);
        const double wt = i64_to_f64_scaled(D[0], E);
        acc[s] = fma(-wt, nb, acc[s]);
        run_step<Q>(D);
      }
  }
  run_start<Q>(P + MC * NPP64<Q>, (unsigned)i0, (unsigned)j, 4u, D);
#pragma unroll
  for (int s = 0; s < RUN64; ++s)
    if (s < cnt) {
      mid.s[p0 + 4 * s + mid.delta] = acc[s] * rcp_i64_scaled(D[0], E);
      run_step<Q>(D);
    }
}

// One run of the FP32 surrogate on shared-memory values: per point the
// weights by Horner from the plane table and the two interleaved partial
// sums of node_update (cell.cu), then the IEEE divide by the centre weight.
template <int Q, bool DEEP>
__device__ __forceinline__ void run32_resident(const LevelView<float>& lv, const float* P, int i0, int j, int k,
                                               int cnt, SlabRef<float> lo, SlabRef<float> mid,
                                               SlabRef<float> hi, const float* ghost_c, const float* f_c) {
  constexpr int NPP = np_pad<Q>();
  const int N = lv.N;
  const int L = N - 1 - j - k, m1 = N - 2 - k, m0 = N - 1 - k;
  const int tc = m1 * (m1 + 1) / 2 - j + 1, bc = -(m0 * (m0 + 1) / 2) + j - 1;
  const int64_t p0 = lin_interior32(i0, j, k, N);
  const float tj = (float)j;
  float a0[RUN64], a1[RUN64];
#pragma unroll
  for (int s = 0; s < RUN64; ++s)
    if (s < cnt) {
      a0[s] = f_c[p0 + 4 * s];
      a1[s] = 0.0f;
    }
#pragma unroll 1
  for (int w = 0; w < 14; ++w) {
    float Pw[NPP];
#pragma unroll
    for (int v = 0; v < NPP; v += 4) {
      const float4 q4 = *reinterpret_cast<const float4*>(P + w * NPP + v);
      Pw[v] = q4.x;
      Pw[v + 1] = q4.y;
      Pw[v + 2] = q4.z;
      Pw[v + 3] = q4.w;
    }
    const int off = neighbour_offset(w, L, tc, bc);
    const int di = DI(w), dj = DJ(w), dk = DK(w);
    const SlabRef<float> sr = pick(dk, lo, mid, hi);
#pragma unroll
    for (int s = 0; s < RUN64; ++s)
      if (s < cnt) {
        const float nb = DEEP ? sr.at(p0 + 4 * s + off)
                              : nb_value(lv, ghost_c, lo, mid, hi, k, i0 + 4 * s + di, j + dj, k + dk);
        const float wt = eval_plane<float, Q>(Pw, (float)(i0 + 4 * s), tj);
        if (w & 1)
          a1[s] = fmaf(-wt, nb, a1[s]);
        else
          a0[s] = fmaf(-wt, nb, a0[s]);
      }
  }
  float Pc[NPP];
#pragma unroll
  for (int v = 0; v < NPP; v += 4) {
    const float4 q4 = *reinterpret_cast<const float4*>(P + MC * NPP + v);
    Pc[v] = q4.x;
    Pc[v + 1] = q4.y;
    Pc[v + 2] = q4.z;
    Pc[v + 3] = q4.w;
  }
#pragma unroll
  for (int s = 0; s < RUN64; ++s)
    if (s < cnt) mid.s[p0 + 4 * s + mid.delta] = (a0[s] + a1[s]) / eval_plane<float, Q>(Pc, (float)(i0 + 4 * s), tj);
}

// The sweep: grid = nC clusters of CS CTAs (cluster rank r holds slab r of
// cell blockIdx.x / CS).  kidx[(g (N + 1) + k) 2 + part]: first item of
// colour g's run list (relative to the colour's segment) in part 0 (deep
// runs) or 1 (runs next to the cell boundary) whose plane is >= k.
template <class T, int Q>
__global__ void __launch_bounds__(RES_THREADS<T>, 1) lsqp_resident_sweep(LevelView<T> lv, T* u, const T* f,
                                                                        const int* __restrict__ kidx) {
  using TE = typename Tab<T>::E;
  constexpr int PD = Tab<T>::template per_dir<Q>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
  const int c = blockIdx.x / CS;
  const int N = lv.N;
  int k0, k1;
  slab_planes(N, CS, r, k0, k1);
  const int64_t P0 = plane_start(N, k0), P1 = plane_start(N, k1);
  const int64_t cbase = lv.off_C + (int64_t)c * lv.n_int;
  // shift: elements between the 16-byte boundary at or below the slab's
  // first value and that value, in global memory; kept in shared memory
  auto shift_of = [&](int64_t p) { return (int)(((uintptr_t)(u + cbase + p) & 15u) / sizeof(T)); };
  const int sh = shift_of(P0);
  T* us = reinterpret_cast<T*>(smem_raw);
  const int64_t n_slab = P1 - P0;
  const int64_t n_vals = (n_slab + 2 * VEC<T> + VEC<T> - 1) / VEC<T> * VEC<T>;
  TE* tab = reinterpret_cast<TE*>(us + n_vals);
  uint64_t* bar = reinterpret_cast<uint64_t*>(tab + (size_t)(k1 - k0) * 15 * PD);

  // aligned middle [pa, pb) by one bulk copy, the ends by plain loads
  const int64_t pa = std::min<int64_t>(P1, P0 + (VEC<T> - sh) % VEC<T>);
  const int64_t pb = std::max<int64_t>(pa, P1 - shift_of(P1));
  const bool bulk = pb > pa;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && bulk) {
    const uint32_t bytes = (uint32_t)((pb - pa) * (int64_t)sizeof(T));
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(us + (pa - P0 + sh), u + cbase + pa, bytes, bar);
  }
  for (int64_t p = P0 + threadIdx.x; p < pa; p += blockDim.x) us[p - P0 + sh] = u[cbase + p];
  for (int64_t p = pb + threadIdx.x; p < P1; p += blockDim.x) us[p - P0 + sh] = u[cbase + p];
  // the slab planes' surrogate table
  if (sizeof(T) == 8) {
    const int64_t n2 = (int64_t)(k1 - k0) * 15 * PD / 2;
    const longlong2* src = reinterpret_cast<const longlong2*>(lv.plane64) +
                           ((int64_t)c * (N - 3) + (k0 - 1)) * 15 * PD / 2;
    longlong2* dst = reinterpret_cast<longlong2*>(tab);
    for (int64_t t = threadIdx.x; t < n2; t += blockDim.x) dst[t] = __ldg(src + t);
  } else {
    constexpr int NP = (Q + 1) * (Q + 2) / 2;
    const float* src = reinterpret_cast<const float*>(lv.plane32) + ((int64_t)c * (N - 3) + (k0 - 1)) * 15 * NP;
    float* dst = reinterpret_cast<float*>(tab);
    const int64_t n = (int64_t)(k1 - k0) * 15 * PD;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      const int e = (int)(t % PD);
      dst[t] = e < NP ? src[(t / PD) * NP + e] : 0.0f;
    }
  }
  bool failed = bulk && !mbar_wait(bar, 0);
  failed = __syncthreads_or(failed);
  if (failed && threadIdx.x == 0) atomicExch(lv.err, 1);

  // this CTA's slab and its neighbours' (distributed shared memory)
  SlabRef<T> mid{us, sh - P0}, lo = mid, hi = mid;
  if (r > 0) {
    int a0, a1;
    slab_planes(N, CS, r - 1, a0, a1);
    const int64_t q0 = plane_start(N, a0);
    lo = SlabRef<T>{cluster.map_shared_rank(us, r - 1), shift_of(q0) - q0};
  }
  if (r + 1 < CS) {
    const int64_t q0 = P1;
    hi = SlabRef<T>{cluster.map_shared_rank(us, r + 1), shift_of(q0) - q0};
  }
  const T* ghost_c = lv.ghost + (int64_t)c * lv.n_full;
  const T* f_c = f + cbase;
  const int E = sizeof(T) == 8 ? lv.cell_e[c] : 0;
  cluster.sync();   // every slab is in shared memory

  for (int g = 0; g < 4; ++g) {
    if (!failed) {
      const int* kx = kidx + (size_t)g * (N + 1) * 2;
      const int d0 = kx[2 * k0], d1 = kx[2 * k1], n0 = kx[2 * k0 + 1], n1 = kx[2 * k1 + 1];
      const int nd = d1 - d0, nt = nd + (n1 - n0);
      const uint2* items = lv.run_nodes + lv.run_off[g];
      for (int e = threadIdx.x; e < nt; e += blockDim.x) {
        const uint2 it = items[e < nd ? d0 + e : n0 + (e - nd)];
        const int i0 = unpack_i(it.x), j = unpack_j(it.x), k = unpack_k(it.x);
        const int cnt = (int)(it.y & 0xffu);
        const TE* P = tab + (size_t)(k - k0) * 15 * PD;
        // planes k - 1 and k + 1 are in this slab except at its ends
        const SlabRef<T> lk = k == k0 ? lo : mid, hk = k + 1 == k1 ? hi : mid;
        if constexpr (sizeof(T) == 8) {
          if (it.y & 0x100u)
            run64_resident<Q, true>(lv, P, E, i0, j, k, cnt, lk, mid, hk, ghost_c, f_c);
          else
            run64_resident<Q, false>(lv, P, E, i0, j, k, cnt, lk, mid, hk, ghost_c, f_c);
        } else {
          if (it.y & 0x100u)
            run32_resident<Q, true>(lv, P, i0, j, k, cnt, lk, mid, hk, ghost_c, f_c);
          else
            run32_resident<Q, false>(lv, P, i0, j, k, cnt, lk, mid, hk, ghost_c, f_c);
        }
      }
    }
    cluster.sync();   // colour g done on every slab; no slab is read after the last one
  }
  if (failed) {
    // a copy that did not complete in time may still land: wait for it
    // (bounded) before the CTA's shared memory is released
    if (threadIdx.x == 0) mbar_wait(bar, 0);
    return;
  }
  for (int64_t p = P0 + threadIdx.x; p < P1; p += blockDim.x) u[cbase + p] = us[p - P0 + sh];
}

// Opt-in shared memory per CTA of the current device (queried once; the
// static's initialisation is thread-safe for the server's worker threads).
int max_smem_optin() {
  static const int v = [] {
    int dev = 0, bytes = 0;
    HHG_CUDA(cudaGetDevice(&dev));
    HHG_CUDA(cudaDeviceGetAttribute(&bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    return bytes;
  }();
  return v;
}

// Smallest cluster size (1, 2, 4 or 8) whose largest slab fits the shared
// memory of one CTA, and that slab's bytes; 0 when none does.
template <class T, int Q>
int resident_cluster(int N, size_t* smem) {
  if (N < 8) return 0;
  const size_t cap = (size_t)max_smem_optin() - 1024;   // headroom for static shared memory
  for (int CS = 1; CS <= 8; CS *= 2) {
    size_t mx = 0;
    bool ok = true;
    for (int r = 0; r < CS; ++r) {
      int k0, k1;
      slab_planes(N, CS, r, k0, k1);
      if (k1 <= k0) ok = false;
      mx = std::max(mx, slab_smem<T, Q>(N, k0, k1));
    }
    if (ok && mx <= cap) {
      if (smem) *smem = mx;
      return CS;
    }
  }
  return 0;
}

template <class T, int Q>
void launch_resident_q(const LevelView<T>& lv, T* u, const T* f, const int* kidx, cudaStream_t st) {
  size_t smem = 0;
  const int CS = resident_cluster<T, Q>(lv.N, &smem);
  HHG_CHECK(CS > 0, HHG_EINVAL, "cell-resident sweep does not fit this level");
  auto kern = lsqp_resident_sweep<T, Q>;
  ensure_smem_limit((const void*)kern, smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(lv.nC * CS), 1, 1);
  cfg.blockDim = dim3(RES_THREADS<T>, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HHG_CUDA(cudaLaunchKernelEx(&cfg, kern, lv, u, f, kidx));
  count_launch();
}

}  // namespace

template <class T>
bool resident_supported(const LevelView<T>& lv) {
  if (lv.q < 1 || lv.q > 3 || lv.nrhs != 1 || lv.run_kidx == nullptr) return false;
  if (sizeof(T) == 8 ? lv.plane64 == nullptr : lv.plane32 == nullptr) return false;
  switch (lv.q) {
    case 1: return resident_cluster<T, 1>(lv.N, nullptr) > 0;
    case 2: return resident_cluster<T, 2>(lv.N, nullptr) > 0;
    default: return resident_cluster<T, 3>(lv.N, nullptr) > 0;
  }
}
template bool resident_supported<double>(const LevelView<double>&);
template bool resident_supported<float>(const LevelView<float>&);

void resident_slab_planes(int N, int CS, int* k_bounds) {
  for (int r = 0; r < CS; ++r) {
    int k0, k1;
    slab_planes(N, CS, r, k0, k1);
    k_bounds[r] = k0;
    k_bounds[r + 1] = k1;
  }
}

template <class T>
int resident_cluster_size(const LevelView<T>& lv) {
  if (!resident_supported(lv)) return 0;
  switch (lv.q) {
    case 1: return resident_cluster<T, 1>(lv.N, nullptr);
    case 2: return resident_cluster<T, 2>(lv.N, nullptr);
    default: return resident_cluster<T, 3>(lv.N, nullptr);
  }
}
template int resident_cluster_size<double>(const LevelView<double>&);
template int resident_cluster_size<float>(const LevelView<float>&);

template <class T>
void launch_resident_sweep(const LevelView<T>& lv, T* u, const T* f, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_resident_q<T, 1>(lv, u, f, lv.run_kidx, st); break;
    case 2: launch_resident_q<T, 2>(lv, u, f, lv.run_kidx, st); break;
    case 3: launch_resident_q<T, 3>(lv, u, f, lv.run_kidx, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}
template void launch_resident_sweep<double>(const LevelView<double>&, double*, const double*, cudaStream_t);
template void launch_resident_sweep<float>(const LevelView<float>&, float*, const float*, cudaStream_t);

}  // namespace hhg
