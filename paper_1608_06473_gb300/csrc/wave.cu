// FP32 surrogate smoother as one plane wavefront per macro cell.
//
// One CTA sweeps one macro cell: the four colour steps of the multicolour
// Gauss-Seidel sweep (colours (i + 2j + 3k) mod 4, Eq. 5.1) run as a
// wavefront over the cell's planes k, colour c on plane k = s + 1 - 2c in
// step s.  A colour-c update on plane k reads planes k - 1 .. k + 1; colour
// c - 1 finished plane k + 1 in step s - 1 and colour c + 1 reaches plane
// k - 1 only in step s + 1, so every update sees the values four separate
// colour sweeps would give it, and the four colour tasks of a step are
// independent: one barrier per step.
//
// u is updated in place in global memory.  A plane is touched by the four
// colours within seven consecutive steps, so after its first read it is
// served from L1 / L2; each step prefetches the u and f planes two steps
// ahead into L2 (prefetch.global.L2 per 128-byte line), so u crosses HBM
// about once per sweep each way and f once: the 12 bytes per update of the
// FP32 smoother.  The cell's per-plane weight polynomials (FP32, paired by
// direction) are staged in shared memory once per launch and evaluated per
// node with packed FP32 FMAs (Sec. 3.4).  No thread waits on anything but
// the CTA barrier.  A step's node-list entries and their f values do not
// depend on u, so each thread loads its first entries of step s + 1 before
// the barrier that ends step s.
#include <algorithm>

#include <cuda_runtime.h>

#include "arith.cuh"
#include "device.cuh"
#include "kernels.h"

namespace hhg {

namespace {

__device__ __forceinline__ int wave_plane_size(int N, int k) { return (N - 2 - k) * (N - 1 - k) / 2; }

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int THREADS>
constexpr int wave_min_blocks() { return 1024 / THREADS; }

template <int Q>
size_t wave_smem(int N) {
  return sizeof(float2) * (size_t)(N - 3) * NPAIR * npp2<Q>();
}

// The colour tasks of step s: colour cc on plane s + 1 - 2 cc, as one pool
// of list entries [0, e4): entries [e_cc, e_cc+1) are task cc, starting at
// list position b_cc.
struct Tasks {
  int b0, b1, b2, b3, e1, e2, e3, e4;
};

__device__ __forceinline__ Tasks step_tasks(const LevelView<float>& lv, int s, int np) {
  Tasks t;
  int e = 0;
  auto one = [&](int cc, int& b) {
    const int k = s + 1 - 2 * cc;
    if (k < 1 || k > np) {
      b = 0;
      return;
    }
    b = lv.plane_off[k * 4 + cc];
    e += lv.plane_off[k * 4 + cc + 1] - b;
  };
  one(0, t.b0);
  t.e1 = e;
  one(1, t.b1);
  t.e2 = e;
  one(2, t.b2);
  t.e3 = e;
  one(3, t.b3);
  t.e4 = e;
  return t;
}

// A list entry of a step (the point packed, its position in the cell's
// block of the vector, -1 for none) with its right-hand side, loaded ahead:
// neither depends on the values the step reads from u.
struct Entry {
  uint32_t p;
  int lin;
  float fv;
};

__device__ __forceinline__ Entry load_entry(const LevelView<float>& lv, const Tasks& t, int s, int idx,
                                            const float* fc) {
  Entry e;
  const int cc = (idx >= t.e1) + (idx >= t.e2) + (idx >= t.e3);
  const int pos = cc == 0 ? t.b0 + idx : (cc == 1 ? t.b1 + idx - t.e1 : (cc == 2 ? t.b2 + idx - t.e2 : t.b3 + idx - t.e3));
  if (idx < t.e4) {
    const uint32_t q = lv.plane_nodes[pos];
    const int k = s + 1 - 2 * cc;
    e.p = pack_ijk(unpack_i(q), unpack_j(q), k);
    e.lin = lin_interior32(unpack_i(q), unpack_j(q), k, lv.N);
    e.fv = fc[e.lin];
  } else {
    e.p = 0u;
    e.lin = -1;
    e.fv = 0.0f;
  }
  return e;
}

template <int Q, int THREADS>
__global__ void __launch_bounds__(THREADS, wave_min_blocks<THREADS>()) lsqp_wave32_smooth(LevelView<float> lv,
                                                                                       float* u, const float* f) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NP2 = npp2<Q>();
  constexpr int B = 2;  // entries per thread in flight
  extern __shared__ __align__(16) float2 s_tab2[];   // [N - 3][NPAIR][NP2]
  const int N = lv.N, np = N - 3;
  const int c = blockIdx.x;
  const int64_t cbase = lv.off_C + (int64_t)c * lv.n_int;
  {
    const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
    float* d = reinterpret_cast<float*>(s_tab2);
    for (int t = threadIdx.x; t < np * NPAIR * NP2 * 2; t += THREADS) {
      const int h = t & 1, e = (t >> 1) % NP2, m = ((t >> 1) / NP2) % NPAIR, k = (t >> 1) / (NP2 * NPAIR);
      const int w = 2 * m + h;
      d[t] = (e < NP && w < 15) ? tab[((int64_t)k * 15 + w) * NP + e] : 0.0f;
    }
  }
  // u plane k is first read in step k - 2, f plane k in step k - 1
  auto prefetch = [&](const float* v, int k) {
    if (k < 1 || k > np) return;
    const float* p = v + cbase + lin_interior32(1, 1, k, N);
    const int n = wave_plane_size(N, k);
    for (int x = threadIdx.x * 32; x < n; x += THREADS * 32) prefetch_l2(p + x);
  };
  for (int k = 1; k <= 3; ++k) prefetch(u, k);
  for (int k = 1; k <= 2; ++k) prefetch(f, k);

  float* uc = u + cbase;          // the cell's block of u and f
  const float* fc = f + cbase;
  // Eq. 5.1 at entry e with its neighbours nb (FP32, paired directions)
  auto update = [&](const Entry& e, const float (&nb)[14]) {
    const int i = unpack_i(e.p), j = unpack_j(e.p), k = unpack_k(e.p);
    const float2* P = s_tab2 + (k - 1) * NPAIR * NP2;
    const float2 Iv = make_float2((float)i, (float)i), Jv = make_float2((float)j, (float)j);
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int m = 0; m < 7; ++m)
      acc = __ffma2_rn(eval_plane2<Q>(P + m * NP2, Iv, Jv), make_float2(nb[2 * m], nb[2 * m + 1]), acc);
    const float wc = eval_plane2<Q>(P + 7 * NP2, Iv, Jv).x;
    uc[e.lin] = div_nr32(e.fv - acc.x - acc.y, wc);
  };
  auto gather = [&](const Entry& e, float (&nb)[14]) {
    const int i = unpack_i(e.p), j = unpack_j(e.p), k = unpack_k(e.p);
    if (deep_interior(i, j, k, N)) {
      int off[14];
      neighbour_offsets(j, k, N, off);
#pragma unroll
      for (int w = 0; w < 14; ++w) nb[w] = uc[e.lin + off[w]];
    } else {
#pragma unroll
      for (int w = 0; w < 14; ++w) nb[w] = load_pt(lv, (const float*)u, c, i + DI(w), j + DJ(w), k + DK(w));
    }
  };

  Tasks T = step_tasks(lv, 0, np);
  Entry ahead[B];
#pragma unroll
  for (int b = 0; b < B; ++b) ahead[b] = load_entry(lv, T, 0, threadIdx.x + b * THREADS, fc);
  __syncthreads();

  for (int s = 0; s <= np + 5; ++s) {
    prefetch(u, s + 4);
    prefetch(f, s + 3);
    for (int base = threadIdx.x; base < T.e4; base += B * THREADS) {
      Entry e[B];
      float nb[B][14];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        e[b] = base == (int)threadIdx.x ? ahead[b] : load_entry(lv, T, s, base + b * THREADS, fc);
        if (e[b].lin >= 0) gather(e[b], nb[b]);
      }
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (e[b].lin >= 0) update(e[b], nb[b]);
    }
    // the next step's first entries and their f, before the barrier
    T = step_tasks(lv, s + 1, np);
#pragma unroll
    for (int b = 0; b < B; ++b) ahead[b] = load_entry(lv, T, s + 1, threadIdx.x + b * THREADS, fc);
    __syncthreads();
  }
}

template <int Q, int THREADS>
void launch_wave(const LevelView<float>& lv, float* u, const float* f, cudaStream_t st) {
  const size_t smem = wave_smem<Q>(lv.N);
  auto kern = lsqp_wave32_smooth<Q, THREADS>;
  ensure_smem_limit((const void*)kern, smem);
  kern<<<lv.nC, THREADS, smem, st>>>(lv, u, f);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <int Q>
void launch_wave_cfg(int cfg, const LevelView<float>& lv, float* u, const float* f, cudaStream_t st) {
  if (cfg == 0) launch_wave<Q, 128>(lv, u, f, st);
  else launch_wave<Q, 256>(lv, u, f, st);
}

int optin_smem_wave() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return optin;
}

}  // namespace

bool wave32_supported(const LevelView<float>& lv, int cfg) {
  if (cfg < 0 || cfg >= WAVE32_CONFIGS) return false;
  if (lv.q < 1 || lv.q > 3 || lv.N < 8 || lv.N > 1023 || lv.plane32 == nullptr || lv.plane_nodes == nullptr)
    return false;
  static const int optin = optin_smem_wave();
  const size_t smem = lv.q == 1 ? wave_smem<1>(lv.N) : (lv.q == 2 ? wave_smem<2>(lv.N) : wave_smem<3>(lv.N));
  return smem <= (size_t)optin;
}

void launch_wave32_smooth(const LevelView<float>& lv, float* u, const float* f, int cfg, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_wave_cfg<1>(cfg, lv, u, f, st); break;
    case 2: launch_wave_cfg<2>(cfg, lv, u, f, st); break;
    case 3: launch_wave_cfg<3>(cfg, lv, u, f, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}

}  // namespace hhg
