// FP32 surrogate smoother with the cell's planes staged in shared memory.
//
// One CTA owns one macro cell and runs the four colour steps of the
// multicolour Gauss-Seidel sweep (colours (i + 2j + 3k) mod 4, Eq. 5.1 on
// every interior node) as a plane wavefront: in step s colour c is updated
// on plane k = s + 1 - c, c = 0..3, with a barrier after each colour.  A
// colour-c update on plane k therefore sees colour c - 1 already done on
// planes k - 1, k, k + 1 and colour c + 1 not yet started there -- the same
// values as four separate colour sweeps.
//
// The interior of plane k is one contiguous run of the cell's block of the
// canonical vector, so it is brought into a ring of shared-memory slots by
// one bulk (TMA) copy, issued three steps before its first update and
// completing on a per-slot mbarrier; the at most three values at each end
// that are not 16-byte aligned come by 4-byte asynchronous copies.  All
// neighbour reads of the updates are shared-memory reads (boundary
// neighbours come from the cell's halo copy); a plane goes back to HBM with
// coalesced stores once its colour-3 update is done.  Every node's u is thus
// read once and written once per sweep, and f is read once: the 12 bytes per
// update of the FP32 smoother.
//
// Weights: per plane k, each direction's polynomial reduced to a polynomial
// in (i, j) (computed in FP64 and rounded once to FP32 at fit time) is read
// into a small ring of shared-memory tables and evaluated per node (Sec. 3.4).
#include <cuda_runtime.h>

#include "arith.cuh"
#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace hhg {

namespace {

// Colour c of plane k is updated in step s = k - 1 + SKEW c.  SKEW = 1 is the
// tightest wavefront (colour c - 1 on plane k + 1 is updated earlier in the
// same step, so the step needs a barrier after each colour); SKEW = 2 moves
// every dependency of a step into earlier steps, so the four colour tasks of a
// step are independent and share one barrier, at the cost of a wider ring.
template <int SKEW>
struct Sched {
  static constexpr int RING = 3 * SKEW + 4;  // u planes s - 3 SKEW .. s + 2 in use, s + 3 in flight
  static constexpr int CTAB = 3 * SKEW + 2;  // tables of planes s + 1 - 3 SKEW .. s + 1 in use, s + 2 filled
};

__host__ __device__ inline int plane_size(int N, int k) { return (N - 2 - k) * (N - 1 - k) / 2; }
// Floats per ring slot: plane 1 (the largest) at an offset of up to 3 floats
// (the slot keeps the plane's global 16-byte phase), rounded up to 16 bytes.
__host__ __device__ inline int slot_floats(int N) { return (plane_size(N, 1) + 3 + 3) & ~3; }

template <int Q, int SKEW>
size_t stage_smem(int N) {
  return sizeof(float) * (size_t)Sched<SKEW>::RING * slot_floats(N) +
         sizeof(float2) * (size_t)Sched<SKEW>::CTAB * NPAIR * npp2<Q>() + sizeof(uint64_t) * Sched<SKEW>::RING +
         sizeof(int) * 2 * (size_t)(N + 2);
}

// Resident CTAs per SM the register budget is sized for (64 registers a thread).
template <int THREADS>
constexpr int stage_min_blocks() { return THREADS >= 1024 ? 1 : 1024 / THREADS; }

template <int Q, int THREADS, int SKEW>
__global__ void __launch_bounds__(THREADS, stage_min_blocks<THREADS>()) lsqp_stage32_smooth(LevelView<float> lv,
                                                                                       float* u, const float* f,
                                                                                       int* err) {
  constexpr int RING = Sched<SKEW>::RING, CTAB = Sched<SKEW>::CTAB;
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NP2 = npp2<Q>();
  extern __shared__ __align__(16) float smem[];
  const int N = lv.N, np = N - 3, S = slot_floats(N);
  float* ring = smem;
  float2* ctab = reinterpret_cast<float2*>(ring + RING * S);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctab + CTAB * NPAIR * NP2);
  int* porg = reinterpret_cast<int*>(bar + RING);  // [N + 2]: ring offset of the first node of plane k
  int* pst = porg + (N + 2);                       // [N + 2]: position of that node in the cell's block
  const int c = blockIdx.x;
  const int64_t cbase = lv.off_C + (int64_t)c * lv.n_int;
  const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
  const float* ghost = lv.ghost + (int64_t)c * lv.n_full;
  const int n_plane = lv.n_plane;
  // set by any thread whose bounded wait gave up; read by all after a barrier
  __shared__ int s_fail;

  // the slot keeps the plane's 16-byte phase in the vector; planes 0 and
  // np + 1 have no interior points (their entries are never read)
  for (int k = threadIdx.x; k <= N + 1; k += THREADS) {
    const int ps = (k >= 1 && k <= np) ? lin_interior32(1, 1, k, N) : 0;
    pst[k] = ps;
    porg[k] = (k >= 1 && k <= np) ? ((k - 1) % RING) * S + (int)((cbase + ps) & 3) : 0;
  }
  if (threadIdx.x == 0) {
    for (int r = 0; r < RING; ++r) mbar_init(&bar[r], 1);
    s_fail = 0;
  }
  __syncthreads();
  auto slot = [](int k) { return (k - 1) % RING; };

  auto issue = [&](int k) {
    if (k < 1 || k > np) return;
    const int64_t g0 = cbase + pst[k], g1 = g0 + plane_size(N, k);
    const int64_t a0 = (g0 + 3) & ~(int64_t)3, a1 = g1 & ~(int64_t)3;
    float* o = ring + porg[k];
    if (threadIdx.x == 0) {
      const uint32_t bytes = a1 > a0 ? (uint32_t)((a1 - a0) * 4) : 0u;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[slot(k)], bytes);
      if (bytes) bulk_g2s(o + (a0 - g0), u + a0, bytes, &bar[slot(k)]);
    }
    const int t = (int)threadIdx.x - 32;  // lanes 0..5 of warp 1: ragged head and tail
    if (t >= 0 && t < 6) {
      const int64_t g = t < 3 ? g0 + t : a1 + (t - 3);
      const bool ok = t < 3 ? g < (a0 < g1 ? a0 : g1) : (g >= (a1 > a0 ? a1 : a0) && g < g1);
      if (ok) cp_async4(o + (g - g0), u + g);
    }
  };
  auto writeback = [&](int k) {
    if (k < 1 || k > np) return;
    float* dst = u + cbase + pst[k];
    const float* o = ring + porg[k];
    const int n = plane_size(N, k);
    for (int x = threadIdx.x; x < n; x += THREADS) dst[x] = o[x];
  };
  auto load_tab = [&](int k) {
    if (k < 1 || k > np) return;
    float* d = reinterpret_cast<float*>(ctab + ((k - 1) % CTAB) * NPAIR * NP2);
    const float* s = tab + (int64_t)(k - 1) * 15 * NP;
    for (int t = threadIdx.x; t < NPAIR * NP2 * 2; t += THREADS) {
      const int h = t & 1, e = (t >> 1) % NP2, m = (t >> 1) / NP2, w = 2 * m + h;
      d[t] = (e < NP && w < 15) ? s[w * NP + e] : 0.0f;
    }
  };
  auto wait_plane = [&](int k) {
    if (k < 1 || k > np) return;
    // the n-th use of a slot (n = (k - 1) / RING) completes phase n
    if (!mbar_wait(&bar[slot(k)], (uint32_t)(((k - 1) / RING) & 1))) s_fail = 1;
  };

  // Eq. 5.1 at list entry e of plane k (all neighbours resident)
  auto update = [&](int k, int e, float fv, uint32_t p, int x) {
    const float2* P = ctab + ((k - 1) % CTAB) * NPAIR * NP2;
    const int om = porg[k];
    const int i = unpack_i(p), j = unpack_j(p);
    const float2 I = make_float2((float)i, (float)i), J = make_float2((float)j, (float)j);
    auto body = [&](auto nb) {
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        const float2 w2 = eval_plane2<Q>(P + m * NP2, I, J);
        acc = __ffma2_rn(w2, make_float2(nb(2 * m), nb(2 * m + 1)), acc);
      }
      const float wc = eval_plane2<Q>(P + 7 * NP2, I, J).x;
      ring[om + x] = div_nr32(fv - acc.x - acc.y, wc);
    };
    if (deep_interior(i, j, k, N)) {
      // L = length of line j in plane k; node (i, j) of plane k + 1 sits
      // j - 1 places before node (i, j) of plane k, of plane k - 1 j - 1 after
      const float* pm = ring + om + x;
      const float* pt = ring + porg[k + 1] + x - j;
      const float* pb = ring + porg[k - 1] + x + j;
      const int L = N - 1 - j - k;
      body([&](int w) -> float {
        switch (w) {
          case ME: return pm[1];
          case MW: return pm[-1];
          case MN: return pm[L];
          case MS: return pm[-L - 1];
          case MNW: return pm[L - 1];
          case MSE: return pm[-L];
          case TC: return pt[1];
          case TW: return pt[0];
          case TS: return pt[1 - L];
          case TSE: return pt[2 - L];
          case BC: return pb[-1];
          case BE: return pb[0];
          case BN: return pb[L];
          default: return pb[L - 1];  // BNW
        }
      });
    } else {
      body([&](int w) -> float {
        const int code = lv.plane_nb[w * n_plane + e];
        if (code < 0) return ghost[code & 0x7fffffff];
        return ring[porg[k + (code >> 29) - 1] + (code & 0x1fffffff)];
      });
    }
  };

  // the colour tasks of step s: colour cc on plane s + 1 - SKEW cc, taken as
  // one pool of list entries (SKEW = 2) or one task per barrier (SKEW = 1)
  auto run_tasks = [&](int s, int c0, int c1) {
    int b0 = 0, b1 = 0, b2 = 0, b3 = 0, p1, p2, p3, p4;  // task starts in the lists; pool prefix sums
    auto task = [&](int cc, int& b) {
      const int k = s + 1 - SKEW * cc;
      if (cc < c0 || cc >= c1 || k < 1 || k > np) return 0;
      b = lv.plane_off[k * 4 + cc];
      return lv.plane_off[k * 4 + cc + 1] - b;
    };
    p1 = task(0, b0);
    p2 = p1 + task(1, b1);
    p3 = p2 + task(2, b2);
    p4 = p3 + task(3, b3);
    constexpr int B = 2;  // entries per thread in flight
    for (int base = threadIdx.x; base < p4; base += B * THREADS) {
      int e[B], kk[B], x[B];
      uint32_t p[B];
      float fv[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int idx = base + b * THREADS;
        const int cc = (idx >= p1) + (idx >= p2) + (idx >= p3);
        const int start = cc == 0 ? b0 : (cc == 1 ? b1 - p1 : (cc == 2 ? b2 - p2 : b3 - p3));
        kk[b] = s + 1 - SKEW * cc;
        e[b] = idx < p4 ? start + idx : -1;
        p[b] = e[b] >= 0 ? lv.plane_nodes[e[b]] : 0u;
        x[b] = e[b] >= 0 ? lv.plane_x[e[b]] : 0;
      }
#pragma unroll
      for (int b = 0; b < B; ++b) fv[b] = e[b] >= 0 ? f[cbase + pst[kk[b]] + x[b]] : 0.0f;
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (e[b] >= 0) update(kk[b], e[b], fv[b], p[b], x[b]);
    }
  };

  issue(1);
  issue(2);
  load_tab(1);
  cp_async_commit();
  wait_plane(1);
  cp_async_wait_all();
  __syncthreads();
  int s = 0;
  for (; s <= np + 3 * SKEW; ++s) {
    // a wait that gave up: no further copies, updates or write-back (u is
    // left partly swept; the caller sees HHG_ETIMEOUT)
    if (s_fail) break;
    writeback(s - 3 * SKEW);  // colour 3 done in step s - 1
    issue(s + 3);             // into the slot of plane s + 3 - RING, last read in step s - 1
    load_tab(s + 2);
    cp_async_commit();
    wait_plane(s + 2);
    if (SKEW == 1) {
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        run_tasks(s, cc, cc + 1);
        if (cc == 3) cp_async_wait_all();
        __syncthreads();
      }
    } else {
      run_tasks(s, 0, 4);
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if (s_fail) {
    // let the copies already issued land before the CTA exits (planes up to
    // s + 2 were issued, the last two possibly not yet waited for), each
    // wait bounded again
    cp_async_wait_all();
    if (threadIdx.x == 0) {
      for (int k = s + 1; k <= s + 2; ++k)
        if (k >= 1 && k <= np) mbar_wait(&bar[slot(k)], (uint32_t)(((k - 1) / RING) & 1));
      atomicExch(err, 1);
    }
  }
}

template <int Q, int THREADS, int SKEW>
void launch_q(const LevelView<float>& lv, float* u, const float* f, int* err, cudaStream_t st) {
  const size_t smem = stage_smem<Q, SKEW>(lv.N);
  auto kern = lsqp_stage32_smooth<Q, THREADS, SKEW>;
  ensure_smem_limit((const void*)kern, smem);
  kern<<<lv.nC, THREADS, smem, st>>>(lv, u, f, err);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

int optin_smem() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return optin;
}

// Launch configurations the tuner chooses from: (SKEW, threads per CTA).
struct Cfg {
  int skew, threads;
};
constexpr Cfg kCfgs[STAGE32_CONFIGS] = {{1, 256}, {1, 1024}, {2, 128}, {2, 512}};

template <int Q>
size_t cfg_smem(int cfg, int N) {
  return kCfgs[cfg].skew == 1 ? stage_smem<Q, 1>(N) : stage_smem<Q, 2>(N);
}

template <int Q>
void launch_cfg(int cfg, const LevelView<float>& lv, float* u, const float* f, int* err, cudaStream_t st) {
  switch (cfg) {
    case 0: launch_q<Q, 256, 1>(lv, u, f, err, st); break;
    case 1: launch_q<Q, 1024, 1>(lv, u, f, err, st); break;
    case 2: launch_q<Q, 128, 2>(lv, u, f, err, st); break;
    default: launch_q<Q, 512, 2>(lv, u, f, err, st); break;
  }
}

size_t smem_of(int q, int cfg, int N) {
  return q == 1 ? cfg_smem<1>(cfg, N) : (q == 2 ? cfg_smem<2>(cfg, N) : cfg_smem<3>(cfg, N));
}

}  // namespace

bool stage32_supported(const LevelView<float>& lv, const float* u, int cfg) {
  if (cfg < 0 || cfg >= STAGE32_CONFIGS) return false;
  if (lv.q < 1 || lv.q > 3 || lv.N < 8 || lv.plane32 == nullptr || lv.err == nullptr || lv.plane_nb == nullptr)
    return false;
  if (reinterpret_cast<uintptr_t>(u) & 15) return false;
  static const int optin = optin_smem();
  return smem_of(lv.q, cfg, lv.N) <= (size_t)optin;
}

void launch_stage32_smooth(const LevelView<float>& lv, float* u, const float* f, int cfg, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_cfg<1>(cfg, lv, u, f, lv.err, st); break;
    case 2: launch_cfg<2>(cfg, lv, u, f, lv.err, st); break;
    case 3: launch_cfg<3>(cfg, lv, u, f, lv.err, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}

}  // namespace hhg
