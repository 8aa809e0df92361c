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

#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace hhg {

namespace {

constexpr int RING = 7;  // u planes s-3 .. s+2 in use during step s, plus s+3 in flight
constexpr int CTAB = 5;  // coefficient tables of planes s-2 .. s+1 in use, s+2 being filled

__host__ __device__ inline int plane_size(int N, int k) { return (N - 2 - k) * (N - 1 - k) / 2; }
// Floats per ring slot: plane 1 (the largest) at an offset of up to 3 floats
// (the slot keeps the plane's global 16-byte phase), rounded up to 16 bytes.
__host__ __device__ inline int slot_floats(int N) { return (plane_size(N, 1) + 3 + 3) & ~3; }

template <int Q>
size_t stage_smem(int N) {
  return sizeof(float) * ((size_t)RING * slot_floats(N) + (size_t)CTAB * 15 * np_pad<Q>()) + sizeof(uint64_t) * RING;
}

// Resident CTAs per SM the register budget is sized for (64 registers a thread).
template <int THREADS>
constexpr int stage_min_blocks() { return THREADS >= 1024 ? 1 : 1024 / THREADS; }

template <int Q, int THREADS>
__global__ void __launch_bounds__(THREADS, stage_min_blocks<THREADS>()) lsqp_stage32_smooth(LevelView<float> lv, float* u, const float* f,
                                                                int* err) {
  constexpr int NP = (Q + 1) * (Q + 2) / 2;
  constexpr int NPP = np_pad<Q>();
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = lv.N, np = N - 3, S = slot_floats(N);
  float* ring = reinterpret_cast<float*>(smem);
  float* ctab = ring + RING * S;
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctab + CTAB * 15 * NPP);
  const int c = blockIdx.x;
  const int64_t cbase = lv.off_C + (int64_t)c * lv.n_int;
  const float* tab = lv.plane32 + (int64_t)c * np * 15 * NP;
  const float* ghost = lv.ghost + (int64_t)c * lv.n_full;
  bool failed = false;

  // first interior node of plane k within the cell's block, and the
  // shared-memory position of that node (the slot keeps the 16-byte phase)
  auto pstart = [&](int k) { return lin_interior32(1, 1, k, N); };
  auto slot = [](int k) { return (k - 1) % RING; };  // planes 1..7 take slots 0..6, 8..14 reuse them
  auto origin = [&](int k) { return ring + slot(k) * S + (int)((cbase + pstart(k)) & 3); };

  if (threadIdx.x == 0)
    for (int r = 0; r < RING; ++r) mbar_init(&bar[r], 1);
  __syncthreads();

  auto issue = [&](int k) {
    if (k < 1 || k > np) return;
    const int64_t g0 = cbase + pstart(k), g1 = g0 + plane_size(N, k);
    const int64_t a0 = (g0 + 3) & ~(int64_t)3, a1 = g1 & ~(int64_t)3;
    float* o = origin(k);
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
    const int64_t g0 = cbase + pstart(k);
    const float* o = origin(k);
    const int n = plane_size(N, k);
    for (int x = threadIdx.x; x < n; x += THREADS) u[g0 + x] = o[x];
  };
  auto load_tab = [&](int k) {
    if (k < 1 || k > np) return;
    float* d = ctab + ((k - 1) % CTAB) * 15 * NPP;
    const float* s = tab + (int64_t)(k - 1) * 15 * NP;
    for (int t = threadIdx.x; t < 15 * NPP; t += THREADS) {
      const int e = t % NPP, w = t / NPP;
      d[t] = e < NP ? s[w * NP + e] : 0.0f;
    }
  };
  auto wait_plane = [&](int k) {
    if (k < 1 || k > np) return;
    // the n-th use of a slot (n = (k - 1) / RING) completes phase n
    if (!mbar_wait(&bar[slot(k)], (uint32_t)(((k - 1) / RING) & 1))) failed = true;
  };

  // colour cc on plane k (all its neighbours are resident)
  auto process = [&](int k, int cc) {
    const int beg = lv.plane_off[k * 4 + cc], end = lv.plane_off[k * 4 + cc + 1];
    const float* P = ctab + ((k - 1) % CTAB) * 15 * NPP;
    float* om = origin(k);
    const float* ot = origin(k + 1);  // used only for interior neighbours (k + 1 <= np)
    const float* ob = origin(k - 1);  // used only for interior neighbours (k - 1 >= 1)
    const int pk = pstart(k);
    const float* fk = f + cbase + pk;
    for (int t = beg + (int)threadIdx.x; t < end; t += THREADS) {
      const uint32_t p = lv.plane_nodes[t];
      const int i = unpack_i(p), j = unpack_j(p);
      const int x = lin_interior32(i, j, k, N) - pk;
      const float fi = (float)i, fj = (float)j;
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
        return eval_plane<float, Q>(Pw, fi, fj);
      };
      auto update = [&](auto nb) {
        float a0 = fk[x], a1 = 0.0f;
#pragma unroll
        for (int w = 0; w < 14; w += 2) {
          a0 = fmaf(-wt(w), nb(w), a0);
          a1 = fmaf(-wt(w + 1), nb(w + 1), a1);
        }
        om[x] = (a0 + a1) / wt(MC);
      };
      if (deep_interior(i, j, k, N)) {
        // plane-local offsets: L = length of line j in plane k; a node (i, j)
        // of plane k + 1 sits j - 1 places before (i, j) of plane k
        const int L = N - 1 - j - k;
        update([&](int w) -> float {
          switch (w) {
            case ME: return om[x + 1];
            case MW: return om[x - 1];
            case MN: return om[x + L];
            case MS: return om[x - L - 1];
            case MNW: return om[x + L - 1];
            case MSE: return om[x - L];
            case TC: return ot[x - j + 1];
            case TW: return ot[x - j];
            case TS: return ot[x - L - j + 1];
            case TSE: return ot[x - L - j + 2];
            case BC: return ob[x + j - 1];
            case BE: return ob[x + j];
            case BN: return ob[x + L + j];
            default: return ob[x + L + j - 1];  // BNW
          }
        });
      } else {
        update([&](int w) -> float {
          const int i2 = i + DI(w), j2 = j + DJ(w), k2 = k + DK(w);
          if (is_interior(i2, j2, k2, N)) {
            const float* o = DK(w) > 0 ? ot : (DK(w) < 0 ? ob : om);
            return o[lin_interior32(i2, j2, k2, N) - pstart(k2)];
          }
          return ghost[lin_full(i2, j2, k2, N)];
        });
      }
    }
  };

  issue(1);
  issue(2);
  load_tab(1);
  cp_async_commit();
  wait_plane(1);
  cp_async_wait_all();
  __syncthreads();
  for (int s = 0; s <= np + 3; ++s) {
    writeback(s - 3);  // final since step s - 1
    issue(s + 3);      // into the slot of plane s - 4, free since step s - 1
    load_tab(s + 2);
    cp_async_commit();
    wait_plane(s + 2);
#pragma unroll 1
    for (int cc = 0; cc < 4; ++cc) {
      const int k = s + 1 - cc;
      if (k >= 1 && k <= np) process(k, cc);
      if (cc == 3) cp_async_wait_all();
      __syncthreads();
    }
  }
  if (failed) atomicExch(err, 1);
}

template <int Q, int THREADS>
void launch_q(const LevelView<float>& lv, float* u, const float* f, int* err, cudaStream_t st) {
  const size_t smem = stage_smem<Q>(lv.N);
  auto kern = lsqp_stage32_smooth<Q, THREADS>;
  HHG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<lv.nC, THREADS, smem, st>>>(lv, u, f, err);
  HHG_CUDA(cudaGetLastError());
  count_launch();
}

template <int Q>
void launch_t(const LevelView<float>& lv, float* u, const float* f, int* err, cudaStream_t st) {
  if (lv.N >= 128)
    launch_q<Q, 1024>(lv, u, f, err, st);
  else if (lv.N >= 64)
    launch_q<Q, 256>(lv, u, f, err, st);
  else
    launch_q<Q, 128>(lv, u, f, err, st);
}

}  // namespace

bool stage32_supported(const LevelView<float>& lv, const float* u) {
  if (lv.q < 1 || lv.q > 3 || lv.N < 8 || lv.plane32 == nullptr || lv.err == nullptr) return false;
  if (reinterpret_cast<uintptr_t>(u) & 15) return false;
  size_t smem = 0;
  switch (lv.q) {
    case 1: smem = stage_smem<1>(lv.N); break;
    case 2: smem = stage_smem<2>(lv.N); break;
    default: smem = stage_smem<3>(lv.N); break;
  }
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  return smem <= (size_t)optin;
}

void launch_stage32_smooth(const LevelView<float>& lv, float* u, const float* f, cudaStream_t st) {
  switch (lv.q) {
    case 1: launch_t<1>(lv, u, f, lv.err, st); break;
    case 2: launch_t<2>(lv, u, f, lv.err, st); break;
    case 3: launch_t<3>(lv, u, f, lv.err, st); break;
    default: throw Error{HHG_ENOTFIT, "surrogate degree not fitted"};
  }
}

}  // namespace hhg
