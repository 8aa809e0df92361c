// C ABI of libhhg: setup of the shell hierarchy, surrogate fit, operator
// application, smoothing, residual and the V-cycle driver.  See
// include/hhg.h for the contract of every entry point.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "device.cuh"
#include "kernels.h"
#include "linalg.h"
#include "mesh.h"
#include "shell.h"

namespace hhg {

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }

void ensure_smem_limit(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> enabled;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : enabled)
    if (e.first == func) {
      if (e.second >= bytes) return;
      HHG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      e.second = bytes;
      return;
    }
  HHG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  enabled.push_back({func, bytes});
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void* Allocator::alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (budget && used + bytes > budget)
    throw Error{HHG_ENOMEM, "HBM budget exceeded: need " + std::to_string(used + bytes) + " of " +
                                std::to_string(budget) + " bytes"};
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? HHG_ENOMEM : HHG_ECUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  }
  used += bytes;
  live.push_back({p, bytes});
  return p;
}

void Allocator::release(void* p) {
  if (!p) return;
  for (size_t n = 0; n < live.size(); ++n)
    if (live[n].first == p) {
      cudaFree(p);
      used -= live[n].second;
      live.erase(live.begin() + n);
      return;
    }
}

void Allocator::release_all() {
  for (auto& a : live) cudaFree(a.first);
  live.clear();
  used = 0;
}

static void check_device_error(hhg_shell* s, cudaStream_t st);

template <class T>
static T* upload(Allocator& A, const std::vector<T>& h, cudaStream_t st) {
  T* d = A.alloc_n<T>(h.size());
  if (!h.empty()) HHG_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  HHG_CUDA(cudaStreamSynchronize(st));
  return d;
}

// ---------------------------------------------------------------------------
// level construction
// ---------------------------------------------------------------------------

// Canonical index of a face-local point with weights (l0, l1, l2) over the
// face's vertices (sum = lay.N), through the face's own edges.
static int64_t face_point_index(const MacroMesh& m, const LevelLayout& lay, int f, int l0, int l1, int l2) {
  const auto& F = m.faces[f];
  const auto& E = m.face_edges[f];
  const int N = lay.N;
  const int mask = (l0 > 0) | ((l1 > 0) << 1) | ((l2 > 0) << 2);
  switch (mask) {
    case 1: return F[0];
    case 2: return F[1];
    case 4: return F[2];
    case 3: return lay.off_E + (int64_t)E[0] * (N - 1) + (l1 - 1);
    case 5: return lay.off_E + (int64_t)E[1] * (N - 1) + (l2 - 1);
    case 6: return lay.off_E + (int64_t)E[2] * (N - 1) + (l2 - 1);
    case 7: return lay.off_F + (int64_t)f * lay.n_face + lin_face(l1, l2, N);
  }
  throw Error{HHG_EINVAL, "face_point_index: empty support"};
}

static int64_t edge_point_index(const MacroMesh& m, const LevelLayout& lay, int e, int l0, int l1) {
  if (l1 == 0) return m.edges[e][0];
  if (l0 == 0) return m.edges[e][1];
  return lay.off_E + (int64_t)e * (lay.N - 1) + (l1 - 1);
}

// Both coarse ends of the coarse edge a fine point (barycentric weights lam
// over d vertices, sum N) is the midpoint of; a coarse-lattice point returns
// itself twice.  Weights returned on the coarse lattice (sum N/2).
static void parents(int d, const int* lam, int* pa, int* pb) {
  int odd[4], no = 0;
  for (int a = 0; a < d; ++a)
    if (lam[a] & 1) odd[no++] = a;
  for (int a = 0; a < d; ++a) pa[a] = pb[a] = lam[a];
  if (no == 2) {
    pa[odd[0]] += 1; pa[odd[1]] -= 1;
    pb[odd[0]] -= 1; pb[odd[1]] += 1;
  } else if (no == 4) {  // (i, j, k) all odd: the coarse edge of direction (1, -1, 1)
    const int dl[4] = {-1, 1, -1, 1};
    for (int a = 0; a < 4; ++a) { pa[a] += dl[a]; pb[a] -= dl[a]; }
  }
  for (int a = 0; a < d; ++a) { pa[a] /= 2; pb[a] /= 2; }
}

// Points of the closed macro cell that are not interior (its faces, edges
// and vertices), in lin_full order, and each full position's slot among them
// (-1 for interior points).
static void boundary_points(int N, std::vector<uint32_t>& bnd_ijk, std::vector<int>& bnd_slot) {
  bnd_ijk.clear();
  bnd_slot.assign((size_t)tet_points(N), -1);
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - j - k; ++i)
        if (!is_interior(i, j, k, N)) {
          bnd_slot[lin_full(i, j, k, N)] = (int)bnd_ijk.size();
          bnd_ijk.push_back(pack_ijk(i, j, k));
        }
}

// Halo sources (canonical index of every cell boundary point, -1 where it is
// a Dirichlet node) and the incidence of the lower nodes in the cells: for
// lower node r, inc_cb[inc_ptr[r] .. inc_ptr[r+1]) are the (cell * n_bnd +
// slot) positions holding it, in ascending cell order.  Dirichlet nodes have
// no incidence.
static void lower_incidence(const MacroMesh& m, const LevelLayout& lay, const std::vector<uint32_t>& bnd_ijk,
                            std::vector<int>& halo_src, std::vector<int64_t>& inc_ptr, std::vector<int>& inc_cb) {
  const int n_bnd = (int)bnd_ijk.size();
  const int64_t nhal = lay.nC * n_bnd;
  halo_src.assign((size_t)nhal, -1);
  inc_ptr.assign((size_t)lay.off_C + 1, 0);
  for (int c = 0; c < lay.nC; ++c)
    for (int b = 0; b < n_bnd; ++b) {
      const uint32_t p = bnd_ijk[b];
      const int64_t idx = cell_node_index(m, lay, c, unpack_i(p), unpack_j(p), unpack_k(p));
      const bool dir = node_dirichlet(m, lay, idx);
      halo_src[(size_t)c * n_bnd + b] = dir ? -1 : (int)idx;
      if (!dir) inc_ptr[idx + 1]++;
    }
  for (int64_t r = 0; r < lay.off_C; ++r) inc_ptr[r + 1] += inc_ptr[r];
  inc_cb.assign((size_t)inc_ptr[lay.off_C], 0);
  std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
  for (int64_t t = 0; t < nhal; ++t)
    if (halo_src[t] >= 0) inc_cb[fill[halo_src[t]]++] = (int)t;
}

// Run lists of the FP64 surrogate kernels and the cell-resident sweep (see
// LevelView): per line, the points of the segment (one colour, stride 4; or
// all, stride 1) split where deep-interior and boundary-adjacent points
// meet, each part into near-equal runs of at most RUN64 points; deep runs
// first, each part in plane order; kidx[(g (N + 1) + k) 2 + part] = first
// item of colour g (relative to off[g]) of the part whose plane is >= k.
// Host only (also reached through hhg_run_lists for host-side tests).
static void build_run_lists(int N, std::vector<uint2>& run_nodes, int off[6], std::vector<int>& run_kidx) {
  auto deep = [N](int i, int j, int k) { return i >= 2 && j >= 2 && k >= 2 && i + j + k <= N - 2; };
  run_nodes.clear();
  for (int g = 0; g < 5; ++g) {
    off[g] = (int)run_nodes.size();
    const int h = g < 4 ? 4 : 1;
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 1; k < N; ++k)
        for (int j = 1; j < N - k; ++j) {
          const int last = N - 1 - j - k;
          int i = 1;
          while (g < 4 && i <= last && (i + 2 * j + 3 * k) % 4 != g) i += 1;
          while (i <= last) {
            const bool d = deep(i, j, k);
            int n_pts = 0;
            while (i + n_pts * h <= last && deep(i + n_pts * h, j, k) == d) ++n_pts;
            const int n_runs = (n_pts + RUN64 - 1) / RUN64;
            for (int r = 0, done = 0; r < n_runs; ++r) {
              const int cnt = (n_pts - done) / (n_runs - r);
              if (d == (pass == 0))
                run_nodes.push_back(make_uint2(pack_ijk(i + done * h, j, k), (uint32_t)cnt | ((uint32_t)d << 8)));
              done += cnt;
            }
            i += n_pts * h;
          }
        }
  }
  off[5] = (int)run_nodes.size();
  run_kidx.assign((size_t)4 * (N + 1) * 2, 0);
  for (int g = 0; g < 4; ++g) {
    const int b = off[g], n_seg = off[g + 1] - b;
    int deep_end = 0;
    while (deep_end < n_seg && (run_nodes[b + deep_end].y & 0x100u)) ++deep_end;
    for (int part = 0; part < 2; ++part) {
      const int lo = part == 0 ? 0 : deep_end, hi = part == 0 ? deep_end : n_seg;
      int e = lo;
      for (int k = 0; k <= N; ++k) {
        while (e < hi && unpack_k(run_nodes[b + e].x) < k) ++e;
        run_kidx[((size_t)g * (N + 1) + k) * 2 + part] = e;
      }
    }
  }
}

static void build_level(hhg_shell* s, int n, cudaStream_t st) {
  const MacroMesh& m = s->mesh;
  Level& L = s->levels[n];
  const int N = 4 << n;
  L.N = N;
  L.lay = make_layout(m, N);
  const LevelLayout& lay = L.lay;
  HHG_CHECK(lay.n_total < (int64_t)INT32_MAX, HHG_EINVAL, "level too large for 32-bit node indices");
  Allocator& A = s->alloc;

  // cell-local tables shared by all cells
  std::vector<uint32_t> plane_nodes;
  std::vector<int> plane_off(4 * (N + 1) + 1, 0);
  // every node list puts the deep-interior points (all 14 neighbours
  // interior) first, so warps take one addressing path
  auto deep = [N](int i, int j, int k) { return i >= 2 && j >= 2 && k >= 2 && i + j + k <= N - 2; };
  for (int k = 0; k <= N; ++k)
    for (int cc = 0; cc < 4; ++cc) {
      plane_off[k * 4 + cc] = (int)plane_nodes.size();
      for (int pass = 0; pass < 2; ++pass)
        for (int j = 1; j <= N - 2 - k; ++j)
          for (int i = 1; i <= N - 1 - j - k; ++i)
            if (k >= 1 && (i + 2 * j + 3 * k) % 4 == cc && deep(i, j, k) == (pass == 0))
              plane_nodes.push_back(pack_ijk(i, j, k));
    }
  plane_off[4 * (N + 1)] = (int)plane_nodes.size();
  // for the staged smoother: each listed point's position within its plane
  // (interior points of plane k, line by line), and for points next to the
  // cell boundary the 14 neighbour codes, [w][entry]: bit 31 set = halo
  // point (low bits: its cell-local full index), else bits 29-30 = dk + 1
  // and the low bits the neighbour's position within plane k + dk
  const int n_plane = (int)plane_nodes.size();
  std::vector<int> plane_x((size_t)n_plane), plane_nb((size_t)14 * n_plane, 0);
  for (int e = 0; e < n_plane; ++e) {
    const uint32_t p = plane_nodes[e];
    const int i = unpack_i(p), j = unpack_j(p), k = unpack_k(p);
    plane_x[e] = (int)(lin_interior(i, j, k, N) - lin_interior(1, 1, k, N));
    if (deep(i, j, k)) continue;
    for (int w = 0; w < 14; ++w) {
      const int i2 = i + dir_di(w), j2 = j + dir_dj(w), k2 = k + dir_dk(w);
      plane_nb[(size_t)w * n_plane + e] =
          is_interior(i2, j2, k2, N)
              ? (int)(((uint32_t)(dir_dk(w) + 1) << 29) |
                      (uint32_t)(lin_interior(i2, j2, k2, N) - lin_interior(1, 1, k2, N)))
              : (int)(0x80000000u | (uint32_t)lin_full(i2, j2, k2, N));
    }
  }
  std::vector<uint32_t> int_ijk;
  for (int k = 1; k < N; ++k)
    for (int j = 1; j < N - k; ++j)
      for (int i = 1; i < N - j - k; ++i) int_ijk.push_back(pack_ijk(i, j, k));
  // colour_nodes: per colour, deep points first; all_nodes: every interior
  // point, deep first (the apply / residual order)
  std::vector<uint32_t> colour_nodes, all_nodes;
  for (int cc = 0; cc < 4; ++cc) {
    L.colour_off[cc] = (int)colour_nodes.size();
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 1; k < N; ++k)
        for (int j = 1; j < N - k; ++j)
          for (int i = 1; i < N - j - k; ++i)
            if ((i + 2 * j + 3 * k) % 4 == cc && deep(i, j, k) == (pass == 0)) colour_nodes.push_back(pack_ijk(i, j, k));
  }
  L.colour_off[4] = (int)colour_nodes.size();
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N - k; ++j)
        for (int i = 1; i < N - j - k; ++i)
          if (deep(i, j, k) == (pass == 0)) all_nodes.push_back(pack_ijk(i, j, k));
  // chunked colour lists: up to CHUNK32 deep points of a line (stride 4),
  // then the points of the colour next to the cell boundary
  std::vector<uint32_t> chunk_nodes;
  for (int cc = 0; cc < 4; ++cc) {
    L.chunk_off[cc] = (int)chunk_nodes.size();
    for (int k = 2; k < N; ++k)
      for (int j = 2; j < N - k; ++j) {
        const int last = N - 2 - j - k;
        int i = 2;
        while ((i + 2 * j + 3 * k) % 4 != cc) ++i;
        for (; i <= last; i += 4 * CHUNK32) {
          const int cnt = std::min(CHUNK32, (last - i) / 4 + 1);
          chunk_nodes.push_back(pack_ijk(i, j, k) | ((uint32_t)(cnt - 1) << 30));
        }
      }
    L.chunk_mid[cc] = (int)chunk_nodes.size();
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N - k; ++j)
        for (int i = 1; i < N - j - k; ++i)
          if (!deep(i, j, k) && (i + 2 * j + 3 * k) % 4 == cc) chunk_nodes.push_back(pack_ijk(i, j, k));
  }
  L.chunk_off[4] = (int)chunk_nodes.size();
  std::vector<uint2> run_nodes;
  std::vector<int> run_kidx;
  build_run_lists(N, run_nodes, L.run_off, run_kidx);
  std::vector<uint32_t> bnd_ijk;
  std::vector<int> bnd_slot;
  boundary_points(N, bnd_ijk, bnd_slot);
  L.n_bnd = (int)bnd_ijk.size();
  L.h_plane_off = plane_off;

  // halo sources and the incidence of lower nodes in cells
  std::vector<int> halo_src;
  std::vector<int64_t> inc_ptr;
  std::vector<int> inc_cb;
  lower_incidence(m, lay, bnd_ijk, halo_src, inc_ptr, inc_cb);

  // lower-primitive colour steps and Dirichlet list
  std::vector<int> steps[6], dirl;
  for (int64_t v = 0; v < lay.nV; ++v) (m.vertex_dirichlet((int)v) ? dirl : steps[0]).push_back((int)v);
  for (int64_t e = 0; e < lay.nE; ++e)
    for (int p = 1; p < N; ++p) {
      const int64_t idx = lay.off_E + e * (N - 1) + p - 1;
      (m.edge_dirichlet((int)e) ? dirl : steps[1 + (p & 1)]).push_back((int)idx);
    }
  for (int64_t f = 0; f < lay.nF; ++f)
    for (int q = 1; q < N - 1; ++q)
      for (int p = 1; p < N - q; ++p) {
        const int64_t idx = lay.off_F + f * lay.n_face + lin_face(p, q, N);
        (m.face_dirichlet((int)f) ? dirl : steps[3 + (p + 2 * q) % 3]).push_back((int)idx);
      }
  L.n_free = lay.n_total - (int64_t)dirl.size();
  // the lower rows are stored in step order (steps 1-6, then the Dirichlet
  // rows): a smoother step reads one contiguous range of the sliced rows
  std::vector<int> perm, pos((size_t)lay.off_C, -1);
  L.max_step = 0;
  for (int t = 0; t < 6; ++t) {
    L.step_beg[t] = (int)perm.size();
    L.step_n[t] = (int)steps[t].size();
    L.max_step = std::max(L.max_step, L.step_n[t]);
    perm.insert(perm.end(), steps[t].begin(), steps[t].end());
  }
  perm.insert(perm.end(), dirl.begin(), dirl.end());
  HHG_CHECK((int64_t)perm.size() == lay.off_C, HHG_EINVAL, "lower rows do not partition into smoother steps");
  for (int64_t p = 0; p < lay.off_C; ++p) pos[perm[p]] = (int)p;
  L.d_low_perm = upload(A, perm, st);
  L.d_low_pos = upload(A, pos, st);
  L.n_dirichlet = (int)dirl.size();
  L.d_dirichlet = upload(A, dirl, st);

  L.d_plane_nodes = upload(A, plane_nodes, st);
  L.d_plane_x = upload(A, plane_x, st);
  L.d_plane_nb = upload(A, plane_nb, st);
  L.n_plane = n_plane;
  L.d_plane_off = upload(A, plane_off, st);
  L.d_int_ijk = upload(A, int_ijk, st);
  L.d_colour_nodes = upload(A, colour_nodes, st);
  L.d_all_nodes = upload(A, all_nodes, st);
  L.d_chunk_nodes = upload(A, chunk_nodes, st);
  L.d_run_nodes = upload(A, run_nodes, st);
  L.d_run_kidx = upload(A, run_kidx, st);
  L.d_bnd_ijk = upload(A, bnd_ijk, st);
  L.d_bnd_slot = upload(A, bnd_slot, st);
  L.d_halo_src = upload(A, halo_src, st);

  // exact lower-primitive rows, assembled on the device in two passes
  LevelView<double> v{};
  v.N = N; v.nC = (int)lay.nC; v.off_E = lay.off_E; v.off_F = lay.off_F; v.off_C = lay.off_C;
  v.n_total = lay.n_total; v.n_int = lay.n_int; v.n_full = lay.n_full; v.n_bnd = L.n_bnd;
  v.geom = s->d_geom; v.bnd_ijk = L.d_bnd_ijk; v.bnd_slot = L.d_bnd_slot; v.halo_src = L.d_halo_src;
  v.low_perm = L.d_low_perm; v.low_pos = L.d_low_pos;
  int64_t* d_inc_ptr = upload(A, inc_ptr, st);
  int* d_inc_cb = upload(A, inc_cb, st);
  int* d_len = A.alloc_n<int>((size_t)std::max<int64_t>(lay.off_C, 1));
  launch_low_assemble(v, 0, d_inc_ptr, d_inc_cb, d_len, nullptr, nullptr, nullptr, nullptr, st);
  std::vector<int> len((size_t)lay.off_C);
  HHG_CUDA(cudaMemcpyAsync(len.data(), d_len, len.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  HHG_CUDA(cudaStreamSynchronize(st));
  L.n_slices = (lay.off_C + 31) / 32;
  std::vector<int64_t> sell_ptr((size_t)L.n_slices + 1, 0);
  for (int64_t sl = 0; sl < L.n_slices; ++sl) {
    int w = 0;
    for (int64_t p = sl * 32; p < std::min<int64_t>(lay.off_C, sl * 32 + 32); ++p) {
      const int r = perm[p];
      HHG_CHECK(len[r] >= 0, HHG_EINVAL, "lower-primitive row wider than the assembly buffer");
      w = std::max(w, len[r]);
    }
    sell_ptr[sl + 1] = sell_ptr[sl] + 32 * (int64_t)w;
  }
  L.d_sell_ptr = upload(A, sell_ptr, st);
  L.d_sell_col = A.alloc_n<int>((size_t)std::max<int64_t>(sell_ptr.back(), 1));
  L.d_sell_val = A.alloc_n<double>((size_t)std::max<int64_t>(sell_ptr.back(), 1));
  L.d_low_diag = A.alloc_n<double>((size_t)std::max<int64_t>(lay.off_C, 1));
  launch_low_assemble(v, 1, d_inc_ptr, d_inc_cb, d_len, L.d_sell_ptr, L.d_sell_col, L.d_sell_val, L.d_low_diag, st);
  HHG_CUDA(cudaStreamSynchronize(st));
  A.release(d_inc_ptr);
  A.release(d_inc_cb);
  A.release(d_len);

  // transfers to the next coarser level (this level as the fine one)
  if (n > 0) {
    const LevelLayout lc = make_layout(m, N / 2);
    std::vector<int> par((size_t)2 * lay.off_C, -1), clf((size_t)lc.off_C, -1);
    auto put = [&](int64_t r, int64_t a, int64_t b) {
      par[2 * r] = node_dirichlet(m, lc, a) ? -1 : (int)a;
      par[2 * r + 1] = node_dirichlet(m, lc, b) ? -1 : (int)b;
    };
    for (int64_t v0 = 0; v0 < lay.nV; ++v0) put(v0, v0, v0);
    for (int64_t e = 0; e < lay.nE; ++e)
      for (int p = 1; p < N; ++p) {
        const int lam[2] = {N - p, p};
        int pa[2], pb[2];
        parents(2, lam, pa, pb);
        put(lay.off_E + e * (N - 1) + p - 1, edge_point_index(m, lc, (int)e, pa[0], pa[1]),
            edge_point_index(m, lc, (int)e, pb[0], pb[1]));
      }
    for (int64_t f = 0; f < lay.nF; ++f)
      for (int q = 1; q < N - 1; ++q)
        for (int p = 1; p < N - q; ++p) {
          const int lam[3] = {N - p - q, p, q};
          int pa[3], pb[3];
          parents(3, lam, pa, pb);
          put(lay.off_F + f * lay.n_face + lin_face(p, q, N), face_point_index(m, lc, (int)f, pa[0], pa[1], pa[2]),
              face_point_index(m, lc, (int)f, pb[0], pb[1], pb[2]));
        }
    L.d_low_par = upload(A, par, st);
    // coarse lower nodes -> their fine position
    for (int64_t v0 = 0; v0 < lc.nV; ++v0)
      if (!m.vertex_dirichlet((int)v0)) clf[v0] = (int)v0;
    for (int64_t e = 0; e < lc.nE; ++e)
      if (!m.edge_dirichlet((int)e))
        for (int p = 1; p < lc.N; ++p) clf[lc.off_E + e * (lc.N - 1) + p - 1] = (int)(lay.off_E + e * (N - 1) + 2 * p - 1);
    for (int64_t f = 0; f < lc.nF; ++f)
      if (!m.face_dirichlet((int)f))
        for (int q = 1; q < lc.N - 1; ++q)
          for (int p = 1; p < lc.N - q; ++p)
            clf[lc.off_F + f * lc.n_face + lin_face(p, q, lc.N)] =
                (int)(lay.off_F + f * lay.n_face + lin_face(2 * p, 2 * q, N));
    s->levels[n - 1].d_coarse_low_fine = upload(A, clf, st);
  }

  // halo copies and work vectors
  L.d_ghost64 = A.alloc_n<double>((size_t)(lay.nC * lay.n_full));
  HHG_CUDA(cudaMemsetAsync(L.d_ghost64, 0, sizeof(double) * lay.nC * lay.n_full, st));
  L.d_r = A.alloc_n<double>((size_t)lay.n_total);
  L.d_tmp = A.alloc_n<double>((size_t)std::max(L.max_step, 1));
  if (n + 2 < s->Lf || n == 0) {
    L.d_u = A.alloc_n<double>((size_t)lay.n_total);
    L.d_f = A.alloc_n<double>((size_t)lay.n_total);
    HHG_CUDA(cudaMemsetAsync(L.d_u, 0, sizeof(double) * lay.n_total, st));
    HHG_CUDA(cudaMemsetAsync(L.d_f, 0, sizeof(double) * lay.n_total, st));
  }
  HHG_CUDA(cudaMemsetAsync(L.d_r, 0, sizeof(double) * lay.n_total, st));
}

template <class T>
static LevelView<T> view(hhg_shell* s, int n);

template <>
LevelView<double> view<double>(hhg_shell* s, int n) {
  Level& L = s->levels[n];
  const LevelLayout& lay = L.lay;
  LevelView<double> v{};
  v.N = L.N; v.nC = (int)lay.nC; v.off_E = lay.off_E; v.off_F = lay.off_F; v.off_C = lay.off_C;
  v.n_total = lay.n_total; v.n_int = lay.n_int; v.n_full = lay.n_full; v.n_bnd = L.n_bnd;
  v.geom = s->d_geom; v.plane_nodes = L.d_plane_nodes; v.plane_off = L.d_plane_off; v.int_ijk = L.d_int_ijk;
  v.plane_x = L.d_plane_x; v.plane_nb = L.d_plane_nb; v.n_plane = L.n_plane;
  v.bnd_ijk = L.d_bnd_ijk; v.bnd_slot = L.d_bnd_slot; v.halo_src = L.d_halo_src; v.ghost = L.d_ghost64;
  v.coef = L.d_coef; v.q = (L.d_coef && L.N >= 8) ? s->q : 0;
  v.plane64 = L.d_plane64; v.cell_e = L.d_cell_e;
  v.colour_nodes = L.d_colour_nodes;
  v.all_nodes = L.d_all_nodes;
  for (int cc = 0; cc < 5; ++cc) v.colour_off[cc] = L.colour_off[cc];
  v.run_nodes = L.d_run_nodes;
  for (int g = 0; g < 6; ++g) v.run_off[g] = L.run_off[g];
  v.run_kidx = L.d_run_kidx;
  v.fp64_kernel = s->fp64_kernel;
  v.sell_ptr = L.d_sell_ptr; v.sell_col = L.d_sell_col; v.sell_val = L.d_sell_val; v.low_diag = L.d_low_diag;
  v.low_perm = L.d_low_perm; v.low_pos = L.d_low_pos;
  v.err = s->d_err;
  v.nrhs = s->nb;
  v.vstride = lay.n_total;
  v.gstride = lay.nC * lay.n_full;
  v.pstride = s->pstride;
  v.tstride = std::max(L.max_step, 1);
  return v;
}

template <>
LevelView<float> view<float>(hhg_shell* s, int n) {
  const LevelView<double> d = view<double>(s, n);
  Level& L = s->levels[n];
  LevelView<float> v{};
  v.N = d.N; v.nC = d.nC; v.off_E = d.off_E; v.off_F = d.off_F; v.off_C = d.off_C;
  v.n_total = d.n_total; v.n_int = d.n_int; v.n_full = d.n_full; v.n_bnd = d.n_bnd;
  v.geom = d.geom; v.plane_nodes = d.plane_nodes; v.plane_off = d.plane_off; v.int_ijk = d.int_ijk;
  v.plane_x = d.plane_x; v.plane_nb = d.plane_nb; v.n_plane = d.n_plane;
  v.bnd_ijk = d.bnd_ijk; v.bnd_slot = d.bnd_slot; v.halo_src = d.halo_src; v.ghost = L.d_ghost32;
  v.coef = L.d_coef32; v.q = d.q; v.plane32 = L.d_plane32;
  v.colour_nodes = d.colour_nodes;
  v.all_nodes = d.all_nodes;
  for (int cc = 0; cc < 5; ++cc) v.colour_off[cc] = d.colour_off[cc];
  v.chunk_nodes = L.d_chunk_nodes;
  for (int cc = 0; cc < 5; ++cc) v.chunk_off[cc] = L.chunk_off[cc];
  for (int cc = 0; cc < 4; ++cc) v.chunk_mid[cc] = L.chunk_mid[cc];
  v.run_nodes = d.run_nodes;
  for (int g = 0; g < 6; ++g) v.run_off[g] = d.run_off[g];
  v.run_kidx = d.run_kidx;
  v.fp64_kernel = d.fp64_kernel;
  v.sell_ptr = d.sell_ptr; v.sell_col = d.sell_col; v.sell_val = L.d_sell_val32; v.low_diag = L.d_low_diag32;
  v.low_perm = d.low_perm; v.low_pos = d.low_pos;
  v.err = d.err;
  v.smooth_cfg = L.tune32 == TUNE_NONE ? -1 : L.tune32;
  v.nrhs = d.nrhs;
  v.vstride = d.vstride;
  v.gstride = d.gstride;
  v.pstride = d.pstride;
  v.tstride = d.tstride;
  return v;
}

// Tuner of the FP32 surrogate smoother: on every fitted level, times the
// per-colour node kernel and each staged configuration that fits (one
// warm-up and three timed cell sweeps each, CUDA events on `st`, on the
// level's own FP32 work vectors) and keeps the fastest.  Runs once the FP32
// buffers exist and again after every fit.
static void tune_smooth32(hhg_shell* s, cudaStream_t st) {
  if (!s->f32_ready || s->q == 0) return;
  cudaEvent_t e0, e1;
  HHG_CUDA(cudaEventCreate(&e0));
  HHG_CUDA(cudaEventCreate(&e1));
  for (size_t n = 0; n < s->levels.size(); ++n) {
    Level& L = s->levels[n];
    if (L.N < 8) continue;
    LevelView<float> v = view<float>(s, (int)n);
    v.nrhs = 1;
    float best_ms = 0.0f;
    int best = -1;
    for (int cfg = -2; cfg < SMOOTH32_CONFIGS; ++cfg) {
      L.tune32_ms[cfg + 2] = -1.0;
      if (cfg >= 0 && !smooth32_supported(v, L.d_u32, cfg)) continue;
      v.smooth_cfg = cfg;
      launch_cell(v, HHG_OP_LSQP, SMOOTH, L.d_u32, L.d_u32, (const float*)L.d_f32, nullptr, st);
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        HHG_CUDA(cudaEventRecord(e0, st));
        launch_cell(v, HHG_OP_LSQP, SMOOTH, L.d_u32, L.d_u32, (const float*)L.d_f32, nullptr, st);
        HHG_CUDA(cudaEventRecord(e1, st));
        HHG_CUDA(cudaEventSynchronize(e1));
        float t = 0.0f;
        HHG_CUDA(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t);
      }
      L.tune32_ms[cfg + 2] = ms;
      if (best_ms == 0.0f || ms < best_ms) {
        best_ms = ms;
        best = cfg;
      }
    }
    L.tune32 = best;
  }
  ++s->gen;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timed sweeps ran on the work vectors: clear them again
  for (auto& L : s->levels) {
    HHG_CUDA(cudaMemsetAsync(L.d_u32, 0, sizeof(float) * L.lay.n_total, st));
    HHG_CUDA(cudaMemsetAsync(L.d_f32, 0, sizeof(float) * L.lay.n_total, st));
  }
  HHG_CUDA(cudaStreamSynchronize(st));
  check_device_error(s, st);
}

// FP32 buffers of every level, allocated on the first FP32 call: halo
// copies, work vectors and FP32 copies of the lower-primitive rows.
static void ensure_f32(hhg_shell* s, cudaStream_t st) {
  if (s->f32_ready) return;
  Allocator& A = s->alloc;
  const int64_t cap = s->cap;
  for (auto& L : s->levels) {
    const LevelLayout& lay = L.lay;
    L.d_ghost32 = A.alloc_n<float>((size_t)(cap * lay.nC * lay.n_full));
    HHG_CUDA(cudaMemsetAsync(L.d_ghost32, 0, sizeof(float) * cap * lay.nC * lay.n_full, st));
    for (float** v : {&L.d_u32, &L.d_f32, &L.d_r32}) {
      *v = A.alloc_n<float>((size_t)(cap * lay.n_total));
      HHG_CUDA(cudaMemsetAsync(*v, 0, sizeof(float) * cap * lay.n_total, st));
    }
    L.d_tmp32 = A.alloc_n<float>((size_t)(cap * std::max(L.max_step, 1)));
    int64_t nsell = 0;
    HHG_CUDA(cudaMemcpyAsync(&nsell, L.d_sell_ptr + L.n_slices, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    HHG_CUDA(cudaStreamSynchronize(st));
    L.d_sell_val32 = A.alloc_n<float>((size_t)std::max<int64_t>(nsell, 1));
    L.d_low_diag32 = A.alloc_n<float>((size_t)std::max<int64_t>(lay.off_C, 1));
    launch_copy_cast<float>(L.d_sell_val, L.d_sell_val32, nsell, st);
    launch_copy_cast<float>(L.d_low_diag, L.d_low_diag32, lay.off_C, st);
  }
  HHG_CUDA(cudaStreamSynchronize(st));
  s->f32_ready = true;
  ++s->gen;
  tune_smooth32(s, st);
}

template <class T>
static T* step_tmp(Level& L);
template <>
double* step_tmp<double>(Level& L) { return L.d_tmp; }
template <>
float* step_tmp<float>(Level& L) { return L.d_tmp32; }

// ---------------------------------------------------------------------------
// diagnostics: CUDA events around the finest-level cell kernels
// ---------------------------------------------------------------------------

struct TimedScope {
  hhg_shell* s;
  int which;
  cudaStream_t st;
  cudaEvent_t b = nullptr, e = nullptr;
  // n = level index, or -1 for classes timed on every level
  // while a V-cycle is captured the events become event-record nodes of the
  // graph (external record), re-recorded by every replay
  TimedScope(hhg_shell* s_, int n, int which_, cudaStream_t st_) : s(s_), which(which_), st(st_) {
    if (!s->timing || (n >= 0 && n != (int)s->levels.size() - 1)) return;
    HHG_CUDA(cudaEventCreate(&b));
    HHG_CUDA(cudaEventCreate(&e));
    HHG_CUDA(cudaEventRecordWithFlags(b, st, s->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  }
  ~TimedScope() {
    if (!b) return;
    cudaEventRecordWithFlags(e, st, s->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    if (s->capturing) s->gtimed.emplace_back(which, b, e);  // an event-record node pair of the graph
    else s->tevents[which].push_back({b, e});
  }
};

static void graph_timed_clear(hhg_shell* s) {
  for (auto& t : s->gtimed) {
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  s->gtimed.clear();
}

// After a graph replay has completed: adds its timed scopes to the totals.
static void graph_timed_accumulate(hhg_shell* s) {
  if (!s->timing) return;
  for (auto& t : s->gtimed) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)) != cudaSuccess) {
      cudaGetLastError();  // timings of graph replays unavailable: the totals cover the launched cycles only
      continue;
    }
    s->gsum[std::get<0>(t)] += ms;
    s->gcnt[std::get<0>(t)] += 1;
  }
  s->cg_iters += s->cg_graph_iters;  // the replayed cycle's coarse solve
}

static void timing_clear(hhg_shell* s) {
  s->cg_iters = 0;
  for (int t = 0; t < HHG_T_COUNT; ++t) {
    s->gsum[t] = 0.0;
    s->gcnt[t] = 0;
  }
  for (auto& v : s->tevents) {
    for (auto& p : v) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    v.clear();
  }
}

// ---------------------------------------------------------------------------
// operators on one level (device vectors, FP64)
// ---------------------------------------------------------------------------

static void check_op(hhg_shell* s, int n, int op) {
  HHG_CHECK(op == HHG_OP_IFEM || op == HHG_OP_LSQP || op == HHG_OP_DD, HHG_EINVAL, "unknown operator");
  if (op != HHG_OP_IFEM && s->levels[n].N >= 8)
    HHG_CHECK(s->levels[n].d_coef != nullptr, HHG_ENOTFIT, "LSQP requested before hhg_fit_surrogate");
}

// Kernels of an operator choice: double discretisation (Sec. 4.1) relaxes
// with the fitted surrogate and computes residuals (and applies) with the
// exact stencils.
static int smooth_op(int op) { return op == HHG_OP_DD ? HHG_OP_LSQP : op; }
static int exact_op(int op) { return op == HHG_OP_DD ? HHG_OP_IFEM : op; }
static int eff_op(hhg_shell* s, int n, int op) { return (s->levels[n].N >= 8) ? op : HHG_OP_IFEM; }

template <class T = double>
static void op_apply(hhg_shell* s, int n, int op, const T* u, T* y, cudaStream_t st) {
  LevelView<T> v = view<T>(s, n);
  launch_halo(v, u, st);
  {
    TimedScope ts(s, n, HHG_T_CELL_APPLY, st);
    launch_cell(v, eff_op(s, n, exact_op(op)), APPLY, const_cast<T*>(u), y, (const T*)nullptr, nullptr, st);
  }
  launch_low(v, APPLY, u, y, (const T*)nullptr, nullptr, low_blocks(v.off_C), st);
}

// Reduction scratch: 64 scalar slots of `cap` entries (slot k, right-hand
// side b at d_red[k cap + b]), then `cap` blocks of pstride partial sums.
static double* scal(hhg_shell* s, int slot) { return s->d_red + (int64_t)slot * s->cap; }
static double* parts(hhg_shell* s) { return s->d_red + 64 * (int64_t)s->cap; }

// r = f - L u for the active right-hand sides; the squared norms land in
// scalar slot `slot` (device).
template <class T = double>
static void op_residual(hhg_shell* s, int n, int op, const T* u, const T* f, T* r, int slot, cudaStream_t st) {
  TimedScope all(s, -1, HHG_T_RESIDUAL, st);
  LevelView<T> v = view<T>(s, n);
  const int nb = low_blocks(v.off_C);
  double* part = parts(s);
  launch_halo(v, u, st);
  {
    TimedScope ts(s, n, HHG_T_CELL_RESIDUAL, st);
    launch_cell(v, eff_op(s, n, exact_op(op)), RESIDUAL, const_cast<T*>(u), r, f, part, st);
  }
  launch_low(v, RESIDUAL, u, r, f, part + v.nC, nb, st);
  launch_sum(part, v.nC + nb, v.nrhs, v.pstride, scal(s, slot), st);
}

template <class T = double>
static void op_smooth(hhg_shell* s, int n, int op, const T* f, T* u, cudaStream_t st) {
  TimedScope all(s, -1, HHG_T_SMOOTH, st);
  LevelView<T> v = view<T>(s, n);
  Level& L = s->levels[n];
  for (int t = 0; t < 6; ++t) launch_low_step(v, L.step_beg[t], L.step_n[t], u, f, step_tmp<T>(L), st);
  launch_halo(v, (const T*)u, st);
  TimedScope ts(s, n, HHG_T_CELL_SMOOTH, st);
  launch_cell(v, eff_op(s, n, smooth_op(op)), SMOOTH, u, u, f, nullptr, st);
}

// Reports (and clears) a bounded device-side wait that gave up since the
// last check (the staged kernels set the shell's error word).
// Word 1 of the error word is soft: a coarse solve inside a captured
// V-cycle stopped at its fixed iteration count before the tolerance; the
// next capture doubles the count (the cycle's correction is still valid).
static void check_device_error(hhg_shell* s, cudaStream_t st) {
  int e[2] = {0, 0};
  HHG_CUDA(cudaMemcpyAsync(e, s->d_err, sizeof(e), cudaMemcpyDeviceToHost, st));
  HHG_CUDA(cudaStreamSynchronize(st));
  if (e[1] != 0) {
    HHG_CUDA(cudaMemsetAsync(s->d_err + 1, 0, sizeof(int), st));
    s->cg_graph_iters *= 2;
  }
  if (e[0] != 0) {
    HHG_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
    throw Error{HHG_ETIMEOUT, "a bounded device-side wait gave up (shared-memory staging did not complete)"};
  }
}

// The active right-hand sides' entries of a scalar slot (waits for the stream).
static std::vector<double> read_scalars(hhg_shell* s, int slot, cudaStream_t st) {
  std::vector<double> h((size_t)s->nb);
  HHG_CUDA(cudaMemcpyAsync(h.data(), scal(s, slot), sizeof(double) * s->nb, cudaMemcpyDeviceToHost, st));
  HHG_CUDA(cudaStreamSynchronize(st));
  return h;
}

// Coarsest level (N = 4): Jacobi-preconditioned conjugate gradients on the
// exact, symmetric operator, pre-assembled at setup (coarse.cu), to
// ||r|| <= 1e-13 ||f|| (the paper uses Gauss-Seidel as coarse solver, Sec. 4;
// an exact solve keeps the cycle independent of that choice).
static void coarse_solve(hhg_shell* s, const double* f, double* x, cudaStream_t st) {
  TimedScope all(s, -1, HHG_T_COARSE, st);
  const CoarseOp& A = *static_cast<CoarseOp*>(s->coarse_op);
  const int64_t n = A.n_total, cap = s->cap;
  double* r = s->d_cg;
  double* z = r + n * cap;
  double* p = z + n * cap;
  double* q = p + n * cap;
  double* part = parts(s);  // 3 CG_BLOCKS partials per right-hand side (pstride >= 3 CG_BLOCKS)
  // scalar slots: 0, 1 = r.z (double-buffered), 2 = r.r, 3 = r0.r0,
  // 4, 5 = r.r double-buffered for fixed-count iterations
  launch_cg_init(A, f, x, r, z, p, part, scal(s, 0), scal(s, 3), s->nb, st);
  if (s->cg_fixed > 0) {
    // no host reads (inside a graph): a fixed number of iterations, each
    // skipping the right-hand sides that have converged
    HHG_CUDA(cudaMemcpyAsync(scal(s, 4), scal(s, 3), sizeof(double) * s->nb, cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < s->cg_fixed; ++it)
      launch_cg_iteration(A, x, r, z, p, q, part, scal(s, it & 1), scal(s, (it + 1) & 1), scal(s, 4 + ((it + 1) & 1)),
                          s->nb, st, scal(s, 4 + (it & 1)), scal(s, 3));
    launch_cg_check(scal(s, 4 + (s->cg_fixed & 1)), scal(s, 3), s->nb, s->d_err + 1, st);
    return;
  }
  const std::vector<double> ff = read_scalars(s, 3, st);
  bool zero = true;
  for (double v : ff) zero = zero && v == 0.0;
  if (zero) return;
  for (int it = 0; it < 20000; ++it) {
    ++s->cg_iters;
    launch_cg_iteration(A, x, r, z, p, q, part, scal(s, it & 1), scal(s, (it + 1) & 1), scal(s, 2), s->nb, st);
    if ((it & 7) == 7) {
      const std::vector<double> rr = read_scalars(s, 2, st);
      bool done = true;
      for (int b = 0; b < s->nb; ++b) {
        if (!std::isfinite(rr[b])) throw Error{HHG_EDIVERGED, "coarse solve diverged"};
        done = done && rr[b] <= 1e-26 * ff[b];
      }
      if (done) {
        s->cg_last = it + 1;
        return;
      }
    }
  }
  throw Error{HHG_ENOCONV, "coarse solve did not reach its tolerance"};
}

static void vcycle_rec(hhg_shell* s, int n, int op, const double* f, double* u, int nu1, int nu2, cudaStream_t st) {
  if (n == 0) {
    coarse_solve(s, f, u, st);
    return;
  }
  Level& L = s->levels[n];
  Level& C = s->levels[n - 1];
  for (int t = 0; t < nu1; ++t) op_smooth(s, n, op, f, u, st);
  op_residual(s, n, op, u, f, L.d_r, 8, st);
  LevelView<double> vf = view<double>(s, n), vc = view<double>(s, n - 1);
  {
    TimedScope tr(s, -1, HHG_T_TRANSFER, st);
    launch_restrict(vf, vc, C.d_coarse_low_fine, (const double*)L.d_r, C.d_f, st);
  }
  HHG_CUDA(cudaMemsetAsync(C.d_u, 0, sizeof(double) * C.lay.n_total * s->nb, st));
  vcycle_rec(s, n - 1, op, C.d_f, C.d_u, nu1, nu2, st);
  {
    TimedScope tr(s, -1, HHG_T_TRANSFER, st);
    launch_halo(vc, (const double*)C.d_u, st);
    launch_prolong_add(vf, vc, L.d_low_par, (const double*)C.d_u, u, st);
  }
  for (int t = 0; t < nu2; ++t) op_smooth(s, n, op, f, u, st);
}

// The inner cycle of the mixed-precision solve: the same V-cycle in FP32 on
// levels N >= 8 (smoothing, residual, transfers), the FP64 coarse solve on
// N = 4 (FP32 right-hand side widened, solution narrowed).
static void vcycle_rec32(hhg_shell* s, int n, int op, const float* f, float* u, int nu1, int nu2, cudaStream_t st) {
  if (n == 0) {
    Level& C = s->levels[0];
    launch_widen(f, C.d_f, C.lay.n_total * s->nb, false, st);
    coarse_solve(s, C.d_f, C.d_u, st);
    launch_copy_cast<float>(C.d_u, u, C.lay.n_total * s->nb, st);
    return;
  }
  Level& L = s->levels[n];
  Level& C = s->levels[n - 1];
  for (int t = 0; t < nu1; ++t) op_smooth<float>(s, n, op, f, u, st);
  op_residual<float>(s, n, op, u, f, L.d_r32, 8, st);
  LevelView<float> vf = view<float>(s, n), vc = view<float>(s, n - 1);
  {
    TimedScope tr(s, -1, HHG_T_TRANSFER, st);
    launch_restrict(vf, vc, C.d_coarse_low_fine, (const float*)L.d_r32, C.d_f32, st);
  }
  HHG_CUDA(cudaMemsetAsync(C.d_u32, 0, sizeof(float) * C.lay.n_total * s->nb, st));
  vcycle_rec32(s, n - 1, op, C.d_f32, C.d_u32, nu1, nu2, st);
  {
    TimedScope tr(s, -1, HHG_T_TRANSFER, st);
    launch_halo(vc, (const float*)C.d_u32, st);
    launch_prolong_add(vf, vc, L.d_low_par, (const float*)C.d_u32, u, st);
  }
  for (int t = 0; t < nu2; ++t) op_smooth<float>(s, n, op, f, u, st);
}

// ---------------------------------------------------------------------------
// surrogate fit
// ---------------------------------------------------------------------------

// ipoly = false: LSQP on S_l = M_{m(l,j)} (Sec. 3.2); ipoly = true: IPOLY
// (Sec. 3.1), interpolation at the m_q nodes of degree q of the macro cell
// shrunk to its interior (for q = 2 the ten points a = N - 3, b = N/2 - 1;
// the square system is solved by the same QR).  unprojected = true samples the stencils of the
// unprojected domain (Phi = Id; constant per cell, so every degree
// reproduces them): the cell-interior rows of the CONS operator (Sec. 4.1).
static void fit(hhg_shell* s, int q, int j, cudaStream_t st, bool ipoly = false, bool unprojected = false) {
  TimedScope all(s, -1, HHG_T_FIT, st);
  const int mq = n_coeffs(q);
  const int64_t nC = s->levels.empty() ? 0 : s->levels[0].lay.nC;
  CellGeom* d_geom_sample = s->d_geom;
  if (unprojected) {  // the cells' geometry with the radii flagged negative (Phi = Id)
    std::vector<CellGeom> g((size_t)nC);
    HHG_CUDA(cudaMemcpyAsync(g.data(), s->d_geom, g.size() * sizeof(CellGeom), cudaMemcpyDeviceToHost, st));
    HHG_CUDA(cudaStreamSynchronize(st));
    for (CellGeom& c : g)
      for (double& r : c.r) r = -std::fabs(r);
    d_geom_sample = upload(s->alloc, g, st);
  }
  for (size_t n = 0; n < s->levels.size(); ++n) {
    Level& L = s->levels[n];
    const int N = L.N;
    if (N < 8) continue;
    const int l = (int)n;  // paper level: N = 2^(l+2)
    std::vector<uint32_t> pts;
    if (ipoly && q == 2) {
      const int a = N - 3, b = N / 2 - 1;
      const int P[10][3] = {{1, 1, 1}, {1, 1, a}, {1, a, 1}, {a, 1, 1}, {1, 1, b},
                            {1, b, 1}, {b, 1, 1}, {1, b, b}, {b, 1, b}, {b, b, 1}};
      for (auto& p : P) pts.push_back(pack_ijk(p[0], p[1], p[2]));
    } else if (ipoly) {
      // the nodes of degree q of the shrunk cell, (1,1,1) + (N-4)(a,b,c)/q,
      // each coordinate rounded to the nearest fine node where (N-4)/q is
      // not an integer
      auto node = [&](int x) { return (int)std::floor(1.0 + (double)(N - 4) * x / q + 0.5); };
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= q - a; ++b)
          for (int c = 0; c <= q - a - b; ++c) pts.push_back(pack_ijk(node(a), node(b), node(c)));
    } else {
      const int mlev = std::min(l, std::max(1, j));
      const int Nm = 4 << mlev, scale = 1 << (l - mlev);
      for (int k = 1; k < Nm; ++k)
        for (int jj = 1; jj < Nm - k; ++jj)
          for (int i = 1; i < Nm - jj - k; ++i) pts.push_back(pack_ijk(i * scale, jj * scale, k * scale));
    }
    const int np = (int)pts.size();
    // sampling matrix in the line-form monomial order (a, d, b): xi^a eta^b zeta^d
    std::vector<double> Am((size_t)np * mq), sc(mq);
    {
      int t = 0;
      for (int a = 0; a <= q; ++a)
        for (int d = 0; d <= q - a; ++d)
          for (int b = 0; b <= q - a - d; ++b) {
            sc[t] = std::ldexp(1.0, -(a + b + d) * (l + 2));  // 1 / N^(a+b+d)
            for (int p = 0; p < np; ++p) {
              const double x = (double)unpack_i(pts[p]) / N, y = (double)unpack_j(pts[p]) / N,
                           z = (double)unpack_k(pts[p]) / N;
              Am[(size_t)p * mq + t] = std::pow(x, a) * std::pow(y, b) * std::pow(z, d);
            }
            ++t;
          }
    }
    const std::vector<double> P = lsq_pinv(Am, np, mq);
    Allocator& A = s->alloc;
    uint32_t* d_pts = upload(A, pts, st);
    double* d_P = upload(A, P, st);
    double* d_sc = upload(A, sc, st);
    const size_t ncoef = (size_t)L.lay.nC * 15 * mq;
    const size_t nplane64 = (size_t)plane64_len(L.lay.nC, N, q);
    if (s->q != q || !L.d_coef) {  // (re)allocate only when the degree changes
      for (void* p : {(void*)L.d_coef, (void*)L.d_coef32, (void*)L.d_plane64, (void*)L.d_cell_e, (void*)L.d_plane32})
        A.release(p);
      L.d_plane32 = A.alloc_n<float>((size_t)plane_table_len((int)L.lay.nC, N, q));
      L.d_coef = A.alloc_n<double>(ncoef);
      L.d_coef32 = A.alloc_n<float>(ncoef);
      L.d_plane64 = A.alloc_n<long long>(nplane64);
      L.d_cell_e = A.alloc_n<int>((size_t)L.lay.nC);
    }
    // sample in chunks of cells so the sample buffer stays below ~1 GB
    const int64_t per_cell = (int64_t)np * 14;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(L.lay.nC, (int64_t)(1 << 27) / per_cell));
    double* d_b = A.alloc_n<double>((size_t)chunk * per_cell);
    LevelView<double> v = view<double>(s, (int)n);
    for (int c0 = 0; c0 < L.lay.nC; c0 += chunk) {
      const int nc = (int)std::min<int64_t>(chunk, L.lay.nC - c0);
      LevelView<double> vc = v;
      vc.geom = d_geom_sample + c0;
      vc.nC = nc;
      launch_sample(vc, d_pts, np, d_b, st);
      launch_fit_coef(nc, mq, np, d_P, d_sc, d_b, L.d_coef + (int64_t)c0 * 15 * mq, L.d_coef32 + (int64_t)c0 * 15 * mq,
                      st);
    }
    launch_plane64_table(v, q, L.d_coef, L.d_cell_e, L.d_plane64, st);
    launch_plane_table(v, q, L.d_coef, L.d_plane32, st);
    HHG_CUDA(cudaStreamSynchronize(st));
    A.release(d_b);
    A.release(d_pts);
    A.release(d_P);
    A.release(d_sc);
  }
  if (unprojected) s->alloc.release(d_geom_sample);
  s->q = q;
  s->j = ipoly ? 0 : j;
  ++s->gen;
  s->cg_graph_iters = 0;
  tune_smooth32(s, st);
}

// ---------------------------------------------------------------------------
// argument helpers
// ---------------------------------------------------------------------------

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Device view of a (possibly host) vector argument of n doubles.
struct Arg {
  const void* user;
  double* dev;   // device address (of doubles or floats, see elem)
  bool host;
  size_t elem;
  float* dev32() const { return reinterpret_cast<float*>(dev); }
};

static Arg stage_in(hhg_shell* s, int slot, const void* p, int64_t n, bool copy, cudaStream_t st,
                    size_t elem = sizeof(double)) {
  HHG_CHECK(p != nullptr, HHG_EINVAL, "NULL vector argument");
  Arg a{p, (double*)p, is_host_ptr(p), elem};
  if (a.host) {
    if (s->stage_len < n) {
      for (auto& d : s->d_stage) { s->alloc.release(d); d = nullptr; }
      s->stage_len = 0;
      for (auto& d : s->d_stage) d = s->alloc.alloc_n<double>((size_t)n);
      s->stage_len = n;
    }
    a.dev = s->d_stage[slot];
    if (copy) HHG_CUDA(cudaMemcpyAsync(a.dev, p, elem * n, cudaMemcpyHostToDevice, st));
  }
  return a;
}

static void stage_out(const Arg& a, int64_t n, cudaStream_t st) {
  if (a.host) {
    HHG_CUDA(cudaMemcpyAsync(const_cast<void*>(a.user), a.dev, a.elem * n, cudaMemcpyDeviceToHost, st));
    HHG_CUDA(cudaStreamSynchronize(st));
  }
}

static int level_index(hhg_shell* s, int L) {
  HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
  HHG_CHECK(L >= 2 && L <= s->Lf, HHG_EINVAL, "level out of range");
  return L - 2;
}

template <class F>
static hhg_status guarded(F&& fn) {
  try {
    fn();
    set_error("");
    return HHG_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return HHG_ENOMEM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HHG_EINVAL;
  }
}

}  // namespace hhg

using namespace hhg;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* hhg_last_error(void) { return g_last_error.c_str(); }

int64_t hhg_launch_count(void) { return g_launches.load(); }

hhg_status hhg_timing(hhg_shell* s, int enable) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    if (!enable) timing_clear(s);
    if (s->timing != (enable != 0)) ++s->gen;  // a captured cycle holds (or lacks) the timers' events
    s->timing = enable != 0;
  });
}

hhg_status hhg_timing_read(hhg_shell* s, int which, double* total_ms, int64_t* launches) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    HHG_CHECK(which >= 0 && which < HHG_T_COUNT, HHG_EINVAL, "unknown timer");
    double tot = 0;
    for (auto& p : s->tevents[which]) {
      HHG_CUDA(cudaEventSynchronize(p.second));
      float ms = 0;
      HHG_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
      tot += ms;
    }
    tot += s->gsum[which];
    if (total_ms) *total_ms = tot;
    if (launches)
      *launches = which == HHG_T_COARSE ? s->cg_iters : (int64_t)s->tevents[which].size() + s->gcnt[which];
  });
}

static hhg_status setup_shells(const hhg_shell_desc* d, int count, void* stream, hhg_shell** out);

hhg_status hhg_setup_shell(const hhg_shell_desc* d, void* stream, hhg_shell** out) {
  return setup_shells(d, 1, stream, out);
}

hhg_status hhg_setup_shells(const hhg_shell_desc* d, int count, void* stream, hhg_shell** out) {
  return setup_shells(d, count, stream, out);
}

hhg_status hhg_shell_part(const hhg_shell* s, int L, int k, int64_t* start, int64_t* count) {
  return guarded([&] {
    const int n = level_index(const_cast<hhg_shell*>(s), L);
    HHG_CHECK(k >= 0 && k < s->n_parts, HHG_EINVAL, "shell index out of range");
    const LevelLayout& lay = s->levels[n].lay;
    const int64_t per_e = lay.N - 1, per_f = lay.n_face, per_c = lay.n_int;
    // every shell of the group has the same numbers of macro vertices, edges,
    // faces and cells; its primitives follow those of the shells before it
    const int64_t nV = lay.nV / s->n_parts, nE = lay.nE / s->n_parts, nF = lay.nF / s->n_parts,
                  nC = lay.nC / s->n_parts;
    const int64_t st4[4] = {k * nV, lay.off_E + k * nE * per_e, lay.off_F + k * nF * per_f, lay.off_C + k * nC * per_c};
    const int64_t ct4[4] = {nV, nE * per_e, nF * per_f, nC * per_c};
    for (int t = 0; t < 4; ++t) {
      if (start) start[t] = st4[t];
      if (count) count[t] = ct4[t];
    }
  });
}

static hhg_status setup_shells(const hhg_shell_desc* dd, int count, void* stream, hhg_shell** out) {
  return guarded([&] {
    HHG_CHECK(dd && out && count >= 1, HHG_EINVAL, "NULL argument or empty group");
    const hhg_shell_desc* d = dd;
    std::vector<std::pair<double, double>> radii;
    for (int k = 0; k < count; ++k) {
      const hhg_shell_desc& e = dd[k];
      HHG_CHECK(e.r_inner > 0 && e.r_outer > e.r_inner, HHG_EINVAL, "need 0 < r_inner < r_outer");
      HHG_CHECK(e.tang_refine == d->tang_refine && e.radial_layers == d->radial_layers &&
                    e.fine_log2_intervals == d->fine_log2_intervals && e.unprojected == d->unprojected,
                HHG_EINVAL, "the shells of a group must share tang_refine, radial_layers and the level");
      radii.push_back({e.r_inner, e.r_outer});
    }
    HHG_CHECK(d->tang_refine >= 0 && d->tang_refine <= 6, HHG_EINVAL, "tang_refine out of range");
    HHG_CHECK(d->radial_layers >= 1 && d->radial_layers <= 4096, HHG_EINVAL, "radial_layers out of range");
    HHG_CHECK(d->fine_log2_intervals >= 2 && d->fine_log2_intervals <= 10, HHG_EINVAL, "level out of range");
    *out = nullptr;
    Star star;
    kuhn_star(&star);
    for (int t = 0; t < 24; ++t)
      for (int a = 0; a < 3; ++a)
        HHG_CHECK(star.t[t][a] == hhg::star(t, a), HHG_EINVAL, "internal star table mismatch");
    cudaStream_t st = (cudaStream_t)stream;
    hhg_shell* s = new hhg_shell();
    try {
      s->alloc.budget = d->hbm_budget_bytes;
      s->mesh = build_shells(radii, d->tang_refine, d->radial_layers);
      s->mesh.blend = d->unprojected == 0;
      s->n_parts = count;
      s->Lf = d->fine_log2_intervals;
      std::vector<CellGeom> geom(s->mesh.nC());
      for (int c = 0; c < s->mesh.nC(); ++c)
        for (int a = 0; a < 4; ++a) {
          const int v = s->mesh.cells[c][a];
          for (int x = 0; x < 3; ++x) geom[c].x[a][x] = s->mesh.vx[v][x];
          geom[c].r[a] = s->mesh.blend ? s->mesh.vr[v] : -1.0;  // negative: no blending
        }
      s->d_geom = upload(s->alloc, geom, st);
      HHG_CUDA(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
      for (cudaEvent_t& e : s->gev) HHG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      s->d_err = s->alloc.alloc_n<int>(4);
      HHG_CUDA(cudaMemsetAsync(s->d_err, 0, 4 * sizeof(int), st));
      s->levels.resize(s->Lf - 1);
      for (int n = 0; n < (int)s->levels.size(); ++n) build_level(s, n, st);
      // reduction scratch: 64 scalar slots, then partial sums (per-cell and
      // per-block residual partials, or the coarse solver's 3 CG_BLOCKS)
      int64_t ps = 3 * CG_BLOCKS;
      for (auto& L : s->levels) ps = std::max<int64_t>(ps, L.lay.nC + low_blocks(L.lay.off_C));
      s->pstride = (int)ps;
      s->red_len = 64 + ps;
      s->d_red = s->alloc.alloc_n<double>((size_t)s->red_len);
      HHG_CUDA(cudaMemsetAsync(s->d_red, 0, sizeof(double) * s->red_len, st));
      {
        const Level& L0 = s->levels[0];
        const int64_t n0 = L0.lay.n_total;
        s->d_cg = s->alloc.alloc_n<double>((size_t)(4 * n0));
        double* dinv = s->alloc.alloc_n<double>((size_t)n0);
        CoarseOp* A = new CoarseOp{};
        s->coarse_op = A;
        A->n_total = n0;
        A->off_C = L0.lay.off_C;
        A->nC = (int)L0.lay.nC;
        A->sell_ptr = L0.d_sell_ptr;
        A->low_pos = L0.d_low_pos;
        A->sell_col = L0.d_sell_col;
        A->sell_val = L0.d_sell_val;
        A->low_diag = L0.d_low_diag;
        int* col = s->alloc.alloc_n<int>((size_t)(14 * L0.lay.nC));
        double* val = s->alloc.alloc_n<double>((size_t)(14 * L0.lay.nC));
        double* diag = s->alloc.alloc_n<double>((size_t)L0.lay.nC);
        launch_coarse_setup(view<double>(s, 0), *A, col, val, diag, dinv, st);
      }
      HHG_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      if (s->gstream) cudaStreamDestroy(s->gstream);
      for (cudaEvent_t e : s->gev)
        if (e) cudaEventDestroy(e);
      s->alloc.release_all();
      delete static_cast<CoarseOp*>(s->coarse_op);
      delete s;
      throw;
    }
    *out = s;
  });
}

hhg_status hhg_destroy(hhg_shell* s) {
  return guarded([&] {
    if (!s) return;
    cudaDeviceSynchronize();
    timing_clear(s);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    graph_timed_clear(s);
    s->d_uprev = nullptr;
    if (s->gstream) cudaStreamDestroy(s->gstream);
    for (cudaEvent_t e : s->gev)
      if (e) cudaEventDestroy(e);
    delete static_cast<CoarseOp*>(s->coarse_op);
    s->alloc.release_all();
    delete s;
  });
}

hhg_status hhg_tuning(const hhg_shell* s, int L, int* cfg, double* ms) {
  return guarded([&] {
    const int n = level_index(const_cast<hhg_shell*>(s), L);
    const Level& Lv = s->levels[n];
    if (cfg) *cfg = Lv.tune32;
    if (ms)
      for (int t = 0; t < 2 + SMOOTH32_CONFIGS; ++t) ms[t] = Lv.tune32 == TUNE_NONE ? -1.0 : Lv.tune32_ms[t];
  });
}

hhg_status hhg_set_graphs(hhg_shell* s, int enable) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    s->graphs = enable != 0;
  });
}

hhg_status hhg_set_tuning(hhg_shell* s, int L, int cfg) {
  return guarded([&] {
    const int n = level_index(s, L);
    HHG_CHECK(cfg >= -2 && cfg < SMOOTH32_CONFIGS, HHG_EINVAL, "unknown smoother configuration");
    s->levels[n].tune32 = cfg;
    ++s->gen;
  });
}

hhg_status hhg_set_fp64_kernel(hhg_shell* s, int variant) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    HHG_CHECK(variant == FP64_NODES || variant == FP64_RUNS || variant == FP64_RESIDENT, HHG_EINVAL,
              "unknown FP64 kernel variant");
    s->fp64_kernel = variant;
    ++s->gen;
  });
}

hhg_status hhg_run_lists(int N, uint32_t* items, int64_t cap, int* off6, int* kidx, int64_t* n_items) {
  return guarded([&] {
    HHG_CHECK(N >= 4 && N <= 1023 && off6 != nullptr, HHG_EINVAL, "need 4 <= N <= 1023 and off6");
    std::vector<uint2> runs;
    std::vector<int> kx;
    build_run_lists(N, runs, off6, kx);
    if (n_items) *n_items = (int64_t)runs.size();
    if (items) {
      HHG_CHECK(cap >= (int64_t)runs.size(), HHG_EINVAL, "run-list buffer too small");
      for (size_t t = 0; t < runs.size(); ++t) {
        items[2 * t] = runs[t].x;
        items[2 * t + 1] = runs[t].y;
      }
    }
    if (kidx) std::copy(kx.begin(), kx.end(), kidx);
  });
}

hhg_status hhg_slab_planes(int N, int cluster, int* k_bounds) {
  return guarded([&] {
    HHG_CHECK(N >= 8 && N <= 1023 && cluster >= 1 && cluster <= 8 && k_bounds != nullptr, HHG_EINVAL,
              "need 8 <= N <= 1023, 1 <= cluster <= 8 and k_bounds");
    resident_slab_planes(N, cluster, k_bounds);
  });
}

hhg_status hhg_fp64_kernel(hhg_shell* s, int L, int* variant, int* cluster) {
  return guarded([&] {
    const int n = level_index(s, L);
    if (variant) *variant = s->fp64_kernel;
    if (cluster) {
      LevelView<double> v = view<double>(s, n);
      v.nrhs = 1;
      *cluster = s->fp64_kernel == FP64_RESIDENT ? resident_cluster_size(v) : 0;
    }
  });
}

hhg_status hhg_num_nodes(const hhg_shell* s, int L, int64_t* n_total, int64_t* n_free) {
  return guarded([&] {
    const int n = level_index(const_cast<hhg_shell*>(s), L);
    if (n_total) *n_total = s->levels[n].lay.n_total;
    if (n_free) *n_free = s->levels[n].n_free;
  });
}

hhg_status hhg_node_coords(const hhg_shell* s, int L, double* xyz) {
  return guarded([&] {
    const int n = level_index(const_cast<hhg_shell*>(s), L);
    HHG_CHECK(xyz != nullptr, HHG_EINVAL, "NULL output");
    level_coords(s->mesh, s->levels[n].lay, xyz);
  });
}

hhg_status hhg_fit_ipoly(hhg_shell* s, void* stream) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    fit(s, 2, 0, (cudaStream_t)stream, true);
  });
}

hhg_status hhg_fit_ipoly_degree(hhg_shell* s, int q, void* stream) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    HHG_CHECK(q >= 1 && q <= 3, HHG_EINVAL, "q must be 1, 2 or 3");
    fit(s, q, 0, (cudaStream_t)stream, true);
  });
}

hhg_status hhg_fit_cons(hhg_shell* s, int q, int j, void* stream) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    HHG_CHECK(q >= 1 && q <= 3, HHG_EINVAL, "q must be 1, 2 or 3");
    HHG_CHECK(j >= 1, HHG_EINVAL, "j must be >= 1");
    fit(s, q, j, (cudaStream_t)stream, false, true);
  });
}

hhg_status hhg_fit_surrogate(hhg_shell* s, int q, int j, void* stream) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    HHG_CHECK(q >= 1 && q <= 3, HHG_EINVAL, "q must be 1, 2 or 3");
    HHG_CHECK(j >= 1, HHG_EINVAL, "j must be >= 1");
    fit(s, q, j, (cudaStream_t)stream);
  });
}

static void check_common(hhg_shell* s, int n, int op, int dtype, int nrhs) {
  HHG_CHECK(dtype == HHG_F64 || dtype == HHG_F32, HHG_EINVAL, "dtype must be HHG_F64 or HHG_F32");
  HHG_CHECK(nrhs >= 1, HHG_EINVAL, "nrhs must be >= 1");
  check_op(s, n, op);
}

// Grows every per-right-hand-side buffer of the shell (halo copies, work
// vectors, step buffers, reduction and coarse-solver scratch) to hold nrhs
// vectors.  Contents are not kept: every operation initialises what it reads.
static void ensure_cap(hhg_shell* s, int nrhs, cudaStream_t st) {
  if (nrhs <= s->cap) return;
  HHG_CUDA(cudaStreamSynchronize(st));
  Allocator& A = s->alloc;
  const int64_t cap = nrhs;
  auto regrow = [&](auto*& p, int64_t per) {
    using E = std::remove_reference_t<decltype(*p)>;
    if (!p) return;
    A.release(p);
    p = nullptr;
    p = A.alloc_n<E>((size_t)(cap * std::max<int64_t>(per, 1)));
    HHG_CUDA(cudaMemsetAsync(p, 0, sizeof(E) * cap * std::max<int64_t>(per, 1), st));
  };
  for (auto& L : s->levels) {
    const int64_t nt = L.lay.n_total, ng = L.lay.nC * L.lay.n_full, ntmp = std::max(L.max_step, 1);
    regrow(L.d_ghost64, ng);
    regrow(L.d_r, nt);
    regrow(L.d_tmp, ntmp);
    regrow(L.d_u, nt);
    regrow(L.d_f, nt);
    regrow(L.d_ghost32, ng);
    regrow(L.d_u32, nt);
    regrow(L.d_f32, nt);
    regrow(L.d_r32, nt);
    regrow(L.d_tmp32, ntmp);
  }
  A.release(s->d_red);
  s->d_red = nullptr;
  s->red_len = (64 + (int64_t)s->pstride) * cap;
  s->d_red = A.alloc_n<double>((size_t)s->red_len);
  HHG_CUDA(cudaMemsetAsync(s->d_red, 0, sizeof(double) * s->red_len, st));
  A.release(s->d_cg);
  s->d_cg = nullptr;
  s->d_cg = A.alloc_n<double>((size_t)(4 * s->levels[0].lay.n_total * cap));
  HHG_CUDA(cudaStreamSynchronize(st));
  s->cap = (int)cap;
  ++s->gen;
}

// Sets the number of right-hand sides the next operations process together
// and restores one on scope exit.
struct Batch {
  hhg_shell* s;
  Batch(hhg_shell* s_, int nb, cudaStream_t st) : s(s_) {
    ensure_cap(s, nb, st);
    s->nb = nb;
  }
  ~Batch() { s->nb = 1; }
};

// All vector arguments in device memory: the batched path (every kernel
// takes all right-hand sides, the surrogate weights of a node are evaluated
// once for all of them); otherwise one right-hand side at a time through the
// staging buffers.
static bool all_device(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (p == nullptr || is_host_ptr(p)) return false;
  return true;
}

hhg_status hhg_apply(hhg_shell* s, int L, hhg_op op, hhg_dtype dtype, const void* u, void* y, int nrhs,
                     void* stream) {
  return guarded([&] {
    const int n = level_index(s, L);
    check_common(s, n, op, dtype, nrhs);
    HHG_CHECK(u != y, HHG_EINVAL, "u and y must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nt = s->levels[n].lay.n_total;
    if (dtype == HHG_F32) ensure_f32(s, st);
    if (nrhs > 1 && all_device({u, y})) {
      Batch bt(s, nrhs, st);
      if (dtype == HHG_F32) op_apply<float>(s, n, op, (const float*)u, (float*)y, st);
      else op_apply(s, n, op, (const double*)u, (double*)y, st);
      return;
    }
    for (int b = 0; b < nrhs; ++b) {
      if (dtype == HHG_F32) {
        Arg au = stage_in(s, 0, (const float*)u + b * nt, nt, true, st, sizeof(float));
        Arg ay = stage_in(s, 1, (float*)y + b * nt, nt, false, st, sizeof(float));
        op_apply<float>(s, n, op, au.dev32(), ay.dev32(), st);
        stage_out(ay, nt, st);
        continue;
      }
      Arg au = stage_in(s, 0, (const double*)u + b * nt, nt, true, st);
      Arg ay = stage_in(s, 1, (double*)y + b * nt, nt, false, st);
      op_apply(s, n, op, au.dev, ay.dev, st);
      stage_out(ay, nt, st);
    }
  });
}

hhg_status hhg_load_vector(hhg_shell* s, int L, const double* f, double* b, void* stream) {
  return guarded([&] {
    const int n = level_index(s, L);
    HHG_CHECK(f != b, HHG_EINVAL, "f and b must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    Level& Lv = s->levels[n];
    const int64_t nt = Lv.lay.n_total;
    if (!Lv.d_inc_ptr) {  // the incidence is rebuilt on the host the first time
      std::vector<uint32_t> bnd_ijk;
      std::vector<int> bnd_slot, halo_src, inc_cb;
      std::vector<int64_t> inc_ptr;
      boundary_points(Lv.N, bnd_ijk, bnd_slot);
      lower_incidence(s->mesh, Lv.lay, bnd_ijk, halo_src, inc_ptr, inc_cb);
      Lv.d_inc_ptr = upload(s->alloc, inc_ptr, st);
      Lv.d_inc_cb = upload(s->alloc, inc_cb, st);
    }
    Arg af = stage_in(s, 0, f, nt, true, st);
    Arg ab = stage_in(s, 1, b, nt, false, st);
    launch_load_vector(view<double>(s, n), Lv.d_inc_ptr, Lv.d_inc_cb, af.dev, ab.dev, st);
    stage_out(ab, nt, st);
  });
}

hhg_status hhg_residual(hhg_shell* s, int L, hhg_op op, hhg_dtype dtype, const void* u, const void* f, void* r,
                        int nrhs, double* norms, void* stream) {
  return guarded([&] {
    const int n = level_index(s, L);
    check_common(s, n, op, dtype, nrhs);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nt = s->levels[n].lay.n_total;
    if (dtype == HHG_F32) ensure_f32(s, st);
    if (nrhs > 1 && all_device({u, f, r})) {
      Batch bt(s, nrhs, st);
      if (dtype == HHG_F32) op_residual<float>(s, n, op, (const float*)u, (const float*)f, (float*)r, 9, st);
      else op_residual(s, n, op, (const double*)u, (const double*)f, (double*)r, 9, st);
      if (norms) {
        const std::vector<double> h = read_scalars(s, 9, st);
        for (int b = 0; b < nrhs; ++b) norms[b] = std::sqrt(h[b]);
      }
      return;
    }
    for (int b = 0; b < nrhs; ++b) {
      if (dtype == HHG_F32) {
        Arg au = stage_in(s, 0, (const float*)u + b * nt, nt, true, st, sizeof(float));
        Arg af = stage_in(s, 1, (const float*)f + b * nt, nt, true, st, sizeof(float));
        Arg ar = stage_in(s, 2, (float*)r + b * nt, nt, false, st, sizeof(float));
        op_residual<float>(s, n, op, au.dev32(), af.dev32(), ar.dev32(), 9, st);
        stage_out(ar, nt, st);
      } else {
        Arg au = stage_in(s, 0, (const double*)u + b * nt, nt, true, st);
        Arg af = stage_in(s, 1, (const double*)f + b * nt, nt, true, st);
        Arg ar = stage_in(s, 2, (double*)r + b * nt, nt, false, st);
        op_residual(s, n, op, au.dev, af.dev, ar.dev, 9, st);
        stage_out(ar, nt, st);
      }
      if (norms) norms[b] = std::sqrt(read_scalars(s, 9, st)[0]);
    }
  });
}

hhg_status hhg_smooth(hhg_shell* s, int L, hhg_op op, hhg_dtype dtype, const void* f, void* u, int sweeps, int nrhs,
                      void* stream) {
  return guarded([&] {
    const int n = level_index(s, L);
    check_common(s, n, op, dtype, nrhs);
    HHG_CHECK(sweeps >= 0, HHG_EINVAL, "sweeps must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    Level& Lv = s->levels[n];
    const int64_t nt = Lv.lay.n_total;
    if (dtype == HHG_F32) ensure_f32(s, st);
    if (nrhs > 1 && all_device({f, u})) {
      Batch bt(s, nrhs, st);
      if (dtype == HHG_F32) {
        launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, (float*)u, nrhs, nt, st);
        for (int t = 0; t < sweeps; ++t) op_smooth<float>(s, n, op, (const float*)f, (float*)u, st);
      } else {
        launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, (double*)u, nrhs, nt, st);
        for (int t = 0; t < sweeps; ++t) op_smooth(s, n, op, (const double*)f, (double*)u, st);
      }
      return;
    }
    for (int b = 0; b < nrhs; ++b) {
      if (dtype == HHG_F32) {
        Arg af = stage_in(s, 1, (const float*)f + b * nt, nt, true, st, sizeof(float));
        Arg au = stage_in(s, 0, (float*)u + b * nt, nt, true, st, sizeof(float));
        launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, au.dev32(), 1, nt, st);
        for (int t = 0; t < sweeps; ++t) op_smooth<float>(s, n, op, af.dev32(), au.dev32(), st);
        stage_out(au, nt, st);
        if (au.host) check_device_error(s, st);
        continue;
      }
      Arg af = stage_in(s, 1, (const double*)f + b * nt, nt, true, st);
      Arg au = stage_in(s, 0, (double*)u + b * nt, nt, true, st);
      launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, au.dev, 1, nt, st);
      for (int t = 0; t < sweeps; ++t) op_smooth(s, n, op, af.dev, au.dev, st);
      stage_out(au, nt, st);
    }
  });
}

// V-cycles for the active right-hand sides (s->nb of them, device vectors f
// and u, nt apart) until every relative residual is <= rtol or max_cycles;
// rel receives the final relative residuals, the return value is the number
// of cycles run.
static int solve_batch(hhg_shell* s, int op, int dtype, const double* f, double* u, int nu1, int nu2, int max_cycles,
                       double rtol, double* rel, cudaStream_t st) {
  const int n = (int)s->levels.size() - 1, nb = s->nb;
  Level& Lv = s->levels[n];
  const int64_t nt = Lv.lay.n_total;
  const bool dd = op == HHG_OP_DD;
  double* uprev = nullptr;
  if (dd) {  // double discretisation stops on the updates u_k - u_{k-1} (Sec. 4.1)
    if (s->uprev_len < nt * s->cap) {
      s->alloc.release(s->d_uprev);
      s->d_uprev = nullptr;
      s->d_uprev = s->alloc.alloc_n<double>((size_t)(nt * s->cap));
      s->uprev_len = nt * s->cap;
      ++s->gen;
    }
    uprev = s->d_uprev;
  }
  launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, u, nb, nt, st);
  op_residual(s, n, op, u, f, Lv.d_r, 10, st);
  std::vector<double> r0 = read_scalars(s, 10, st);
  std::vector<double> d0((size_t)nb, -1.0);
  // per-right-hand-side stopping: copy a right-hand side's iterate out at the
  // cycle where it first meets rtol (see hhg_shell::freeze_host)
  const bool freeze = s->freeze_host != nullptr;
  std::vector<char> frozen((size_t)nb, 0);
  auto freeze_out = [&](int b, int c) {
    launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, u, nb, nt, st);
    HHG_CUDA(cudaMemcpyAsync(s->freeze_host + (int64_t)b * nt, u + (int64_t)b * nt, sizeof(double) * nt,
                             cudaMemcpyDeviceToHost, st));
    HHG_CUDA(cudaStreamSynchronize(st));
    s->freeze_cycle[b] = c;
    frozen[b] = 1;
  };
  bool todo = false;
  for (int b = 0; b < nb; ++b) {
    r0[b] = std::sqrt(r0[b]);
    HHG_CHECK(std::isfinite(r0[b]), HHG_EDIVERGED, "initial residual is not finite");
    rel[b] = r0[b] > 0 ? 1.0 : 0.0;
    if (freeze && rel[b] <= rtol) freeze_out(b, 0);
    todo = todo || rel[b] > rtol;
  }
  if (dtype == HHG_F32) ensure_f32(s, st);
  auto cycle = [&](cudaStream_t cs) {
    if (dd) HHG_CUDA(cudaMemcpyAsync(uprev, u, sizeof(double) * nt * nb, cudaMemcpyDeviceToDevice, cs));
    if (dtype == HHG_F32) {
      // iterative refinement: e = one FP32 V-cycle on L e = r (e0 = 0), u += e;
      // double discretisation checks updates, not residuals, so r is formed here
      if (dd) op_residual(s, n, op, u, f, Lv.d_r, 11, cs);
      launch_copy_cast<float>(Lv.d_r, Lv.d_f32, nt * nb, cs);
      HHG_CUDA(cudaMemsetAsync(Lv.d_u32, 0, sizeof(float) * nt * nb, cs));
      vcycle_rec32(s, n, op, Lv.d_f32, Lv.d_u32, nu1, nu2, cs);
      launch_widen(Lv.d_u32, u, nt * nb, true, cs);
    } else {
      vcycle_rec(s, n, op, f, u, nu1, nu2, cs);
    }
  };
  // The first cycle runs launch by launch (its coarse solve is host-driven
  // and sets the iteration count); later cycles replay one CUDA graph of the
  // whole cycle, captured once per key, with fixed-count coarse iterations.
  // Graphs are captured and launched on the shell's own stream, ordered
  // after and before the caller's stream by events.
  const bool graphs = s->graphs;
  int cyc = 0;
  while (todo && cyc < max_cycles) {
    if (!graphs || cyc == 0) {
      cycle(st);
      if (cyc == 0 && s->cg_graph_iters == 0) s->cg_graph_iters = std::max(32, (s->cg_last * 3 / 2 + 16 + 7) / 8 * 8);
    } else {
      const hhg_shell::GraphKey key{f, u, nb, op, dtype, nu1, nu2, s->cg_graph_iters, s->gen};
      if (!s->graph_exec || !(s->graph_key == key)) {
        if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
        s->graph_exec = nullptr;
        cudaGraph_t g = nullptr;
        graph_timed_clear(s);
        HHG_CUDA(cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeRelaxed));
        s->cg_fixed = s->cg_graph_iters;
        s->capturing = true;
        const int64_t l0 = hhg_launch_count();
        try {
          cycle(s->gstream);
        } catch (...) {
          s->cg_fixed = 0;
          s->capturing = false;
          cudaStreamEndCapture(s->gstream, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        s->graph_launches = hhg_launch_count() - l0;
        count_launch((int)-s->graph_launches);  // counted per replay instead
        s->cg_fixed = 0;
        s->capturing = false;
        HHG_CUDA(cudaStreamEndCapture(s->gstream, &g));
        const cudaError_t ie = cudaGraphInstantiate(&s->graph_exec, g, 0);
        cudaGraphDestroy(g);
        HHG_CUDA(ie);
        s->graph_key = key;
      }
      HHG_CUDA(cudaEventRecord(s->gev[0], st));
      HHG_CUDA(cudaStreamWaitEvent(s->gstream, s->gev[0], 0));
      HHG_CUDA(cudaGraphLaunch(s->graph_exec, s->gstream));
      count_launch((int)s->graph_launches);
      HHG_CUDA(cudaEventRecord(s->gev[1], s->gstream));
      HHG_CUDA(cudaStreamWaitEvent(st, s->gev[1], 0));
    }
    if (dd) {
      launch_diff_norm(u, uprev, nt, nb, parts(s), s->pstride, scal(s, 10), st);
    } else {
      op_residual(s, n, op, u, f, Lv.d_r, 10, st);
    }
    const std::vector<double> rn = read_scalars(s, 10, st);
    if (graphs && cyc > 0) graph_timed_accumulate(s);
    check_device_error(s, st);
    todo = false;
    for (int b = 0; b < nb; ++b) {
      if (frozen[b]) continue;
      const double v = std::sqrt(rn[b]);
      HHG_CHECK(std::isfinite(v), HHG_EDIVERGED, "residual norm became NaN or Inf");
      if (dd) {
        if (d0[b] < 0) d0[b] = v;  // the first update
        rel[b] = d0[b] > 0 ? v / d0[b] : 0.0;
      } else {
        rel[b] = r0[b] > 0 ? v / r0[b] : 0.0;
      }
      if (freeze && rel[b] <= rtol) freeze_out(b, cyc + 1);
      todo = todo || rel[b] > rtol;
    }
    ++cyc;
  }
  launch_zero_list(Lv.d_dirichlet, Lv.n_dirichlet, u, nb, nt, st);
  if (freeze)
    for (int b = 0; b < nb; ++b)
      if (!frozen[b]) freeze_out(b, cyc);  // not converged within max_cycles
  return cyc;
}

hhg_status hhg_vcycle(hhg_shell* s, hhg_op op, hhg_dtype dtype, const void* f, void* u, int nu1, int nu2,
                      int max_cycles, double rtol, int nrhs, double* relres_out, int* cycles_out, void* stream) {
  return guarded([&] {
    HHG_CHECK(s != nullptr, HHG_EINVAL, "NULL shell");
    const int n = (int)s->levels.size() - 1;
    check_common(s, n, op, dtype, nrhs);
    for (int m = 0; m <= n; ++m) check_op(s, m, op);
    HHG_CHECK(nu1 >= 0 && nu2 >= 0 && max_cycles >= 0, HHG_EINVAL, "negative cycle parameter");
    cudaStream_t st = (cudaStream_t)stream;
    Level& Lv = s->levels[n];
    const int64_t nt = Lv.lay.n_total;
    std::vector<double> rel((size_t)nrhs, 0.0);
    int cycles_max = 0;
    if (nrhs > 1 && all_device({f, u})) {
      Batch bt(s, nrhs, st);
      cycles_max = solve_batch(s, op, dtype, (const double*)f, (double*)u, nu1, nu2, max_cycles, rtol, rel.data(), st);
    } else {
      for (int b = 0; b < nrhs; ++b) {
        Arg af = stage_in(s, 1, (const double*)f + b * nt, nt, true, st);
        Arg au = stage_in(s, 0, (double*)u + b * nt, nt, true, st);
        const int cyc = solve_batch(s, op, dtype, af.dev, au.dev, nu1, nu2, max_cycles, rtol, &rel[b], st);
        stage_out(au, nt, st);
        cycles_max = std::max(cycles_max, cyc);
      }
    }
    HHG_CUDA(cudaStreamSynchronize(st));
    bool all_conv = true;
    for (int b = 0; b < nrhs; ++b) {
      if (relres_out) relres_out[b] = rel[b];
      all_conv = all_conv && rel[b] <= rtol;
    }
    if (cycles_out) *cycles_out = cycles_max;
    if (!all_conv) throw Error{HHG_ENOCONV, "max_cycles reached before rtol"};
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Residual without allocation: partial sums in a fixed device array
// ---------------------------------------------------------------------------

namespace {

// The array itself.  In host code its name is only a host-side stand-in;
// kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[HHG_NOALLOC_SCRATCH];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (with that device current).
double* noalloc_scratch() {
  int dev = 0;
  HHG_CUDA(cudaGetDevice(&dev));
  HHG_CHECK(dev >= 0 && dev < kMaxDevices, HHG_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    HHG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" hhg_status hhg_residual_noalloc(hhg_shell* s, int L, hhg_op op, const double* u, const double* f,
                                           double* r, double* norm2_dev, void* stream) {
  return guarded([&] {
    const int n = level_index(s, L);
    check_op(s, n, op);
    HHG_CHECK(u && f && r && norm2_dev, HHG_EINVAL, "NULL argument");
    for (const void* p : {(const void*)u, (const void*)f, (const void*)r, (const void*)norm2_dev})
      HHG_CHECK(!is_host_ptr(p), HHG_EINVAL, "hhg_residual_noalloc takes device pointers only");
    LevelView<double> v = view<double>(s, n);
    v.nrhs = 1;
    const int nb = low_blocks(v.off_C);
    HHG_CHECK((int64_t)v.nC + nb <= HHG_NOALLOC_SCRATCH, HHG_EINVAL,
              "level needs " + std::to_string((int64_t)v.nC + nb) + " partial slots, more than HHG_NOALLOC_SCRATCH (" +
                  std::to_string(HHG_NOALLOC_SCRATCH) + ")");
    double* part = noalloc_scratch();
    cudaStream_t st = (cudaStream_t)stream;
    launch_halo(v, u, st);
    launch_cell(v, eff_op(s, n, exact_op(op)), RESIDUAL, const_cast<double*>(u), r, f, part, st);
    launch_low(v, RESIDUAL, u, r, f, part + v.nC, nb, st);
    launch_sum(part, v.nC + nb, 1, 0, norm2_dev, st);
  });
}
