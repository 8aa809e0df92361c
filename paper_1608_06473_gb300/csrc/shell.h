// Internal state of an hhg_shell: the macro mesh, and per refinement level
// the device index maps, pre-assembled lower-primitive stencils, surrogate
// coefficients, halo copies and work vectors.
#pragma once

#include <cstdint>
#include <tuple>
#include <vector>

#include "common.h"
#include "mesh.h"

namespace hhg {

// FP32 surrogate smoother configurations the tuner chooses from besides the
// per-colour node kernels: 0..3 staged (stage.cu), 4..5 wavefront (wave.cu),
// 6 chunked per-colour (cell.cu), 7 cell-resident sweep (resident.cu)
constexpr int SMOOTH32_CONFIGS = 8;
constexpr int TUNE_NONE = -9;           // FP32 smoother of a level not tuned yet

// Geometry of one macro cell: its 4 vertices (ascending global id) and the
// radii that rho interpolates (Sec. 2.2, blending map Phi).
struct CellGeom {
  double x[4][3];
  double r[4];
};

// Byte-budgeted device allocator: refuses before cudaMalloc when a request
// would exceed the budget (HHG_ENOMEM).
struct Allocator {
  size_t budget = 0;  // 0 = unlimited
  size_t used = 0;
  std::vector<std::pair<void*, size_t>> live;
  void* alloc(size_t bytes);
  void release(void* p);
  void release_all();
  template <class T>
  T* alloc_n(size_t n) { return static_cast<T*>(alloc(n * sizeof(T))); }
};

// Deep-interior points per chunked work item of the FP32 smoother.
constexpr int CHUNK32 = 4;
// Most points per run item of the FP64 surrogate kernels (run lists below).
constexpr int RUN64 = 8;
// FP64 surrogate kernel variants (hhg_set_fp64_kernel): weights per node by
// Horner (default, the fastest measured), or by forward differences along
// runs of a line, one launch per colour or as the cell-resident sweep.
constexpr int FP64_NODES = 0;       // per-node kernels
constexpr int FP64_RUNS = 1;        // per-colour run kernels
constexpr int FP64_RESIDENT = 2;    // run kernels, smoother as the cell-resident sweep where it fits

// Packed cell-local point: i | j << 10 | k << 20 (N <= 1023).
HD uint32_t pack_ijk(int i, int j, int k) { return (uint32_t)i | ((uint32_t)j << 10) | ((uint32_t)k << 20); }
HD int unpack_i(uint32_t p) { return (int)(p & 1023u); }
HD int unpack_j(uint32_t p) { return (int)((p >> 10) & 1023u); }
HD int unpack_k(uint32_t p) { return (int)(p >> 20); }

// Device-side view of one level, passed to kernels by value.
template <class T>
struct LevelView {
  int N;
  int nC;
  int64_t off_E, off_F, off_C, n_total, n_int, n_full;
  int n_bnd;
  const CellGeom* geom;          // [nC]
  const uint32_t* plane_nodes;   // interior points (packed) by (k, colour), deep-interior ones first
  const int* plane_off;          // start of (k, colour) in plane_nodes, [4 (N + 1) + 1]
  const int* plane_x;            // [n_plane] position of each listed point within its plane
  const int* plane_nb;           // [14 * n_plane] neighbour codes of the points next to the cell boundary
  int n_plane;
  const uint32_t* int_ijk;       // [n_int] interior points in canonical order
  const uint32_t* bnd_ijk;       // [n_bnd] boundary points of a cell
  const int* bnd_slot;           // [n_full] boundary slot of a cell-local point, -1 = interior
  const int* halo_src;           // [nC * n_bnd] canonical index of each cell's boundary point, -1 = Dirichlet
  T* ghost;                      // [nC * n_full] per-cell copies of boundary values
  const T* coef;                 // [nC * 15 * m_q] surrogate coefficients (raw index monomials)
  int q;                         // surrogate degree (0 = not fitted)
  // FP64 surrogate: per cell, plane k and direction, the coefficients of
  // the polynomial in (i, j) as integers scaled by 2^cell_e[c]
  // ([nC][N - 3][15][npp64(q)] int64)
  const long long* plane64;
  const int* cell_e;             // [nC]
  const float* plane32;          // FP32 surrogate: per cell, plane and direction the polynomial in (i, j)
  const uint32_t* colour_nodes;  // interior points (packed) per colour, deep-interior ones first
  const uint32_t* all_nodes;     // all interior points, deep-interior ones first
  int colour_off[5];             // start of each colour in colour_nodes
  // chunked colour lists of the FP32 smoother: per colour cc, items
  // [chunk_off[cc], chunk_mid[cc]) cover up to CHUNK32 deep-interior points
  // i0, i0 + 4, .. of one line (pack_ijk(i0, j, k) | (count - 1) << 30), items
  // [chunk_mid[cc], chunk_off[cc + 1]) are single points next to the cell
  // boundary (pack_ijk)
  const uint32_t* chunk_nodes;
  int chunk_off[5], chunk_mid[4];
  // run lists of the FP64 surrogate kernels: segment g = 0..3 holds the runs
  // of colour g (points i0, i0 + 4, ..), segment 4 the runs over all interior
  // points (i0, i0 + 1, ..), items [run_off[g], run_off[g + 1]).  A run is
  // up to RUN64 points of one line (j, k), all deep-interior or all next to
  // the cell boundary, deep runs first: x = pack_ijk(i0, j, k),
  // y = count | deep << 8
  const uint2* run_nodes;
  int run_off[6];
  // run_kidx[(g (N + 1) + k) 2 + part]: first item of colour g's runs
  // (relative to run_off[g]) among the deep (part 0) or boundary-adjacent
  // (part 1) runs whose plane is >= k, k = 0 .. N
  const int* run_kidx;
  int fp64_kernel;               // FP64_NODES, FP64_RUNS or FP64_RESIDENT
  // lower primitives: canonical rows 0 .. off_C-1 in sliced ELL (32-row
  // slices, column-major inside a slice), Dirichlet rows have diag 0
  // rows stored in smoother-step order: position p holds canonical row
  // low_perm[p], canonical row r sits at position low_pos[r]; slice p >> 5
  const int64_t* sell_ptr;       // [n_slices + 1]
  const int* sell_col;           // canonical column, -1 = padding
  const T* sell_val;
  const int* low_perm;           // [off_C]
  const int* low_pos;            // [off_C]
  const T* low_diag;             // [off_C]
  int* err;                      // device error word: set to 1 when a bounded wait gives up
  int smooth_cfg;                // FP32 surrogate smoother: -1 / -2 = per-colour node kernel (1 / 2 nodes per thread in flight), 0..3 = staged, 4..5 = wavefront, 6 = chunked, 7 = cell-resident
  // right-hand sides processed together: vector b of a level lives at
  // v + b vstride, its halo copy at ghost + b gstride, its residual partials
  // at partial + b pstride, its lower-step buffer at tmp + b tstride
  int nrhs;
  int64_t vstride, gstride;
  int pstride, tstride;
};

struct Level {
  LevelLayout lay;
  int N = 0;
  int n_bnd = 0;
  uint32_t* d_bnd_ijk = nullptr;
  int* d_bnd_slot = nullptr;
  int* d_halo_src = nullptr;
  uint32_t* d_plane_nodes = nullptr;
  int* d_plane_off = nullptr;
  int* d_plane_x = nullptr;
  int* d_plane_nb = nullptr;
  int n_plane = 0;
  std::vector<int> h_plane_off;
  uint32_t* d_int_ijk = nullptr;
  // lower primitives
  int64_t n_slices = 0;
  int64_t* d_sell_ptr = nullptr;
  int* d_sell_col = nullptr;
  double* d_sell_val = nullptr;
  double* d_low_diag = nullptr;
  float* d_sell_val32 = nullptr;
  float* d_low_diag32 = nullptr;
  int* d_low_perm = nullptr;      // lower rows in step order (see LevelView)
  int* d_low_pos = nullptr;
  int step_beg[6] = {0, 0, 0, 0, 0, 0};   // first position of each smoother step
  int step_n[6] = {0, 0, 0, 0, 0, 0};
  int max_step = 0;
  int* d_dirichlet = nullptr;    // Dirichlet lower nodes
  // incidence of the lower nodes in the cells (load vector; built on first use)
  int64_t* d_inc_ptr = nullptr;
  int* d_inc_cb = nullptr;
  int n_dirichlet = 0;
  int64_t n_free = 0;
  // transfers: coarse parents of this level's lower nodes (this level fine),
  // and the fine position of this level's lower nodes (this level coarse)
  int* d_low_par = nullptr;          // [2 * off_C], -1 = Dirichlet parent
  int* d_coarse_low_fine = nullptr;  // [off_C], -1 = Dirichlet
  // surrogate
  double* d_coef = nullptr;
  float* d_coef32 = nullptr;
  long long* d_plane64 = nullptr;
  float* d_plane32 = nullptr;
  int* d_cell_e = nullptr;
  uint32_t* d_colour_nodes = nullptr;
  uint32_t* d_all_nodes = nullptr;
  int colour_off[5] = {0, 0, 0, 0, 0};
  uint32_t* d_chunk_nodes = nullptr;   // chunked colour lists (see LevelView)
  int chunk_off[5] = {0, 0, 0, 0, 0}, chunk_mid[4] = {0, 0, 0, 0};
  uint2* d_run_nodes = nullptr;        // FP64 run lists (see LevelView)
  int run_off[6] = {0, 0, 0, 0, 0, 0};
  int* d_run_kidx = nullptr;
  // FP32 surrogate smoother chosen by the tuner (TUNE_NONE = not tuned, -1 =
  // per-colour node kernel, -2 = the same with two nodes per thread in flight,
  // 0..3 = staged, 4..5 = wavefront, 6 = chunked configuration) and the candidates' times
  // (ms; index cfg + 2)
  int tune32 = TUNE_NONE;
  double tune32_ms[2 + SMOOTH32_CONFIGS] = {};
  // halo copies and work vectors (allocated on demand)
  double* d_ghost64 = nullptr;
  float* d_ghost32 = nullptr;
  double* d_u = nullptr;
  double* d_f = nullptr;
  double* d_r = nullptr;
  double* d_tmp = nullptr;  // step buffer for simultaneous lower-primitive updates
  // FP32 work vectors of the mixed-precision cycle (allocated on first use)
  float* d_u32 = nullptr;
  float* d_f32 = nullptr;
  float* d_r32 = nullptr;
  float* d_tmp32 = nullptr;
};

// Number of monomials of total degree <= q in three variables (Eq. 3.2).
HD int n_coeffs(int q) { return (q + 1) * (q + 2) * (q + 3) / 6; }

// int64 per direction in the FP64 plane table: the (q + 1)(q + 2) / 2
// coefficients of a polynomial in (i, j), rounded up to an even count
// (16-byte aligned records).
HD int npp64(int q) { return ((q + 1) * (q + 2) / 2 + 1) / 2 * 2; }
// FP64 plane table length (int64 values) for nC cells.
HD int64_t plane64_len(int64_t nC, int N, int q) { return nC * (N - 3) * 15 * npp64(q); }

}  // namespace hhg

struct hhg_shell {
  hhg::MacroMesh mesh;
  int Lf = 0;                          // finest log2(N)
  int n_parts = 1;                     // shells of the group (disjoint components of the macro mesh)
  std::vector<hhg::Level> levels;      // levels[n]: N = 4 << n
  hhg::CellGeom* d_geom = nullptr;
  hhg::Allocator alloc;
  int q = 0, j = 0;                    // surrogate degree and sampling choice, q = 0: not fitted
  double* d_red = nullptr;             // reduction scratch (partials + results)
  int64_t red_len = 0;
  double* d_cg = nullptr;              // coarse-solver vectors
  double* d_uprev = nullptr;           // previous iterate of double-discretisation cycles
  int64_t uprev_len = 0;
  // per-right-hand-side stopping (continuous batching of the solve server):
  // when set, each right-hand side's iterate is copied to freeze_host + b *
  // n_total at the first cycle where it meets rtol (its cycle count to
  // freeze_cycle[b]), it no longer keeps the cycle loop going, and its
  // relative residual stays the one of that cycle
  double* freeze_host = nullptr;
  int* freeze_cycle = nullptr;
  int* d_err = nullptr;                // device error word of the staged kernels (0 = ok)
  // batches: work vectors, halo copies, step buffers, reduction and coarse
  // solver scratch hold `cap` right-hand sides; `nb` of them are active in
  // the current call
  int cap = 1;
  int nb = 1;
  // CUDA-graph V-cycles: the captured cycle of the last key, the
  // coarse-solver iteration count it was captured with, and a generation
  // counter bumped whenever captured kernels or buffers change
  bool graphs = true;
  int fp64_kernel = hhg::FP64_NODES;  // FP64 surrogate kernel variant (hhg_set_fp64_kernel)
  int64_t gen = 0;
  int cg_fixed = 0;          // > 0 while capturing: fixed-count coarse iterations
  int cg_graph_iters = 0;    // iterations the next capture uses
  int cg_last = 0;           // iterations of the last host-driven coarse solve
  struct GraphKey {
    const void* f;
    const void* u;
    int nb, op, dtype, nu1, nu2, iters;
    int64_t gen;
    bool operator==(const GraphKey& o) const {
      return f == o.f && u == o.u && nb == o.nb && op == o.op && dtype == o.dtype && nu1 == o.nu1 && nu2 == o.nu2 &&
             iters == o.iters && gen == o.gen;
    }
  } graph_key{};
  cudaGraphExec_t graph_exec = nullptr;
  bool capturing = false;
  int64_t graph_launches = 0;          // kernels in the captured cycle (counted again per replay)
  // timed scopes captured into the graph (class, begin, end): re-recorded by
  // every replay and accumulated after it into gsum / gcnt
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> gtimed;
  double gsum[HHG_T_COUNT] = {};
  int64_t gcnt[HHG_T_COUNT] = {};
  cudaStream_t gstream = nullptr;      // capture and replay stream of the graphs
  cudaEvent_t gev[2] = {nullptr, nullptr};
  int pstride = 0;                     // residual partials per right-hand side
  void* coarse_op = nullptr;           // hhg::CoarseOp of the N = 4 level (owned)
  double* d_stage[3] = {nullptr, nullptr, nullptr};  // staging for host-pointer arguments
  bool f32_ready = false;              // FP32 resources allocated
  int64_t stage_len = 0;

  // diagnostics: CUDA-event pairs around timed kernel launches
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tevents[HHG_T_COUNT];
  int64_t cg_iters = 0;

  hhg::Level& level_of(int L) { return levels.at(L - 2); }
};
