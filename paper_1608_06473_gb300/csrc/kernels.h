// Host-side launchers of the CUDA kernels (implemented in cell.cu, low.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "shell.h"

namespace hhg {

enum Mode { APPLY = 0, RESIDUAL = 1, SMOOTH = 2 };

// Raises the dynamic shared memory limit of kernel `func` to at least
// `bytes` (never lowers it, so concurrent host threads launching the same
// kernel with different sizes stay valid).
void ensure_smem_limit(const void* func, size_t bytes);

// ---- cell interiors (cell.cu) ----------------------------------------------
// One CTA per macro cell (grid = nC).
//   APPLY:    out = L u on the interior nodes
//   RESIDUAL: out = f - L u, partial[c] = sum of out^2 over cell c (nC slots)
//   SMOOTH:   the four colour steps (i + 2j + 3k) mod 4 = 0..3 of Eq. 5.1,
//             u updated in place (one launch per colour, or for FP32 the
//             staged one-launch sweep where the tuner chose it, lv.smooth_cfg).
// lv.nrhs right-hand sides per call (RESIDUAL partials at b pstride + c).
// op: 0 = IFEM (on-the-fly exact stencils), 1 = LSQP (surrogate).
template <class T>
void launch_cell(const LevelView<T>& lv, int op, Mode mode, T* u, T* out, const T* f, double* partial,
                 cudaStream_t st);
template <>
void launch_cell<double>(const LevelView<double>& lv, int op, Mode mode, double* u, double* out, const double* f,
                         double* partial, cudaStream_t st);
template <>
void launch_cell<float>(const LevelView<float>& lv, int op, Mode mode, float* u, float* out, const float* f,
                        double* partial, cudaStream_t st);

// FP32 surrogate smoother with shared-memory plane staging (stage.cu): the
// four cell colour steps in one launch per sweep.  `cfg` (0 ..
// STAGE32_CONFIGS - 1) picks the wavefront skew and the CTA size; a
// configuration is supported when the surrogate is fitted, u is 16-byte
// aligned and its plane ring fits in shared memory.  A bounded wait that
// gives up sets *lv.err.
constexpr int STAGE32_CONFIGS = 4;
bool stage32_supported(const LevelView<float>& lv, const float* u, int cfg);
void launch_stage32_smooth(const LevelView<float>& lv, float* u, const float* f, int cfg, cudaStream_t st);

// FP32 surrogate smoother as a plane wavefront per cell (wave.cu): the four
// cell colour steps in one launch per sweep, u updated in place through the
// caches, one barrier per step.  cfg 0, 1: 128, 256 threads per CTA.  A
// configuration is supported when the surrogate is fitted and the cell's
// plane table fits in shared memory.
constexpr int WAVE32_CONFIGS = 2;
bool wave32_supported(const LevelView<float>& lv, int cfg);
void launch_wave32_smooth(const LevelView<float>& lv, float* u, const float* f, int cfg, cudaStream_t st);

// Chunked per-colour FP32 smoother (cell.cu): configuration 6, each colour
// one launch over all cells.
constexpr int CHUNK32_CONFIGS = 1;
bool chunk32_supported(const LevelView<float>& lv);

// Cell-resident sweep (resident.cu): the four cell colour steps of the
// surrogate smoother in one launch, each cell's interior held in the shared
// memory of a cluster of 1..8 CTAs (FP64, and FP32 configuration 7).
// Supported for one right-hand side when the surrogate is fitted and the
// largest slab fits one CTA's shared memory.  A bounded wait that gives up
// sets *lv.err and leaves u unchanged.
constexpr int RESIDENT32_CONFIGS = 1;
template <class T>
bool resident_supported(const LevelView<T>& lv);
template <class T>
void launch_resident_sweep(const LevelView<T>& lv, T* u, const T* f, cudaStream_t st);
// Planes [k_bounds[r], k_bounds[r + 1]) of slab r, r < CS, of a cell at N
// (host; the kernel computes the same split).
void resident_slab_planes(int N, int CS, int* k_bounds);
// Cluster size (CTAs per cell) the sweep uses on this level, 0 if unsupported.
template <class T>
int resident_cluster_size(const LevelView<T>& lv);
static_assert(STAGE32_CONFIGS + WAVE32_CONFIGS + CHUNK32_CONFIGS + RESIDENT32_CONFIGS == SMOOTH32_CONFIGS,
              "tuner table size");

// Whether smoother configuration cfg >= 0 (staged 0..3, wavefront 4..5,
// chunked 6, cell-resident 7) can run on this level and vector.
inline bool smooth32_supported(const LevelView<float>& lv, const float* u, int cfg) {
  if (cfg < STAGE32_CONFIGS) return stage32_supported(lv, u, cfg);
  if (cfg < STAGE32_CONFIGS + WAVE32_CONFIGS) return wave32_supported(lv, cfg - STAGE32_CONFIGS);
  if (cfg < STAGE32_CONFIGS + WAVE32_CONFIGS + CHUNK32_CONFIGS) return chunk32_supported(lv);
  return resident_supported(lv);
}

// FP64 surrogate plane table (fit time): per cell the scale exponent E and,
// per plane k and direction, the (q+1)(q+2)/2 coefficients of the
// polynomial in (i, j), times 2^E, rounded to int64.
void launch_plane64_table(const LevelView<double>& lv, int q, const double* coef, int* cell_e, long long* table,
                          cudaStream_t st);

// FP32 surrogate plane table (fit time): per cell, plane k and direction the
// (q+1)(q+2)/2 coefficients of the polynomial in (i, j), rounded to FP32.
void launch_plane_table(const LevelView<double>& lv, int q, const double* coef, float* table, cudaStream_t st);
inline int64_t plane_table_len(int nC, int N, int q) { return (int64_t)nC * (N - 3) * 15 * ((q + 1) * (q + 2) / 2); }

// Exact stencils (14 off-centre weights) at cell-local points of every cell:
// b[(c * n_pts + p) * 14 + w] (Table 4.3 "t_sample").
void launch_sample(const LevelView<double>& lv, const uint32_t* pts, int n_pts, double* b, cudaStream_t st);

// coef[c][w][t] = scale[t] * sum_p aplus[t][p] b[c][p][w] for w < 14 and the
// centre coef[c][14][t] = -sum_w coef[c][w][t]; optional float copy.
void launch_fit_coef(int nC, int mq, int n_pts, const double* aplus, const double* scale, const double* b,
                     double* coef, float* coef32, cudaStream_t st);

// ---- lower primitives, halos, transfers, reductions (low.cu) ---------------
template <class T>
void launch_halo(const LevelView<T>& lv, const T* u, cudaStream_t st);

template <class T>
void launch_low(const LevelView<T>& lv, Mode mode, const T* u, T* out, const T* f, double* partial,
                int n_partial_blocks, cudaStream_t st);
int low_blocks(int64_t rows);

// One smoother step over the n rows at positions pbeg .. pbeg + n - 1.
template <class T>
void launch_low_step(const LevelView<T>& lv, int pbeg, int n, T* u, const T* f, T* tmp, cudaStream_t st);

template <class T>
void launch_zero_list(const int* list, int n, T* v, int nrhs, int64_t vstride, cudaStream_t st);

template <class T>
void launch_prolong_add(const LevelView<T>& fine, const LevelView<T>& coarse, const int* low_par, const T* ec,
                        T* uf, cudaStream_t st);

template <class T>
void launch_restrict(const LevelView<T>& fine, const LevelView<T>& coarse, const int* coarse_low_fine,
                     const T* rf, T* rc, cudaStream_t st);

// out[b] = ||a_b - b_b||^2 over n entries per right-hand side (vectors n
// apart), through partial (pstride per right-hand side, fixed order).
void launch_diff_norm(const double* a, const double* b, int64_t n, int nrhs, double* partial, int pstride,
                      double* out, cudaStream_t st);
// out[b] = sum of partial[b pstride .. b pstride + n - 1], b < nrhs (fixed
// order, one block per right-hand side).
void launch_sum(const double* partial, int n, int nrhs, int pstride, double* out, cudaStream_t st);

template <class T>
void launch_copy_cast(const double* src, T* dst, int64_t n, cudaStream_t st);
// dst = (double) src, or dst += (double) src when add
void launch_widen(const float* src, double* dst, int64_t n, bool add, cudaStream_t st);

// ---- coarsest-level conjugate gradients (coarse.cu) -------------------------
constexpr int CG_BLOCKS = 128;
struct CoarseOp {                // exact operator of the N = 4 level
  int64_t n_total, off_C;
  int nC;
  const int64_t* sell_ptr;       // lower-primitive rows (the level's sliced ELL, step order)
  const int* low_pos;            // position of a canonical row
  const int* sell_col;
  const double* sell_val;
  const double* low_diag;
  const int* int_col;            // [14 nC] interior row of each cell, -1 = Dirichlet column
  const double* int_val;         // [14 nC]
  const double* int_diag;        // [nC]
  const double* dinv;            // [n_total] inverse diagonal, 0 on Dirichlet rows
};
// Assembles the interior rows and the inverse diagonal (setup).
void launch_coarse_setup(const LevelView<double>& lv, CoarseOp& A, int* col, double* val, double* diag, double* dinv,
                         cudaStream_t st);
// nrhs systems at once: vectors n_total apart, part 3 CG_BLOCKS doubles per
// right-hand side, scalars rz / rr one per right-hand side (contiguous).
void launch_cg_init(const CoarseOp& A, const double* f, double* x, double* r, double* z, double* p, double* part,
                    double* rz_out, double* rr_out, int nrhs, cudaStream_t st);
// With rr_cur != nullptr (fixed-count iterations, e.g. inside a CUDA graph)
// a right-hand side whose rr_cur <= 1e-26 ff is left unchanged and its
// scalars are carried to rz_next / rr_out.
void launch_cg_iteration(const CoarseOp& A, double* x, double* r, double* z, double* p, double* q, double* part,
                         const double* rz_cur, double* rz_next, double* rr_out, int nrhs, cudaStream_t st,
                         const double* rr_cur = nullptr, const double* ff = nullptr);
// *flag = 1 when some rr[b] > 1e-26 ff[b].
void launch_cg_check(const double* rr, const double* ff, int nrhs, int* flag, cudaStream_t st);

// Lower-primitive stencil assembly (setup): pass 0 counts columns per row,
// pass 1 fills the sliced ELL rows and the diagonal.
void launch_low_assemble(const LevelView<double>& lv, int pass, const int64_t* inc_ptr, const int* inc_cb,
                         int* row_len, int64_t* sell_ptr, int* sell_col, double* sell_val, double* diag,
                         cudaStream_t st);

// Load vector b = V f of the accuracy study (vertex quadrature; load.cu).
void launch_load_vector(const LevelView<double>& lv, const int64_t* inc_ptr, const int* inc_cb, const double* f,
                        double* b, cudaStream_t st);

}  // namespace hhg
