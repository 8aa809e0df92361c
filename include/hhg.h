/*
 * hhg.h -- C ABI of the GB300 two-scale HHG multigrid library (libhhg.so).
 *
 * Method: Bauer, Mohr, Ruede, Weismueller, Wittmann, Wohlmuth, "A two-scale
 * approach for efficient on-the-fly operator assembly in massively parallel
 * high performance multigrid codes" (arXiv:1608.06473).
 *
 * Problem (Sec. 2.1, Eq. 2.1): -Laplace(u) = f on the thick spherical shell
 * r1 < |x| < r2, u = 0 on both spheres, P1 finite elements on a regularly
 * refined tetrahedral macro mesh whose nodes are moved by the blending map
 * Phi(x) = rho(x) x/|x| (Sec. 2.2).  The fine operator is applied matrix-free:
 * either the exact stencil assembled on the fly from the 24 element matrices
 * around every node (IFEM, Sec. 4.2.1), or the two-scale surrogate whose 15
 * stencil weights are least-squares polynomials per macro cell (LSQP,
 * Sec. 3.2-3.4), evaluated along fine-grid lines (Sec. 3.4, Eq. 5.4).
 *
 * Levels.  `L` is log2 of N, the number of intervals per macro edge
 * (N = 2^L, L >= 2).  The paper's level l is L - 2 (N = 2^(l+2), Sec. 2.2).
 * The coarsest level of every hierarchy is L = 2 (N = 4, one interior node
 * per macro cell).
 *
 * Vectors.  A vector of level L holds one value per fine node in the
 * canonical order: the macro vertices, then the N-1 nodes of every macro
 * edge, then the (N-1)(N-2)/2 interior nodes of every macro face, then the
 * (N-1)(N-2)(N-3)/6 interior nodes of every macro cell (i fastest, then j,
 * then k).  hhg_num_nodes gives its length n_total.  `nrhs` vectors are
 * stacked contiguously with stride n_total.  Entries at Dirichlet nodes (on
 * r1 or r2) are ignored on input and written as 0 on output.
 *
 * Pointers.  Every vector argument may be device memory (e.g. a torch
 * tensor's data_ptr) or host memory; host vectors are copied through
 * library-owned device buffers on `stream`, and the call returns after the
 * results have reached the host.  Device vectors are used in place and the
 * call returns once the work is enqueued on `stream`, except where a host
 * scalar output (norms, relres, cycles) is requested: then the call waits
 * for the stream.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *
 * Ownership.  The caller owns every vector.  The library owns the hierarchy
 * (index maps, halo copies, pre-assembled lower-primitive stencils,
 * surrogate coefficients, per-level work vectors) and frees it in
 * hhg_destroy.  All library allocations are charged against
 * hbm_budget_bytes; a call that would exceed it returns HHG_ENOMEM without
 * allocating.
 *
 * Errors.  Every call returns an hhg_status; on failure hhg_last_error()
 * returns a message for the calling thread.  A CUDA error leaves the shell
 * usable only for hhg_destroy.  Kernels that stage data in shared memory
 * wait on it with bounded waits; one that gives up sets a device error word
 * that the next call waiting for the stream reports as HHG_ETIMEOUT (the
 * results of the affected work are then undefined).
 *
 * Threads.  One shell may be used from one host thread at a time; calls on
 * the same shell that overlap on the GPU (different streams) race on its
 * work vectors.
 */
#ifndef HHG_H
#define HHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hhg_shell hhg_shell;

typedef enum {
  HHG_OK = 0,
  HHG_EINVAL = -1,     /* bad argument or descriptor */
  HHG_ENOMEM = -2,     /* the HBM budget (or the device) has no room */
  HHG_ECUDA = -3,      /* a CUDA call failed */
  HHG_ENOTFIT = -4,    /* the surrogate was requested before hhg_fit_surrogate */
  HHG_ENOCONV = -5,    /* max_cycles reached before rtol */
  HHG_EDIVERGED = -6,  /* a residual norm became NaN or Inf */
  HHG_ETIMEOUT = -7    /* a bounded device-side wait gave up */
} hhg_status;

typedef enum {
  HHG_OP_IFEM = 0,     /* exact stencils, assembled on the fly (Sec. 4.2.1) */
  HHG_OP_LSQP = 1,     /* the fitted surrogate stencils: LSQP (Sec. 3.2) or IPOLY (Sec. 3.1) */
  HHG_OP_DD = 2        /* double discretisation (Sec. 4.1): relaxation with the
                          fitted surrogate, residuals and apply with the exact
                          stencils; hhg_vcycle stops on the updates */
} hhg_op;

/* Arithmetic of a call.  hhg_apply / hhg_residual / hhg_smooth: the vectors
 * and the arithmetic are FP64 or FP32.  hhg_vcycle: f and u are always FP64
 * vectors; HHG_F64 runs FP64 V-cycles, HHG_F32 runs mixed precision --
 * iterative refinement with an FP64 residual (the stopping test is on it),
 * each correction from one V-cycle whose smoothing, residuals and transfers
 * are FP32 and whose coarsest solve is FP64.  The surrogate fit is FP64. */
typedef enum {
  HHG_F64 = 0,
  HHG_F32 = 1
} hhg_dtype;

/* Macro mesh and hierarchy (Sec. 2.2; macro counts of Sec. 4.1).
 * The surface is an icosahedron refined `tang_refine` times (1:4 splits,
 * midpoints projected to the sphere); `radial_layers` uniform layers between
 * r_inner and r_outer; every prism is cut into three tetrahedra:
 * 60 macro cells for (0, 1), 480 for (1, 2), 3840 for (2, 4). */
typedef struct {
  double r_inner;                /* r1 > 0 */
  double r_outer;                /* r2 > r1 */
  int tang_refine;               /* >= 0 */
  int radial_layers;             /* >= 1 */
  int fine_log2_intervals;       /* finest L (N = 2^L), 2..10 */
  size_t hbm_budget_bytes;       /* 0 = no limit beyond the device */
  int unprojected;               /* 0: nodes blended onto the shell (Phi, Sec. 2.2);
                                    1: the unprojected polyhedral domain Omega_H
                                    (Phi = Id), the paper's CONS operator (Sec. 4.1) */
} hhg_shell_desc;

/* Builds the macro mesh, its primitive graph and, for every level L = 2 ..
 * fine_log2_intervals, the index maps, the halo maps and the exact stencils
 * of all vertex, edge and face nodes (assembled from the element matrices of
 * the adjacent macro cells, Sec. 2.3: lower primitives keep exact stencils).
 * Work is enqueued on `stream` and completed before return. */
hhg_status hhg_setup_shell(const hhg_shell_desc* desc, void* stream, hhg_shell** out);

/* Several shells in one hierarchy: count descriptors that share
 * tang_refine, radial_layers and fine_log2_intervals but may differ in their
 * radii.  The shells become the disjoint components of one macro mesh, so
 * every kernel of every call spans all of them (one launch where a single
 * shell has one), and a V-cycle solves all of them together (its stopping
 * test is on the residual of the whole group).  The budget of desc[0]
 * applies to the group.  hhg_shell_part gives where shell k's nodes sit in
 * the canonical vectors. */
hhg_status hhg_setup_shells(const hhg_shell_desc* desc, int count, void* stream, hhg_shell** out);

/* Shell k of a group on level L: start[t] and count[t] (nullable, 4 entries)
 * of its nodes among the macro vertices (t = 0), edge nodes (1), face nodes
 * (2) and cell-interior nodes (3) of the canonical vector; each range is
 * contiguous and in the order of a single shell's canonical vector. */
hhg_status hhg_shell_part(const hhg_shell* shell, int L, int k, int64_t* start, int64_t* count);

/* Frees everything the shell owns (NULL is accepted). */
hhg_status hhg_destroy(hhg_shell* shell);

/* n_total: vector length of level L; n_free: unknowns (non-Dirichlet). */
hhg_status hhg_num_nodes(const hhg_shell* shell, int L, int64_t* n_total, int64_t* n_free);

/* Mapped positions Phi(x) of all nodes of level L, canonical order, written
 * to a host array of 3 * n_total doubles (x, y, z per node). */
hhg_status hhg_node_coords(const hhg_shell* shell, int L, double* xyz_host);

/* LSQP setup (Sec. 3.2, Table 4.3): for every macro cell and level L >= 3
 * (paper l >= 1), the exact stencils at the sampling set
 * S_l = M_{m(l,j)}, m(l,j) = min{l, max{1, j}} (Eq. 3.3) are evaluated on the
 * GPU and the 14 off-centre least-squares polynomials of total degree <= q
 * are fitted (Householder QR, FP64); the centre polynomial is minus their
 * sum (Lemma of Sec. 3.4).  q in 1..3, j >= 1.  L = 2 keeps the exact
 * stencil (Sec. 3, first paragraph).  May be called again to refit. */
hhg_status hhg_fit_surrogate(hhg_shell* shell, int q, int j, void* stream);

/* IPOLY setup (Sec. 3.1): the quadratic (q = 2) polynomials interpolating the
 * exact stencils at ten points of every macro cell and level L >= 3 -- the
 * quadratic nodes of the cell shrunk to its interior, (1,1,1), (1,1,a),
 * (1,a,1), (a,1,1), (1,1,b), (1,b,1), (b,1,1), (1,b,b), (b,1,b), (b,b,1) with
 * a = N - 3, b = N/2 - 1.  Replaces any previous fit; HHG_OP_LSQP and
 * HHG_OP_DD then use these polynomials. */
hhg_status hhg_fit_ipoly(hhg_shell* shell, void* stream);

/* IPOLY of degree q in 1..3 (Sec. 3.1, Table 4.1): interpolation at the m_q
 * nodes of degree q of the cell shrunk to its interior, (1,1,1) +
 * (N-4)(a,b,c)/q for a+b+c <= q, each coordinate rounded to the nearest fine
 * node where (N-4)/q is not an integer (q = 3 at N = 8, 32, 128).  q = 2 is
 * hhg_fit_ipoly. */
hhg_status hhg_fit_ipoly_degree(hhg_shell* shell, int q, void* stream);

/* CONS stencils as the cell-interior surrogate (Sec. 4.1, "CONS DD"): the
 * polynomials of hhg_fit_surrogate fitted to the stencils of the unprojected
 * domain Omega_H (Phi = Id), which are constant per macro cell and so
 * reproduced by every q.  Replaces any previous fit.  With HHG_OP_DD the
 * relaxation then uses these stencils in the cell interiors (vertex, edge
 * and face rows stay exact) and the residuals the exact operator. */
hhg_status hhg_fit_cons(hhg_shell* shell, int q, int j, void* stream);

/* Load vector of the accuracy study (Sec. 4): b_I = V_I f_I for every
 * unknown I of level L, with V_I the sum of |T| / 4 over the fine tetrahedra
 * T containing node I (vertex quadrature on each tetrahedron of the blended
 * mesh; of the straight mesh for an unprojected shell), and b_I = 0 at
 * Dirichlet nodes.  f holds the values of the right-hand-side function at
 * the nodes (canonical order, n_total doubles; host or device); b the same
 * size; f and b must not overlap.  The first call per level builds the
 * incidence of the lower nodes in the cells on the host (kept until
 * hhg_destroy). */
hhg_status hhg_load_vector(hhg_shell* shell, int L, const double* f, double* b, void* stream);

/* y = L_L u (op = IFEM) or y = L~_L u (op = LSQP) on level L, for nrhs
 * vectors (Sec. 3.4, the operator of Eq. 3.4).  u and y must not overlap. */
hhg_status hhg_apply(hhg_shell* shell, int L, hhg_op op, hhg_dtype dtype,
                     const void* u, void* y, int nrhs, void* stream);

/* r = f - L u on level L; if norms_host is not NULL, the Euclidean norm of
 * each returned r is written there (waits for the stream). */
hhg_status hhg_residual(hhg_shell* shell, int L, hhg_op op, hhg_dtype dtype,
                        const void* u, const void* f, void* r, int nrhs,
                        double* norms_host, void* stream);

/* `sweeps` multicolour hybrid Gauss-Seidel sweeps on level L, u updated in
 * place (Eq. 5.1 on every node).  One sweep is 10 steps, each updating its
 * node set simultaneously from the values at the start of the step:
 * (1) macro vertices, (2,3) edge nodes with even / odd position,
 * (4-6) face nodes with (p + 2q) mod 3 = 0, 1, 2, (7-10) cell-interior nodes
 * with (i + 2j + 3k) mod 4 = 0..3 (no two of them coupled). */
hhg_status hhg_smooth(hhg_shell* shell, int L, hhg_op op, hhg_dtype dtype,
                      const void* f, void* u, int sweeps, int nrhs, void* stream);

/* V(nu1, nu2) cycles on the finest level (Sec. 4): smooth, residual,
 * restriction R = P^T, recursion down to L = 2 (solved by FP64 conjugate
 * gradients to 1e-13 relative residual), prolongation (linear along the
 * coarse edges), smooth.  Coarse operators are re-discretised (their own
 * surrogate for op = LSQP).  u holds the initial guess and returns the
 * iterate; cycles stop once ||f - L u||_2 <= rtol ||f - L u_0||_2 for every
 * right-hand side or after max_cycles (HHG_ENOCONV).  relres_out (nullable,
 * nrhs) receives the final relative residuals, cycles_out (nullable) the
 * number of cycles run.  op = HHG_OP_DD (double discretisation, Sec. 4.1):
 * smoothing with the surrogate, residuals with the exact stencils, and the
 * stopping test on the updates instead of the residual,
 * ||u_k - u_{k-1}||_2 <= rtol ||u_1 - u_0||_2, as that section recommends;
 * relres_out then holds that ratio.  With HHG_F32 the FP64 refinement forms
 * the exact residual every cycle and the FP32 cycle relaxes with the
 * surrogate: that is defect correction, whose fixed point is the solution of
 * the exact operator, not the fixed point of the FP64 double-discretisation
 * cycle (the two differ by the inconsistency between the operators). */
hhg_status hhg_vcycle(hhg_shell* shell, hhg_op op, hhg_dtype dtype,
                      const void* f, void* u, int nu1, int nu2, int max_cycles,
                      double rtol, int nrhs, double* relres_out, int* cycles_out,
                      void* stream);

/* CUDA graphs in hhg_vcycle (enable != 0, the default): the first cycle of
 * a call runs launch by launch and its coarsest solve sets an iteration
 * count; every later cycle replays one CUDA graph of the whole V-cycle
 * (captured once per vector pointers, batch size and cycle parameters, and
 * again after a fit or tuning change), on a stream of the shell ordered
 * after `stream` by events.  Inside the graph the coarsest solve runs that
 * fixed number of conjugate-gradient iterations, each leaving converged
 * right-hand sides unchanged; should it stop short of the tolerance the
 * cycle's correction is kept and the next capture doubles the count.
 * enable = 0 runs every cycle launch by launch. */
hhg_status hhg_set_graphs(hhg_shell* shell, int enable);

/* ---- Serving: a request loop over resident hierarchies -----------------
 * Not a construct of the paper: a solve service for streams of shell
 * problems.  Requests (a shell geometry, a level, 1..n right-hand sides) are
 * queued by hhg_server_submit and admitted in arrival order as soon as one
 * of `max_inflight` slots is free and the request fits the HBM budget.  A
 * request runs on its slot's own CUDA stream and host worker thread, so
 * admitted requests overlap on the device.  Hierarchies (index maps, halo
 * copies, pre-assembled lower-primitive rows) and their surrogate
 * coefficients stay resident in a cache keyed by the geometry and level;
 * a request reuses an idle cached hierarchy of its key, else a new one is
 * built and fitted, evicting idle hierarchies (least recently used first)
 * when the budget requires.  Each request is solved by the batched V-cycle
 * (all of its right-hand sides together, as hhg_vcycle with device vectors)
 * to the server's tolerance; its result does not depend on what else is in
 * flight (every kernel and reduction has a fixed order; only the FP32
 * smoother configuration, chosen per hierarchy by timing, may change the
 * rounding of mixed-precision solves).
 *
 * Continuous batching (max_batch_rhs > 1): when a slot takes a request, the
 * requests queued behind it for the same geometry and level join it, up to
 * max_batch_rhs right-hand sides in total, and run as one batched solve on
 * one hierarchy (the weights of every node are evaluated once for all of
 * them).  Every right-hand side is then stopped on its own: its iterate is
 * taken at the first cycle where its relative residual meets rtol, so a
 * request's result equals that of the same request solved alone with the
 * same setting (to the batched kernels' rounding, 1e-10 relative in FP64). */
typedef struct hhg_server hhg_server;

typedef struct {
  size_t hbm_budget_bytes;  /* resident hierarchies + request vectors; 0 = no limit */
  int max_inflight;         /* concurrent requests (slots), >= 1 */
  int q, j;                 /* surrogate degree and sampling (hhg_fit_surrogate) */
  int nu1, nu2;             /* V(nu1, nu2) */
  int max_cycles;
  double rtol;              /* stop at ||r|| <= rtol ||r0|| for every right-hand side */
  hhg_dtype dtype;          /* HHG_F64 or HHG_F32 (mixed precision, see hhg_vcycle) */
  int max_batch_rhs;        /* continuous batching: right-hand sides per merged solve; 0 or 1 = off */
} hhg_server_desc;

/* One request's geometry and level (as hhg_shell_desc; L = fine_log2_intervals). */
typedef struct {
  double r_inner, r_outer;
  int tang_refine, radial_layers, L;
} hhg_problem;

/* Per-request record: times in seconds since the server was created. */
typedef struct {
  double t_submit, t_start, t_end;
  int cycles;               /* V-cycles run (with continuous batching: until its last right-hand side stopped) */
  int reused;               /* 1 if a resident hierarchy served it, 0 if one was built */
  hhg_status status;
  int batch_rhs;            /* right-hand sides of the solve it ran in (its own, plus merged requests') */
} hhg_request_info;

/* Vector length and unknown count of a problem (no GPU work). */
hhg_status hhg_problem_nodes(const hhg_problem* p, int64_t* n_total, int64_t* n_free);

hhg_status hhg_server_create(const hhg_server_desc* desc, hhg_server** out);

/* Queues a request; f_host holds nrhs vectors of hhg_problem_nodes' n_total
 * doubles (copied before return).  *ticket identifies it. */
hhg_status hhg_server_submit(hhg_server* srv, const hhg_problem* p, const double* f_host, int nrhs,
                             int64_t* ticket);

/* Waits for a request; copies its solutions (nrhs vectors) to u_host and the
 * final relative residuals to relres (both nullable) and returns the
 * request's own status (HHG_ENOCONV, HHG_ENOMEM when it can never fit the
 * budget, ...).  A ticket can be waited for once. */
hhg_status hhg_server_wait(hhg_server* srv, int64_t ticket, double* u_host, double* relres,
                           hhg_request_info* info);

/* Resident hierarchies and their bytes, and the hierarchies built and
 * evicted since hhg_server_create (diagnostics; every pointer nullable). */
hhg_status hhg_server_stats(hhg_server* srv, int* n_resident, size_t* bytes_resident, int64_t* n_built,
                            int64_t* n_evicted);

/* Waits for every queued request, then frees all hierarchies. */
hhg_status hhg_server_destroy(hhg_server* srv);

/* ---- Residual without allocation (no counterpart in the paper) ----------
 * Some callers cannot allocate device memory at the moment they need a
 * residual: code in a latency-critical loop that must not stall on the
 * device-wide synchronisation cudaMalloc/cudaFree can imply, and processes
 * whose device memory is reserved up front by a pool allocator (a framework's
 * caching allocator), where a raw cudaMalloc fails or fragments the pool.
 * For them this entry
 * point computes the same r = f - L u and ||r||^2 as hhg_residual without
 * allocating anything: the per-block partial sums of the norm go to a fixed
 * array of HHG_NOALLOC_SCRATCH doubles (128 KiB) that lives in the library
 * image; every GPU that loads the library holds it until the process exits.
 *   - FP64, one right-hand side, device pointers only (host pointers would
 *     need staging buffers: HHG_EINVAL);
 *   - norm2_dev: device address of one double that receives ||r||_2^2;
 *     nothing is copied to the host and the call does not wait;
 *   - a level needs (macro cells + lower-primitive blocks) partial slots;
 *     levels that need more than HHG_NOALLOC_SCRATCH are rejected with
 *     HHG_EINVAL (the 3840-cell shell needs 7936);
 *   - the first call on a device looks up the array's device address and
 *     caches it; make that first call before any stream capture;
 *   - all calls share the array and it keeps the last call's partial sums:
 *     calls whose work overlaps on the GPU (different streams, or different
 *     host threads) race on it and must be serialised by the caller.  Each
 *     call overwrites every slot it reads, so no clearing is needed. */
#define HHG_NOALLOC_SCRATCH 16384
hhg_status hhg_residual_noalloc(hhg_shell* shell, int L, hhg_op op, const double* u,
                                const double* f, double* r, double* norm2_dev, void* stream);

/* ---- Diagnostics (not part of the method) ------------------------------ */

/* Number of CUDA kernels this library has launched in this process. */
int64_t hhg_launch_count(void);

/* Kernel classes timed by hhg_timing. */
typedef enum {
  HHG_T_CELL_SMOOTH = 0,     /* finest-level cell-interior smoother (4 colours) */
  HHG_T_CELL_RESIDUAL = 1,   /* finest-level cell-interior residual */
  HHG_T_CELL_APPLY = 2,      /* finest-level cell-interior apply */
  HHG_T_COARSE = 3,          /* coarsest-level solves; count = CG iterations */
  HHG_T_FIT = 4,             /* hhg_fit_surrogate calls */
  HHG_T_SMOOTH = 5,          /* full sweeps on every level (all 10 steps) */
  HHG_T_RESIDUAL = 6,        /* residuals on every level */
  HHG_T_TRANSFER = 7,        /* restrictions and prolongations */
  HHG_T_COUNT = 8
} hhg_timer;

/* enable != 0: from now on every launch of a timed class is bracketed by
 * CUDA events on the stream it runs on; enable = 0 stops and clears the
 * record.  hhg_timing_read waits for the recorded events and returns the
 * summed stream time (ms) and the number of bracketed calls (for
 * HHG_T_COARSE: the number of conjugate-gradient iterations). */
hhg_status hhg_timing(hhg_shell* shell, int enable);
hhg_status hhg_timing_read(hhg_shell* shell, int which, double* total_ms, int64_t* launches);

/* Launch configuration the tuner chose for the FP32 surrogate smoother on
 * level L (the tuner times the candidates on the device once the FP32
 * buffers exist and after every fit): *cfg = -1 for the per-colour
 * thread-per-node kernel, -2 for the same with two nodes per thread in
 * flight, 0..3 for the shared-memory staged one-launch kernel with
 * (wavefront skew, threads per CTA) = (1, 256), (1, 1024), (2, 128),
 * (2, 512), 4..5 for the plane-wavefront one-launch kernel (u in place
 * through the caches) with 128 and 256 threads per CTA, 6 for the
 * per-colour kernel over chunks of up to 4 points of a line, 7 for the
 * cell-resident sweep (each cell's interior held in the shared memory of a
 * cluster of 1..8 CTAs for the four colour steps); -9 if not
 * tuned.  ms (nullable, 10 entries) receives each candidate's best time for one cell
 * sweep, candidate cfg at ms[cfg + 2] (-1 = not run).  The FP32 apply and
 * residual use the two-nodes variant when the smoother does.  Batched calls
 * (nrhs > 1) smooth with the per-colour kernel that forms every node's
 * weights once for all right-hand sides. */
hhg_status hhg_tuning(const hhg_shell* shell, int L, int* cfg, double* ms);

/* Pins the FP32 surrogate smoother of level L to configuration cfg (-2, -1,
 * a staged configuration 0..3, a wavefront configuration 4..5, the
 * chunked configuration 6 or the cell-resident configuration 7 as above)
 * until the next fit; a one-launch configuration that does not fit the
 * level falls back to the per-colour kernel at launch.  HHG_EINVAL for an
 * unknown cfg. */
hhg_status hhg_set_tuning(hhg_shell* shell, int L, int cfg);

/* Kernels of the single-right-hand-side FP64 surrogate apply, residual and
 * smoother (Sec. 3.4).  variant 0 (the default): a thread per point, each
 * weight evaluated by integer Horner from the plane table, one launch per
 * colour.  variant 1: a thread per run of up to 8 points of one line (one
 * colour, or consecutive points), each weight reached by exact integer
 * forward differences along the run (Eq. 5.4), one launch per colour.
 * variant 2: the run kernels, with the smoother's four colour steps as one
 * cell-resident sweep (each cell's interior held in the shared memory of a
 * cluster of CTAs) where the cell fits.  All give bitwise the same results;
 * the choice only changes speed (on a GB300 the default is the fastest).
 * HHG_EINVAL for another value. */
hhg_status hhg_set_fp64_kernel(hhg_shell* shell, int variant);

/* Host-side tables of the run and cell-resident kernels (the paper has no
 * counterpart; no GPU work, for host-side tests).  hhg_run_lists: the run
 * lists of a cell at N (4 <= N <= 1023): items (nullable, 2 uint32 per run,
 * cap runs) = packed (i0 | j << 10 | k << 20, count | deep << 8); off6 (6
 * ints) = start of colour 0..3 (points i0, i0 + 4, ..) and of all points
 * (i0, i0 + 1, ..), off6[5] = total; kidx (nullable, 8 (N + 1) ints) = per
 * colour g, plane k = 0..N and part (0 deep-interior runs, 1 runs next to
 * the cell boundary) the first run of the part on a plane >= k, relative to
 * off6[g]; *n_items (nullable) = the number of runs.  HHG_EINVAL for N out
 * of range or a buffer too small.  hhg_slab_planes: the planes [k_bounds[r],
 * k_bounds[r + 1]) held by cluster rank r of the cell-resident sweep with
 * `cluster` CTAs per cell (1..8) at N (8 <= N <= 1023), k_bounds of
 * cluster + 1 ints; HHG_EINVAL otherwise. */
hhg_status hhg_run_lists(int N, uint32_t* items, int64_t cap, int* off6, int* kidx, int64_t* n_items);
hhg_status hhg_slab_planes(int N, int cluster, int* k_bounds);

/* The FP64 kernel variant in effect and, for level L, the CTAs per cluster
 * of the cell-resident smoother sweep (0 when the smoother runs one launch
 * per colour: another variant, no fit yet, or a cell too large for the
 * shared memory of 8 CTAs). */
hhg_status hhg_fp64_kernel(hhg_shell* shell, int L, int* variant, int* cluster);

/* Throughput of one arithmetic pipe on the current device (the paper has
 * no counterpart: these are the roofline denominators of the FP64 and FP32
 * stencil kernels).  kind 0: FP64 fused multiply-add, 1: FP32 fused
 * multiply-add, 2: INT32 multiply-add.  A kernel of 8 independent
 * multiply-add chains per thread, 8 CTAs of 256 threads per SM, runs for
 * about 150 ms (calibrated), best of three; *ops_per_s receives the
 * multiply-adds per second (one FMA = 2 flops), *ms (nullable) the time of
 * the best run.  Waits for the stream; allocates a small output buffer on
 * it (stream-ordered). */
hhg_status hhg_peak_rate(int kind, double* ops_per_s, double* ms, void* stream);

/* The hand-written arithmetic helpers of the surrogate kernels applied
 * elementwise to n device values (the paper has no counterpart; tests
 * compare them with the IEEE operations):
 *   which 0: out[t] = a[t] / b[t], FP32, reciprocal estimate + one
 *            Newton-Raphson step (the staged FP32 smoother's divide);
 *   which 1: out[t] = 2^E / W with W = ((const int64_t*) a)[t] != 0 and
 *            E = ((const int*) b)[t]: the integer-pipe reciprocal of the
 *            FP64 surrogate's centre weight (FP32 estimate, two fixed-point
 *            Newton-Raphson steps);
 *   which 2: out[t] = W 2^-E (W, E as for 1), integer-pipe conversion with
 *            the scale undone, truncated toward zero.
 * Device pointers; does not wait. */
hhg_status hhg_check_arith(int which, const void* a, const void* b, void* out, int64_t n, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* hhg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HHG_H */
