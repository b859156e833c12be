/*
 * mg.h -- C ABI of the GB300 additive multilevel Helmholtz solver.
 *
 * The library solves the p-dimensional Helmholtz model
 *     [-Laplace - phi] psi = chi   on (0,1)^d, zero Dirichlet boundary,
 * (Section 2, Eq. pHelmholtz, phi = k^2) with d-linear finite elements on the
 * regular levels l = 1..L of a tripartitioned spacetree (Section 3) and
 * complex grid spacing h e^{i theta} inside an exterior scaling layer
 * (Section 2 "complex scaled grid", Section 7.3-7.4).  One call of mg_cycle
 * is one additive FAS cycle (Algorithm 2 / Appendix A Algorithm 4):
 * residual and hierarchical residual on every level, restriction to every
 * coarser level, damped Jacobi on all levels at once, then correction and
 * prolongation back to the fine grid.
 *
 * Conventions shared by every call
 *  - d is 2, 3 or 4; level l has n = 3^l cells per axis and (n+1)^d
 *    vertices including the Dirichlet ring.  Vertex arrays are row-major with
 *    x fastest: index = x + (n+1)*(y + (n+1)*(z + (n+1)*w)).  Complex values
 *    are interleaved (re, im) FP64 pairs (mg_c128).  Boundary entries are
 *    zero.
 *  - d = 4 (p = 4 of Section 7.1) takes a constant k2_field and depth <= 4,
 *    runs mg_set_rhs/_vector, mg_set_solution, mg_get_solution, mg_get_level,
 *    mg_cycle, mg_residual_norm/_max, mg_last_cycle_norm, mg_solve and
 *    mg_set_precision; the other calls return MG_ERR_INVALID for it.
 *  - A host pointer to page-locked memory (cudaHostAlloc, cudaHostRegister)
 *    is read or written by kernels directly over the host link; pageable
 *    memory is staged through cudaMemcpyAsync.
 *  - Pointers marked "host or device" are read on the host when the
 *    accompanying on_device flag is 0 and as device pointers of the current
 *    CUDA device otherwise.  The caller keeps ownership of every array it
 *    passes; the library copies what it needs before returning.
 *  - Every call returns an MG_* status and never aborts; no C++ exception
 *    crosses the ABI.  Arguments are validated before any device work.
 *    mg_last_error returns a human-readable message of the last failure of
 *    a context.  Device work is enqueued on the context's stream;
 *    asynchronous device errors surface as MG_ERR_CUDA at the next
 *    synchronising call (mg_residual_norm, mg_solve, mg_get_solution with a
 *    host destination).
 *  - A context owns every device buffer it allocates and frees them in
 *    mg_destroy.  Contexts are not thread-safe; distinct contexts are
 *    independent.
 */
#ifndef MG_H
#define MG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;
typedef struct { double re, im; } mg_c128;

enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,    /* bad argument; nothing was enqueued               */
  MG_ERR_CUDA = 2,       /* a CUDA runtime call failed                       */
  MG_ERR_OOM = 3,        /* device allocation failed                         */
  MG_DIVERGED = 4,       /* relative residual > 1e6, NaN or Inf (Table 2 bottom) */
  MG_NOT_CONVERGED = 5,  /* max_cycles reached above tol                     */
  MG_ERR_TIMEOUT = 6     /* a bounded device-side wait gave up               */
};

/* Relaxation variant (Section 5.2): MG_HB masks the Jacobi update at
 * c-points, Eq. hb-omega.  Transfer: MG_DLINEAR adds the update as is
 * (T = id); MG_HIERARCHICAL adds only its hierarchical surplus
 * T = (id - P I), the BPX prolongation of Appendix A.  MG_BPX is
 * MG_ADD with MG_HIERARCHICAL. */
enum { MG_ADD = 0, MG_HB = 1, MG_BPX = 2 };
enum { MG_DLINEAR = 0, MG_HIERARCHICAL = 1 };
/* Arithmetic of the cycles: complex128 throughout, or complex64 cycles with
 * FP32 accumulation inside an FP64 defect-correction loop (fine residual,
 * solution update and norms in FP64). */
enum { MG_C128 = 0, MG_C64_REFINE = 1 };
/* Relaxation schemes of the Section 5.1 table (succ = L - l on a regular grid). */
enum { MG_OMEGA_JACOBI = 0, MG_OMEGA_UCG = 1, MG_OMEGA_LGRID = 2, MG_OMEGA_EXP = 3,
       MG_OMEGA_TRANSITION = 4 };

/* Creates a solver for the hierarchy of depth L = depth (levels 1..L).
 *  k2_field   host, (3^L+1)^d FP64 values of phi = k^2 at the fine vertices
 *             (Section 4: phi is a per-vertex weight).  Coarse levels sample
 *             it at their own vertices (injection); a cell uses the mean of
 *             its 2^d vertex values.  A constant field takes a faster path.
 *  theta      rotation angle of the complex spacing, 0 <= theta < pi/2.
 *  layer_width  0 <= w <= 0.5: along each axis, a cell whose centre lies
 *             closer than w to a face has spacing h e^{i theta}
 *             (coordinate-wise exterior scaling); w = 0.5 rotates every cell
 *             (the complex scaled grid of Section 7.3).
 * The solution starts at zero and the rhs at zero.
 * Errors: MG_ERR_INVALID (d not in {2,3,4}, depth < 1 or too deep for the
 * device, theta or w out of range, a varying k2_field with d = 4, NULL
 * pointers), MG_ERR_OOM, MG_ERR_CUDA. */
int mg_create(int d, int depth, const double* k2_field, double theta,
              double layer_width, mg_ctx** out);

/* Same as mg_create with a general coordinate-wise scaling (the channel
 * problem of Section 7.4: a 30 degree layer at the two open faces and an
 * interior rotation theta applied independently of it).  Along every axis a
 * cell whose centre c satisfies c < width_lo or 1 - c < width_hi lies in the
 * layer and has spacing h e^{i theta_layer}; every other cell has spacing
 * h e^{i theta_interior}.  Layers that together cover the axis
 * (width_lo + width_hi >= 1) rotate every cell.  mg_create(d, depth, k2,
 * theta, w) is mg_create_ecs(d, depth, k2, theta, 0, w, w).
 *  theta_layer, theta_interior   in [0, pi/2)
 *  width_lo, width_hi            in [0, 1]
 * A rotated interior makes every stencil row complex, so the fast kernels
 * that take the interior rows as real are not used.
 * Errors: as mg_create. */
int mg_create_ecs(int d, int depth, const double* k2_field, double theta_layer,
                  double theta_interior, double width_lo, double width_hi,
                  mg_ctx** out);

/* A solver on an adaptive spacetree with hanging vertices (the adaptive
 * Cartesian grids of Section 3; hanging vertices and FAS injection of
 * Section 4).  Level 1 has all 3^d cells; a level-l cell flagged in refine
 * splits into 3^d level-(l+1) cells.  A vertex whose 2^d cells of its level
 * do not all exist is hanging: its value is the d-linear interpolation from
 * the next coarser level.  The cycle is the additive correction scheme on
 * the hierarchical generating system (the form Lemma 2 / Theorem 2 prove
 * the FAS cycle equal to): every level's residual is the cell-wise residual
 * of its leaves plus the restricted residual of the next finer level
 * (including the partial residuals of hanging vertices).  Relaxation factors
 * are per vertex (Section 5.1 table): mg_cycle's omega[depth - 1 - s] is the
 * factor of the vertices with succ(v) = s, where succ(v) = 0 unless all 2^d
 * cells around v are refined, else 1 + the minimum of succ over v's children
 * that carry unknowns; on a fully refined tree succ = depth - l, the regular
 * grid's level factors.
 *  d          2 or 3;  k2_field, theta_layer, theta_interior, width_lo,
 *             width_hi: as mg_create_ecs.
 *  refine     host, the flags of levels 1..depth-1 concatenated: level l's
 *             (3^l)^d bytes (x fastest), nonzero = refine; flags of cells
 *             that do not exist are ignored.  The deepest levels may hold
 *             no cells yet (mg_adapt can fill them).
 * Runs mg_set_rhs, mg_set_solution and mg_get_solution (nodal values on the
 * uniform finest grid; mg_get_solution returns the fine-grid function, d-
 * linear on each leaf), mg_get_level (which = 0: the level's values, 1: its
 * residual of the last cycle), mg_cycle, mg_residual_norm and mg_residual_max
 * (over the fine-grid vertices: unknowns with no unknown at the same point on
 * the next finer level), mg_last_cycle_norm, mg_solve in complex128,
 * mg_adapt and mg_get_refinement; the other calls return MG_ERR_INVALID.
 * Arrays are dense over every level's full grid; kernels run over the
 * bounding box of each level's existing vertices.
 * Errors: as mg_create_ecs, and MG_ERR_INVALID for a NULL refine or d = 4. */
int mg_create_adaptive(int d, int depth, const double* k2_field, double theta_layer,
                       double theta_interior, double width_lo, double width_hi,
                       const unsigned char* refine, mg_ctx** out);

/* One step of feature-based dynamic refinement and erasing (Section 5.3) on
 * an adaptive context, all on the device but for choosing the bins:
 *  1. s(v) = max over the axes of |u(v - e) - 2 u(v) + u(v + e)| (undivided
 *     second differences of the level's values) at every fine-grid vertex;
 *  2. the span [min s, max s] is split into `bins` equal subranges; the k top
 *     bins whose vertex count is closest to refine_frac x (fine-grid
 *     vertices) are refined, the k' bottom bins closest to erase_frac x
 *     (fine-grid vertices) erased (the smallest k, k' on ties; a vertex in
 *     both sets is refined);
 *  3. vetoes: |r(v) / H_l[v, v]| > veto (the vertex still changes: r is the
 *     current generating-system residual; with veto_relative nonzero, >
 *     veto |u(v)|: the update exceeds that fraction of the value), refining
 *     on level depth (h_min),
 *     and erasing below min_level + 1 (h_max: min_level is the level of the
 *     coarsest admissible grid, whose cells stay);
 *  4. refining a vertex refines its 2^d cells; a refined cell of level
 *     l >= min_level loses its children when they are leaves, none is being
 *     refined and every fine-grid vertex of level l + 1 on the closed cell is
 *     erased (one level of coarsening per step);
 *  5. vertices that exist after the step and did not carry an unknown both
 *     before and after it take P u_(l-1) (zero hierarchical surplus), then
 *     coarse copies of finer unknowns are injected.  Pure refinement leaves
 *     the fine-grid function unchanged.
 *  refine_frac, erase_frac   in [0, 1] (the paper: 0.1, 0.02)
 *  bins                      in [1, 64] (the paper: 20)
 *  veto                      > 0 (the paper: 1e-2; +inf disables it)
 *  veto_relative             0: absolute bound, nonzero: relative to |u(v)|
 *  min_level                 in [1, depth]
 *  stats                     host long long[4] or NULL: vertices selected for
 *                            refining, for erasing, fine-grid vertices after
 *                            the step, finest level holding cells.
 * Synchronises the stream once (counts and new bounding boxes); the step and
 * the cycles run as CUDA graphs again once they repeat on the same finest
 * level and grid capacities.  The reference residual of mg_solve and
 * mg_residual_norm (the first one after mg_set_rhs or mg_set_solution) is
 * kept across steps, so relative residuals compare with the start grid.
 * Errors: MG_ERR_INVALID (not adaptive, arguments out of range),
 * MG_DIVERGED (a non-finite indicator: the grid is left as it is),
 * MG_ERR_CUDA. */
int mg_adapt(mg_ctx* ctx, double refine_frac, double erase_frac, int bins, double veto, int veto_relative,
             int min_level, long long* stats);

/* The current refine flags of an adaptive context in mg_create_adaptive's
 * layout (levels 1..depth-1 concatenated, x fastest, 1 = refined).
 *  refine   host, sum over l < depth of (3^l)^d bytes.  Synchronising.
 * Errors: MG_ERR_INVALID (NULL, not adaptive), MG_ERR_CUDA. */
int mg_get_refinement(mg_ctx* ctx, unsigned char* refine);

/* Releases every device buffer of the context (NULL is ignored). */
void mg_destroy(mg_ctx* ctx);

/* Enqueues all later work on this cudaStream_t (0 = legacy default stream). */
int mg_set_stream(mg_ctx* ctx, void* cuda_stream);

/* Nodal right-hand side f (host or device, fine-vertex layout).  The library
 * forms b_L = M_L f with the consistent, complex-scaled mass matrix
 * (Section 4: chi holds the weight of the discretised right-hand side).
 * Resets the reference residual used by relative norms. */
int mg_set_rhs(mg_ctx* ctx, const mg_c128* f_nodal, int on_device);

/* Sets the fine solution u (host or device); boundary entries are ignored.
 * Clears any pending correction and the reference residual. */
int mg_set_solution(mg_ctx* ctx, const mg_c128* u, int on_device);

/* Writes the current fine solution, with every correction of the cycles
 * run so far applied, to out (host or device, fine-vertex layout).
 * Synchronises the stream when out is a host pointer. */
int mg_get_solution(mg_ctx* ctx, mg_c128* out, int on_device);

/* One additive FAS cycle (Algorithm 2; Appendix A Algorithm 4) on levels
 * 1..L.  omega_per_level: host, L complex relaxation factors, index l-1
 * (Section 5.1: one factor per level; on an adaptive context entry
 * L - 1 - s serves the vertices with succ(v) = s, see mg_create_adaptive).
 * variant MG_ADD/MG_HB/MG_BPX and transfer MG_DLINEAR/MG_HIERARCHICAL as
 * above.  Asynchronous. */
int mg_cycle(mg_ctx* ctx, int variant, const mg_c128* omega_per_level, int transfer);

/* Euclidean norm of the fine residual b - H u over the fine vertices and
 * its ratio to the residual of the starting solution (Section 7 norms; on a
 * regular grid the h-weighted norm gives the same ratio).  Synchronising. */
int mg_residual_norm(mg_ctx* ctx, double* abs_l2, double* rel_l2);

/* Maximum modulus of the fine residual b - H u over the vertices (the max
 * norm of the Section 7.4 table), computed on the device; a non-finite
 * entry gives +infinity.  The first call allocates one fine-size complex128
 * buffer (an adaptive context: the max over its fine-grid vertices, fused
 * into the residual pass, no allocation).  Synchronises the stream.
 * Errors: MG_ERR_INVALID (NULL), MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_TIMEOUT. */
int mg_residual_max(mg_ctx* ctx, double* abs_max);

/* Residual norm of the iterate that entered the last complex128 cycle, as
 * fused into that cycle's finest-level sweep (no extra pass); rel_l2 is -1
 * when no reference residual exists yet.  Synchronising. */
int mg_last_cycle_norm(mg_ctx* ctx, double* abs_l2, double* rel_l2);

/* Runs cycles until the relative residual is <= tol (MG_OK), max_cycles
 * were run (MG_NOT_CONVERGED) or the iteration diverged (MG_DIVERGED).
 * With precision MG_C128 every cycle is the plain complex128 cycle; with
 * MG_C64_REFINE see mg_set_precision.  cycles_done counts fine-grid cycles
 * (inner cycles for the refinement form); rel_res is the final relative
 * FP64 residual.  Either output pointer may be NULL. */
int mg_solve(mg_ctx* ctx, int variant, const mg_c128* omega, int transfer, double tol,
             int max_cycles, int* cycles_done, double* rel_res);

/* Selects the arithmetic of mg_solve.  MG_C64_REFINE: each outer step forms
 * r = b - H u in FP64, runs inner_cycles complex64 cycles on H e = r from
 * e = 0, and adds e to u in FP64. */
int mg_set_precision(mg_ctx* ctx, int precision, int inner_cycles);

/* Grid unfolding (Section 5 remark on FMG; Section 7.1): stages s = 1..L-1
 * solve on levels 1..s with b_s = M_s f_s and run cycles_per_stage cycles,
 * each stage starting from the d-linear interpolation of the previous one;
 * the fine solution is then set to the interpolation of stage L-1.  Level
 * l of stage s uses omega[l-1 + L-s].  Needs mg_set_rhs first. */
int mg_fmg(mg_ctx* ctx, int variant, const mg_c128* omega, int transfer, int cycles_per_stage);

/* Host helper: fills out[0..depth-1] with the relaxation factors of one
 * Section 5.1 scheme, succ = depth - l: Jacobi only, undamped coarse grid,
 * undamped L-grid (l_grid), exponential omega_s^(succ+1) or transition
 * omega_s^((1-1/iter_n)(succ+1)). */
int mg_omega_scheme(int scheme, mg_c128 omega_s, int depth, int iter_n, int l_grid,
                    mg_c128* out);

/* Copies one per-level device array to out (host or device) for inspection:
 * which = 0 solution (fine: with pending corrections applied; coarse: the
 * injected copy the last cycle used), 1 right-hand side b_l.  Synchronises
 * when out is a host pointer. */
int mg_get_level(mg_ctx* ctx, int level, int which, mg_c128* out, int on_device);

/* ---- adjoint (far-field functional) form; not in the paper ----------------
 * Forward problem H(V) u = M f with k^2 = E - V; functional
 * s = sum_q w_q u(x_q) (d-linear samples of the fine solution), J = |s|^2. */

/* Replaces the fine k^2 field (fine-vertex layout, (3^depth+1)^d values, x
 * fastest) of a context that was created with a varying field; coarse levels
 * and cell shifts follow (a cell takes the mean of its vertex values, coarse
 * levels sample the field at their own vertices).  on_device = 0: k2_field is
 * host memory, checked for finite values (MG_ERR_INVALID otherwise),
 * synchronising.  on_device = 1: k2_field is device memory; it is copied and
 * the cell shifts are formed on the context's stream, with no host round
 * trip and no synchronisation (the pointer must stay valid until the stream
 * reaches the call; values are not checked: a non-finite field shows up as a
 * diverged or non-finite solve).  MG_ERR_INVALID for contexts created with a
 * constant field, d = 4 and adaptive contexts. */
int mg_set_k2(mg_ctx* ctx, const double* k2_field, int on_device);

/* Sets the fine right-hand side vector b_L itself (host or device), instead
 * of M f; boundary entries are ignored. */
int mg_set_rhs_vector(mg_ctx* ctx, const mg_c128* b, int on_device);

/* s = sum_q w_q u(x_q) of the current fine solution; xyz: host, npts points
 * of d coordinates in [0,1] (x first); w: host weights; out: host.
 * Synchronising. */
int mg_sample(mg_ctx* ctx, int npts, const double* xyz, const mg_c128* w, mg_c128* out);

/* Sets b_L = a with a_v = sum_q w_q psi_v(x_q): the adjoint right-hand side
 * of the sampled functional (the transpose of mg_sample; unconjugated). */
int mg_set_rhs_samples(mg_ctx* ctx, int npts, const double* xyz, const mg_c128* w);

/* Gradients of J = |s|^2 from the forward solution u and the adjoint
 * solution lambda of H lambda = a (device arrays, fine layout; H is
 * complex-symmetric, so H^T = H):
 *   dJdV[v] = 2 Re( conj(s) * (-2^-d) sum_{cells c at v} lambda_c^T M_c u_c )
 *   dJdf[v] = 2 Re( conj(s) * (M lambda)_v )          (real nodal f)
 * for every fine vertex (boundary included), device outputs (either may be
 * NULL).  Asynchronous. */
int mg_adjoint_grad(mg_ctx* ctx, const mg_c128* u, const mg_c128* lambda, mg_c128 s,
                    double* dJdV, double* dJdf);

/* ---- batched form; not in the paper (its multichannel idea, Section 7.5) --
 * n independent 2D problems of any depths, each with a constant k^2, solved
 * together: every outer defect-correction step of every problem (FP64
 * residual, inner_cycles complex64 cycles, FP64 update) runs in ONE
 * persistent launch whose work items (problem, stage, tile) are taken from a
 * queue in dependency order, replayed as a CUDA graph. */
typedef struct mg_batch mg_batch;

/* Creates n contexts (arrays d, depth, theta, layer_width of n entries; k2:
 * n host pointers to fine k^2 fields that must each be constant).  The batch
 * owns the contexts.  MG_ERR_INVALID for 3D or varying-k^2 problems. */
int mg_batch_create(int n, const int* d, const int* depth, const double* const* k2,
                    const double* theta, const double* layer_width, mg_batch** out);
void mg_batch_destroy(mg_batch* batch);

/* Context of problem p (owned by the batch): set its rhs, solution, read
 * its solution or run single-problem calls on it with the mg_* API. */
int mg_batch_get_ctx(mg_batch* batch, int p, mg_ctx** out);

/* Enqueues the batch's work (and its contexts' work) on this stream. */
int mg_batch_set_stream(mg_batch* batch, void* cuda_stream);

/* Solves every problem to relative FP64 residual tol (relative to its
 * residual at the start of the call), at most max_outer outer steps of
 * inner_cycles complex64 cycles each.  Each step measures the residual of
 * the iterate entering it, so a problem leaves the batch after the step
 * whose entering residual is at most tol; that step is still applied to it
 * (and counted).  omega: n host pointers, problem p's has depth_p entries.
 * Per problem: status (MG_OK / MG_NOT_CONVERGED / MG_DIVERGED, the first
 * two from the FP64 residual of the returned solution), inner cycles run and
 * final relative residual (any output may be NULL).  Returns MG_OK unless
 * the call itself failed. */
int mg_batch_solve(mg_batch* batch, int variant, const mg_c128* const* omega, int transfer,
                   double tol, int max_outer, int inner_cycles, int* status, int* cycles,
                   double* rel_res);

/* Autotuner: times one outer step of the batch for every candidate fine tile
 * (4 or 8 coarse cells per edge) and persistent residency (2, 4 or 8 blocks
 * per SM), keeps the fastest for later solves and restores the solutions.
 * Outputs (may be NULL): chosen tile, residency, its time per outer step. */
int mg_batch_autotune(mg_batch* batch, int variant, const mg_c128* const* omega, int transfer,
                      int inner_cycles, int* tile_out, int* blocks_per_sm_out, double* ms_out);

/* Persistent launches issued by the batch so far. */
long long mg_batch_launches(const mg_batch* batch);
const char* mg_batch_last_error(const mg_batch* batch);

/* Bound on every device-side wait of the persistent launches, in polls
 * (default 2^22, about a second; each poll sleeps 64-256 ns).  When a wait
 * runs out, the kernel records it and finishes without hanging; the next
 * synchronising call returns MG_ERR_TIMEOUT and the results of the affected
 * cycles are invalid.  polls >= 1. */
int mg_set_spin_limit(mg_ctx* ctx, unsigned polls);

/* Diagnostic for failure handling: while enabled, the first item of every
 * coarse-chain launch also waits on a device counter that nothing ever
 * increments, so the wait must run out (use a small mg_set_spin_limit).  The
 * launch still completes; the next synchronising call reports
 * MG_ERR_TIMEOUT.  2D contexts with a constant shift (the persistent path). */
int mg_debug_unsatisfiable_wait(mg_ctx* ctx, int enable);

/* Instrumentation.  mg_set_timing(ctx, 1) makes every later cycle record a
 * CUDA event pair around its finest-level sweep kernel on the context's
 * stream.  mg_get_stats synchronises the stream and returns, since the last
 * mg_get_stats call: the number of kernels the context launched, the number
 * of timed fine sweeps and their summed device time in milliseconds; it
 * then resets all three.  Any output pointer may be NULL. */
int mg_set_timing(mg_ctx* ctx, int enable);
int mg_get_stats(mg_ctx* ctx, long long* kernel_launches, int* fine_sweeps,
                 double* fine_sweep_ms);

/* Per-item trace of the persistent launches (2D FP64 path): with tracing on,
 * every tile of the finest-level sweep and every item of the coarse chain
 * records {taken, dependencies met, done, SM id} (globaltimer ns) into a
 * device buffer, overwritten by each cycle.  mg_get_trace synchronises and
 * copies fine_slots fine-sweep records (indexed by queue position) followed by
 * chain_slots chain records (indexed by item) to out (host, 4 x u64 each).
 * Both counts are at most 65536.  Turning tracing on or off drops captured
 * cycle graphs. */
int mg_set_trace(mg_ctx* ctx, int enable);
int mg_get_trace(mg_ctx* ctx, unsigned long long* out, int fine_slots, int chain_slots);

/* Allocation-free fine residual (the paper has no counterpart; it serves
 * callers that cannot allocate device memory when they need a residual, such
 * as frameworks that reserve the whole device for their own pool, or
 * time-critical loops that cannot take the implicit synchronisation of
 * cudaMalloc/cudaFree).  u and b are device arrays in the fine-vertex layout
 * (u's Dirichlet ring must hold zeros); r (device, may be NULL) receives
 * b - H_L u on the interior and zero on the boundary; norm2 (device, one
 * double) receives the FP64 sum of |r|^2 over the interior vertices.  Work is
 * enqueued on the context's stream; the call allocates nothing.
 * Scratch: the per-block partial sums and the completion ticket live in a
 * file-scope device array of 16384 doubles + 256 bytes that every GPU which
 * loads the library holds until exit.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with the device
 * current), so make the first call on each device before any stream capture;
 * later calls outside capture look it up again (a device reset may move it),
 * calls during capture use the cached address.  The context's device (the
 * one current at mg_create) must be current: MG_ERR_INVALID otherwise.
 * Every call shares the array and it keeps the last call's contents (the
 * call clears the ticket itself); calls whose kernels overlap on the GPU
 * race on it.  Limit: one block per 256 vertices and one partial per block,
 * so fine grids above 16384 * 256 = 4,194,304 vertices (2D depth >= 7,
 * 3D depth >= 5) are rejected with MG_ERR_INVALID. */
int mg_residual_noalloc(mg_ctx* ctx, const mg_c128* u, const mg_c128* b, mg_c128* r,
                        double* norm2);

/* Message of the last failure on this context ("" if none); ctx may be NULL
 * for failures of mg_create. */
const char* mg_last_error(const mg_ctx* ctx);

/* ---- coupled multichannel form (Section 7.5, Eq. coupledHelmholtz) -------
 * c channels of the Helmholtz problem fused into one grid: every vertex
 * carries a C^c tuple, and the operator keeps the couplings inside the
 * block (the matrix A-hat of Section 7.5):
 *     (A u)_i = K u_i - sum_j Phi_ij M u_j,
 * i.e. H_ii = K - phi_i M on the diagonal and A_ij = -kappa_ij M (a constant
 * coupling potential times the mass matrix) off it, with the complex-scaled
 * d-linear K and M of the single-channel form (coordinate-wise layer of
 * width layer_width and angle theta).  One cycle is Algorithm 4 on tuples
 * with damped block-Jacobi smoothing, du_v = omega_l D_v^{-1} r_v, D_v the
 * c x c diagonal block of A at v; restriction, prolongation, injection, the
 * hb mask and the BPX transfer act channel by channel.  It runs the plain
 * (not single-touch pipelined) form of the cycle.
 * Layout: tuple arrays hold (3^depth+1)^d vertices x c channels, channel
 * fastest (index = vertex * c + channel), vertices as in the single-channel
 * form.  d is 2 or 3; c is 1, 2, 3, 4, 8 or 16. */
typedef struct mg_mc_ctx mg_mc_ctx;

/* phi: host, c x c complex matrix, row-major (phi_i = Phi_ii, kappa_ij =
 * Phi_ij); finite values.  The same Phi serves every level.  MG_ERR_INVALID
 * for d, depth, c, theta or layer_width out of range or a singular diagonal
 * block; MG_ERR_OOM when the arrays do not fit. */
int mg_mc_create(int d, int depth, int channels, const mg_c128* phi, double theta, double layer_width,
                 mg_mc_ctx** out);
int mg_mc_set_stream(mg_mc_ctx* ctx, void* cuda_stream);
/* b = M f channel by channel from nodal f (host or device, tuple layout);
 * resets the reference residual. */
int mg_mc_set_rhs(mg_mc_ctx* ctx, const mg_c128* f_nodal, int on_device);
/* u (host or device, tuple layout); the Dirichlet ring is taken as zero. */
int mg_mc_set_solution(mg_mc_ctx* ctx, const mg_c128* u, int on_device);
/* the current fine solution (host or device); synchronising for host out. */
int mg_mc_get_solution(mg_mc_ctx* ctx, mg_c128* out, int on_device);
/* one cycle; variant MG_ADD / MG_HB, transfer MG_DLINEAR / MG_HIERARCHICAL
 * (MG_BPX = MG_ADD with MG_HIERARCHICAL), omega_per_level[depth] (index l-1). */
int mg_mc_cycle(mg_mc_ctx* ctx, int variant, const mg_c128* omega_per_level, int transfer);
/* FP64 Euclidean norm of b - A u over all interior vertices and channels,
 * and the same relative to the first norm taken after the last set_rhs /
 * set_solution; synchronising. */
int mg_mc_residual_norm(mg_mc_ctx* ctx, double* abs_l2, double* rel_l2);
const char* mg_mc_last_error(const mg_mc_ctx* ctx);
void mg_mc_destroy(mg_mc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
