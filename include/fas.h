/*
 * fas.h -- C ABI of the GB300 matrix-free FAS multigrid library (libfasmg.so).
 *
 * The library solves  A u = f  with  A u = alpha u - beta div_h(kappa grad_h u)  on a uniform
 * cell-centred grid (Sec. 2.1-2.2 of the paper: cells x_i = (i - 1/2) h, one ghost layer, the
 * 5-point / 7-point operator L_h), by the FAS multigrid of Algorithm 1 with its recursive
 * multilevel remark, X-MCGS smoothing (Sec. 2.3, Eqs. FCGS-1..4; 3D sets of Appendix B), and the
 * average restriction / piecewise-constant prolongation of Appendix C.
 *
 * Conventions shared by every entry point
 *   Layout     Fields are dense C-order arrays with x fastest: 2D index j*nx + i, 3D index
 *              (l*ny + j)*nx + i, 0-based. No ghost cells are stored; boundary conditions are
 *              folded into the point equations (homogeneous Neumann: ghost = adjacent cell;
 *              homogeneous Dirichlet: ghost = -adjacent cell, Eqs. boundry1-2).
 *   Ownership  Field pointers passed to fas_vcycle / fas_solve / fas_heat_run are DEVICE pointers
 *              owned by the caller and must stay valid until the call returns (the library may
 *              enqueue work on the stream that reads them; calls return after that work is
 *              complete unless stated otherwise). The library owns only the coarse levels and
 *              scratch it allocates in fas_create and frees in fas_destroy.
 *              The *_host entry points take HOST pointers and do the copies themselves.
 *   Alignment  Every DEVICE field pointer must be 16-byte aligned (the kernels move fields in
 *              16-byte vectors). cudaMalloc and PyTorch allocations are; a view that starts at an
 *              odd element is not. A misaligned pointer is rejected with FAS_EINVAL before any
 *              work is enqueued.
 *   Streams    All device work is enqueued on the cudaStream_t given to fas_create (NULL = the
 *              legacy default stream).
 *   Errors     Every call returns a fas_status; nothing aborts or throws. fas_last_error() gives a
 *              thread-local message for the last failing call on the calling thread.
 *   Threads    A fas_ctx must not be used by two threads at once.
 */
#ifndef FAS_H
#define FAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FAS_OK = 0,
  FAS_EINVAL = 1,        /* invalid argument (sizes not powers of two, h <= 0, nu < 0, ...)  */
  FAS_ENOMEM = 2,        /* device or host allocation failed                                  */
  FAS_ENOTCONV = 3,      /* kmax cycles done without reaching tol; info is filled            */
  FAS_ENONFINITE = 4,    /* residual became NaN/Inf                                           */
  FAS_ETIMEOUT = 5,      /* a bounded device-side wait expired (fas_debug_bounded_wait)       */
  FAS_ECUDA = 6,         /* a CUDA runtime call failed (message in fas_last_error)            */
  FAS_EUNSUPPORTED = 7   /* valid request this build does not implement                       */
} fas_status;

/* Boundary kinds per face. NEUMANN: homogeneous, ghost = adjacent cell. DIRICHLET: homogeneous,
 * ghost = -adjacent cell (Eqs. boundry1-2; values through fas_fold_dirichlet). PERIODIC: the grid wraps
 * around along the axis, as in the grain-growth example of Sec. 3.3.1 (the paper writes no ghost
 * relation for it; here the ghost of the first cell is the last cell and vice versa, and the face
 * between them is an interior face). Both faces of an axis must be PERIODIC or neither; periodic axes
 * need cell-centred unknowns and a constant kappa (FAS_EUNSUPPORTED otherwise) and run the
 * per-operation kernels. With alpha = 0 and no Dirichlet face the operator is singular and is handled
 * like the all-Neumann pressure solve (mean-free right-hand side, mean removed after every cycle). */
typedef enum { FAS_BC_NEUMANN = 0, FAS_BC_DIRICHLET = 1, FAS_BC_PERIODIC = 2 } fas_bc;
typedef enum { FAS_FP64 = 0, FAS_MIXED = 1 } fas_precision;

/* Where the unknowns sit (Sec. 4.1, the MAC staggered grid). FAS_CELL: cell centres (Sec. 2.1).
 * FAS_FACE_X / _Y / _Z: one velocity component on the faces normal to x / y / z. A face field has
 * the cell-field shape: along its own axis, slot s holds face s+1 (faces 1..n-1 are the unknowns)
 * and the last slot holds the far wall face, whose value is 0 and is never changed; the near wall
 * face is not stored and is 0. Every wall is no-slip: the normal component is 0 on its own walls,
 * tangential walls act as homogeneous Dirichlet ghosts (ghost = -adjacent value, Sec. 4.1), so bc[]
 * must be all FAS_BC_DIRICHLET. Smoothing uses the X-MCGS sets by the parity of the face index and
 * the cell indices (Eqs. FCGS-1..4 on faces); restriction and prolongation are those of Appendix D. */
typedef enum { FAS_CELL = 0, FAS_FACE_X = 1, FAS_FACE_Y = 2, FAS_FACE_Z = 3 } fas_location;

/* Problem and solver parameters (the paper's user parameters s, kMax, tol, meshLevel of
 * Algorithm 1's symbol table, plus the operator of Sec. 2.2 generalised to alpha, beta, kappa). */
typedef struct {
  int dim;               /* 2 or 3                                                             */
  int n[3];              /* cells along x, y, z (n[2] ignored in 2D); each a power of two >= 2  */
  double h;              /* uniform spacing on every axis (Sec. 2.1: h = (b-a)/M = (d-c)/N)      */
  double alpha, beta;    /* A u = alpha u - beta div(kappa grad u); heat step: alpha 1, beta dt  */
  const double* kappa;   /* DEVICE pointer to a per-cell diffusivity field, or NULL            */
  double kappa_const;    /* diffusivity used when kappa == NULL                                 */
  int bc[6];             /* fas_bc per face: x_lo, x_hi, y_lo, y_hi, z_lo, z_hi                  */
  int nu1, nu2;          /* pre- and post-smoothing sweeps (the paper's s; default 2, 2)        */
  int nu_coarse;         /* sweeps on the coarsest level (paper: s); <= 0 means nu1             */
  int kmax;              /* maximum V-cycles per solve (kMax)                                  */
  int coarsest;          /* cells along the shortest axis of the coarsest level (>= 2)          */
  int coarse_exact;      /* 0: smooth the coarsest level (paper); 1: dense direct solve         */
  double tol;            /* stopping tolerance                                                 */
  int tol_relative;      /* 1: ||f - A u||_2 <= tol ||f||_2 ; 0: h^{d/2}||f - A u||_2 <= tol    */
  int precision;         /* fas_precision: FP64, or FP32 inner cycles in FP64 refinement        */
  int inner_cycles;      /* FAS_MIXED: FP32 V-cycles per refinement step (default 1)          */
  int use_graph;         /* 1: capture repeated launch sequences in CUDA graphs (default 1)     */
  int path;              /* 0: sweep-fused kernels where the level allows and they pay (default);
                          * 1: one kernel per operation everywhere, the 3D restriction and tau
                          *    correction one cell per thread (reference path);
                          * 2: sweep-fused kernels on every level they handle, whatever its size */
  int seg_rows;          /* rows per warp segment in the fused 2D kernels (0: default 128)      */
  int location;          /* fas_location (default FAS_CELL). Face grids need kappa == NULL and
                          * coarse_exact 0; they run the per-operation kernels                  */
  int ordering;          /* fas_ordering of the X-MCGS sweeps (default FAS_ORDER_FORWARD)       */
} fas_params;

/* X-MCGS sweep orderings (Sec. 2.3, the smoother comparison). FORWARD ("1234-1234"): every sweep
 * updates the parity sets in the paper's order, sets 1-2 (2D; 1-4 in 3D: odd index sum) then the
 * rest. SYMMETRIC ("1234-4321"): the sweeps of each smoothing step alternate forward and backward
 * (sets in reverse order), the symmetric Gauss-Seidel analogue; cell-centred unknowns only, and it
 * runs the per-operation kernels. */
typedef enum { FAS_ORDER_FORWARD = 0, FAS_ORDER_SYMMETRIC = 1 } fas_ordering;

/* Per-solve report. res0/res are ||f - A u||_2 before the first and after the last cycle
 * (the paper's h-weighted value when tol_relative == 0); rel = res / ||f||_2; rho is the mean
 * contraction (res/res0)^(1/cycles). */
typedef struct {
  int cycles;
  int converged;
  double res0, res, rel, rho;
} fas_info;

typedef struct fas_ctx fas_ctx;

/* Fill *p with the defaults: V(2,2), kmax 20, coarsest 4, tol 1e-10 relative, FP64, Neumann. */
void fas_default_params(fas_params* p);

/* Validate the parameters, build the level hierarchy (Sec. 2.1: each coarser grid halves every
 * axis and doubles h) and allocate its device storage. stream is a cudaStream_t (may be NULL).
 * Errors: FAS_EINVAL (bad sizes or parameters), FAS_ENOMEM, FAS_ECUDA. */
fas_status fas_create(const fas_params* p, void* stream, fas_ctx** out);

/* Free everything fas_create allocated. NULL is accepted. */
fas_status fas_destroy(fas_ctx* ctx);

/* Number of levels (finest = 0) and the cell count of a level. */
int fas_num_levels(const fas_ctx* ctx);

/* Exactly one V-cycle in place on device field u with right-hand side f (one pass of Algorithm
 * 1's k loop with recursion), then the residual norm into info (may be NULL). */
fas_status fas_vcycle(fas_ctx* ctx, double* u, const double* f, fas_info* info);

/* V-cycles on u (initial guess, overwritten) until the residual test of Algorithm 1 passes or
 * kmax cycles are done. FP64 or mixed precision per the context's parameters.
 * Returns FAS_ENOTCONV (info filled) if tol was not reached, FAS_ENONFINITE on NaN/Inf. */
fas_status fas_solve(fas_ctx* ctx, double* u, const double* f, fas_info* info);

/* Backward-Euler heat stepping (the paper's time-dependent use, the new step overwriting the
 * old): for n in 0..nsteps-1 solve (I - dt div(kappa grad)) u^{n+1} = u^n + dt fsrc from the
 * initial guess u^n. The context must have alpha = 1 and beta = dt. fsrc may be NULL (no
 * source). infos (may be NULL) receives one fas_info per step. */
fas_status fas_heat_run(fas_ctx* ctx, double* u, const double* fsrc, double dt, int nsteps,
                        fas_info* infos);

/* Adjoint of fas_heat_run (not in the paper): given dL/du^N for a loss L of the final state of
 * nsteps backward-Euler steps from u0 (device fields), computes the gradients of L with respect to
 * u0, the source fsrc and the per-cell diffusivity of the context (the field passed as kappa to
 * fas_create; with a constant kappa g_kappa is the gradient with respect to a per-cell field at that
 * value). A = I - dt div(kappa grad) is symmetric, so each backward step is a solve with the same
 * multigrid:  mu = A^{-1} lambda,  g_f += dt mu,  g_kappa += -(d(mu^T A u^{n+1})/d kappa),
 * lambda <- mu, starting from lambda = dL/du^N; g_u0 = lambda at the end. Forward states are kept
 * every ckpt_every steps (<= 0: every step) and recomputed segment by segment in the backward sweep.
 * uT (may be NULL) receives u^N; g_u0, g_f, g_kappa may each be NULL. fsrc may be NULL (no source).
 * The context must have alpha = 1 and beta = dt. All pointers are DEVICE pointers. */
fas_status fas_heat_adjoint(fas_ctx* ctx, const double* u0, const double* fsrc, double dt, int nsteps,
                            const double* dL_duT, double* uT, double* g_u0, double* g_f, double* g_kappa,
                            int ckpt_every);

/* Inhomogeneous Dirichlet values (Sec. 2.1, Eq. boundry1 with a value g on the face): with the ghost
 * 2g - u of such a face, the point equation of the cell next to it gains the constant 2 beta kappa g /
 * h^2 (kappa of that cell), which this call adds to f. Every face of fas_params.bc that is
 * FAS_BC_DIRICHLET takes values[face] (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi; values of Neumann faces
 * are ignored); the solves then use the homogeneous operator. Faces are added to each cell in the
 * order z, y, x (low side first). f: DEVICE float64, nx*ny(*nz). Cell-centred contexts only. For a
 * heat run, whose right-hand side is u^n + dt fsrc with beta = dt, pass values g / dt and fsrc. */
fas_status fas_fold_dirichlet(fas_ctx* ctx, double* f, const double values[6]);

/* fas_heat_run with HOST buffers: copies u0_host and fsrc_host (may be NULL) to device buffers the
 * context keeps between calls, runs nsteps steps and copies the result to uT_host (may equal
 * u0_host). Returns after the result is on the host. Page-locked buffers that the GPU can address
 * (cudaHostAlloc / PyTorch pin_memory under unified addressing, 16-byte aligned) are copied by the
 * GPU's own loads and stores over the host link; other buffers by cudaMemcpyAsync. */
fas_status fas_heat_run_host(fas_ctx* ctx, const double* u0_host, double* uT_host,
                             const double* fsrc_host, double dt, int nsteps, fas_info* infos);

/* --- many independent problems ----------------------------------------------------------------
 * Solve count independent problems, problem k on device fields u[k], f[k] with context ctxs[k]
 * (each context its own size, diffusivity, dt, precision; contexts must be distinct and on the
 * current device), in ONE launch of one CUDA graph on `stream` (a cudaStream_t, NULL = legacy
 * default): every problem's solve -- its norms, its initial residual and a device-side while loop
 * of cycles until its own tolerance or kmax -- is an independent branch of the graph, so small and
 * large problems run concurrently. The graph is built on the first call for a given list of
 * (ctx, u, f) and reused afterwards. infos[k] (may be NULL) receives problem k's report. Returns
 * FAS_ENOTCONV if any problem missed its tolerance, FAS_ENONFINITE if any residual was not finite.
 * Not in the paper (its problems run one at a time). */
fas_status fas_solve_batched(fas_ctx* const* ctxs, int count, double* const* u, const double* const* f,
                             fas_info* infos, void* stream);

/* Autotuning of a context's launch parameters: float32 cycles per refinement step (mixed precision,
 * 1..3) and the row-segment length of the sweep-fused kernels (auto, 16, 32, 64, 128), chosen by
 * the time of full solves of f from u = 0 (u is overwritten; a scratch field of the finest size).
 * Results are cached per (dim, n, precision) for the process, so contexts of a size already tuned
 * take the cached choice without timing. out (may be NULL) receives the choice and its time. */
typedef struct {
  int inner_cycles, seg_rows;
  double ms;           /* time of one solve with the chosen parameters                           */
  int candidates;      /* number of parameter sets timed (0 when the cached choice was used)      */
} fas_tune_result;

fas_status fas_autotune(fas_ctx* ctx, double* u_scratch, const double* f, fas_tune_result* out);

/* --- single operators, for testing each kernel against the oracle ---------------------------- */

/* out = f - A u on level `level` (Sec. 2.2, r = f - L_h p), norm2 (may be NULL) = ||out||_2; out
 * may be NULL when only the norm is wanted.
 * Level 0 fields are the caller's; level > 0 operates on caller fields of that level's size. */
fas_status fas_residual(fas_ctx* ctx, int level, const double* u, const double* f, double* out,
                        double* norm2);

/* The refinement residual of the mixed-precision solve on level 0, as the solve computes it:
 * r32 = (float)(f - A u) rounded to nearest even, norm2 (may be NULL) = ||r32||_2. With a constant
 * kappa the point equation is evaluated as fma(c, S, fma(-alpha, u, f)), c = beta kappa / h^2, where
 * S = sum_nb u_nb - M u (M the diagonal's neighbour count plus boundary multiplicities) is summed
 * exactly in integer arithmetic on the significands and rounded once; cells whose stencil holds a
 * zero, a subnormal or non-finite value, or values more than 2^5 apart in exponent, use the float64
 * expression of fas_residual (2D levels with nx a multiple of 128 decide per row of 128 cells, and
 * also take that expression for rows holding values of both signs). r32 is reproducible bit for bit;
 * norm2 sums float32 partials whose grouping depends on how the GPU scheduled the work, so its last
 * bits may vary between calls. u, f DEVICE float64, r32 DEVICE float32, nx*ny(*nz) each. */
fas_status fas_residual_ir(fas_ctx* ctx, const double* u, const double* f, float* r32, double* norm2);

/* `sweeps` X-MCGS sweeps in place on u of level `level` (Sec. 2.3 / Appendix B). */
fas_status fas_smooth(fas_ctx* ctx, int level, double* u, const double* f, int sweeps);

/* uc = R(u) (Appendix C average of 2^d children; on a face grid the Appendix D face restriction),
 * u of level `level`, uc of level + 1. */
fas_status fas_restrict(fas_ctx* ctx, int level, const double* u, double* uc);

/* u += P(c) (Appendix C piecewise-constant prolongation; on a face grid the Appendix D face
 * prolongation), c of level + 1, u of level `level`. */
fas_status fas_prolong_add(fas_ctx* ctx, int level, double* u, const double* c);

/* --- kernel timing (CUDA events on the context's stream) ------------------------------------ */

/* Kernel families for fas_prof_read. */
typedef enum {
  FAS_K_SMOOTH = 0,      /* X-MCGS sweeps (colour phases or fused sweeps)                       */
  FAS_K_RESIDUAL = 1,    /* residual (+ restriction + tau correction when fused)                */
  FAS_K_RESTRICT = 2,    /* restriction of u and r                                              */
  FAS_K_TAU = 3,         /* coarse source term f_c = R(r) + A_c R(u)                             */
  FAS_K_PROLONG = 4,     /* prolongation of the correction (+ post-smoothing when fused)         */
  FAS_K_COARSE = 5,      /* single-CTA V-cycle over the small levels                             */
  FAS_K_IR = 6,          /* mixed precision: float64 residual r = b - A u, rounded to float32    */
  FAS_K_NORM = 7,        /* norms and means                                                     */
  FAS_K_OTHER = 8,       /* right-hand sides, fills, conversions                                */
  FAS_K_UPDATE = 9,      /* mixed precision: float64 u += e (alone or fused into the post-smoothing) */
  FAS_K_NFAMILIES = 10
} fas_kernel_family;

/* Per (family, level) totals since the last fas_prof_enable(ctx, 1). */
typedef struct {
  int family, level;
  long long launches;
  double ms;             /* sum of CUDA-event durations of the launches                        */
  double units;          /* cells of that level processed by the launches (per launch summed)   */
} fas_prof_record;

/* Start (on != 0: clears previous records) or stop recording an event pair around every launch. */
fas_status fas_prof_enable(fas_ctx* ctx, int on);

/* Synchronise the stream and write up to `cap` aggregated records; *count receives the number of
 * (family, level) pairs seen (may exceed cap). */
fas_status fas_prof_read(fas_ctx* ctx, fas_prof_record* out, int cap, int* count);

/* --- solving without allocating ---------------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory when they need a solve: programs whose allocator has reserved all device memory up
 * front and hands it out itself, applications that give a solver a fixed budget and only device
 * pointers to work in, and real-time loops that cannot take an allocation's latency or failure.
 *
 * fas_vcycle_small_static runs ncycles V-cycles (the V-cycle of fas_vcycle, float64, constant kappa,
 * coarsest level smoothed) on device field u in place, for right-hand side f, with no context and no
 * allocation: the whole level hierarchy is held in one CTA's shared memory, and the only global
 * scratch -- the level descriptors and the residual-norm slot, about 27 KB -- is a static device
 * array that every GPU loading the library keeps until the process exits.
 *   p         problem and smoothing parameters as for fas_create (kappa must be NULL, coarse_exact 0,
 *             precision FAS_FP64; kmax, tol, inner_cycles, use_graph, path, seg_rows are ignored)
 *   u, f      DEVICE pointers of the caller, dense C order (x fastest), nx*ny(*nz) float64 each
 *   res_host  HOST pointer (may be NULL) receiving ||f - A u||_2 after the last cycle; when given,
 *             the call waits for the stream, otherwise it returns with the work enqueued
 *   stream    cudaStream_t (NULL: legacy default stream)
 * Limits: at most 16 levels and a hierarchy (u and f on every level, the restricted start below the
 * top, plus descriptors) of at most 200 KB of shared memory: float64 grids up to 64 x 64 in 2D or
 * 16 x 16 x 16 in 3D. Larger grids return FAS_EINVAL with the needed size in fas_last_error().
 * The first call on a device looks up the static array's device address (once per device, with that
 * device current); make that first call before any stream capture begins, and do not use the entry
 * point on a device after cudaDeviceReset in the same process. The level descriptors are written by
 * small kernels that take them by value. All calls share the array, and each call leaves its own
 * descriptors and norm in it, so calls that overlap on the GPU race (for example on two streams);
 * the caller must serialise them (one stream, or events). */
fas_status fas_vcycle_small_static(const fas_params* p, double* u, const double* f, int ncycles,
                                   double* res_host, void* stream);

/* Self-test of the integer-arithmetic float32 <-> float64 conversions that the float64 kernels use
 * instead of the hardware conversions (no counterpart in the paper): converts a fixed list of special
 * values and, for each of `count` seeded pseudo-random draws, a raw 64-bit pattern, three doubles in
 * and around float32's exponent range (random, exact-tie and tie +- 1 significands) and two floats,
 * and compares each result with the hardware conversion (float64 -> float32 both by the general
 * routine and, inside float32's normal range, by the shorter one the residual kernels use). *mismatches (HOST) receives the number of
 * results that differ in any bit (two NaNs count as equal). Runs on the current device and stream 0. */
fas_status fas_selftest_conversions(long long count, unsigned long long seed, long long* mismatches);

/* Measured float64 FMA throughput of the current device (no counterpart in the paper): times a kernel
 * of independent DFMA chains on every SM with CUDA events (best of three launches after a warm-up) and
 * writes the rate in TFLOP/s (an FMA counts as two operations) to *tflops (HOST). It is the FP64-pipe
 * denominator of the roofline of the float64 kernels. Runs on the current device and stream 0 and
 * waits for it; FAS_ECUDA if a CUDA call fails. */
fas_status fas_probe_fp64_rate(double* tflops);

/* Test hook of the bounded device waits (no counterpart in the paper). The 3D refinement residual and
 * the sweep-fused 3D smoother stream their planes into shared memory with TMA tile copies and wait for
 * each on an mbarrier; a wait gives up after limit_ns nanoseconds (default 1e9), the kernel stops its
 * work and sets an error word, and the call that launched it returns FAS_ETIMEOUT (the context stays
 * usable). limit_ns sets that deadline for later launches; withhold_next = 1 makes the next launch of
 * the refinement residual, 2 the next launch of the fused sweep, withhold one copy (the first of
 * block 0), so that its waits run out; 0 withholds nothing. The request applies to the next launch
 * enqueued, and a launch captured into a solve's CUDA graph keeps it on every replay, so the hook is
 * meant for contexts with use_graph 0 or for calls that are not captured (fas_residual_ir).
 * Process-wide; FAS_EINVAL if limit_ns <= 0 or withhold_next is not 0, 1 or 2. */
fas_status fas_debug_bounded_wait(long long limit_ns, int withhold_next);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* fas_last_error(void);

/* Number of kernel launches this context has issued since creation or the last reset (for the
 * benchmark's launch count; a captured graph counts each of its kernel nodes per replay). */
long long fas_launch_count(const fas_ctx* ctx, int reset);

#ifdef __cplusplus
}
#endif

#endif /* FAS_H */
