/*
 * grain.h -- C ABI of the grain-growth step (Sec. 3.3.1 of the paper, the multi-order-parameter
 * Allen-Cahn system of Fan and Chen), part of libfasmg.so. Every linear solve runs through the FAS
 * multigrid of fas.h on a periodic grid.
 *
 * Model (Sec. 3.3.1, Eq. grain-growth-equations): q order parameters eta_1..eta_q with
 *     d eta_i / dt = -L ( -alpha eta_i + beta eta_i^3 + 2 gamma eta_i sum_{j != i} eta_j^2 - kappa Lap eta_i ),
 * periodic in every direction (the paper's constants: L = 1, alpha = beta = gamma = 1, kappa = 2,
 * h = 2, dt = 0.25). The paper prints no time discretisation; the step here is linearly implicit
 * backward Euler (diffusion implicit, the local terms explicit with the old values):
 *     (1 - dt L kappa Lap_h) eta_i^{n+1} = eta_i^n - dt L ( -alpha eta_i^n + beta (eta_i^n)^3
 *                                           + 2 gamma eta_i^n (phi^n - (eta_i^n)^2) ),
 *     phi^n = sum_j (eta_j^n)^2,
 * so each order parameter is one solve of A = I - dt L kappa Lap_h (fas.h with alpha 1, beta dt L kappa,
 * constant diffusivity, FAS_BC_PERIODIC on every face) from the initial guess eta_i^n: q independent
 * problems of one size, solved as batches of concurrent graph branches (fas_solve_batched).
 *
 * Layout     eta is ONE DEVICE array of q fields, field i at eta + i * cells (cells = nx*ny(*nz)),
 *            each a dense C-order float64 field with x fastest; 16-byte aligned; owned by the caller.
 * Ownership  The context owns the right-hand sides of the q solves (q fields) and the multigrid
 *            contexts of one batch, allocated in gg_create.
 * Errors     fas_status codes as in fas.h; fas_last_error() has the message.
 */
#ifndef GRAIN_H
#define GRAIN_H

#include "fas.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gg_ctx gg_ctx;

/* Model constants of Sec. 3.3.1 (the paper's values: 1, 1, 1, 1, 2). */
typedef struct {
  double L, alpha, beta, gamma, kappa;
} gg_model;

/* Create a grain-growth context.
 *   dim, n[3], h   periodic grid (n[2] ignored in 2D), each n a power of two >= 4, spacing h
 *   dt             time step
 *   q              number of order parameters (>= 1)
 *   model          model constants (NULL: the paper's values)
 *   solver         multigrid parameters of the q solves (NULL: fas_default_params); only nu1, nu2,
 *                  nu_coarse, kmax, coarsest, tol, tol_relative, precision, inner_cycles and use_graph
 *                  are taken, the operator and boundary fields are set here
 *   batch          problems per graph launch (<= 0: min(q, 128)); the context keeps that many
 *                  multigrid contexts and runs the q solves in ceil(q / batch) launches
 *   stream         cudaStream_t for all work (NULL: legacy default stream)
 * Errors: FAS_EINVAL (bad sizes or constants), FAS_ENOMEM, FAS_ECUDA. */
fas_status gg_create(int dim, const int n[3], double h, double dt, int q, const gg_model* model,
                     const fas_params* solver, int batch, void* stream, gg_ctx** out);

/* One time step of all q order parameters in place: the right-hand sides from the old values (one
 * pass over the q fields for phi, one for the right-hand sides), then the q solves, each from its old
 * field. infos (HOST, may be NULL) receives q reports. Returns FAS_ENOTCONV if a solve missed its
 * tolerance within kmax (the step is still complete), FAS_ENONFINITE on a non-finite residual.
 * Returns after the step is complete. */
fas_status gg_step(gg_ctx* ctx, double* eta, fas_info* infos);

/* The right-hand sides of the step only (for testing): rhs = q fields as eta. DEVICE pointers. */
fas_status gg_rhs(gg_ctx* ctx, const double* eta, double* rhs);

/* Free everything gg_create allocated. NULL is accepted. */
fas_status gg_destroy(gg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GRAIN_H */
