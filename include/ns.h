/*
 * ns.h -- C ABI of the projection step for incompressible Navier-Stokes on the MAC staggered grid
 * (Sec. 4 of the paper), part of libfasmg.so. Every linear solve runs through the FAS multigrid of
 * fas.h: the velocity components on face grids (fas_location FAS_FACE_*), the pressure on cells.
 *
 * Domain, unknowns and boundaries (Sec. 4.1): a box of n[0] x n[1] (x n[2]) cells of spacing h,
 * velocity component c on the faces normal to axis c, pressure at cell centres. Walls are no-slip:
 * the normal component is 0 on its own walls; the tangential velocity on the wall is 0 except on
 * the lid, the top wall of the last axis (y in 2D, z in 3D), which moves with velocity lid[c].
 *
 * Layout     Every field is a dense C-order float64 array of nx*ny(*nz) values with x fastest, the
 *            cell-field shape. A velocity field of component c stores, along axis c, face s+1 at
 *            slot s (faces 1..n-1 are the unknowns) and the far wall face, which must be 0 and stays
 *            0, at slot n-1; the near wall face is not stored (it is 0).
 * Fields     fields[8] = { U_new, U_old, V_new, V_old, W_new, W_old, P_new, P_old }, DEVICE pointers
 *            owned by the caller, each 16-byte aligned (in 2D the W entries are ignored and may be
 *            NULL). These are the
 *            paper's memory-efficient assignments of the schemes to eight resident fields.
 *            First order (Sec. 4.2): on entry *_old hold u^n and p^n, *_new are work fields; after
 *            the call *_old hold u^{n+1}, p^{n+1}, *_new the intermediate velocity and the pressure
 *            increment.
 *            Second order (Sec. 4.3, lagged update): on entry U_new/V_new/W_new hold u^n and
 *            U_old/V_old/W_old hold u^{n-1} (both u^0 before the first step), P_old holds p^n; after
 *            the call the velocity *_new hold u^{n+1}, the velocity *_old hold u^n, P_old p^{n+1} and
 *            P_new the pressure increment.
 * Ownership  The context owns the multigrid hierarchies of the four solves and one scratch field
 *            (the right-hand side of the current solve), allocated in ns_create.
 * Errors     fas_status codes as in fas.h; fas_last_error() has the message.
 */
#ifndef NS_H
#define NS_H

#include "fas.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_ctx ns_ctx;

/* Create a projection-step context.
 *   dim, n[3], h   grid (n[2] ignored in 2D); each n a power of two >= 4
 *   Re, dt         Reynolds number and time step; the viscous operator is I - (dt/Re) Lap
 *   order          time order of the projection scheme: 1 (Sec. 4.2, Scheme first-1..4: backward Euler
 *                  viscous step, WENO3 convection of u^n) or 2 (Sec. 4.3, Scheme second-1..4:
 *                  Crank-Nicolson viscous step, WENO3 convection of the extrapolated (3u^n - u^{n-1})/2
 *                  with advecting components already solved in the step averaged as (u^n + u~^{n+1})/2);
 *                  other values return FAS_EUNSUPPORTED
 *   lid[3]         tangential velocity of the top wall of the last axis (lid[dim-1] is ignored)
 *   solver         multigrid parameters of the viscous solves (NULL: defaults with kmax 40); only nu1,
 *                  nu2, nu_coarse, kmax, coarsest, tol, tol_relative, precision, inner_cycles and
 *                  use_graph are taken, the operator fields are set here
 *   pressure       the same for the pressure solve (NULL: defaults with coarse_exact 1, kmax 60)
 *   stream         cudaStream_t for all work (NULL: legacy default stream) */
fas_status ns_create(int dim, const int n[3], double h, double Re, double dt, int order, const double lid[3],
                     const fas_params* solver, const fas_params* pressure, void* stream, ns_ctx** out);

/* One time step of the projection scheme of the context's order. First order (Sec. 4.2):
 *   f_c = c^n - dt (u^n . grad) c^n - dt (grad p^n)_c + dt F_c   (third-order WENO convection)
 *   (I - dt/Re Lap) c~ = f_c        from the initial guess c^n, into C_new, for every component
 *   -dt Lap p~ = -div u~            homogeneous Neumann, mean 0, into P_new (zero initial guess)
 *   c^{n+1} = c~ - dt (grad p~)_c   into C_old;   p^{n+1} = p^n + p~ into P_old.
 * Second order (Sec. 4.3): f_c = c^n - dt (a . grad) cbar + (dt/2Re) Lap c^n - dt (grad p^n)_c + dt F_c,
 * C_old <- C_new, (I - dt/2Re Lap) c~ = f_c from c^n into C_new, the same pressure step, and
 * c^{n+1} = c~ - dt (grad p~)_c in place in C_new.
 * force (may be NULL, as may each entry): DEVICE pointers to the body force F_c of each component on
 * its faces (the face-field layout above) for this step: F at t^{n+1} for the first-order scheme, the
 * step average (F(t^n) + F(t^{n+1}))/2 for the second-order scheme, e.g. the source of a
 * manufactured solution.
 * info (may be NULL) receives 4 reports: the solves of U, V, W (zeroed in 2D) and of the pressure.
 * div_max (HOST pointer, may be NULL) receives max |div u^{n+1}| over the cells.
 * A solve that stops at kmax without reaching its tolerance does not stop the step: the step is
 * completed and FAS_ENOTCONV returned. Non-finite residuals return FAS_ENONFINITE at once. */
fas_status ns_projection_step(ns_ctx* ns, double* const fields[8], const double* const force[3], fas_info info[4],
                              double* div_max);

/* Kernel launches issued by the context and its solvers since creation or the last reset. */
long long ns_launch_count(ns_ctx* ns, int reset);

/* Free the context (NULL accepted). */
fas_status ns_destroy(ns_ctx* ns);

#ifdef __cplusplus
}
#endif

#endif /* NS_H */
