/*
 * helm.h -- C ABI of the GB300 semi matrix-free twogrid-preconditioned FGMRES
 * solver for the Helmholtz problem with an impedance boundary.
 *
 * The method (arXiv 2104.01439):
 *   -Lap u - k^2 u = f in (0,1)^d,  du/dn - i k u = g on the boundary (Sec. 2,
 *   eq. Helmholtz). Lagrange FE discretisation gives A(k,eps) u = F with
 *   A(k,eps) = K - (k^2 + i eps) M - i k B  (Sec. 2, eq. sys_matrix).
 *   FGMRES (Saad 1993) solves A0 P_eps^{-1} (P_eps u) = F with A0 = A(k,0);
 *   P_eps^{-1} is one twogrid V(nu,nu)-cycle on A_eps = A(k,eps): damped
 *   Jacobi smoothing, restriction P^T, a direct coarse solve on the 2h mesh,
 *   prolongation P (Sec. 4, Algorithm 1). Fine-level operators are applied
 *   matrix-free; the coarse matrix is factored once per (k, h, order, shift)
 *   (Sec. 6: "semi matrix-free").
 *
 * Discretisation of this library: P1 or P2 Lagrange elements on the uniform
 * right-triangle mesh of the unit square (each cell split along its main
 * diagonal), or P1 on Kuhn's six-tetrahedra subdivision of the unit cube.
 * DoFs are numbered lexicographically, x fastest: (order*n + 1)^dim of them.
 *
 * Conventions for every entry point:
 *   - complex vectors are interleaved (re, im) pairs of double (complex128);
 *   - "device" pointers are CUDA device memory owned by the caller, used on
 *     the handle's stream and never retained after the call returns;
 *   - "host" pointers are host memory owned by the caller;
 *   - return value: HELM_OK (0) or a negative HELM_E* code; nothing calls
 *     exit(), prints, or traps on the device. After an error the handle stays
 *     valid unless the code is HELM_ECUDA (the CUDA context may be lost).
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define HELM_OK 0
#define HELM_EINVAL (-1)     /* bad argument (sizes, order, dim, null pointer) */
#define HELM_ENOMEM (-2)     /* device allocation failed */
#define HELM_ECUDA (-3)      /* a CUDA runtime call failed */
#define HELM_EZEROPIVOT (-4) /* coarse factorisation met a zero/non-finite pivot (eps = 0 can) */
#define HELM_ETIMEOUT (-5)   /* a bounded device-side wait ran out */
#define HELM_ENOTSUP (-6)    /* configuration the library or the device does not support */
#define HELM_ESCRATCH (-7)   /* problem too large for the fixed scratch of helm_coarse_solve_noalloc */

/* ---- helm_result.status (non-fatal outcome of a solve) --------------- */
#define HELM_CONVERGED 0     /* true relative residual <= tol */
#define HELM_MAXIT 1         /* iteration cap reached; x holds the last iterate */
#define HELM_BREAKDOWN 2     /* h_{j+1,j} = 0 (happy breakdown); x is the Krylov solution */
#define HELM_NONFINITE 3     /* NaN/Inf met in the residual; x is not meaningful */

/* ---- precision of the preconditioner (opts.precision) ---------------- */
/* Element families: Lagrange P_order on the cells split into triangles / Kuhn tetrahedra
 * (helm_setup), or tensor-product Q_order on squares / cubes (helm_setup_q; Sec. 2). */
#define HELM_SIMPLICES 0
#define HELM_TENSOR 1

#define HELM_FP64 0          /* everything in complex128 (Gram-Schmidt arithmetic in
                                double-float pairs) */
#define HELM_MIXED 1         /* V-cycle (smoother, transfers, coarse triangular
                                solves) in complex64; outer apply, Arnoldi basis
                                and coarse factorisation in double-float pairs
                                (~48 significant bits), the orthogonalising second
                                Gram-Schmidt pass too (the first pass's projections
                                in float); Hessenberg, Givens and the true residual
                                in complex128 */

typedef struct helm_ctx* helm_t;

typedef struct {
  int dim;          /* 2 or 3 (3 only with order 1)                      */
  double omega;     /* Jacobi damping (paper: 2/3, Sec. 4; default 0.6)   */
  int nu;           /* pre- and post-smoothing steps of V(nu,nu), 1..8    */
  int restart;      /* FGMRES restart length m, 1..512                    */
  int maxit;        /* cap on total Arnoldi columns (paper: 500, Sec. 6)  */
  double tol;       /* on the TRUE relative residual ||F - A0 x||/||F||   */
  int precision;    /* HELM_FP64 or HELM_MIXED                            */
  void* stream;     /* cudaStream_t for all work of this handle (NULL = legacy default) */
} helm_opts;

typedef struct {
  int iters;            /* total finished Arnoldi columns (each one preconditioner
                           application; the orthogonalisation finishes a column one
                           step late, so a converged cycle may apply it once more) */
  int cycles;           /* FGMRES cycles (restarts + 1)                      */
  int status;           /* HELM_CONVERGED / HELM_MAXIT / HELM_BREAKDOWN / HELM_NONFINITE */
  double relres_true;   /* ||F - A0 x|| / ||F|| recomputed in FP64 at the end */
  double relres_est;    /* last Givens residual estimate |g_{j+1}| / ||F||    */
  float solve_ms;       /* device time of the solve (CUDA events)            */
  int kernels;          /* kernel launches issued by the solve (graph nodes included) */
} helm_result;

/* Defaults: dim 2, omega 0.6, nu 2, restart 50, maxit 500, tol 1e-8, FP64, stream NULL. */
void helm_default_opts(helm_opts* opts);

/*
 * Set up a solver for A(k, shift) on the mesh with h = 1/n (1/h must be an
 * even integer >= 4) and Lagrange order 1 or 2 (Sec. 2; Sec. 4 two levels).
 * Builds the per-DoF-class stencil coefficients of A0 and A_eps, the Jacobi
 * diagonal, the transfer weights, and factors the coarse matrix A_eps^(2h)
 * (block tridiagonal over grid lines / planes; the explicit inverses of the
 * diagonal Schur blocks are formed by Gauss-Jordan without pivoting, in
 * complex128; for shift > 0 every leading principal minor is non-zero because
 * Im(x^H A x) < 0). Allocates all device state on the opts' stream.
 * shift >= 0 is the paper's epsilon (Sec. 2, eq. Helmholtz_shift).
 * Returns HELM_EZEROPIVOT if a pivot is zero or not finite (possible for shift = 0).
 */
int helm_setup(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out);

/*
 * A handle with the fine-level operators only: the per-class stencils of A0 and A_eps,
 * the Jacobi diagonal and the smoother's workspaces, but no coarse factor and no Krylov
 * storage (set-up cost independent of the coarse solve). helm_apply and helm_smooth work
 * on it; helm_solve, helm_solve_host, helm_batch_solve, helm_vcycle and the coarse solves
 * return HELM_EINVAL. Same arguments and checks as helm_setup.
 */
int helm_operator_setup(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out);

/*
 * helm_setup with the paper's own elements: tensor-product Lagrange Q_order on the squares
 * (cubes) of the uniform grid, order 1 or 2 in 2D and 1 in 3D (Sec. 2: "standard Q_p"; the
 * lattice points are the Gauss-Lobatto points, equispaced for these orders). The lattice, DoF
 * numbering, buffers and every other call are those of helm_setup; the stencils, transfers
 * and load vectors are the Q_order ones. Same checks and errors as helm_setup.
 */
int helm_setup_q(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out);

/*
 * Heterogeneous wavenumber k(x) (Sec. 2 with k in L^inf; Sec. 6, where k(x) = k_max mu(x) comes
 * from a velocity model): helm_setup for the operators
 *   A(k, eps) = K - sum_e (k_e^2 + i eps) M_e - i sum_F k_F B_F    (eq. sys_matrix)
 * with one wavenumber per element, on the fine mesh and, rediscretised from the coarse
 * elements' own values, on the 2h mesh (Sec. 4). elements: HELM_SIMPLICES or HELM_TENSOR;
 * k_fine: one k >= 0 per element of the mesh of spacing h, k_coarse: one per element of the
 * 2h mesh, both in the element order of helm_host_het_row (copied; the caller keeps them). A
 * boundary facet takes its element's k. shift: one real eps >= 0 for the whole domain (eq.
 * Helmholtz_shift). The shifted operator's class stencils hold K - i eps M, and the
 * k-dependent part -M_k - i B_k is added from per-DoF rows (complex64 in the V-cycle of the
 * HELM_MIXED form, complex128 in the outer apply and in the coarse factorisation), with a
 * per-DoF Jacobi diagonal. The coarse factorisation factors every block (no reuse of
 * converged inverses). Everything else is as for helm_setup. HELM_EINVAL for a null or
 * non-finite k array or a mesh helm_setup refuses.
 */
int helm_setup_het(int elements, const double* k_fine, const double* k_coarse, double h, int order, double shift,
                   const helm_opts* opts, helm_t* out);

/* Load vector of the paper's point source (Sec. 6): f = 2 exp(-1000 |x - s|^2), g = 0, F = M f
 * interpolated at the DoFs (host, complex128[N]). Works on every handle. */
int helm_rhs_source(helm_t h, double sx, double sy, double sz, void* F_host);

/* Number of complex DoFs N = (order/h + 1)^dim of the fine space. */
int helm_num_dofs(helm_t h, int64_t* n);

/* Number of complex DoFs of the 2h (coarse) space. */
int helm_num_coarse_dofs(helm_t h, int64_t* n);

/* Device milliseconds helm_setup spent in the coarse factorisation (CUDA
 * events) and the number of kernels it launched. Either pointer may be NULL. */
int helm_setup_info(helm_t h, float* ms, int* kernels);

/*
 * Coarse factorisation (Sec. 6: the coarse LU is computed once per (k, h, shift) and reused
 * by every iteration) as block elimination along two chains of coarse blocks. The interior
 * blocks of the coarse operator are all alike, so each chain's Schur complement follows one
 * recurrence; where it has converged (the relative change of the block inverse stays below
 * 1e-7 for the complex64 form's double-float factor, which the solve rounds to complex64, and
 * 1e-11 for the FP64 form, two steps in a row) the remaining blocks of that chain take the
 * converged inverse instead of being
 * factored. This happens for large shifts (e.g. eps = k^2 / 2) and not for small ones.
 * Reports how many of the nb coarse blocks were factored and how many reused (either
 * pointer may be NULL). HELM_EINVAL for an operator-only handle.
 */
int helm_factor_info(helm_t h, int* factored, int* reused);

/*
 * Solve A0 x = F (Sec. 4: FGMRES right-preconditioned by the twogrid
 * V-cycle on A_eps). F, x: device complex128[N], caller-owned; x is
 * overwritten (x0 = 0 is used, any input content is ignored).
 * The call is synchronous with respect to the host (it reads the convergence
 * state). res may be NULL.
 */
int helm_solve(helm_t h, const void* F, void* x, helm_result* res);

/*
 * Same as helm_solve with HOST buffers: copies F host->device, solves, copies
 * x device->host, all on the handle's stream. F_host, x_host: complex128[N].
 */
int helm_solve_host(helm_t h, const void* F_host, void* x_host, helm_result* res);

/*
 * Solve `count` independent problems concurrently (each handle keeps its own
 * stream; their iterations are interleaved by one host loop so that the
 * device overlaps them). F[i], x[i]: device complex128 of handle i's size.
 * res: array of count results (may be NULL). Handles must be distinct.
 */
int helm_batch_solve(int count, const helm_t* hs, const void* const* F, void* const* x,
                     helm_result* res);

/* Free every device resource of the handle. NULL is ignored. */
void helm_destroy(helm_t h);

/* Static string for a return code. */
const char* helm_strerror(int code);

/* Name of the last CUDA runtime error this thread met inside the library
 * ("none" if there was none); the detail behind a HELM_ECUDA / HELM_ENOMEM. */
const char* helm_last_cuda_error(void);

/* ---- right-hand sides (host output, complex128[N]) --------------------- */

/*
 * Load vector of the plane wave u = exp(i k d.x), d = (cos theta, sin theta[, 0]):
 * f = 0 and impedance data g = i k (d.n - 1) u on each boundary facet with
 * that facet's outward normal (Sec. 2, F(v) = int f v + int_dOmega g v). HELM_EINVAL for a
 * handle of helm_setup_het (no single k).
 */
int helm_rhs_planewave(helm_t h, double theta, void* F_host);

/* Load vector of f = exp(-|x - c|^2 / (2 sigma^2)) with g = 0: F = M (I_h f). */
int helm_rhs_gaussian(helm_t h, double sigma, double cx, double cy, double cz, void* F_host);

/* The same two load vectors without a handle (host only), for the mesh of
 * (dim, order, h): F_host receives complex128[(order/h + 1)^dim]. HELM_EINVAL for a
 * mesh helm_setup would refuse (1/h not an even integer >= 4, dim/order not supported,
 * 2^30 DoFs or more), a null F_host, k <= 0 or sigma <= 0; nothing is written then. */
int helm_load_planewave(int dim, int order, double h, double k, double theta, void* F_host);
int helm_load_gaussian(int dim, int order, double h, double sigma, double cx, double cy, double cz, void* F_host);
/* The same with the element family given (HELM_SIMPLICES as above, or HELM_TENSOR for the
 * Q_order meshes of helm_setup_q). */
int helm_load_planewave_e(int dim, int order, int elements, double h, double k, double theta, void* F_host);
int helm_load_gaussian_e(int dim, int order, int elements, double h, double sigma, double cx, double cy, double cz,
                         void* F_host);

/* ---- host-only inspection of the operator tables (no GPU work) ----------- */

/* Row `dof` of the unit-coefficient matrices K (stiffness), M (mass) and B (boundary mass)
 * of the solver for the mesh of (dim, order, h): level 0 is that mesh, level 1 its coarse
 * mesh of spacing 2h (the twogrid coarse level, built by the solver from these tables). The
 * row is read from the per-class tables that the matrix-free kernels use (Sec. 2,
 * eq. discreteproblem): coefficient o belongs to the neighbour at per-axis offset
 * d_ax = (o / (2R+1)^ax) mod (2R+1) - R, x first, R = order; neighbours outside the lattice get
 * 0. K, M, B: caller arrays of (2*order+1)^dim doubles. dof: lexicographic lattice index of that
 * level, x fastest. Besides the meshes helm_setup takes, HELM_TENSOR accepts order 3 in 2D here
 * (Q3 at the Gauss-Lobatto points; tables only, no solver). HELM_EINVAL for a mesh refused, an
 * element family not supported, a level other than 0 or 1, a dof out of range or a null array. */
int helm_host_stencil_row(int dim, int order, int elements, double h, int level, int64_t dof, double* K,
                          double* M, double* B);

/* Heterogeneous wavenumber k(x) = k_max mu(x) (Sec. 2 with k in L^inf; Sec. 6): row `dof` of
 * K, M_k = sum_e k_e^2 M_e (the k-weighted mass), M and B_k = sum_F k_F B_F (the k-weighted
 * boundary mass) on level 0 or 1 of the mesh of (dim, order, h), in the box layout of
 * helm_host_stencil_row. k_elem: one wavenumber per element of that level (n = 1/h or 1/(2h)
 * cells per side), cells in lexicographic order, x fastest, and within a cell its simplices in
 * the order (0,0)-(1,0)-(1,1), (0,0)-(1,1)-(0,1) (2D) or the Kuhn tetrahedra of the axis
 * permutations in lexicographic order (3D); one element per cell for HELM_TENSOR. A boundary
 * facet takes its element's value. HELM_EINVAL as for helm_host_stencil_row. */
int helm_host_het_row(int dim, int order, int elements, double h, int level, const double* k_elem, int64_t dof,
                      double* K, double* Mk, double* M, double* Bk);

/* Row `fine_dof` of the canonical interpolation P from the 2h space to the h space (Sec. 4,
 * the matrix I^(l)), read from the per-class weights the transfer kernels use: *count entries,
 * coarse lattice indices in cols (x fastest) and weights in w (arrays of (order+1)^dim).
 * HELM_EINVAL as for helm_host_stencil_row. */
int helm_host_prolongation_row(int dim, int order, int elements, double h, int64_t fine_dof, int64_t* cols,
                               double* w, int* count);

/* ---- individual hot-path steps (device complex128 buffers) ------------- */

/* y = A x with A = A0 (which = 0) or A_eps (which = 1), matrix-free, FP64 (Sec. 6).
 * x, y: device complex128[N], not overlapping. Stream-ordered: the kernel is enqueued on
 * the handle's stream (opts.stream) and the call returns without waiting for it; a
 * launch failure returns HELM_ECUDA. */
int helm_apply(helm_t h, int which, const void* x, void* y);

/*
 * u = nu damped-Jacobi sweeps on A_eps applied to f from u^0 = 0 (the presmoothing of
 * Algorithm 1: u^{i+1} = u^i + omega D^{-1} (f - A_eps u^i)), in the handle's precision
 * (the sweeps of the mixed form run in complex64, the last one writes complex128).
 * f, u: device complex128[N], not overlapping; 2 <= nu <= 8 (else HELM_EINVAL).
 * Stream-ordered like helm_apply. Works on full and operator-only handles.
 */
int helm_smooth(helm_t h, const void* f, void* u, int nu);

/*
 * u = one twogrid V(nu,nu)-cycle on A_eps applied to f with u^0 = 0
 * (Algorithm 1), in the handle's precision. f, u: device complex128[N].
 */
int helm_vcycle(helm_t h, const void* f, void* u);

/*
 * uc = A_eps^(2h)^{-1} rc with the stored coarse factor (Algorithm 1, direct
 * coarse solve), in the handle's precision. rc, uc: device complex128[Nc],
 * lexicographic order of the 2h mesh's DoFs.
 */
int helm_coarse_solve(helm_t h, const void* rc, void* uc);

/*
 * Coarse solve that allocates no device memory. The paper has no counterpart;
 * this entry point only serves callers that must not allocate when they call:
 * code running under a fixed device-memory budget with no headroom left, code
 * that has handed all device memory to its own allocator, and latency-bound
 * loops that cannot afford the implicit device synchronisation a cudaMalloc
 * or cudaFree may cause. It computes exactly what helm_coarse_solve computes
 * (same arguments, same kernels), but its temporary block-padded coarse
 * vectors live in one fixed array of 4 MiB that is part of the library's
 * device image (every GPU that loads the library holds it until the process
 * exits) instead of the handle's own buffers.
 *   - Limit: 2 * (coarse blocks) * (padded block length) complex values of the
 *     handle's precision must fit in 4 MiB (complex128: 131072 values, e.g. the
 *     coarse grid of P1 h=1/512; complex64: twice that). Larger problems get
 *     HELM_ESCRATCH and nothing is launched.
 *   - The first call on a device looks up the array's device address for that
 *     device and keeps it; make that first call outside any stream capture. The
 *     kept address does not survive cudaDeviceReset: do not call this entry
 *     point again after a reset of the device in the same process.
 *   - The device current at the call must be the one the handle was set up
 *     on; otherwise the call returns HELM_EINVAL and launches nothing.
 *   - All calls share the one array and it keeps the previous call's contents
 *     (every entry a call reads is written by that call first). Calls whose
 *     work overlaps on the GPU -- several streams, several host threads -- race
 *     on it: serialise them. Calls on different handles share only this array;
 *     each handle's own state (its error word, the segment workspace of the
 *     complex64 form) is still per handle.
 * rc, uc: device complex128[Nc] as for helm_coarse_solve; synchronous.
 */
int helm_coarse_solve_noalloc(helm_t h, const void* rc, void* uc);

/*
 * Runtime statistics of the last solve's kernels: fills up to `cap` entries
 * of names/ms (device time per phase, summed over the solve) and returns the
 * count through *n. Used by the benchmark for the roofline of each kernel.
 */
int helm_last_profile(helm_t h, int cap, const char** names, double* ms, int* calls, int* n);

/* Enable (1) / disable (0) per-phase CUDA-event timing inside helm_solve (default off). */
int helm_set_profiling(helm_t h, int on);

/* ---- request server: continuous batching of independent solves ----------
 *
 * A solve request carries its own (k, h, order, shift, opts). The server
 * admits requests first-in first-out while the sum of their device-memory
 * estimates (helm_request_bytes) stays within the budget and fewer than
 * max_active are in flight; each admitted request gets its own CUDA stream and
 * handle (operators, coarse factor, Krylov basis), its set-up runs on a setup
 * thread, and one stepping thread advances every admitted solve without
 * blocking (the captured FGMRES iterations of different requests overlap on
 * the device). A finished request's solution is copied to its host buffer,
 * its handle is destroyed and its memory returns to the budget, which admits
 * the next waiting requests. This is the loop a shift-map study needs: many
 * sample solves of different (k, h, shift) in flight at once (Sec. 5, data
 * generation). The paper itself solves one problem at a time.
 * Every result is the same as the result of the same request solved alone:
 * the kernels, launch shapes and reductions do not depend on the mix.
 */
typedef struct helm_server* helm_server_t;

typedef struct {
  double k;         /* wavenumber > 0                                        */
  double h;         /* mesh size: 1/h an even integer >= 4                   */
  int order;        /* 1 or 2 (order 1 only in 3D)                           */
  double shift;     /* epsilon >= 0 of A(k, eps)                             */
  helm_opts opts;   /* dim, omega, nu, restart, maxit, tol, precision; the
                       server owns the streams (opts.stream is ignored)      */
} helm_request;

typedef struct {
  int rc;               /* HELM_OK, or the error that ended this request     */
  helm_result res;      /* the solve's result (valid when rc == HELM_OK)     */
  float setup_ms;       /* device time of the coarse factorisation           */
  double t_submit;      /* host times in seconds since helm_server_create:   */
  double t_admit;       /*   submitted, admitted (memory reserved),          */
  double t_start;       /*   set up and solving,                             */
  double t_done;        /*   finished (solution in x_host)                   */
  size_t bytes;         /* device bytes reserved for the request             */
} helm_ticket_info;

/* Peak device bytes of one request (set-up workspace included); host only. */
int helm_request_bytes(const helm_request* r, size_t* bytes);

/* Device bytes currently held by a handle. */
int helm_device_bytes(helm_t h, size_t* bytes);

/* Start a server on the current CUDA device. budget_bytes > 0; max_active >= 1. */
int helm_server_create(size_t budget_bytes, int max_active, helm_server_t* out);

/*
 * Queue a request. F_host: host complex128[N] load vector, copied before the
 * call returns. x_host: host complex128[N] that receives the solution when the
 * request finishes (NULL: discard); it must stay valid until then.
 * A request whose estimate exceeds the whole budget fails at once with
 * HELM_ENOMEM (in its ticket); invalid parameters return HELM_EINVAL here.
 */
int helm_server_submit(helm_server_t s, const helm_request* r, const void* F_host, void* x_host,
                       int64_t* ticket);

/* Non-blocking: *done = 1 and info filled when the ticket has finished. */
int helm_server_poll(helm_server_t s, int64_t ticket, int* done, helm_ticket_info* info);

/* Block until the ticket has finished; fills info (may be NULL). */
int helm_server_wait(helm_server_t s, int64_t ticket, helm_ticket_info* info);

/* Block until every submitted request has finished. */
int helm_server_drain(helm_server_t s);

/* Drain, stop the server's threads and free everything. NULL is ignored. */
void helm_server_destroy(helm_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
