/*
 * rsc.h -- C ABI of the GB300 library for convection in a rotating spherical
 * shell with implicit Coriolis integration (Gonzalez Sembla, Rambert, Feudel,
 * Tuckerman, "Convection in a Rapidly Rotating Spherical Shell: Newton's
 * Method Using Implicit Coriolis Integration", Mathematics 13, 2113, 2025).
 *
 * Model (Sec. 2.1, Eqs. Navier-Stokes, temp, div, BCs): Boussinesq convection
 * between r_in = eta/(1-eta) and r_out = 1/(1-eta), no-slip walls, T = 1 at
 * r_in and T = 0 at r_out, gravity proportional to r, rotation about z.
 *
 * State layout (Sec. 3.1, Eq. expansion).  Every state or direction vector is
 * a contiguous array of n = 3 * P * Nr * 2 doubles in DEVICE memory unless a
 * name ends in _host:
 *     v[((field * P + pair) * Nr + k) * 2 + part]
 *   field 0 = toroidal potential e, 1 = poloidal potential f, 2 = total
 *   temperature T (U = curl(e r_hat) + curl curl(f r_hat));
 *   pair  = (m, l) with m = 0, Ms, 2Ms, ... <= L and, inside each m,
 *           l = m .. L; P is the number of pairs;
 *   k     = Chebyshev degree of x = 2r - r_in - r_out, k < Nr;
 *   part  = 0 real, 1 imaginary.
 * Spherical harmonics follow Eq. Ylm_norm (no Condon-Shortley phase) and a
 * real field is sum_l a_l0 Y_l^0 + 2 Re sum_{m>0} a_lm Y_l^m.  The imaginary
 * parts of m = 0 coefficients and the entries of e_00, f_00 are zero in every
 * state the library writes.
 *
 * Ownership.  The caller owns every state / vector buffer (for example
 * torch tensors).  The library owns its tables, factorisations, Krylov basis
 * and workspace: allocated by rsc_create (and by the first call with a new
 * time step), released by rsc_destroy.
 *
 * Streams.  Device work is issued on the stream given to rsc_create.  Calls
 * that return numbers to the host (rsc_newton_rw, rsc_norm2, *_host)
 * synchronise that stream; the others are asynchronous.  A context must not be
 * used from two threads at once.
 *
 * Errors.  Every call returns an rsc_status; none aborts or traps.  The text
 * of the last error is available from rsc_last_error.
 */
#ifndef RSC_H
#define RSC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSC_ABI_VERSION 9

typedef struct rsc_ctx rsc_ctx;

typedef enum {
  RSC_OK = 0,
  RSC_EINVAL = 1,      /* bad argument: null pointer, size out of range      */
  RSC_ENOMEM = 2,      /* device or host allocation failed                    */
  RSC_ECUDA = 3,       /* a CUDA runtime call failed                          */
  RSC_ENOCONV = 4,     /* Newton or GMRES reached its iteration cap           */
  RSC_ENAN = 5,        /* a non-finite residual or Krylov norm                */
  RSC_ESINGULAR = 6,   /* zero pivot while factorising the implicit operator  */
  RSC_ETIMEOUT = 7,    /* a bounded device wait gave up                       */
  RSC_ERESOLUTION = 8  /* a continuation stopped on an under-resolved state   */
} rsc_status;

typedef enum {
  RSC_FP64 = 0,        /* every stage in FP64                                 */
  RSC_MIXED = 1        /* transforms and products in FP32 (Legendre sums on
                          tcgen05 tensor cores, 3xTF32), and so the right-hand
                          side of Jacobian actions; the right-hand side of steps
                          and residuals, the temperature solve, Newton residual
                          and update in FP64;
                          the e/f chain solve of Jacobian actions and steps
                          and the GMRES orthogonalisation in double-float
                          arithmetic (FP32 hi + lo pairs, 48-bit significand)
                          unless rsc_tuning chain_df / krylov_split = 0 select
                          the FP64 kernels; the Newton residual step always
                          solves in FP64                                       */
} rsc_precision;

/* Physical parameters and truncation (Sec. 2.1 parameters; Sec. 3.1 grids).
 * Ra is the rotational Rayleigh number, Ek the Ekman number, Pr the Prandtl
 * number, eta = r_in / r_out.  The triangular truncation keeps l <= L and
 * m <= L with m a multiple of Ms (the azimuthal sector 0 <= phi < 2 pi/Ms).
 * Nr Chebyshev coefficients per radial profile, 4 <= Nr <= 128, L <= 255.  */
typedef struct {
  double Ra, Ek, Pr, eta;
  int L, Ms, Nr;
  int precision;       /* rsc_precision */
  int explicit_coriolis; /* 0: Coriolis in the implicit operator (Sec. 3.2, the method);
                            1: Coriolis in the explicit part with a block-diagonal implicit
                            operator (Eqs. expcor_e/f), the comparison scheme of Sec. 5   */
} rsc_params;

/* Newton-GMRES controls (Sec. 3.3: GMRES relative tolerance 1e-10, Newton
 * pseudo-timestep dt = 200).                                                 */
typedef struct {
  double tol;          /* stop when ||B(U) - U||_2 < tol                      */
  int max_newton;      /* Newton iteration cap                                */
  int kmax;            /* GMRES iteration cap (no restart), <= 2048           */
  double gmres_tol;    /* relative GMRES tolerance                            */
  double dt_newton;    /* pseudo-timestep of the Stokes preconditioner        */
} rsc_newton_opts;

#define RSC_MAX_HISTORY 64
typedef struct {
  int iterations;                         /* Newton iterations taken          */
  int gmres_total;                        /* Jacobian actions in all GMRES    */
  double residual;                        /* final ||B(U) - U||_2             */
  double C;                               /* final drift speed                */
  double residual_history[RSC_MAX_HISTORY];
  int gmres_history[RSC_MAX_HISTORY];
  double seconds;                         /* wall time of the call            */
} rsc_newton_report;

/* Create a context for `params` on the CUDA stream `stream` (a cudaStream_t;
 * NULL = legacy default stream) of the current device.  Builds the Gauss-
 * Legendre, associated-Legendre and Chebyshev tables (Sec. 3.1) and uploads
 * them.  Factorisations are built on first use of each time step.          */
rsc_status rsc_create(const rsc_params* params, void* stream, rsc_ctx** out);

/* Release every resource of the context (waits for its stream).            */
rsc_status rsc_destroy(rsc_ctx* ctx);

/* Change the parameters.  A new Ra only changes the explicit part (Sec. 4.2
 * notes that Ra appears only on the right-hand side); Ek, Pr or eta drop the
 * cached factorisations, as does a change of explicit_coriolis; L, Ms, Nr
 * and precision cannot change.                                              */
rsc_status rsc_set_params(rsc_ctx* ctx, const rsc_params* params);

/* Number of doubles n in a state vector, and the number of pairs P.        */
rsc_status rsc_state_size(const rsc_ctx* ctx, size_t* n_real, int* n_pairs);

/* Write the conductive state U = 0, T = r_out r_in / r - r_in (Sec. 2.1) as
 * the steady solution of the discrete temperature equation.                */
rsc_status rsc_conductive_state(rsc_ctx* ctx, double* U);

/* nsteps IMEX Euler steps in place, U <- B(U) (Eq. discrete), with the drift
 * term C d/dphi in the explicit part (Sec. 3.4; C = 0 for plain time
 * stepping).  The implicit operator holds diffusion and Coriolis
 * (Eqs. impcor_e_final, impcor_f_final); it is factorised once per dt.     */
rsc_status rsc_step(rsc_ctx* ctx, double* U, double C, double dt, int nsteps);

/* nsteps second-order steps in place in the laboratory frame (no drift term),
 * the time-stepping scheme of Sec. 5 (a Runge-Kutta predictor-corrector with
 * the linear operator treated implicitly; Table 1 measures its drift error).
 * Reading: Crank-Nicolson for the implicit operator K (diffusion, plus
 * Coriolis unless explicit_coriolis) and Heun's predictor-corrector for the
 * explicit terms N:
 *   (M/dt + K/2) x*      = (M/dt - K/2) x^n + N(x^n)
 *   (M/dt + K/2) x^{n+1} = (M/dt - K/2) x^n + (N(x^n) + N(x*))/2.
 * U must satisfy the boundary conditions (every state the library writes
 * does).  The implicit operator is factorised at dt/2.                      */
rsc_status rsc_step2(rsc_ctx* ctx, double* U, double dt, int nsteps);

/* Same as rsc_step on a HOST buffer: copies to the device, steps, copies
 * back (synchronous).  For end-to-end timing.                              */
rsc_status rsc_step_host(rsc_ctx* ctx, double* U_host, double C, double dt, int nsteps);

/* Explicit terms N(U) at the collocation radii, layout of a state vector:
 * e-rows e_r.curl F, f-rows e_r.curl curl F (F = Ek U x omega + Ra T r/r_out),
 * T-rows -U.grad T (Sec. 3.2, Eq. defineFimp).  Boundary rows hold the
 * unprojected values.  A diagnostic of the transform pipeline.             */
rsc_status rsc_explicit_terms(rsc_ctx* ctx, const double* U, double* N);

/* The implicit solve of one step on its own: x = (M/dt + K)^{-1} rhs, with K the
 * implicit operator of Sec. 3.2 (diffusion and, unless explicit_coriolis, the
 * Coriolis terms of Eqs. impcor_e_final / impcor_f_final, coupling l to l +- 1
 * in two block-tridiagonal chains per m, Fig. blocks) and M the mass operators
 * (Sec. 3.3).  rhs and x are device vectors in the state layout whose entries
 * are values at the Nr collocation radii (not Chebyshev coefficients): row k
 * of a pair is the equation at radius r_k; the boundary rows (k = 0, Nr - 1
 * for e and T; also 1, Nr - 2 for f) hold the boundary-condition values, the
 * rows of e_00 and f_00 hold 0, and x receives Chebyshev coefficients.  rhs
 * and x may be the same buffer.  On a mixed-precision context the e/f chains
 * are solved like its Jacobian actions (chain_df).  Factorises dt on first
 * use.  Returns RSC_EINVAL for a null pointer or dt <= 0.                   */
rsc_status rsc_implicit_solve(rsc_ctx* ctx, const double* rhs, double* x, double dt);

/* One block of the factorisation of dt (built first if needed), copied to the host
 * (synchronous).  which = 0, 1, 2: G, H, W of block `index` (chains in the order
 * (m index, class), blocks l = m .. L inside a chain; Nr x Nr complex row-major, 2 Nr^2
 * doubles): the twisted block Thomas factors of Sec. 3.2 with G = D'^-1, H = D'^-1 A,
 * W = D'^-1 C above the middle block of a chain, G = E'^-1, H = E'^-1 C, W = E'^-1 A
 * below it, and G = Z, H = Z A, W = Z C at the middle block (A, C the couplings to
 * l - 1, l + 1).  which = 3: the inverse of the temperature operator of degree
 * l = index (Nr^2 doubles).  Mixed contexts with implicit Coriolis, the odd-even reduced
 * chains of rsc_tuning chain_cr (built if needed): which = 4: D_i^-1 of odd block `index`
 * (the odd blocks i = 1, 3, ... of every chain, chains in order); which = 5, 6, 7: G', H',
 * W' of reduced block `index` (the even blocks of every chain), the twisted factors of
 * the reduced chains with the conventions above; read from their double-float copies
 * (hi + lo, about 2^-48 relative).  For checks of the factorisation.                */
rsc_status rsc_factor_block(rsc_ctx* ctx, double dt, int which, long index, double* out_host);

/* Wall time (s) of the context's last factorisation and whether it ran on the GPU. */
rsc_status rsc_factor_time(const rsc_ctx* ctx, double* seconds, int* on_gpu);
/* The same for the context's last factorisation of the odd-even reduced chains
 * (rsc_tuning chain_cr; 0 s until one has run).                                  */
rsc_status rsc_factor_time_cr(const rsc_ctx* ctx, double* seconds, int* on_gpu);

/* Jacobian action of Sec. 3.3-3.4 for `count` directions:
 *   out_i = (B_U - I) u_i with the drift unknown c = u_i[J] (Sec. 3.4):
 *   c is read, u_i[J] set to zero in a private copy, c i m M U added to the
 *   explicit part, homogeneous boundary conditions applied.
 * J < 0 gives the steady-state action (no drift unknown).  u and out hold
 * `count` vectors of n doubles back to back; U is the base state.          */
rsc_status rsc_apply_jacobian(rsc_ctx* ctx, const double* U, double C, long J,
                              const double* u, double* out, int count, double dt);

/* Newton-GMRES for a rotating wave (Secs. 3.3-3.4, Eq. twNewton): solves
 * (B_U - I)(u, c) = B(U) - U with matrix-free GMRES, then U <- U - u,
 * C <- C - c, until ||B(U) - U||_2 < opts->tol.  J >= 0 is the frozen phase
 * slot; J < 0 solves for a steady state (C unchanged).  U and *C are updated
 * in place.  Returns RSC_ENOCONV when max_newton is reached.               */
rsc_status rsc_newton_rw(rsc_ctx* ctx, double* U, double* C, long J,
                         const rsc_newton_opts* opts, rsc_newton_report* report);

/* Natural-parameter continuation in Ra (Sec. 4.3).  Points are Newton solves
 * (Sec. 3.4) at successive Rayleigh numbers; the paper adds no equation to
 * Newton's method and only chooses the next Ra and the initial estimate:
 *   Ra^(i+1) = Ra^(i) + alpha (Ra^(i) - Ra^(i-1))              (Eq. new_Ra)
 *   alpha = (n_opt + 1) / (N^(i) + 1), N^(i) the Newton iterations of the
 *   last point                                                   (Eq. alpha_cont)
 *   U^(i+1) = a U^(i) + b U^(i-1) + c U^(i-2) (and C likewise) with (a, b, c)
 *   the Lagrange weights of the new Ra at the last three Ra    (Eq. lagrange)
 * and near turning points (Eqs. tp_detection_Ra, quad_extra_Ra): while
 * |Delta U_J / U_J| > gamma |Delta Ra / Ra|, with J the element of largest
 * |U - U_cond| of the last point, U_J is extrapolated instead and
 * Ra^(i+1) = a Ra^(i) + b Ra^(i-1) + c Ra^(i-2).  Two points give linear
 * weights.  A Newton failure retries the step with alpha halved.           */
typedef struct {
  double Ra0, Ra1;     /* the first two points are solved at these Ra              */
  double Ra_end;       /* stop once a point passes Ra_end in the direction Ra0->Ra1 */
  int n_opt;           /* target Newton iterations (the paper uses 4 to 6)         */
  double gamma;        /* turning-point switch factor (the paper uses 10 to 100)   */
  int max_points;      /* capacity of the points array                             */
  int retries;         /* halvings of alpha after a Newton failure                 */
  rsc_newton_opts newton;
} rsc_continuation_opts;

typedef struct {
  double Ra, C;                 /* parameter and drift of the converged wave           */
  double KE, Nu_in, Nu_out;     /* rsc_diagnostics of the wave                         */
  double residual;              /* final Newton residual                               */
  int newton_iterations, gmres_total;
  int mode;                     /* predictor: 0 Ra independent, 1 U_J independent      */
} rsc_continuation_point;

/* Prediction step of the continuation (host only, no GPU): Ra[0..npts) and
 * s[0..npts) are the last Rayleigh numbers and U_J values, most recent first
 * (npts = 2 or 3; s at the most recent point's J).  Writes the mode (0: Ra,
 * 1: U_J independent), the new Ra and the weights w[3] of the last states.
 * Returns RSC_EINVAL for npts < 2 or null pointers.                        */
rsc_status rsc_continuation_predict(const double* Ra, const double* s, int npts, int n_its,
                                    int n_opt, double gamma, double alpha_scale, int* mode,
                                    double* Ra_new, double* w);

/* Follow a rotating-wave branch.  U (device) holds the initial estimate at
 * Ra0 and returns the last converged wave; *C its drift; J the frozen phase
 * slot (Sec. 3.4).  points[0..*npoints) receive the branch.  The context's Ra
 * is left at the last point.  Returns RSC_OK when the branch reached Ra_end
 * or max_points, RSC_ENOCONV when a step failed after all retries (the points
 * so far are kept).                                                         */
rsc_status rsc_continue_ra(rsc_ctx* ctx, double* U, double* C, long J,
                           const rsc_continuation_opts* opts, rsc_continuation_point* points,
                           int* npoints);

/* Continuation in the Ekman number (Sec. 4.4): the same procedure as
 * rsc_continue_ra with log10 Ek as the parameter (Eq. new_EK; the paper uses
 * n_opt = 3 and gamma 400 to 500).  Every new Ek refactorises the implicit
 * operator.  With ra_coef > 0, Ra = ra_coef Ek^(-1/3) at every point, which
 * keeps the distance to onset (the paper's Ra = 6.5 Ek^(-1/3)); ra_coef = 0
 * keeps the context's Ra.  Grid refinement: when tail_threshold > 0 and a
 * converged point's spectral tail (rsc_spectral_tail) exceeds it, the call
 * returns RSC_ERESOLUTION with that point in U; the caller then creates a
 * finer context (rsc_refine_params), moves U there (rsc_regrid) and resumes
 * from the last Ek (the paper recomputes the last step on the finer grid).  */
typedef struct {
  double Ek0, Ek1;     /* the first two points are solved at these Ek              */
  double Ek_end;       /* stop once a point passes Ek_end in the direction Ek0->Ek1 */
  double ra_coef;      /* > 0: Ra = ra_coef Ek^(-1/3); 0: Ra unchanged              */
  int n_opt;
  double gamma;
  int max_points;
  int retries;
  double tail_threshold;   /* > 0: stop on an under-resolved point (paper: 1e-6)   */
  rsc_newton_opts newton;
} rsc_ek_continuation_opts;

typedef struct {
  double Ek, Ra, C, KE, Nu_in, Nu_out, residual;
  double cheb_tail, sh_tail;    /* rsc_spectral_tail of the wave                     */
  int newton_iterations, gmres_total, mode;
} rsc_ek_point;

rsc_status rsc_continue_ek(rsc_ctx* ctx, double* U, double* C, long J,
                           const rsc_ek_continuation_opts* opts, rsc_ek_point* points,
                           int* npoints);

/* Under-resolution measure of Sec. 4.4: with A the largest |coefficient| of
 * U - U_cond (all fields, complex magnitude), cheb = the largest at the last
 * Chebyshev degree k = Nr - 1 divided by A, sh = the largest at the last
 * spherical-harmonic degree l = L divided by A (synchronous).               */
rsc_status rsc_spectral_tail(rsc_ctx* ctx, const double* U, double* cheb, double* sh);

/* Spectral interpolation between two contexts of the same Ms and eta: every
 * coefficient of U_dst is the one of U_src with the same (field, m, l, k), or
 * zero where the source truncation has none (Fourier interpolation by zero
 * fill, exact for the represented function; coarser targets truncate).
 * Asynchronous on dst's stream; U_src must be ready there.                  */
rsc_status rsc_regrid(const rsc_ctx* src, const double* U_src, rsc_ctx* dst, double* U_dst);

/* Refinement rule of Sec. 4.4: Nr grows by `growth` (the paper: 1.2) when
 * cheb_tail > threshold, L when sh_tail > threshold (caps 128 and 255);
 * *refined = 1 (radial) | 2 (angular), 0 when nothing changed.  Host only.   */
rsc_status rsc_refine_params(const rsc_params* p, double cheb_tail, double sh_tail,
                             double threshold, double growth, rsc_params* out, int* refined);

/* Newton-GMRES on a HOST state (copies in and out inside the call, through a
 * device buffer the context allocated at creation: nothing is allocated).   */
rsc_status rsc_newton_rw_host(rsc_ctx* ctx, double* U_host, double* C, long J,
                              const rsc_newton_opts* opts, rsc_newton_report* report);

/* Batches of instances: the continuation points in Ra of a branch and waves
 * of different azimuthal symmetries M_s (hence different active-m counts),
 * each a full context on a stream of its own that the batch creates and
 * owns.  The parameters of instance i are params[i] (any L, Ms, Nr, Ra, Ek).
 * rsc_batch_apply_jacobian issues the Jacobian actions of every instance as
 * one CUDA graph (captured on the first call with a given set of pointers,
 * drifts, slots, count and dt, replayed afterwards) whose branches run the
 * instances concurrently; rsc_batch_newton_rw runs every instance's
 * Newton-GMRES at once (one host thread per instance, each on its stream).
 * The streams of the instances are ordered after `stream` only inside
 * rsc_batch_apply_jacobian; synchronise the contexts (rsc_batch_context)
 * before reading their results otherwise.  Instances with the same operator
 * (L, Ms, Nr, Ek, Pr, eta, precision, Coriolis treatment; Ra may differ, since
 * it enters only the explicit part) share one set of factorisations per time
 * step (Sec. 3.2: the factors depend on Ek and dt, not on Ra), built by the
 * first instance that needs it; an instance whose Ek changes (rsc_set_params)
 * or that uses partitioned chains factorises on its own.                    */
typedef struct rsc_batch rsc_batch;

rsc_status rsc_batch_create(const rsc_params* params, int n, void* stream, rsc_batch** out);
rsc_status rsc_batch_destroy(rsc_batch* batch);
rsc_status rsc_batch_size(const rsc_batch* batch, int* n);
/* The context of instance i (owned by the batch; do not destroy it).        */
rsc_status rsc_batch_context(rsc_batch* batch, int i, rsc_ctx** ctx);
const char* rsc_batch_last_error(const rsc_batch* batch);

/* For every instance i: out[i][q] = (B_{U[i]} - I) u[i][q], q < count, with
 * drift C[i] and slot J[i] (< 0: none), as rsc_apply_jacobian; u[i], out[i]
 * hold count vectors of that instance's length back to back.  All pointer
 * arrays are host arrays of n device pointers.  Asynchronous on `stream`.   */
rsc_status rsc_batch_apply_jacobian(rsc_batch* batch, const double* const* U, const double* C,
                                    const long* J, const double* const* u, double* const* out,
                                    int count, double dt);

/* rsc_autotune on the first instance of each distinct shape (L, Ms, Nr,
 * precision, Ek, Pr, Coriolis treatment), rsc_set_tuning on the others.       */
rsc_status rsc_batch_autotune(rsc_batch* batch);

/* rsc_newton_rw for every instance concurrently; reports (may be NULL) and
 * status are arrays of n.  Returns the first hard error, else RSC_ENOCONV if
 * any instance did not converge, else RSC_OK.                               */
rsc_status rsc_batch_newton_rw(rsc_batch* batch, double* const* U, double* C, const long* J,
                               const rsc_newton_opts* opts, rsc_newton_report* reports,
                               rsc_status* status);

/* Launch shapes of the transform, right-hand-side and chain kernels (no
 * counterpart in the paper: GPU tiling).  [2] = [FP64 path, mixed path].     */
typedef struct {
  int products_warps[2];   /* warps per block of the DFT + grid products kernel       */
  int products_lats[2];    /* latitudes per warp of that kernel                       */
  int analysis_radii[2];   /* radii per block of the Legendre analysis                */
  int analysis_chunk[2];   /* latitudes per staged chunk of the analysis tables       */
  int synth_radii;         /* radii per block of the CUDA-core (FP64) synthesis       */
  int rhs_pairs[2];        /* (l, m) pairs per block of the right-hand-side kernel    */
  int chain_cluster;       /* CTAs per thread-block cluster of the chain sweeps       */
  int analysis_tc;         /* 1: tensor-core (tcgen05, 3xTF32) Legendre analysis on the
                              mixed path; 0: CUDA-core FP32 analysis                   */
  int chain_async;         /* 0: one warp per 4 rows, a cluster barrier per block;
                              1 / 2: two / four warps per 4 rows (column parts), rows
                              sent with st.async to mbarriers (changes the order of the
                              row sums)                                                */
  int chain_df;            /* mixed path (Jacobian actions and mixed steps): 0 = the FP64
                              chain solve; 2 / 4 = the chain solve in double-float
                              arithmetic (factor blocks and vectors as FP32 hi + lo
                              pairs, Dot2 row sums; about 1e-8 relative from FP64) with
                              two / four warps per 4 rows.  The FP64 residual step
                              always uses the FP64 solve.                              */
  int chain_df_cluster;    /* CTAs per thread-block cluster of the double-float sweeps */
  int krylov_split;        /* 1: GMRES keeps the Krylov basis also as FP32 hi + lo pairs
                              and orthogonalises in double-float arithmetic (inner
                              products within about 1e-14 of FP64); 0: FP64 passes.
                              Not changed by rsc_autotune.                             */
  int chain_parts;         /* 1 to 4: parts per chain of the double-float solve (parts of
                              at least 8 blocks): the parts are swept concurrently and
                              joined through spikes and a reduced system per chain
                              (SPIKE-type), which cuts the sweeps' sequential depth; the
                              factorisation then also computes the spikes on the host.
                              Changing it rebuilds the factorisations.  Not changed by
                              rsc_autotune.                                            */
  int factor_gpu;          /* 1 (default): factorise the implicit operator on the GPU
                              (FP64 block LU with row equilibration and partial
                              pivoting inside each block, Sec. 3.2) when Nr <= 96 and
                              chain_parts = 1; 0: on the host CPU (the same factors to
                              rounding).  Changing it rebuilds the factorisations.     */
  int refine;              /* 0 to 2 (default 1): steps of iterative refinement after every
                              FP64 e/f chain solve (steps, Newton residuals, Jacobian actions
                              of the FP64 path, rsc_implicit_solve on an FP64 context):
                              r = b - (M/dt + K) x in FP64, x += solve(r).  The sweeps
                              multiply by explicit block inverses, which at Ek = 1e-5 leaves
                              relative errors up to 1e-8 in the small poloidal field of
                              the m = 0 chains; one step removes them.  The double-float
                              solve of the mixed path is not refined.                  */
  int synth_pipe;          /* tensor-core synthesis (mixed path): 1 = the table tile and
                              operand of the next (parity, table) phase are staged while
                              the MMAs of the current one run (two tile stages; only
                              where they fit in shared memory, padded K <= 72); 0 = the
                              phases one after another.  Same arithmetic.              */
  int chain_cr;            /* double-float solve of the mixed path: 1 = one level of
                              odd-even (cyclic) reduction of every chain first (the odd
                              blocks eliminated with their inverses D_i^-1, the reduced
                              chain of the even blocks swept as the full chains are;
                              the couplings applied from the Chebyshev tables), which
                              halves the sequential depth of the sweeps and reads 2.5
                              instead of 3 factor blocks per block pair; its factors are
                              computed on first use, on the GPU where factor_gpu puts
                              the FP64 factorisation (chain_parts = 1 and implicit
                              Coriolis only).  Default 1 on a mixed context; 0 = the
                              unreduced chains.  Changes the order of the arithmetic.   */
  double ms[6];            /* after rsc_autotune: best times (ms) of products +
                              analysis (mixed), FP64 synthesis, RHS (mixed), FP64 chain
                              solve, double-float chain solve (0 if none ran); zero
                              otherwise                                               */
} rsc_tuning;

/* Autotuner: times every feasible candidate of each shape on this context's
 * workspace (the conductive state as input; 3 launches after a warm-up) and
 * keeps the fastest; factorises dt = 200 if needed.  Synchronous, a few
 * hundred launches.  `out` (may be NULL) receives the choice.               */
rsc_status rsc_autotune(rsc_ctx* ctx, rsc_tuning* out);
rsc_status rsc_get_tuning(const rsc_ctx* ctx, rsc_tuning* out);
/* Apply shapes (for example tuned on another context of the same size);
 * RSC_EINVAL if one is infeasible here.                                     */
rsc_status rsc_set_tuning(rsc_ctx* ctx, const rsc_tuning* t);

/* Tracing.  Kernel identifiers of rsc_profile_query / rsc_kernel_name.     */
enum {
  RSC_K_RADIAL = 0,    /* Chebyshev evaluation on the de-aliased radii        */
  RSC_K_SYNTH = 1,     /* Legendre synthesis                                  */
  RSC_K_PRODUCTS = 2,  /* inverse DFT, grid products, forward DFT             */
  RSC_K_ANALYSIS = 3,  /* Legendre analysis                                   */
  RSC_K_RHS = 4,       /* curl projections, mass, drift and boundary rows     */
  RSC_K_CHAIN = 5,     /* chain solve, parallel part g = D'^{-1} b per block  */
  RSC_K_TEMP = 6,      /* per-l temperature solve                             */
  RSC_K_DOTS = 7,      /* GMRES dot products and their reduction              */
  RSC_K_AXPY = 8,      /* GMRES multi-vector updates                          */
  RSC_K_BLAS = 9,      /* other vector operations                             */
  RSC_K_CHAIN_SEQ = 10,/* chain solve, forward / backward sweeps (clusters)   */
  RSC_K_CHAIN_RED = 11,/* odd-even reduced chain solve, the passes over every
                          block (odd blocks, reduced right-hand side, odd blocks
                          from their neighbours)                               */
  RSC_NUM_KERNELS = 12
};

/* Start (mask != 0) or stop collecting per-kernel timings: CUDA events are
 * recorded around the launches of the kernels whose bit (1 << kernel_id) is
 * set in `mask`, on the context stream.  Clears the counters.  While tracing
 * is on, Jacobian actions run as individual launches instead of a replayed
 * CUDA graph.                                                               */
rsc_status rsc_profile_enable(rsc_ctx* ctx, int mask);

/* Accumulated device time (ms), launches, algorithmic bytes and flops of one
 * kernel since rsc_profile_enable (synchronises the stream).                */
rsc_status rsc_profile_query(rsc_ctx* ctx, int kernel_id, double* ms, long* launches,
                             double* bytes, double* flops);

/* Name of a kernel identifier.                                              */
const char* rsc_kernel_name(int kernel_id);

/* Number of kernel launches issued by this context since rsc_create.        */
rsc_status rsc_launch_count(const rsc_ctx* ctx, long* count);

/* Diagnostics of the bifurcation diagrams (Secs. 4-5), synchronous:
 *   KE     = (1/V) int |U|^2 / 2 dV over the shell, V = 4 pi (r_out^3 - r_in^3)/3,
 *            from the potentials by Parseval's identity (Sec. 2.1, Eq. Ylm_norm)
 *            and a Gauss-Legendre rule of 2 Nr + 16 radii;
 *   Nu_in, Nu_out = d_r of the spherical mean temperature at r_in, r_out divided
 *            by the conductive gradient -r_out r_in / r^2 there (1 for the
 *            conductive state of Sec. 2.1).
 * U is a device state; any of KE, Nu_in, Nu_out may be NULL (host pointers).
 * Returns RSC_EINVAL when ctx or U is NULL.                                 */
rsc_status rsc_diagnostics(rsc_ctx* ctx, const double* U, double* KE, double* Nu_in,
                           double* Nu_out);

/* Euclidean norm of a device vector of n doubles (synchronous).            */
rsc_status rsc_norm2(rsc_ctx* ctx, const double* v, size_t n, double* out);

/* Allocation-free variant of rsc_norm2 (the paper has no counterpart).
 * Some callers cannot call cudaMalloc: hosts whose device memory is wholly
 * owned by their own pool allocator, and long-running services that forbid
 * allocation after start-up.  This entry point needs no context and
 * allocates nothing: it writes ||v||_2 of the n doubles at device pointer v
 * to out[0] (a device pointer the caller owns), asynchronously on `stream`
 * (a cudaStream_t; NULL = legacy default stream) of the current device.
 * Its scratch is a fixed array of RSC_NORM2_NOALLOC_MAX_N / 4096 doubles
 * (16 KiB) in device memory, held by every GPU that loads the library until
 * the process exits.  The first call on a device looks the array up (once
 * per device, with that device current), so make that first call before any
 * stream capture.  The looked-up address belongs to the device's primary
 * context: after cudaDeviceReset (or anything else that destroys that
 * context) it is stale, and a later call would write through it, so do not
 * use this entry point in a process that resets its devices.  All calls on
 * a device share the array: calls whose
 * kernels overlap on the GPU (other streams, other host threads) race and
 * may return wrong sums; serialise them.  Returns RSC_EINVAL when v or out
 * is NULL or n > RSC_NORM2_NOALLOC_MAX_N, RSC_ECUDA when the look-up or
 * launch fails.                                                            */
#define RSC_NORM2_NOALLOC_MAX_N 8388608
rsc_status rsc_norm2_noalloc(const double* v, size_t n, double* out, void* stream);

/* Text of the last error on this context (never NULL).                     */
const char* rsc_last_error(const rsc_ctx* ctx);

/* Name of a status code.                                                   */
const char* rsc_status_string(int status);

/* ABI version of the loaded library (RSC_ABI_VERSION).                     */
int rsc_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RSC_H */
