/*
 * polyflood.h -- C ABI of the GB300 Newton step for fully implicit polymer
 * flooding (water, oil and polymer mass conservation under Darcy's law,
 * upstream-weighted two-point finite volumes, backward Euler), after
 * H. Liu, Z. Chen et al., arXiv 1807.05298.
 *
 * Conventions shared by every call
 *   - Units are SI: Pa, m, m^2, s, kg, Pa*s; concentrations kg/m^3.
 *   - The grid is Cartesian, nx * ny * nz cells of dx * dy * dz; cell (i,j,k)
 *     has the natural index i + nx*(j + ny*k) (Sec. 3 "natural ordering");
 *     k grows with depth; `top` is the depth of the top face of layer 0.
 *   - Unknowns are block-wise (Sec. 3.4): per cell (P_o, S_w, C), cells in
 *     natural order, then one bottom-hole pressure per well.  Residual rows
 *     are per cell (oil, water, polymer) masses [kg], then one row per well.
 *   - Every call returns pf_status.  On failure pf_last_error() gives a
 *     message (thread-local, owned by the library, valid until the next call
 *     on the same thread).  No C++ exception crosses this boundary.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Host
 *     arrays passed out are written by the library and must have the stated
 *     length.  Calls that take or return host arrays synchronise the stream.
 *   - A pf_sim is bound to the CUDA device current at pf_create and to the
 *     stream given there (NULL = the legacy default stream).  Calls on one
 *     pf_sim must not overlap from several threads.
 *   - After PF_ECUDA the pf_sim is unusable except for pf_destroy.
 */
#ifndef POLYFLOOD_H
#define POLYFLOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pf_status;
enum {
  PF_OK = 0,
  PF_EINVAL = 1,          /* invalid argument; nothing was changed or allocated */
  PF_ENOMEM = 2,          /* device or host allocation failed */
  PF_ENOT_CONVERGED = 3,  /* Newton or the Krylov solve hit its iteration cap */
  PF_ETIMEOUT = 4,        /* a bounded device wait gave up */
  PF_ECUDA = 5,           /* CUDA runtime error; the object is unusable */
  PF_EBUSY = 6            /* request cannot be admitted (serving) */
};

enum { PF_WELL_INJECTOR = 0, PF_WELL_PRODUCER = 1 };
enum { PF_DIR_X = 0, PF_DIR_Y = 1, PF_DIR_Z = 2 };
/* Well constraints, Sec. 2.4: fixed bottom-hole pressure, fixed water rate,
 * fixed oil rate, fixed liquid rate.  Rates are positive volume rates at
 * reference conditions [m^3/s] (formation volume factor 1). */
enum { PF_CTRL_BHP = 0, PF_CTRL_WRATE = 1, PF_CTRL_ORATE = 2, PF_CTRL_LRATE = 3 };
enum { PF_PREC_FP64 = 0, PF_PREC_MIXED = 1 };
enum { PF_PC_BJACOBI = 0, PF_PC_CPR = 1 };
/* Local (first-stage) solve of the preconditioner: the restricted additive
 * Schwarz step of CPR-FP (Alg. 2) with one subdomain per GPU, solved by
 * block-Jacobi (3x3 diagonal blocks) or by block ILU(0) in red-black order
 * (cells coloured by (i + j + k) mod 2; no fill between cells of a colour). */
enum { PF_S1_BJACOBI = 0, PF_S1_ILU0 = 1 };
enum { PF_MIX_NONLINEAR = 0, PF_MIX_LINEAR = 1 };

/* Rock, fluid, relative permeability and polymer constants (Sec. 2.1-2.3).
 *   phi(P) = phi_r + c_r (P - p_r)                                  Sec. 2.1
 *   rho_a(P_a) = rho_a (1 + c_a (P_a - p_ref))     (reading: linear law)
 *   Corey: Sn = (S - swc)/(1 - swc - sor) clipped to [0,1],
 *          k_rw = krw_max Sn^nw, k_ro = kro_max (1-Sn)^no,
 *          P_c = P_o - P_w = pc_e (1-Sn)^pc_n                       Sec. 2.2
 *   Langmuir A_d = ads_a C / (1 + ads_b C) [kg/m^3 rock], A_d,max = a/b;
 *   R_k = 1 + (rrf - 1) A_d / A_d,max                               Sec. 2.3
 *   beta = C / c_ref; mu_m linear or nonlinear mixing rule of mu_w, mu_p0;
 *   Todd-Longstaff mu_p,e, mu_w,partial, mu_w,e with mixing parameter omega
 *   and alpha = clip(C/c_ref, 0, 1)                                 Sec. 2.3
 *   Inaccessible pore volume ipv scales the polymer's pore space.    Sec. 2.3 */
typedef struct pf_physics {
  double rho_w, rho_o;      /* reference densities [kg/m^3] */
  double c_w, c_o;          /* fluid compressibilities [1/Pa] */
  double p_ref;             /* reference pressure of the density law [Pa] */
  double mu_w, mu_o;        /* water and oil viscosities [Pa s] */
  double c_r, p_r;          /* rock compressibility [1/Pa], reference pressure [Pa] */
  double swc, sor, nw, no, krw_max, kro_max;
  double pc_e, pc_n;        /* capillary entry pressure [Pa] and exponent */
  double ads_a, ads_b;      /* Langmuir constants */
  double rrf, ipv;          /* residual resistance factor, inaccessible pore volume */
  double omega, mu_p0, c_ref;
  int mixing;               /* PF_MIX_NONLINEAR or PF_MIX_LINEAR */
  double g;                 /* gravity [m/s^2] */
} pf_physics;

/* One well: perforated cells (natural indices, the first one is the datum of
 * the hydrostatic wellbore, Sec. 2.4), the direction of each perforation for
 * the Peaceman index (Sec. 2.4), and the index parameters.  A cell
 * may carry at most one perforation over all wells. */
typedef struct pf_well_desc {
  int kind;                 /* PF_WELL_INJECTOR or PF_WELL_PRODUCER */
  int n_perf;
  const int64_t* cells;     /* host [n_perf] */
  const int* dirs;          /* host [n_perf] PF_DIR_*, or NULL for all z */
  double rw, skin, gf, f, fh;
  double pb0;               /* initial bottom-hole pressure [Pa] */
} pf_well_desc;

typedef struct pf_model_desc {
  int nx, ny, nz;
  double dx, dy, dz, top;
  const double *kx, *ky, *kz;   /* host [N] permeability [m^2] */
  const double* phi;            /* host [N] reference porosity phi_r */
  const double *p0, *s0, *c0;   /* host [N] initial P_o, S_w, C */
  pf_physics phys;
  int n_wells;
  const pf_well_desc* wells;    /* host [n_wells] */
  /* Optional tables (Sec. 2.2: relative permeability and capillary pressure
   * as functions of saturation; Sec. 2.3: adsorption "in the form of a table"
   * and the water viscosity multiplier of the polymer solution).  Between
   * knots the value is the segment's straight line (its slope is the
   * derivative, also at a knot); below the first and from the last knot on,
   * the end value with derivative 0.  At most PF_MAX_KNOTS knots each; the
   * abscissae strictly increase.  n_sat = 0: the Corey curves of phys. */
  int n_sat;
  const double* sat_table;      /* host [n_sat][4]: S_w in [0, 1], k_rw >= 0, k_ro >= 0, P_c [Pa] */
  /* n_poly = 0: Langmuir and the mixing rule of phys.  Otherwise
   * mu_m = mu_w * multiplier(C), A_d = A_d(C) [kg/m^3 rock] and
   * A_d,max = the largest tabulated A_d (for R_k). */
  int n_poly;
  const double* poly_table;     /* host [n_poly][3]: C >= 0, multiplier > 0, A_d >= 0 */
} pf_model_desc;

#define PF_MAX_KNOTS 64

typedef struct pf_solver_opts {
  int precision;        /* PF_PREC_FP64: all arithmetic FP64.  PF_PREC_MIXED:
                           FP32 Jacobian storage and assembly derivatives,
                           FP32 preconditioner; residual, norms, Krylov basis
                           and orthogonalisation stay FP64. */
  int precond;          /* PF_PC_BJACOBI (the local solve alone) or PF_PC_CPR (Alg. 2) */
  int gmres_restart;    /* Krylov basis size m (default 30) */
  int gmres_max_iter;   /* cap on Krylov iterations per linear solve (default 300) */
  int newton_max_iter;  /* cap on Newton iterations per step (default 25) */
  int use_forcing;      /* 1: linear tolerance eta from the Sec. 3.3 forcing term in the form
                           forcing_form selects; 0: fixed lin_rtol */
  double lin_rtol;      /* fixed relative linear tolerance (default 1e-12) */
  double newton_tol;    /* scaled residual tolerance (default 1e-10) */
  double ds_max;        /* per-iteration saturation change limit (default 0.2) */
  double dc_frac;       /* per-iteration concentration change limit as a fraction of c_ref (default 0.5) */
  int amg_pre_sweeps, amg_post_sweeps;   /* CPR pressure smoother sweeps on the finest level (default 1, 1) */
  int amg_coarse_size;  /* coarsen until at most this many cells, <= 64 (default 32) */
  int amg_cycle;        /* 1: V-cycle, 2: W-cycle below the finest level (default 1) */
  int autotune;         /* 1: pf_create tunes the per-cell kernels' block sizes (pf_autotune) (default 0) */
  int forcing_form;     /* which choice of the Sec. 3.3 forcing term, all restricted to [0.01, 0.1],
                           first Newton iteration of a step 0.1 (default 3):
                           1: |b^l - r^{l-1}| / |b^{l-1}|, r^{l-1} = b^{l-1} - J dx^{l-1}
                              the residual the previous linear solve left (one
                              extra device vector and one SpMV per iteration);
                           2: (|b^l| - |r^{l-1}|) / |b^{l-1}| (one extra SpMV);
                           3: 0.5 (|b^l| / |b^{l-1}|)^((1 + sqrt 5) / 2), the
                              paper's choice.  b = -R; 2-norms over all unknowns. */
  int stage1;           /* PF_S1_BJACOBI or PF_S1_ILU0: the local solve, alone (PF_PC_BJACOBI)
                           or as the first stage of CPR (default PF_S1_ILU0) */
  int amg_coarse_sweeps;  /* pre- and post-smoothing sweeps on the levels below the finest;
                             -1: the finest level's counts (default 2) */
  double reorth_eta;    /* classical Gram-Schmidt takes its second pass when the first one left less
                           than reorth_eta of |w| (default 0.2: a single pass leaves the new vector
                           orthogonal to within about eps |w| / |w'| <= 5 eps; 0: never, 1: always) */
  double ilu_guard;     /* ILU(0) pivot guard: a black cell whose Schur-updated diagonal block has
                           det(D') / det(D) <= ilu_guard keeps D (default 0.1; a large negative
                           value disables the guard) */
  double newton_div;    /* Newton gives up on the step (PF_ENOT_CONVERGED) once the scaled residual
                           exceeds newton_div times its value at the step's first iteration
                           (default 1e6; 0: only the iteration cap) */
  int ilu_store;        /* ILU(0) sweeps read 0: J itself (whose cache lines also hold the other
                           colour's rows), 1: a compact copy of each colour's off-diagonal blocks
                           in J's precision, 2: the same copy in BF16 (mixed precision only);
                           made at each preconditioner set-up.  -1 (default): 2 in mixed and 1 in
                           FP64 precision from 1,000,000 cells on, else 0.  Any value but 0 also
                           gives the finest multigrid smoother per-colour copies of its stencil
                           and 1/diag (in the preconditioner's precision).  The black colour's copy
                           holds J_bj D_j^-1 (the set-up's products with the red inverses) in place
                           of J_bj, so the solve needs no diagonal red sweep; it then differs from
                           the solve without the copies in rounding only.  In FP64 precision the
                           copies also keep the ILU(0) diagonal block inverses per colour slot, in
                           place of the per-cell array */
  int krylov_lookahead; /* 1 (default): while Arnoldi step j runs, enqueue step j + 1 before the host
                           reads step j's Hessenberg column, unless the residual extrapolated from
                           the previous steps says step j may meet the tolerance; 0: enqueue each
                           step after the previous one is checked.  A step enqueued after the
                           solve has converged runs but is not used: the result is the same
                           either way, only the host round trip between steps differs */
} pf_solver_opts;

typedef struct pf_well_control {
  int ctrl;             /* PF_CTRL_* */
  double target;        /* Pa for BHP, else m^3/s at reference conditions */
  double limit;         /* BHP limit [Pa] or 0 for none (see pf_step: applied by switching) */
  double c_inj;         /* injected polymer concentration [kg/m^3] */
} pf_well_control;

typedef struct pf_iter_report {
  double res_scaled;    /* dimensionless max-norm of the residual before the update */
  double res_norm2;     /* 2-norm of the residual [kg] */
  double eta;           /* linear tolerance used */
  double lin_rel_res;   /* achieved relative linear residual */
  int krylov_iters;
  int converged;        /* 1 if res_scaled <= newton_tol (no update was made) */
} pf_iter_report;

typedef struct pf_step_report {
  int newton_iters, krylov_iters, converged;
  double res_scaled;
} pf_step_report;

/* Process-wide: launch the solver's kernels with programmatic dependent
 * launch (a kernel may be scheduled while its predecessor in the stream
 * drains; it waits for that grid's completion before reading anything).  Off
 * by default (measured 1-3% slower on this solver's short kernels); results
 * do not depend on it.  Affects launches and graphs captured after the call. */
pf_status pf_set_programmatic_launch(int on);

/* Library version string (static storage). */
const char* pf_version(void);
/* Message of the last failed call on this thread (static thread-local storage). */
const char* pf_last_error(void);
/* Fills o with the defaults stated in pf_solver_opts. */
pf_status pf_default_opts(pf_solver_opts* o);

typedef struct pf_sim pf_sim;

/* Model loading, grid set-up and initialisation (Sec. 3, steps 1-3): copies
 * the description, computes transmissibilities (Sec. 3.2, harmonic k and
 * geometry) and Peaceman well indices (Sec. 2.4) on the host,
 * uploads everything to device memory owned by the returned object.
 * stream: a cudaStream_t borrowed for the life of the object (NULL allowed).
 * Errors: PF_EINVAL (sizes, NaN, doubly perforated cell), PF_ENOMEM, PF_ECUDA. */
pf_status pf_create(const pf_model_desc* m, const pf_solver_opts* o, void* stream, pf_sim** out);
/* Frees all device and host memory of s; NULL is accepted. */
pf_status pf_destroy(pf_sim* s);
/* Host-side fault injection for tests of pf_create's failure paths (the
 * paper has no counterpart).  Arms the next pf_create (on any thread) so that
 * its k-th CUDA runtime call reports an error instead of running, without
 * touching the GPU: call 1 is the device arena's allocation and call 2 the
 * pinned host buffer (both reported as PF_ENOMEM), then the capture stream,
 * the two step events, the uploads and the closing synchronisation (PF_ECUDA).
 * pf_create then frees everything it had allocated, leaves *out NULL and
 * returns that status with the failed call in pf_last_error().  The hook
 * disarms when it fires and at the end of a pf_create that made fewer than k
 * calls; k = 0 disarms it.  PF_EINVAL for k < 0. */
pf_status pf_inject_create_failure(int k);
/* Well constraints for the next steps (Sec. 3, step 4(b): unchanged within a
 * step).  c[nwells], nwells must equal the model's well count. */
pf_status pf_set_controls(pf_sim* s, const pf_well_control* c, int nwells);

/* Starts a backward-Euler step of length dt [s] from the current state: keeps
 * x^n, evaluates the old masses M^n and the lagged wellbore unit weights. */
pf_status pf_begin_step(pf_sim* s, double dt);
/* One Newton iteration of Alg. 1 at the current iterate: property evaluation,
 * residual and Jacobian assembly, convergence test, linear tolerance from
 * the forcing term of Sec. 3.3, preconditioner set-up, Krylov solve, update.  Requires
 * pf_begin_step.  rep may be NULL. */
pf_status pf_newton_iteration(pf_sim* s, pf_iter_report* rep);
/* pf_begin_step + Newton iterations to convergence (Alg. 1), controls fixed
 * within the step (Sec. 3 step 4(b)).  BHP limits of rate wells (the limit
 * field of pf_well_control, Sec. 4.1.2 "constrained with its bottom hole
 * pressure"): after convergence a rate well whose BHP crossed its limit
 * (injector above, producer below) is moved onto BHP = limit and the step is
 * re-solved from x^n; a switched well whose rate at the limit exceeds its
 * target returns to rate control; at most two re-solves per step.  The
 * switched state persists across steps until the well's constraint changes
 * in pf_set_controls.  On PF_ENOT_CONVERGED the state is restored to x^n (the
 * caller cuts dt, Sec. 3 step 4(a)). */
pf_status pf_step(pf_sim* s, double dt, pf_step_report* rep);
/* Step pieces for callers that drive Newton one iteration at a time:
 * pf_end_step after pf_newton_iteration reported convergence applies the BHP
 * limit check of pf_step; *resolve = 1 means a switch changed, the state was
 * restored to x^n and the step must be solved again (pf_begin_step with the
 * same dt).  pf_abort_step restores x^n after a failed step. */
pf_status pf_end_step(pf_sim* s, int* resolve);
pf_status pf_abort_step(pf_sim* s);
/* Per-well mass rates into the reservoir (positive for injection) [kg/s] of
 * water, oil and polymer (the perforation rates of Sec. 2.4) at the current
 * state with the wellbore weight of the current step, and the reference BHP [Pa]; host arrays of the
 * well count, any may be NULL. */
pf_status pf_well_rates(pf_sim* s, double* q_w, double* q_o, double* q_p, double* pb);
/* switched[w] = 1 if rate well w currently runs on its BHP limit. */
pf_status pf_well_switched(const pf_sim* s, int* switched);

/* Test hooks.  pf_assemble evaluates R and J at the current iterate (after
 * pf_begin_step).  pf_export_system copies them to the host:
 *   R[3N + W];
 *   Jc[7 * 9 * N]: block slot s (0 diagonal, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z,
 *     6 +z), entry e = 3*row + col within the 3x3 block (rows oil, water,
 *     polymer; cols P, S, C), cell i at Jc[(s*9 + e)*N + i]; slots that leave
 *     the grid hold 0;
 *   Jw_b[3 * Pf]: dR_cell/dP_b per perforation (perforations in well order);
 *   Jw_c[3 * Pf]: dR_well/dx_cell per perforation;  Jw_d[W]: dR_well/dP_b.
 * Any output pointer may be NULL to skip it. */
pf_status pf_assemble(pf_sim* s);
pf_status pf_export_system(pf_sim* s, double* R, double* Jc, double* Jw_b, double* Jw_c, double* Jw_d);
/* y = J x with the assembled Jacobian (host x[3N+W], host y[3N+W]). */
pf_status pf_apply_jacobian(pf_sim* s, const double* x, double* y);
/* z = M^-1 v with the configured preconditioner, set up from the assembled
 * Jacobian (host v, z of length 3N+W; a test hook). */
pf_status pf_apply_preconditioner(pf_sim* s, const double* v, double* z);
/* Solves J x = b with the configured preconditioned Krylov method to relative
 * tolerance rtol (host b, x of length 3N+W).  *iters and *rel_res may be NULL. */
pf_status pf_solve_linear(pf_sim* s, const double* b, double* x, double rtol, int* iters, double* rel_res);

/* Host copies of the state (checkpoint / resume).  P, S, C [N]; Pb [W];
 * any pointer may be NULL. */
pf_status pf_get_state(pf_sim* s, double* P, double* S, double* C, double* Pb);
pf_status pf_set_state(pf_sim* s, const double* P, const double* S, const double* C, const double* Pb);
/* Number of cells, wells and perforations of s. */
pf_status pf_sizes(const pf_sim* s, int64_t* n_cells, int* n_wells, int64_t* n_perf);
/* Device-resident state pointers (valid for the life of s): x is the
 * interleaved unknown vector [3N + W] (FP64). */
pf_status pf_device_state(pf_sim* s, double** x_dev);
/* Host copies of the whole interleaved unknown vector x[3N + W] (block-wise
 * order), straight between the caller's buffer (pinned or pageable) and the
 * device state. */
pf_status pf_get_x(pf_sim* s, double* x);
pf_status pf_set_x(pf_sim* s, const double* x);
/* Opt-in CUDA-event timing of kernel classes on the sim's stream: enabling
 * (or disabling) resets the counters; pf_kernel_timing returns the launches
 * and summed device time [ms] of one class since then. */
enum { PF_KT_SPMV = 0, PF_KT_PROPS, PF_KT_FACE, PF_KT_GATHER, PF_KT_WELLS, PF_KT_ORTHO, PF_KT_PRECOND,
       PF_KT_COUNT };
pf_status pf_kernel_timing_enable(pf_sim* s, int on);
pf_status pf_kernel_timing(pf_sim* s, int which, int64_t* launches, double* total_ms);
/* Launch-shape tuner (not in the paper: a GB300 launch detail).  Times block
 * sizes 64, 128 and 256 for the per-cell kernels (properties, face flux,
 * gather, SpMV, stage 2, finest-level smoother) and the two- or three-launch
 * ILU(0) solve on s's own data and keeps the fastest (the smoother's block
 * sizes and the two ILU(0) forms, timed as whole preconditioner applications,
 * take turns over five rounds and each keeps its fastest round).  The FP64 SpMV also tries one thread per block row (reported
 * as a negative spmv: -96, -192 or -384 threads per block).  Each row's
 * arithmetic does not depend on the launch shape, so results are
 * bit-identical whatever is chosen; reduction grids are never tuned for the
 * same reason.  Overwrites scratch (call between Newton iterations, not
 * inside one); out may be NULL. */
typedef struct pf_tuning {
  int props, face, gather, spmv, stage2, rbgs;
  int block_cells;  /* CPR: multigrid levels of at most this many cells (and all coarser ones) run in
                       one thread block (default 512 in FP64, 4096 in FP32; the tuner keeps it) */
  int ilu_fused;    /* ILU(0) solve in two launches, the diagonal red sweep folded into the black
                       sweep (1), or three launches (0); the same arithmetic either way.  No
                       effect with the per-colour copies (ilu_store), where the solve is always
                       two launches through the set-up's products J_bj D_j^-1 */
  int cluster_cells;  /* CPR: larger levels of at most this many cells (<= 16384) run in one
                         thread-block cluster of up to 16 blocks with cluster barriers between
                         phases; 0: none.  The same arithmetic as the per-level kernels. */
} pf_tuning;
pf_status pf_autotune(pf_sim* s, pf_tuning* out);
/* Sets the launch shapes directly (for example a shape pf_autotune chose
 * earlier): every block size a multiple of 32 in [32, 256]; spmv may also be
 * -96, -192 or -384 (one thread per block row) in FP64 precision; block_cells
 * in [1, 65536]; ilu_fused 0 or 1; cluster_cells in [0, 16384].  Results do not depend on the shapes.  PF_EINVAL for any
 * other value. */
pf_status pf_set_tuning(pf_sim* s, const pf_tuning* t);
/* The launch shapes s uses now (chosen by pf_autotune, given by pf_set_tuning,
 * or the defaults); launches nothing.  PF_EINVAL for a NULL t. */
pf_status pf_get_tuning(const pf_sim* s, pf_tuning* t);
/* Kernel launches issued by s so far (monotone counter). */
pf_status pf_launch_count(const pf_sim* s, int64_t* count);

/* ---------------------------------------------------------------------------
 * Time loop, batch engine and serving loop (host runtime, pf_runtime.cu)
 * ------------------------------------------------------------------------- */

/* A schedule: periods of n_steps fixed steps of length dt [s] under fixed
 * well controls (controls[n_wells] host array), Sec. 3 step 4(b). */
typedef struct pf_period {
  int n_steps;
  double dt;
  const pf_well_control* controls;
} pf_period;
typedef struct pf_schedule {
  int n_periods;
  const pf_period* periods;
} pf_schedule;
typedef struct pf_run_report {
  int steps, newton_iters, krylov_iters, cuts;
  pf_status status;
  double seconds;      /* host wall time of the run */
} pf_run_report;

/* Runs the whole schedule on s: per step pf_step, halving the step on Newton
 * failure (Sec. 3 step 4(a)) at most max_cuts times per step; after each
 * accepted sub-step the step doubles again, capped by the period's dt and by
 * what is left of the step (step 4(c)-(d)); the next step starts from the full
 * dt.  rep may be NULL. */
pf_status pf_run_schedule(pf_sim* s, const pf_schedule* sched, int max_cuts, pf_run_report* rep);
/* Message of the last failed runtime call (pf_run_schedule, pf_batch_*, pf_server_*) on this thread. */
const char* pf_runtime_last_error(void);

/* Capillary-gravity equilibrium initial state (Sec. 4.1.3): fills p0 (oil
 * pressure) and s0 (water saturation), host arrays [N], for the grid, rock,
 * fluid and capillary data of m (its own p0, s0, c0 and wells are ignored
 * and may be NULL / 0).
 *   - Oil pressure: from (datum_depth, datum_p) to the centre of the layer
 *     holding the datum along dP/dz = g rho_o(P) (closed form for the linear
 *     density law), then layer to layer in each column so that the discrete
 *     oil potential difference of every vertical face is zero with the
 *     discretisation's face density (reference-pore-volume weighted).
 *   - Water pressure: P_w = P_o at contact_depth (the free water level), then
 *     the same construction for water.
 *   - S_w = the largest S in [0, 1] with P_c(S) >= P_o - P_w (P_c must not
 *     increase with S), or the first saturation knot / swc when no S
 *     qualifies; where P_c(S_w) exceeds P_o - P_w (below the contact) the oil
 *     pressure is set to P_w + P_c(S_w).
 * With layers of uniform porosity and no wells, the state is a rest state of
 * the discrete equations.  Host code only (no device work).  PF_EINVAL on
 * invalid data or an increasing P_c, with the message in pf_last_error. */
pf_status pf_equilibrium_init(const pf_model_desc* m, double datum_depth, double datum_p, double contact_depth,
                              double* p0, double* s0);

/* Device bytes pf_create would allocate for this model and these options
 * (one arena per simulator; used for admission by footprint). */
pf_status pf_footprint(const pf_model_desc* m, const pf_solver_opts* o, size_t* bytes);

/* Batch engine: n scenarios, each a pf_sim with its own stream and CUDA
 * graphs on the current device; pf_batch_run drives them from n_threads host
 * threads so their kernels overlap on the GPU.  schedules[n], reports[n]
 * (may be NULL).  Returns the first failing member's status.  o may be NULL
 * (defaults); its krylov_lookahead is ignored (members run with 0, since their
 * overlapping work already fills the gaps it would hide; the same holds for
 * pf_server). */
typedef struct pf_batch pf_batch;
pf_status pf_batch_create(const pf_model_desc* const* models, int n, const pf_solver_opts* o, int n_threads,
                          pf_batch** out);
pf_status pf_batch_run(pf_batch* b, const pf_schedule* const* schedules, int max_cuts, pf_run_report* reports);
pf_status pf_batch_member(pf_batch* b, int i, pf_sim** out);
pf_status pf_batch_destroy(pf_batch* b);

/* Packed assembly for the batch (the paper has no counterpart: it runs one
 * simulation at a time).  With on = 1 every member's assembly (cell
 * properties, face fluxes, gather, wells) goes through a shared packer: the
 * members that reach an assembly together are assembled by one launch per
 * kernel over all their cells (up to 24 members per launch, several launches
 * beyond that), on a stream of the batch that is ordered after each member's
 * stream and before its next work.  The first member to arrive waits up to
 * window_us microseconds for the others that are inside pf_batch_run (0: pack
 * whoever is waiting now).  Results are bit-identical to the members' own
 * launches.  on = 0 detaches the packer.  Call it only while no pf_batch_run
 * is in progress; PF_EINVAL for a negative window, PF_ECUDA if the stream or
 * events cannot be created.  The batch owns the packer until
 * pf_batch_destroy. */
pf_status pf_batch_set_packing(pf_batch* b, int on, double window_us);
/* Packs launched and members assembled through them since packing was last
 * turned on (their ratio is the mean pack size); either pointer may be NULL. */
pf_status pf_batch_packing_stats(pf_batch* b, int64_t* packs, int64_t* members);

/* Serving loop: requests (a model and a schedule, deep-copied at submit) are
 * queued in arrival order; n_workers host threads admit the first queued
 * request whose footprint fits the free part of hbm_budget, create its pf_sim
 * (device state stays resident for the whole run), run its schedule, keep
 * the final state on the host and free the device memory.  Requests that
 * arrive while others run are admitted as memory and workers free up, and
 * their work overlaps on the GPU.  PF_EBUSY at submit: the request can never
 * fit the budget.  Times are host steady-clock seconds. */
enum { PF_REQ_QUEUED = 0, PF_REQ_RUNNING = 1, PF_REQ_DONE = 2, PF_REQ_FAILED = 3 };
typedef struct pf_result {
  int state;           /* PF_REQ_* */
  pf_status status;
  pf_run_report report;
  double t_submit, t_start, t_end;
  size_t footprint;
} pf_result;
typedef struct pf_server pf_server;
pf_status pf_server_create(size_t hbm_budget, int n_workers, const pf_solver_opts* o, int max_cuts,
                           pf_server** out);
pf_status pf_server_submit(pf_server* srv, const pf_model_desc* m, const pf_schedule* sched, uint64_t* ticket);
pf_status pf_server_poll(pf_server* srv, uint64_t ticket, pf_result* out);
/* Blocks until the request is done or failed (PF_ETIMEOUT after timeout_s). */
pf_status pf_server_wait(pf_server* srv, uint64_t ticket, double timeout_s, pf_result* out);
/* Final P, S, C [N] and Pb [W] of a finished request (host arrays, any NULL). */
pf_status pf_server_fetch_state(pf_server* srv, uint64_t ticket, double* P, double* S, double* C, double* Pb);
pf_status pf_server_stats(pf_server* srv, size_t* in_use, int* running, int* queued);
/* Stops the workers after their current requests; queued requests are dropped. */
pf_status pf_server_destroy(pf_server* srv);

/* Residual norms without any device allocation.  The paper has no
 * counterpart.  Some callers of this library cannot call cudaMalloc: a host
 * framework that hands out every byte of device memory from its own pool and
 * treats any other allocation as an error, or a loop with a fixed time budget
 * per iteration that cannot afford an allocation (which may synchronise the
 * device) once it has started.  For them this entry point computes what the
 * residual-norm step of pf_newton_iteration computes, from caller-owned
 * device buffers:
 *   out[0] = max over cells of |R_oil| / (V phi_r rho_o), |R_water| /
 *            (V phi_r rho_w), |R_polymer| / (V phi_r c_ref) and over wells of
 *            |R_well| / well_denom, the Newton convergence measure;
 *   out[1] = 2-norm of R, the measure the forcing term uses.
 * Arguments (device pointers unless stated): R[3 n_cells + n_wells] block-wise
 * residual; inv_pv[n_cells] = 1 / (V phi_r); well_denom[n_wells] the well
 * rows' scale (dt * W * 1e5 Pa for a BHP row, dt * rho_ref * |target| for a
 * rate row; may be NULL without wells); rho_o, rho_w, c_ref host scalars;
 * out[2] device output; stream a cudaStream_t of the CUDA device that is
 * current on the calling thread (NULL = its legacy stream); a stream of
 * another device is rejected with PF_EINVAL.
 * Limits: n_cells <= 16,777,216 and n_wells <= 4096 (PF_EINVAL with a message
 * from pf_noalloc_last_error() otherwise).  Its scratch is one fixed 64 KiB
 * device array per GPU that loads the library, held until the process exits;
 * the function calls no cudaMalloc, cudaFree or allocating library routine.
 * The first call on each device resolves the array's device address (a
 * symbol lookup, no allocation) and keeps it for later calls; make that
 * first call before any stream capture.  The kept address is void after
 * cudaDeviceReset.  All calls on a device share the array, which holds the
 * last call's partial results; each call clears the counter it needs, and
 * calls that overlap on the GPU (other streams, concurrent host threads) race
 * on the array: serialise them.  Asynchronous: out is written in stream
 * order. */
pf_status pf_residual_norms_noalloc(int64_t n_cells, int n_wells, const double* R, const double* inv_pv,
                                    const double* well_denom, double rho_o, double rho_w, double c_ref,
                                    double* out, void* stream);
/* Message of the last failed pf_residual_norms_noalloc call on this thread. */
const char* pf_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POLYFLOOD_H */
