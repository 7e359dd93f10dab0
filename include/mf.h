/*
 * mf.h -- C interface of the GB300 (sm_103a) library for the FFT-based method-of-lines
 * solution of thin-film (2D) and bulk (3D) magnetization problems of type-II
 * superconductors, after L. Prigozhin and V. Sokolovsky, "FFT-based solution of 2D and 3D
 * magnetization problems in type-II superconductivity" (arXiv:1801.04869).
 *
 * All quantities are dimensionless as in Section 2.3 (film: lengths / l, t / t0,
 * e / e0, j / jc, h_z / jc, g / (jc l), t0 = mu0 jc l / e0) and Section 3.2, Eq. 19 (bulk:
 * h / (jc l), t0 = mu0 jc l^2 / e0), so mu0 = 1; e0 and jc default to 1.
 *
 * Grid: nx x ny (x nz) cells, cell-centred, on the periodic box
 * D = [-Lx, Lx] x [-Ly, Ly] (x [-Lz, Lz]) (Section 2.2, Section 3.1); x is the fastest
 * index.  Each extent must be a power of two: film 8..2048 per axis, bulk 8..512 per axis.
 *
 * State vectors (device, float64):
 *   film  g, the stream function of the sheet current (Eq. 2), nx*ny values
 *   bulk  h, the magnetic field, 3*nx*ny*nz values, component-major (h_x block, h_y, h_z)
 *
 * Ownership: the caller owns every device buffer it passes, including the workspace
 * (mf_workspace_bytes() bytes, 256-byte aligned).  The problem handle is host memory owned by
 * the library until mf_destroy().  No call allocates device memory.  All work is queued on
 * the stream given to mf_create(); calls that return a status synchronise that stream.
 *
 * Errors: every call returns an mf_status; no C++ exception crosses this interface.
 * mf_last_error() gives a message for the most recent failing call on a handle.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MF_OK = 0,
  MF_ERR_ARG = 1,             /* invalid argument or unsupported size */
  MF_ERR_CUDA = 2,            /* a CUDA call failed (message in mf_last_error) */
  MF_ERR_NOCONV = 3,          /* outside iteration did not reach iter_tol in iter_max steps */
  MF_ERR_NONFINITE = 4,       /* a NaN or infinity appeared in a derivative */
  MF_ERR_STEP_UNDERFLOW = 5,  /* adaptive step fell below h_min */
  MF_ERR_WORKSPACE = 6,       /* workspace too small or misaligned */
  MF_ERR_BARRIER = 7          /* a grid barrier timed out; the launch stopped early */
} mf_status;

typedef struct mf_problem mf_problem;

/* Problem description.  Fill with mf_default_params() first. */
typedef struct {
  int dim;                    /* 2 = thin film (state g), 3 = bulk (state h) */
  int nx, ny, nz;             /* grid; nz = 1 for a film */
  double Lx, Ly, Lz;          /* half extents of D */
  const uint8_t* mask;        /* host, nx*ny*nz: 0 = free space (Ohm law rho_out, the outside
                                 iteration acts here), 1 = superconductor (power law),
                                 2 = normal conductor, Ohm law, not iterated (filled hole in a
                                 film, Section 2.2; cutting layer in a bulk body, Section 3.1) */
  const double* jc_map;       /* host, nx*ny*nz critical current per cell, or NULL (use jc) */
  double jc, n, e0;           /* power law rho = (e0/jc) |j/jc|^(n-1), Eq. 3 / Eq. 13 */
  double rho_out;             /* fictitious resistivity of free space and normal cells */
  double sigma;               /* Gaussian filter width; <= 0: sqrt(dx^2+dy^2(+dz^2)) */
  double lambda;              /* film relaxation of Eq. 12 (0.7, Section 2.2) */
  double iter_tol;            /* film: absolute bound on mean |g_dot| over free space
                                 (2e-4, Section 2.3); bulk: delta_it of Section 3.1.
                                 <= 0: run exactly iter_max iterations */
  int iter_max;               /* cap on outside iterations per right-hand side */
  int precision;              /* 0: FP64 transforms; 1: FP32 transforms and power law with
                                 FP64 state, error norm and iteration residual */
  double rtol, atol;          /* BS23 tolerances */
  double h0;                  /* first step; <= 0: min(1e-3, 0.01 (t1 - t0)) */
  double h_min;               /* smallest step before MF_ERR_STEP_UNDERFLOW */
  const double* he_t;         /* host, he_knots increasing times of a piecewise-linear h_e(t) */
  const double* he_v;         /* host, values at the knots */
  int he_knots;               /* 0: use the sinusoid below */
  double he_sin_amp, he_sin_period;   /* h_e = amp sin(2 pi t / period) */
  double he_dir[3];           /* bulk: direction of the uniform applied field (default z) */
  /* Other current-voltage laws of the same method (the conclusion of the paper names
     anisotropic and field-dependent relations as drop-in replacements for Eq. 3 / Eq. 13).
     Both act in the superconductor (mask 1) only; the defaults give Eq. 3 / Eq. 13. */
  double gamma;               /* anisotropy > 0 (default 1): the elliptic power law
                                 e = rho(j_eff) A j,  rho(s) = (e0/jc) (s/jc)^(n-1),
                                 j_eff^2 = j^T A j,  A = diag(1, 1/gamma^2) for a film (the
                                 critical current along y is gamma jc) and
                                 diag(1, 1, 1/gamma^2) for a bulk body (along z) */
  double b0;                  /* bulk only: > 0 gives the Kim-type critical current
                                 jc / (1 + |h| / b0), |h| the local field of the state;
                                 0 (default): none.  A film with b0 > 0 is MF_ERR_ARG. */
} mf_params;

/* One attempted BS23 step (lock-step log). */
typedef struct {
  double t, h, t_new, err;
  int outcome;                /* 0 rejected (error), 1 accepted, 2 rejected (iteration failed) */
  int iters[4];               /* outside iterations of stages k1..k4, -1 if not evaluated */
  int pad;
} mf_step_log;

/* Counters and integrator state. */
typedef struct {
  double t, h;
  long long n_attempts, n_accepted, n_rejected, n_rhs, n_iters, n_noconv, log_count;
  int last_iters;
  double last_r, last_err;
  int grid, threads, smem_bytes, rows_per_item;
  long long workspace_used;
} mf_info;

enum { MF_READ_HZ = 0, MF_READ_MOMENT = 1, MF_READ_J = 2, MF_READ_E = 3 };

/* Defaults: dim 2, n 19, jc = e0 = 1, rho_out 1, lambda 0.7, iter_tol 2e-4, iter_max 1000,
   precision 0, rtol = atol = 1e-6, h_min 1e-12, he_dir (0,0,1), gamma 1, b0 0. */
void mf_default_params(mf_params* p);

/* Device workspace needed by mf_create for these parameters (0 if they are invalid). */
size_t mf_workspace_bytes(const mf_params* p);

/* Set up a problem in a caller-owned device workspace: copies the mask, jc map, knots and
   transform tables, and precomputes the free-space responses used by the outside iteration.
   `stream` is a cudaStream_t (NULL = legacy default stream).  The integrator starts at t = 0
   with a zero state; use mf_set_state() to change it. */
mf_status mf_create(const mf_params* p, void* d_workspace, size_t bytes, void* stream,
                    mf_problem** out);

/* One right-hand side f(t, y) (Section 2.2 for films: Eqs. 9-12; Section 3.1 for bulk
   bodies: Eqs. 13-18).  d_y and d_ydot are device float64 state vectors.  The outside
   iteration starts from a previous free-space solution (Section 2.2): for films, that of the
   last evaluation of the integrator's most recent accepted step (the previous time step) once
   mf_advance/mf_step has accepted one, else that of the previous call; for bulk bodies, that
   of the previous call.  Returns MF_ERR_NOCONV when the iteration did not converge (d_ydot then
   holds the last iterate).  *iters_out (may be NULL) receives the number of iterations. */
mf_status mf_rhs(mf_problem* pb, double t, const double* d_y, double* d_ydot, int* iters_out);

/* As mf_rhs, with an explicit h_e segment (-2: from t) and, when force_iters > 0, exactly
   force_iters outside iterations (for lock-step comparison with another implementation). */
mf_status mf_rhs_ex(mf_problem* pb, double t, int seg, const double* d_y, double* d_ydot,
                    int force_iters, int* iters_out);

/* Time limit of one grid-barrier wait inside the persistent launches (seconds; <= 0 restores
   the default of 4 s).  A launch whose wait runs out raises an abort flag that every CTA polls,
   so all CTAs leave promptly and the call returns MF_ERR_BARRIER; the problem stays usable (call
   mf_reset_warm before relying on the warm start again).  This bounds every wait so that a CTA
   that never arrives (which a cooperative launch rules out) cannot hang the GPU.  The paper has
   no counterpart: it is part of the library's failure detection. */
mf_status mf_set_barrier_timeout(mf_problem* pb, double seconds);

/* Forget the warm starts (previous call and previous time step): the next right-hand side
   starts from h_e_dot on free space. */
mf_status mf_reset_warm(mf_problem* pb);

/* Set the integrator state: time t, next step h (<= 0: default), state d_y (device, copied).
   Clears the first-same-as-last derivative and the step log. */
mf_status mf_set_state(mf_problem* pb, double t, double h, const double* d_y);

/* Copy the current state to d_y (device, may be NULL) and return t and h. */
mf_status mf_get_state(mf_problem* pb, double* t, double* h, double* d_y);

/* Advance with adaptive BS23 steps until t reaches t_target exactly or max_attempts step
   attempts were made (one launch; every decision is taken on the device).  Steps are
   clipped to end on t_target and on h_e knots. */
mf_status mf_advance(mf_problem* pb, double t_target, long long max_attempts);

/* Advance n independent problems (films or bulk bodies) to t_targets[i] (as mf_advance), at
   the same time.  Films (dim 2) of one device and precision are arranged as mf_batch_plan
   describes: a film whose own launch fills the GPU gets that launch, on its own stream; the
   others share persistent launches, one after the other on the stream of the first of them,
   each launch's CTAs cut into one consecutive range per film, and every range runs the
   one-film code with that film's descriptor, grid barrier and partial sums, so each film's
   result is identical to its mf_advance.  Work already queued on a film's own stream is waited
   for first.  Bulk bodies get one launch each on their own streams, all enqueued before any is
   waited for.  Batching has no counterpart in the paper: it is how many independent
   magnetization problems (a parameter or geometry sweep) share one GPU.  statuses (may be
   NULL) receives each problem's status; the return value is the first non-OK one (MF_OK if
   all succeeded).  n = 0 does nothing and returns MF_OK.  MF_ERR_ARG, before any work: pbs or
   t_targets NULL, n < 0, a NULL or a repeated problem.  Returns when every problem has
   finished. */
mf_status mf_advance_batch(mf_problem* const* pbs, int n, const double* t_targets,
                           long long max_attempts, mf_status* statuses);

/* The arrangement mf_advance_batch uses for n films of one device and precision (host only, no
   GPU work): nx, ny are the films' grids, own_grid[i] the CTAs of film i's own launch
   (mf_info.grid), work[i] > 0 its expected work (NULL: cells x log2 cells), coresident the CTAs
   that fit the GPU at once.  mf_advance_batch passes cells x log2 cells times the film's field
   passes per step attempt (19 per right-hand side, 14 per outside iteration) measured in its
   previous batch call, else averaged over its history.  Films are ordered by work, most first,
   into order[0..n-1].  A film with own_grid >= coresident gets launch[i] = -1 (a launch of its
   own, ctas[i] = coresident).  The others fill shared launches 0, 1, ... in that order, at
   most 256 films each, a launch being closed before a film whose share of the grid in
   proportion to its work would be below one CTA; ctas[i] is film i's CTA count in its launch
   (1 <= ctas[i] <= own_grid[i], a launch's CTAs sum to at most coresident, and the largest
   work per CTA of a launch is as small as whole CTAs allow), its range following the launch's
   earlier films in `order`.  Returns the number of shared launches, or -1 for invalid
   arguments. */
int mf_batch_plan(int n, const int* nx, const int* ny, const int* own_grid, const double* work,
                  int coresident, int* order, int* launch, int* ctas);

/* One BS23 step attempt towards t_max; *accepted (may be NULL) is 1 if it was accepted. */
mf_status mf_step(mf_problem* pb, double t_max, int* accepted);

/* Integrate from the current state to each time in t_out (increasing) and record readouts:
   h_m_out (host, may be NULL) gets the magnetization (film: m_z, 1 value per time; bulk:
   m, 3 values per time); d_hz_out (device, may be NULL) gets h_z (film) or j (bulk, 3 fields)
   per output time.  An unset first step (mf_params.h0 <= 0, nothing integrated yet) is chosen
   for the whole span up to the last output time: min(1e-3, 0.01 (t_out[n_out-1] - t)). */
mf_status mf_run_ramp(mf_problem* pb, int n_out, const double* t_out, double* h_m_out,
                      double* d_hz_out);

/* Readout of the current state: MF_READ_HZ (film: h_z = h_e + F^-1[(|k|/2) F g], end of
   Section 2.1; nx*ny values), MF_READ_MOMENT (film: m_z = integral of g; bulk:
   m = 1/2 integral of r x j over the conductor; 1 or 3 values), MF_READ_J (bulk:
   j = curl h, 3 fields), MF_READ_E (the electric field e = rho(|j|) j of Eq. 3 (film, j from
   Eq. 2; 2 fields e_x, e_y) or Eq. 13 (bulk; 3 fields), Ohm law rho_out j outside the
   superconductor, with the Gaussian-smoothed derivatives of Section 2.2 / Section 3.1; the
   transform precision's power law).  d_out is device memory (float64, fields back to back),
   except for MF_READ_MOMENT where it is host memory. */
mf_status mf_readout(mf_problem* pb, int what, double* out);

/* Same readouts of an arbitrary device state vector d_y at time t. */
mf_status mf_readout_of(mf_problem* pb, int what, double t, const double* d_y, double* out);

/* Counters, state and launch configuration. */
mf_status mf_get_info(mf_problem* pb, mf_info* out);

/* Transpose of a film's outside iteration (Eqs. 10-12), the linear core of the right-hand
   side's vector-Jacobian product: with a cold start (free-space h_dot = h_e_dot) and exactly
   `iters` iterations the iteration maps (h_dot_in, h_e_dot) linearly to g_dot; given the
   cotangent d_v of g_dot (device FP64, nx*ny), this writes the cotangent of h_dot_in to
   d_hin_bar (device FP64, nx*ny, zero on free space) and that of h_e_dot to *sbar (host, may be
   NULL).  One persistent launch on the problem's stream; waits for it.  Uses the warm start's
   buffers and clears the warm start.  MF_ERR_ARG for a bulk problem or a film without free
   space.  The adjoint has no counterpart in the paper. */
mf_status mf_film_outside_vjp(mf_problem* pb, int iters, const double* d_v, double* d_hin_bar,
                              double* sbar);

/* Vector-Jacobian product of a film's right-hand side f(g; jc, h_e_dot) (Eqs. 2-4 and 9-12)
   with a cold-started, fixed-count outside iteration (as mf_film_outside_vjp): given the state
   d_g and the cotangent d_v of f (device FP64, nx*ny each), writes the cotangents of g to
   d_gbar and of the per-cell critical current density to d_jcbar (device FP64, nx*ny; zero
   outside the superconductor), and that of h_e_dot to *sbar (host, may be NULL).  The power law
   is linearised as de/dj = rho (I + (n-1) j^ j^T) in the film (rho_out I elsewhere) and
   de/djc = -(n/jc) e.  One persistent launch on the problem's stream; waits for it; clears the
   warm start.  MF_ERR_ARG for a bulk problem or a film without free space.  The adjoint has no
   counterpart in the paper. */
mf_status mf_film_rhs_vjp(mf_problem* pb, int iters, const double* d_g, const double* d_v,
                          double* d_gbar, double* d_jcbar, double* sbar);

/* Vector-Jacobian product of one warm-started film right-hand side with a fixed outside
   iteration count, as the integrator runs it (Section 2.2: each call starts from the previous
   call's last free-space iterate).  Besides g, jc and h_e_dot the call has a fourth input, the
   warm start (free-space h_dot), and a second output, its last iterate.  Given the state d_g,
   the cotangent d_v of f and d_wbar_out of the last iterate (device FP64, nx*ny each; free-space
   values used; NULL = 0), writes the cotangents of g (d_gbar), of the jc map (d_jcbar, zero
   outside the superconductor), of the warm start (d_wbar_in, zero on the conductor; may be
   NULL) and of h_e_dot (*sbar, host, may be NULL).  The power law is linearised as in
   mf_film_rhs_vjp.  One persistent launch; waits; clears the warm start.  The adjoint has no
   counterpart in the paper. */
mf_status mf_film_rhs_vjp_warm(mf_problem* pb, int iters, const double* d_g, const double* d_v,
                               const double* d_wbar_out, double* d_gbar, double* d_jcbar,
                               double* d_wbar_in, double* sbar);

/* Replace the per-cell critical current density (device FP64, nx*ny[*nz]) of a problem that was
   created with a jc map (MF_ERR_ARG otherwise), or the knot values of a piecewise-linear h_e
   (host, n_values entries, which must equal the problem's he_knots, else MF_ERR_ARG; the knot
   times stay).  Both wait for the problem's stream; later calls use the new values.  They let a
   gradient's parameters change without a new problem. */
mf_status mf_set_jc_map(mf_problem* pb, const double* d_jc);
mf_status mf_set_knot_values(mf_problem* pb, const double* h_values, int n_values);

/* Loss and gradient of a film solve with frozen decisions.  The map is the one the integrator
   evaluates once its decisions are fixed: from the state d_g0 (device FP64, nx*ny), n_steps
   Bogacki-Shampine steps with the given times and sizes (host t_steps[i], h_steps[i]; every step
   inside one segment of the h_e knots, all accepted: y <- y + h (2/9 k1 + 1/3 k2 + 4/9 k3)), each
   right-hand side (k1, k2, k3 of step i are calls 3i, 3i+1, 3i+2) running exactly iters[call]
   outside iterations (host, 3 n_steps counts >= 1: e.g. those the Section 2.3 stop test chose
   in a forward run) from the previous call's last iterate; the first call starts from d_warm0
   (device FP64 free-space field) or, if NULL, cold from h_e_dot.  The loss is
   L = 1/2 dx dy sum (h_z(T) - target)^2 with h_z = h_e + F^-1[(|k|/2) F g] (end of Section 2.1),
   T = t_steps[n-1] + h_steps[n-1], d_target device FP64 (nx*ny).  Writes *loss (host) and, when
   d_jcbar is not NULL, dL/djc per cell to d_jcbar (device FP64, nx*ny; zero outside the
   superconductor), dL/dv_k for the n_knots knot values of h_e to knots_bar (host; n_knots must
   equal he_knots) and, when d_warm0_bar is not NULL, dL/d(first warm start) (device FP64).
   d_jcbar = knots_bar = d_warm0_bar = NULL computes the loss alone (forward only).  d_hz_T
   (device FP64, nx*ny, may be NULL) receives h_z(T) of the forward.  Memory: the
   forward keeps a checkpoint (state and warm start) every ckpt_every steps in d_work (device, at
   least mf_film_solve_gradient_work_bytes(pb, n_steps, ckpt_every) bytes); the reverse sweep
   recomputes each segment's stage inputs from its checkpoint and runs mf_film_rhs_vjp_warm three
   times per step, carrying the warm-start cotangent from call to call.  Runs on the problem's
   stream and waits; the solver's state is untouched, its warm start is cleared and its counters
   count these evaluations.  MF_ERR_ARG for a bulk problem, a film without free space, a
   sinusoidal h_e, a step across a knot, a count below 1 or a knot-count mismatch;
   MF_ERR_WORKSPACE for a short work buffer.  The adjoint has no counterpart in the paper. */
size_t mf_film_solve_gradient_work_bytes(const mf_problem* pb, int n_steps, int ckpt_every);
mf_status mf_film_solve_gradient(mf_problem* pb, int n_steps, const double* t_steps,
                                 const double* h_steps, const int* iters, int ckpt_every,
                                 const double* d_g0, const double* d_warm0, const double* d_target,
                                 void* d_work, size_t work_bytes, double* d_jcbar, double* knots_bar,
                                 int n_knots, double* d_warm0_bar, double* d_hz_T, double* loss);

/* Checkpoints: everything a continuation reads — the integrator state and counters, the six
   FP64 state/derivative buffers (with the first-same-as-last derivative), the outside
   iteration's warm start, the step log, and the work-item shape and launch width.  Restoring a
   checkpoint into a problem created with the same parameters makes its next calls identical,
   bit for bit, to the saved problem's.  The blob has mf_checkpoint_bytes bytes, in host or
   device memory owned by the caller; save and restore run on the problem's stream and wait for
   it.  Restore returns MF_ERR_ARG (and changes nothing) if the blob's grid, dimension or
   precision differ.  Checkpoints have no counterpart in the paper. */
size_t mf_checkpoint_bytes(const mf_problem* pb);
mf_status mf_checkpoint_save(mf_problem* pb, void* dst);
mf_status mf_checkpoint_restore(mf_problem* pb, const void* src);

/* Result of mf_autotune. */
typedef struct {
  int rows_per_item;          /* rows of the film row passes / bulk x pass per work item */
  int zs_per_item;            /* bulk y pass z-lines per item (films: two-field row pass rows) */
  int grid;                   /* CTAs of the persistent launch */
  int candidates;             /* configurations timed */
  double ms_per_rhs;          /* best time of one right-hand side with the forced iterations */
  double ms_per_rhs_default;  /* the same for the configuration chosen at mf_create */
} mf_tuning;

/* Time one right-hand side of the current state (force_iters outside iterations, reps timed
   launches after one warm-up) for every work-item shape and launch width the kernels accept
   for this grid, and keep the fastest; *out (may be NULL) receives it.  The candidates are the
   power-of-two rows (and z-lines) per item that fit the shared-memory batch, times the launch
   widths {size rule, all co-resident CTAs, half of them}.  Results change at rounding level
   with the item shape (the reductions are summed per item), not with the launch width.  The
   state, step size and counters are kept; the warm start of the outside iteration and the
   first-same-as-last derivative are cleared (as mf_reset_warm and mf_set_state do).  The
   tuning has no counterpart in the paper: it adapts the FFT passes' tiling to the grid. */
mf_status mf_autotune(mf_problem* pb, int reps, int force_iters, mf_tuning* out);

/* Copy up to cap logged step attempts (host memory); *count gets the number logged. */
mf_status mf_get_log(mf_problem* pb, mf_step_log* out, long long cap, long long* count);

const char* mf_last_error(const mf_problem* pb);
void mf_destroy(mf_problem* pb);

/* Film right-hand side that allocates nothing.  (The paper has no counterpart: this is a
   service for callers that cannot allocate device memory, such as an application that owns
   all device memory through its own pool and forbids cudaMalloc, or a latency-critical loop
   that must not take an allocation's implicit device synchronisation.)
   Evaluates f(t, y) like mf_rhs for a thin film (p->dim == 2) described by p, on `stream`,
   without a problem handle or a caller workspace: all intermediate buffers live in one static
   device array of 8 MiB that every GPU loading this library holds until the process exits.
   Limits: p->nx, p->ny <= 256, otherwise MF_ERR_WORKSPACE with a message in err.
   d_y, d_ydot: device float64, nx*ny values; force_iters as in mf_rhs_ex; *iters_out (may be
   NULL) gets the outside iterations; err (may be NULL) gets err_len bytes of message.
   The first call on a device looks up the array's device address with that device current.
   Every call copies its tables, mask, jc map and state into the array from the host and
   synchronises `stream` several times (and once more to read the status back), so no call can
   be captured into a CUDA graph.  Every call shares the array and leaves its contents behind;
   each call restarts the outside iteration cold (no warm start), and calls whose GPU work
   overlaps in time race on the array. */
mf_status mf_film_rhs_noalloc(const mf_params* p, double t, const double* d_y, double* d_ydot,
                              int force_iters, void* stream, int* iters_out, char* err,
                              size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
