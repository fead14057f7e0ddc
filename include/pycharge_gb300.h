/*
 * pycharge_gb300.h -- C ABI of a GB300 (sm_103a) implementation of the data-parallel hot path of
 * PyCharge (Filipovich & Hughes, arXiv 2107.12437): retarded Lienard-Wiechert fields of point
 * charges with stored trajectories, and the self-consistent Lorentz-oscillator (LO) loop.
 *
 * Conventions for every entry point
 *   - SI units, float64 inputs.
 *   - Array arguments named "device" are CUDA device pointers on the context's device; the caller
 *     owns them and keeps them alive until the call returns.  Small descriptors (the structs
 *     below) live in host memory and are read during the call only.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).  Every call
 *     ends by reading the device status word back, so when it returns the outputs are complete.
 *   - Errors are returned as pc_status; no call aborts, traps or falls back to the CPU.  On error
 *     the content of the outputs is unspecified.
 *   - A context must not be used by two host threads at once (it owns one workspace).
 */
#ifndef PYCHARGE_GB300_H
#define PYCHARGE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PC_OK = 0,
  PC_ERR_ARG = 1,       /* invalid argument (null pointer, non-positive size, bad enum, |axis| != 1) */
  PC_ERR_CUDA = 2,      /* a CUDA runtime call failed (allocation, launch) */
  PC_ERR_HISTORY = 3,   /* a retarded time falls outside a charge's stored samples (Eq. ret_t) */
  PC_ERR_VELOCITY = 4,  /* a dipole charge exceeded v_max (Sec. 3.2, default c/100) */
  PC_ERR_CAUSALITY = 5, /* dt exceeds a light-crossing time between dipoles (Sec. 3.2) */
  PC_ERR_NOCONV = 6,    /* the retarded-time solve or the energy fit did not converge */
  PC_ERR_TIMEOUT = 7    /* reserved: no kernel of this library waits on another (every ordering
                           between blocks goes through kernel or graph-node boundaries), so no
                           call returns it */
} pc_status;

/* field kind, Sec. 3.2 (calculate_E / calculate_B select total, Coulomb or radiation field) */
enum { PC_TOTAL = 0, PC_COULOMB = 1, PC_RADIATION = 2 };

/* arithmetic of the field sum */
enum {
  PC_F64 = 0,  /* every step in float64; float64 outputs */
  PC_MIXED = 1 /* float64 delays per tile, float32 per-pair algebra with dipole pairs in difference
                  form and compensated summation; float32 outputs */
};

typedef struct pc_ctx pc_ctx;

/*
 * Point charges with predefined trajectories (Sec. 3.1: Charge objects), sampled at t0 + k dt,
 * k = 0..S-1, linearly interpolated between samples (Sec. 3.1).
 */
typedef struct {
  int32_t M;             /* number of charges (0 = none) */
  int64_t S;             /* samples per charge, >= 2 */
  double t0, dt;         /* time of sample 0, sample spacing (s) */
  const double *q;       /* device [M] charge (C) */
  const double *pos;     /* device [M][S][3] position (m) */
  const double *vel;     /* device [M][S][3] velocity (m/s), |vel| < c */
  const double *acc;     /* device [M][S][3] acceleration (m/s^2) */
  int32_t static_before; /* 1: before t0 a charge rests at its sample-0 position; 0: PC_ERR_HISTORY */
} pc_charges;

/*
 * Dipoles as field sources (Sec. 3.1: Dipole objects): two charges +q (mass m1) and -q (mass m2)
 * about the centre of mass `origin`, with moment d(t) along the fixed unit `axis`:
 *   r_1 = R + m2/(m1+m2) (d/q) axis,  r_2 = R - m1/(m1+m2) (d/q) axis   (Eqs. r_1, r_2).
 * d, d', d'' are sampled at t0 + n dt and linearly interpolated; before t0 the dipole is at rest
 * with moment d[0] (Sec. 3.2).  This is also the layout pc_dipoles_run writes, so a run's output
 * can be passed here directly (per configuration).
 */
typedef struct {
  int32_t N;                /* number of dipoles (0 = none) */
  int64_t S;                /* samples per dipole, 2 <= S <= 2^30 */
  double t0, dt;
  const double *origin;     /* device [N][3] (m) */
  const double *axis;       /* device [N][3] unit vectors */
  const double *q;          /* device [N] charge magnitude (C), > 0 */
  const double *m1, *m2;    /* device [N] masses of the positive and negative charge (kg) */
  const double *d;          /* device [N][S] moment along axis (C m) */
  const double *d_dot;      /* device [N][S] (C m / s) */
  const double *d_ddot;     /* device [N][S] (C m / s^2) */
} pc_dipole_sources;

/* Outputs of pc_fields; any pointer may be NULL to skip that output.
 * PC_F64 writes double, PC_MIXED writes float.  Layout [T][P][...] with the point index fastest. */
typedef struct {
  void *E;       /* device [T][P][3] electric field (V/m) */
  void *B;       /* device [T][P][3] magnetic field (T) */
  void *phi;     /* device [T][P] scalar potential (V) */
  void *A;       /* device [T][P][3] vector potential (V s/m) */
  uint8_t *mask; /* device [T][P]: 1 where some charge was within r_excl of the point at its
                    retarded time; that charge then contributes nothing */
} pc_field_out;

/* Plane grid: point (iu, iv) = origin + iu*eu + iv*ev, output index iu*nv + iv (meshgrid 'ij'). */
typedef struct {
  double origin[3], eu[3], ev[3];
  int64_t nu, nv;
} pc_plane;

/* Context: owns the workspace (device status word, float32 history mirrors, run scratch). */
pc_status pc_ctx_create(pc_ctx **out, int device);
pc_status pc_ctx_destroy(pc_ctx *ctx);
const char *pc_status_string(pc_status s);

/*
 * pc_fields -- E, B, phi, A of all sources at P points and T times (Sec. 2.2).
 *
 * For every (point r, time t, charge) the retarded time t' = t - |r - r_s(t')|/c (Eq. ret_t) is
 * solved against the charge's piecewise-linear history, the Lienard-Wiechert potentials and fields
 * (Eqs. V, A, E, B; `kind` selects Eq. E, ECoulomb or Eradiation for E and B) are evaluated there,
 * and the contributions of all charges are summed (Sec. 2.2).  Vector potential: A = (v/c^2) phi.
 *   ch, dp      sources (either may be NULL or empty, not both)
 *   points      device [P][3] (m); P >= 0
 *   times       host [T] evaluation times (s); T >= 1
 *   r_excl      a charge closer than r_excl (m) at its retarded position is skipped and masked;
 *               r_excl = 0 masks exact coincidence only
 * Errors: PC_ERR_ARG, PC_ERR_HISTORY (retarded time outside the samples), PC_ERR_NOCONV,
 * PC_ERR_CUDA.
 */
pc_status pc_fields(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const double *points,
                    int64_t P, const double *times, int32_t T, int32_t kind, int32_t precision, double r_excl,
                    const pc_field_out *out, void *stream);

/* Point charges on analytic trajectories (Sec. 2.2, Sec. 3.1: the paper's predefined charges).
 * par holds 12 doubles per charge; unused entries are ignored:
 *   PC_TRAJ_STATIONARY   r0[3]                                     r(t) = r0
 *   PC_TRAJ_OSCILLATING  r0[3], u[3] (unit), A, w, phi            r(t) = r0 + A cos(w t + phi) u
 *   PC_TRAJ_CIRCULAR     c[3], e1[3], e2[3] (orthonormal), a, w, phi
 *                                                                  r(t) = c + a (cos(w t + phi) e1 + sin(w t + phi) e2)
 *   PC_TRAJ_ACCELERATING r0[3], v0[3], acc[3], ta                 r(t) = r0 + v0 s + acc s^2 / 2, s = t - ta >= 0;
 *                                                                  r0 + v0 s for s < 0 (uniform motion)
 * Velocities and accelerations are the exact derivatives.  All arrays on the device. */
enum { PC_TRAJ_STATIONARY = 0, PC_TRAJ_OSCILLATING = 1, PC_TRAJ_CIRCULAR = 2, PC_TRAJ_ACCELERATING = 3 };
typedef struct {
  int32_t M;
  const int32_t *kind; /* [M] */
  const double *q;     /* [M] (C) */
  const double *par;   /* [M][12] */
} pc_param_charges;

/*
 * pc_fields_param -- E, B, phi, A of point charges on analytic trajectories at P points and T times
 * (float64 outputs).  The retarded time (Eq. ret_t) is solved on the exact trajectory (bracketed
 * Newton iteration to rounding), the fields follow Eqs. V, A, E, B with the exact velocity and
 * acceleration, so no history interpolation enters; `kind` selects Eq. E, ECoulomb or Eradiation.
 * The charges must stay slower than light.
 *   points  device [P][3];  times host [T];  r_excl, out as for pc_fields (PC_F64 layout)
 * Errors: PC_ERR_ARG (also for a kind outside PC_TRAJ_*, found on the device), PC_ERR_NOCONV (no
 * bracket or no convergence), PC_ERR_CUDA.
 */
pc_status pc_fields_param(pc_ctx *ctx, const pc_param_charges *ch, const double *points, int64_t P,
                          const double *times, int32_t T, int32_t kind, double r_excl, const pc_field_out *out,
                          void *stream);

/* Tile shape of the PC_MIXED plane evaluation: tile_rows x tile_cols points (256 with one point
 * per thread, or 512 with two per thread: each thread's points in rows r and r + tile_rows/2,
 * evaluated together in the lanes of packed float32 registers; used for grids of dipoles alone,
 * other calls take the one-point tile of the same columns), tile_cols a power of two up to 256;
 * sources_per_stage = 32 or 64 sources staged in shared memory at a time. */
typedef struct {
  int32_t tile_rows, tile_cols, sources_per_stage;
} pc_plane_tiling;

/*
 * pc_autotune_plane -- picks the tile shape of the PC_MIXED plane evaluation for this workload and
 * keeps it in the context for later pc_fields_plane / pc_fields_plane_to_host calls: one-point tiles
 * of 8 x 32, 16 x 16 (the default) or 32 x 8 rows x columns, two-point tiles of 16 x 32, 32 x 16 or
 * 64 x 8 (grids of dipoles alone), each with 64 (the default) and with 32 sources per stage.  Each
 * shape runs once to warm up and once timed on the given arguments (those of pc_fields_plane with
 * PC_MIXED; `out` receives the fields of the last run).  Writes the chosen shape to *chosen (or
 * NULL).  The results of every shape agree to float32 rounding (the tile anchor enters the delays).
 * Errors: those of pc_fields_plane.
 */
pc_status pc_autotune_plane(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const pc_plane *grid,
                            const double *times, int32_t T, int32_t kind, double r_excl, const pc_field_out *out,
                            pc_plane_tiling *chosen, void *stream);

/*
 * pc_set_plane_tiling -- sets the PC_MIXED plane tile shape directly (what pc_autotune_plane
 * chooses).
 * Errors: PC_ERR_ARG for a shape outside those described at pc_plane_tiling.
 */
pc_status pc_set_plane_tiling(pc_ctx *ctx, const pc_plane_tiling *tiling);

/*
 * pc_fields_to_host / pc_fields_plane_to_host -- pc_fields / pc_fields_plane with the outputs
 * delivered to HOST memory: out_host holds host pointers ([T][P][...] as in pc_field_out), each
 * covering its whole array.  When every requested output is page-locked (cudaHostAlloc,
 * cudaHostRegister) and mapped for the device (always so under unified addressing), the kernels
 * store the fields into them directly, so the transfer runs inside the computation.  Otherwise
 * the frames are computed in chunks of about 256 MB of outputs into two alternating device buffers
 * owned by the context, and each chunk is copied to the host on a second stream while the next
 * chunk computes; with pageable buffers those copies are serialized.  The results are identical
 * in both modes.  The call returns when every output has landed.  Sources and points stay on the
 * device.  Errors: those of pc_fields.
 */
pc_status pc_fields_to_host(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const double *points,
                            int64_t P, const double *times, int32_t T, int32_t kind, int32_t precision,
                            double r_excl, const pc_field_out *out_host, void *stream);
pc_status pc_fields_plane_to_host(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp,
                                  const pc_plane *grid, const double *times, int32_t T, int32_t kind,
                                  int32_t precision, double r_excl, const pc_field_out *out_host, void *stream);

/* pc_fields on a plane grid (P = nu*nv points generated on the device); same semantics. */
pc_status pc_fields_plane(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const pc_plane *grid,
                          const double *times, int32_t T, int32_t kind, int32_t precision, double r_excl,
                          const pc_field_out *out, void *stream);

/*
 * Lorentz-oscillator configurations for pc_dipoles_run: B independent configurations of N dipoles
 * each (Sec. 2.3, Sec. 4.2).  Dipole (b, i): centre `origin`, unit `axis`, charges +-q with masses
 * m1 (positive) and m2 (negative), natural angular frequency omega0, initial moment d0 along the
 * axis (d = q r_dip).  All device arrays, [B][N] or [B][N][3].
 */
typedef struct {
  int32_t B, N;
  const double *origin, *axis;
  const double *q, *m1, *m2, *omega0, *d0;
} pc_dipoles;

typedef struct {
  double v_max;        /* maximum charge speed (m/s); <= 0 selects c/100 (Sec. 3.2) */
  int32_t ed_mode;     /* 0: E_d at every RK4 stage time (default); 1: E_d held at t over the step */
  int32_t fit;         /* 1: fit Eq. KE per dipole after the run (outputs gamma, omega) */
  int64_t first_index; /* first step used by the fit (Sec. 3.4: after 10 000 steps) */
  int32_t precision;   /* PC_F64 or PC_MIXED for the driving-field sum */
  double near_f64;     /* PC_MIXED: source dipoles whose centre lies closer than this distance (m)
                        * to the receiver's are summed in float64 (0: none).  The decay rate of
                        * near-field-coupled dipoles sits in a part of their field ~(k R)^3 below
                        * the near field, which float32 rounding swamps: with PC_MIXED alone the
                        * fitted gamma of a pair is off by ~0.3 gamma0 at 1 nm and 1e-3 gamma0 at
                        * 6 nm (omega0 = 2 pi 200 THz); 10e-9 keeps it below 1e-4 gamma0 */
  const double *state_in; /* device, or NULL: resume from this state (written by an earlier call's
                           * state_out for the same dipoles and dt); the call then advances from the
                           * state's step s to s + n_steps, its outputs' sample 0 being step s */
  double *state_out;      /* device, or NULL: receives the state at the call's last step;
                           * pc_dipoles_state_size gives its length */
  int64_t checkpoint_every; /* adjoints (pc_dipoles_adjoint, pc_dipoles_rates_adjoint): 0 keeps the
                           * whole forward history; K > 0 keeps the run's state every K steps and
                           * recomputes each segment of K steps during the reverse sweep */
} pc_run_opts;

/* Outputs of pc_dipoles_run; layout [B][N][n_steps+1] (time fastest); every pointer may be NULL
 * (not wanted).  When d, d_dot and d_ddot are all given (and the run does not resume a state) they
 * are also the history store the run reads back at retarded times; otherwise the run keeps its
 * history in a ring of the context holding only the samples a causal block can still reach
 * (2^k >= D + 18 slots per dipole, D the largest delay between two dipoles in samples plus a margin),
 * so that its memory does not grow with n_steps. */
typedef struct {
  double *d, *d_dot, *d_ddot; /* device */
  double *energy;             /* device [B][N][n_steps+1] Eq. dipoleE, or NULL */
  double *Ed;                 /* device [B][N][n_steps+1] driving field at t_n (V/m), or NULL */
  double *gamma;              /* device [B][N] fitted energy decay rate (1/s), or NULL */
  double *omega;              /* device [B][N] fitted angular frequency (rad/s); delta = omega - omega0 */
} pc_run_out;

/*
 * pc_dipoles_run -- Algorithm 1 for B configurations at once.
 *
 * Each dipole obeys d'' + gamma0 d' + omega0^2 d = (q^2/m) E_d(R, t) (Eq. LO_equation) with
 * m = m1 m2/(m1+m2) (Eq. eff_mass), gamma0 = q^2 omega0^2/(6 pi eps0 c^3 m) and E_d the component
 * along its axis of the retarded field of every other dipole of its configuration at its origin
 * (Sec. 2.3).  RK4 from t = 0 to n_steps*dt; the dipoles rest at d0 for t <= 0 (Sec. 3.2); after
 * each step d'' is set from the equation of motion at the step end.  Optionally the kinetic energy
 * m d'^2/(2 q^2) from first_index on is fitted to Eq. KE (Levenberg-Marquardt), giving gamma and
 * omega per dipole.
 * Configurations of more than 64 dipoles run as grid-wide launches per causal block, the block
 * loop one CUDA graph with a device-side while node; where that node is unavailable, or when the
 * environment variable PYCHARGE_GB300_HOST_LOOP is "1" (for profilers that do not descend into
 * conditional graph nodes), the same launches are issued from the host, with identical results.
 * Errors: PC_ERR_ARG (also B > 65535 with N > 64), PC_ERR_CAUSALITY (two dipoles closer than
 * c dt), PC_ERR_VELOCITY, PC_ERR_NOCONV, PC_ERR_CUDA.
 */
pc_status pc_dipoles_run(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps, const pc_run_opts *opts,
                         const pc_run_out *out, void *stream);

/*
 * pc_autotune_run -- picks the launch shape of the oscillator run for this workload and keeps it in
 * the context for later pc_dipoles_run / adjoint calls: configurations of more than 64 dipoles run as
 * grid-wide launches in which each receiver's sources are split into slices summed in a fixed order;
 * each candidate slice count (powers of two up to min(64, N / 8) and the occupancy heuristic's choice)
 * runs the caller's configuration (dp, dt, opts; no fit, no state) for probe_steps steps once to warm
 * up and once timed, and the fastest is kept.  Writes the chosen count to *chosen (or NULL); smaller
 * configurations run as one CTA each and have nothing to tune (*chosen = 1).  Results of different
 * slice counts agree to the rounding of the driving-field sum (its terms are added in another order).
 * Errors: those of pc_dipoles_run; PC_ERR_ARG for probe_steps < 1 or opts with a fit or a state.
 */
pc_status pc_autotune_run(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t probe_steps, const pc_run_opts *opts,
                          int32_t *chosen, void *stream);

/* pc_set_run_tiling -- sets the source slices per receiver of the grid path directly (0: the
 * occupancy heuristic, 1..64: that many, capped at N / 8).  Errors: PC_ERR_ARG outside 0..64. */
pc_status pc_set_run_tiling(pc_ctx *ctx, int32_t source_slices);

/*
 * Launch timing of the oscillator run (device time of its kernels, measured with CUDA events on the
 * run's stream).  pc_set_run_timing(ctx, 1) clears the counters and makes later pc_dipoles_run /
 * pc_dipoles_run_moving calls of this context record them: the grid path (more than 64 dipoles per
 * configuration) then launches its causal-block loop from the host instead of as one CUDA graph
 * (same kernels, same order, bitwise the same results) with an event pair around every drive
 * (phase A: the driving fields of a block) and RK4 (phase B) launch, and the persistent path (64 or
 * fewer) one around its single launch.  The calls synchronise their stream every 64 blocks to read
 * the events back, so timed runs are for measurement, not production.  pc_set_run_timing(ctx, 0)
 * turns it off; pc_get_run_timing copies the counters accumulated since the last enable.  The drive
 * launches counted are those of whole and partial causal blocks (not the E_d(0) evaluation of a
 * fresh run).  Errors: PC_ERR_ARG (null context or output, enable not 0 or 1), PC_ERR_CUDA.
 */
typedef struct {
  int64_t drive_launches; /* grid path: phase-A launches timed */
  double drive_ms;        /* their summed device time (ms) */
  int64_t rk4_launches;   /* grid path: phase-B launches timed */
  double rk4_ms;
  int64_t run_launches;   /* persistent path: time-loop launches timed (one per call) */
  double run_ms;
} pc_run_timing;

pc_status pc_set_run_timing(pc_ctx *ctx, int32_t enable);
pc_status pc_get_run_timing(pc_ctx *ctx, pc_run_timing *out);

/*
 * pc_dipoles_state_size -- the length (float64 values) of a run state of these dipoles at this dt
 * (pc_run_opts.state_in / state_out): a header (step, depth D, B N), E_d of every dipole at the state's
 * step and d, d', d'' of its last D + 1 samples, D the deepest sample a causal block can reach behind
 * its start (Algorithm 1 needs the retarded history, not only the present state, to continue).
 * A state resumes the run exactly: the continued run equals the uninterrupted one bit for bit when
 * the state's step is a multiple of the causal block length, and to rounding otherwise.
 * Errors: PC_ERR_ARG, PC_ERR_CUDA.
 */
pc_status pc_dipoles_state_size(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t *n_doubles, void *stream);

/* Moving dipoles (Sec. 4.3): the origin of every dipole as a function of time, sampled at the half
 * steps t = h dt / 2, h = 0 .. 2 n_steps, device [B][N][2 n_steps + 1][3] each (m, m/s, m/s^2). */
typedef struct {
  const double *pos, *vel, *acc;
} pc_dipole_motion;

/*
 * pc_dipoles_run_moving -- pc_dipoles_run with moving origins (Sec. 4.3), PC_F64 or PC_MIXED.
 * The driving field of each RK4 stage is evaluated at the receiver's origin at that stage's time
 * (half-step samples 2n, 2n+1, 2n+2); each source charge sits at its origin plus its offset along
 * the axis, with the origin's whole-step samples (even h) joining the moment in the linearly
 * interpolated history (Sec. 3.1) and adding its velocity and acceleration to the charge's; for
 * t <= 0 the origins rest at their first sample.  dp->origin holds the origins at t = 0 (the
 * first samples of pos); the causal block length accounts for the closest approach of the origins
 * over the run and their largest speed.
 * opts->precision PC_MIXED: each source's two charges in float32 in difference form, as in
 * pc_dipoles_run, with the origin's motion added: within the history segment of the origin's own
 * retarded time the origin moves linearly, each charge's retarded time is solved relative to the
 * origin's, and the two charges' fields are differenced term by term (the origin's velocity and
 * acceleration join the charges').  Sources whose retarded times fall before sample 1 or leave that
 * segment by more than 0.1 sample (and, with opts->near_f64 > 0, sources closer than near_f64) take
 * the float64 pair.  The context keeps a float32 copy of the origin samples for the run (48 bytes
 * per dipole and half step).  The moment, the RK4 state and the stored histories stay float64.
 * Errors: those of pc_dipoles_run.
 */
pc_status pc_dipoles_run_moving(pc_ctx *ctx, const pc_dipoles *dp, const pc_dipole_motion *motion, double dt,
                                int64_t n_steps, const pc_run_opts *opts, const pc_run_out *out, void *stream);

/*
 * pc_ke_fit -- Levenberg-Marquardt fit of Eq. KE (Sec. 2.4) to K series of kinetic energies.
 *   ke        device [K][S] samples at spacing dt; samples first_index..S-1 are fitted
 *   gamma     device [K] out: energy decay rate (1/s)
 *   omega     device [K] out: angular frequency (rad/s)
 *   amp, phase device [K] out or NULL: A and phi of Eq. KE with time counted from sample first_index
 * Errors: PC_ERR_ARG, PC_ERR_NOCONV (fewer than two kinetic-energy minima in the window).
 */
pc_status pc_ke_fit(pc_ctx *ctx, const double *ke, int32_t K, int64_t S, double dt, int64_t first_index,
                    double *gamma, double *omega, double *amp, double *phase, void *stream);

/*
 * pc_fields_noalloc -- pc_fields on a point list in PC_MIXED precision (float32 outputs) that
 * allocates nothing.  The paper has no counterpart; this entry point exists for callers that may
 * not allocate device memory: code inside a framework that owns the whole device pool through its
 * own allocator, and latency-critical loops where cudaMalloc/cudaFree (which can synchronise the
 * device) or an allocation failure in mid-run are not acceptable.  It needs no pc_ctx.
 *
 * Scratch: the float32 history mirrors, the point-charge reference positions and the status word
 * live in one static device array of 16 MiB (plus a 256-byte header) that the library reserves on
 * every GPU that loads it and keeps until the process exits.  The sources must fit it:
 *   16 * N * S_dipoles + 64 * N + 48 * M * S_charges + 24 * M  <=  16 MiB  (bytes),
 * otherwise the call returns PC_ERR_ARG without touching the device.
 * Set-up: the first call on a device resolves the array's device address (cudaGetSymbolAddress)
 * with that device current.  A failed lookup
 * returns PC_ERR_CUDA and is retried by the next call.  The device used is the caller's current
 * device; `points` must be device memory of that device (PC_ERR_ARG otherwise).
 * Every call shares the one array and leaves its contents behind: each call clears the status word
 * and rewrites the mirrors it reads, so calls in sequence are independent, but calls that overlap
 * on the GPU (other streams, other host threads) race on the array and must not be issued.
 * Arguments, outputs and errors are those of pc_fields with precision = PC_MIXED.
 */
pc_status pc_fields_noalloc(const pc_charges *ch, const pc_dipole_sources *dp, const double *points, int64_t P,
                            const double *times, int32_t T, int32_t kind, double r_excl, const pc_field_out *out,
                            void *stream);

/* Gradient outputs of pc_dipoles_adjoint (device arrays, overwritten). */
typedef struct {
  double *origin; /* [B][N][3] dL/d origin (1/m units of L) */
  double *omega0; /* [B][N]    dL/d omega0 */
  double *d0;     /* [B][N]    dL/d d0 (initial dipole moment, C m) */
} pc_dipole_grads;

/*
 * pc_dipoles_adjoint -- reverse-mode gradient of L = sum_{b,i} w_{b,i} E_{b,i}(T) through the whole
 * run of pc_dipoles_run, E the dipole energy of Eq. dipoleE at the last step T = n_steps dt and
 * w = dL_dEnergyFinal (device [B][N]).  The paper has no adjoint; it differentiates the same
 * discrete computation as pc_dipoles_run with precision PC_F64 and ed_mode 0: RK4 of
 * Eq. LO_equation, the Lienard-Wiechert driving field (Eqs. E, r_1, r_2) at the retarded time of
 * Eq. ret_t on the piecewise-linear history.  The retarded time is differentiated through its
 * defining equation (implicit-function theorem), the history interpolation exactly; a kink of the
 * loss where a retarded time crosses a sample is not smoothed.
 * The call first repeats the forward run, keeping the whole history and the half-step fields in
 * the context (8 doubles per dipole and step), then sweeps the causal blocks in reverse.  With
 * opts->precision PC_MIXED the forward run takes the mixed driving field (as pc_dipoles_run with
 * PC_MIXED, about 30 times faster on large configurations) and the float64 reverse differentiates
 * along that trajectory; its moment histories agree with the float64 run's to about 1e-8, and so
 * do the gradients.
 *   dp, dt, n_steps, opts   as for pc_dipoles_run; opts->precision PC_F64 or PC_MIXED (the
 *                           forward), opts->ed_mode 0 (PC_ERR_ARG otherwise); the fit is not run
 *   g                       gradients (device)
 * Errors: those of pc_dipoles_run; PC_ERR_ARG also when the source windows of one causal block
 * exceed shared memory (more than about 8 500 steps between the nearest and the farthest
 * dipole of a configuration); PC_ERR_NOCONV when a retarded time leaves its window.
 */
pc_status pc_dipoles_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps, const pc_run_opts *opts,
                             const double *dL_dEnergyFinal, const pc_dipole_grads *g, void *stream);

/* Gradients of the origin samples of a moving run, device [B][N][2 n_steps + 1][3] each (any may
 * be NULL: not wanted), laid out as pc_dipole_motion. */
typedef struct {
  double *pos, *vel, *acc;
} pc_dipole_motion_grads;

/*
 * pc_dipoles_adjoint_moving -- pc_dipoles_adjoint for the run of pc_dipoles_run_moving (Sec. 4.3,
 * origins on given trajectories): gradients of L = sum w E(T) with respect to every origin sample
 * (position, velocity, acceleration at the half steps), omega0 and d0.  The paper has no adjoint.
 * A receiver's origin enters at its stage time (its half-step sample), a source's origin through
 * the linear interpolation of its whole-step samples at the charge's retarded time, whose
 * dependence on the origin samples is taken through its defining equation (Eq. ret_t, implicit-
 * function theorem) as in pc_dipoles_adjoint.  g->origin receives zeros: the static origins do not
 * enter a moving run.
 *   dp, motion, dt, n_steps, opts   as for pc_dipoles_run_moving (ed_mode 0; opts->precision PC_F64
 *                                    or PC_MIXED selects the forward's driving field, the reverse is
 *                                    float64 as in pc_dipoles_adjoint)
 *   dL_dEnergyFinal                  device [B][N]
 *   g, gm                            gradients (device); the call clears gm's arrays first
 * Errors: those of pc_dipoles_adjoint and of pc_dipoles_run_moving.
 */
pc_status pc_dipoles_adjoint_moving(pc_ctx *ctx, const pc_dipoles *dp, const pc_dipole_motion *motion, double dt,
                                    int64_t n_steps, const pc_run_opts *opts, const double *dL_dEnergyFinal,
                                    const pc_dipole_grads *g, const pc_dipole_motion_grads *gm, void *stream);

/*
 * pc_dipoles_rates_adjoint -- reverse-mode gradient of L = sum_{b,i} (dL_dgamma gamma + dL_domega omega)
 * where gamma and omega are the Eq. KE fit (Sec. 2.4) of each dipole's kinetic energy
 * m d'^2/(2 q^2) from first_index on, after the float64 run of pc_dipoles_run (ed_mode 0).  The
 * paper has no adjoint.  The fit is differentiated through its optimum by the implicit-function
 * theorem (full Hessian of the least-squares cost, residual term included), which turns
 * (dL/dgamma, dL/domega) into a cotangent on every d' sample of the fit window; the run is then
 * reversed as in pc_dipoles_adjoint.  delta omega = omega - omega0 has dL/domega0 one less than
 * the omega0 gradient returned here.
 *   dp, dt, n_steps, opts  as for pc_dipoles_run; opts->precision PC_F64, opts->ed_mode 0,
 *                          opts->first_index the first fitted step
 *   dL_dgamma, dL_domega   device [B][N] cotangents (either may be NULL, not both)
 *   gamma, omega           device [B][N] out: the fitted values (or NULL)
 *   g                      gradients (device)
 * Errors: those of pc_dipoles_adjoint; PC_ERR_NOCONV when a fit fails (fewer than two
 * kinetic-energy minima in the window) or its Hessian is singular.
 */
pc_status pc_dipoles_rates_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                   const pc_run_opts *opts, const double *dL_dgamma, const double *dL_domega,
                                   double *gamma, double *omega, const pc_dipole_grads *g, void *stream);

/*
 * pc_dipoles_fields_adjoint -- reverse-mode gradient of a loss on the fields of the oscillators
 * themselves: L = sum over configurations, frames and points of <cE, E> + <cB, B> + cphi phi +
 * <cA, A>, where E, B, phi, A are the fields of configuration b's dipoles (Sec. 2.2, Eqs. E, B,
 * V, A, both charges of every dipole) at the points and times, on the history of the float64 run
 * of pc_dipoles_run from t = 0 (the moments rest at d0 before).  The paper has no adjoint.  Each
 * field term is reversed through the Lienard-Wiechert expressions, the interpolation and the
 * retarded time (implicit-function theorem); the resulting adjoints of the dipoles' history
 * samples and origins seed the reverse sweep of pc_dipoles_adjoint, which carries them to the
 * origins, omega0 and d0.
 *   dp, dt, n_steps, opts   as for pc_dipoles_adjoint (PC_F64 or PC_MIXED forward, ed_mode 0)
 *   points                  device [P][3]; times host [T], 0 <= t (retarded times must fall
 *                           inside the run's samples)
 *   cot                     device float64 cotangents [B][T][P][3] (E, B, A) and [B][T][P] (phi),
 *                           any may be NULL; cot->mask must be NULL
 *   g                       gradients (device)
 * Errors: those of pc_dipoles_adjoint; PC_ERR_HISTORY for times past the run; PC_ERR_NOCONV when
 * the points' delays from a source span more than 8 500 samples.
 */
pc_status pc_dipoles_fields_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                    const pc_run_opts *opts, const double *points, int64_t P, const double *times,
                                    int32_t T, const pc_field_out *cot, const pc_dipole_grads *g, void *stream);

/*
 * pc_alu_peaks -- measures this GPU's float32 and float64 fused-multiply-add throughput (FMA/s)
 * with dependent-chain kernels; used as roofline denominators.  Writes fp32_fma_per_s,
 * fp64_fma_per_s (host pointers).
 */
pc_status pc_alu_peaks(pc_ctx *ctx, double *fp32_fma_per_s, double *fp64_fma_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif
