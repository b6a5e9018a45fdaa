/*
 * fsd.h — C ABI of the GB300 (sm_103a) library for the per-time-step
 * saddle-point solve of fast Stokesian dynamics for rigid multi-bead
 * aggregates (arxiv 2607.25161).
 *
 * The operation (Sec. 2.3.3, Eq. spm_agg; Algorithm 1 steps 1, 4, 5):
 *
 *   [ M_inf        B Sigma^T ] [ F      ]   [ (E.(x - X) ; 0) ; E_inf        ]
 *   [ Sigma B^T   -RR_FU^nf  ] [ U-U_inf] = [ -(FF^P + RR_FE^nf : E_inf)     ]
 *
 * M_inf is the periodic FTS-level RPY mobility applied matrix-free by the
 * positively split Ewald method (real-space pair sum + Gaussian spreading,
 * FFT, Green's function, interpolation; Sec. 2.2), RR^nf = Sigma R^nf Sigma^T
 * the near-field lubrication resistance of bead pairs on different bodies
 * (Sec. 2.3.2), Sigma the rigid-body constraint (Eq. gc, Eq. sigma).  GMRES
 * with the block-triangular preconditioner of Table 1 (M_inf ~ I/zeta,
 * block-diagonal Schur complement, one 6x6 LU per aggregate) solves it.
 *
 * Units: any consistent set; the defaults are a = 1, eta = 1.
 * Imposed flow: simple shear, flow along x, gradient along y (Sec. 3.1.1):
 *   u_inf = gamma y e_x,  E_inf = gamma/2 (e_x e_y + e_y e_x),
 *   Omega_inf = -gamma/2 e_z, origin of y at 0.
 *
 * Pointers: every array argument may be HOST or DEVICE memory (detected with
 * cudaPointerGetAttributes).  Device arrays are read / written on the
 * context's stream (ready when that stream is); host arrays are copied
 * synchronously.  The caller owns every array it passes; the library never
 * keeps a caller pointer after a call returns.  The context owns all device
 * workspace.
 *
 * Orderings: beads are identified by their index in the bead_pos array given
 * to fsd_setup, aggregates by their id (dense 0..N-1).  Every input and output
 * uses those orderings; internally beads are regrouped per aggregate and
 * aggregates sorted spatially.
 *
 * Errors: every call returns an fsd_status; no exception or abort crosses
 * the ABI; fsd_last_error() gives a message.  FSD_ENOCONV still writes the
 * best iterate and the stats.  FSD_EOVERLAP is a warning (beads of different
 * aggregates closer than 2a (1 - 1e-6)); all outputs are still written.
 */
#ifndef FSD_H
#define FSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsd_ctx fsd_ctx;

typedef enum {
  FSD_OK = 0,
  FSD_EINVAL = 1,   /* invalid argument; nothing was changed            */
  FSD_ENOMEM = 2,   /* device or host allocation failed                 */
  FSD_ECUDA = 3,    /* a CUDA runtime call failed                       */
  FSD_ENOCONV = 4,  /* Krylov solve did not reach tol within max_iter   */
  FSD_ENUMERIC = 5, /* NaN / Inf, or a singular per-aggregate 6x6 block */
  FSD_EOVERLAP = 6, /* warning: overlapping beads of different bodies   */
  FSD_ETIMEOUT = 7  /* a bounded device wait gave up                    */
} fsd_status;

/* Near-field Brownian samplers (fsd_params.nf_sampler). */
enum { FSD_NF_LANCZOS = 0, FSD_NF_PAIRWISE = 1 };

/* Precision of the operator applications inside the solve. */
enum { FSD_FP64 = 0, FSD_MIXED = 1 };

/* Flags. */
enum {
  FSD_FLAG_WARM_START = 1, /* start each solve from the previous solution */
  FSD_FLAG_COMOVING = 2,   /* fsd_step advances the bodies by the disturbance
                              motion only: X += (U - U_inf(X)) dt and q by
                              Omega - Omega_inf.  A cubic periodic box has no
                              sheared (Lees-Edwards) images, so the imposed
                              affine motion would drive bodies across the y
                              boundary into each other; each solve is still
                              the full sheared problem */
  FSD_FLAG_GRAPH = 4,      /* run each solve (and fsd_step's update) as one
                              captured CUDA graph: the GMRES restart cycles,
                              Arnoldi steps and refinement sweeps are
                              conditional graph nodes and the Givens
                              least-squares update runs on the device, so a
                              solve makes no host round trip.  The geometry
                              (neighbour lists, lubrication blocks, LUs) is
                              still prepared before the launch.  Same
                              arithmetic as the host-driven loop.  Ignored
                              while the profiler is on */
  FSD_FLAG_AUTOTUNE = 8,   /* at set-up, when xi, rc and grid are all left
                              to the rules: time each candidate splitting xi
                              in {0.30 .. 0.70}/a, and (small boxes) 1.02,
                              1.25 and 1.6 times the smallest xi whose R_c
                              stays below L/2 (R_c and the grid from the
                              accuracy rules of Sec. 3.2, P from xerr) and
                              each real-space tile on the device, with the
                              operator the Krylov iterations apply, and keep
                              the fastest.  Costs about eight set-ups */
  FSD_FLAG_LEES_EDWARDS = 16, /* sheared periodic box for shear runs: fsd_step
                              moves the bodies by their full velocity and
                              advances the box offset `tilt` by shear_rate L dt
                              (wrapped to [-L/2, L/2)), so each body's images
                              across y move with the imposed flow.  Excludes
                              FSD_FLAG_COMOVING.  The operator kernels read the
                              offset from device memory, so one captured graph
                              serves every step */
  FSD_FLAG_FP32_KRYLOV = 32  /* mixed precision only: the inner GMRES keeps its
                              Krylov bases V and Z in FP32 and orthogonalises
                              with FP32 products and in-warp sums (FP64
                              cross-warp sums, Hessenberg, Givens rotations,
                              refinement residual and LU stay FP64).  Off by
                              default: the Arnoldi orthogonalisation is FP64.
                              On this part FP64 runs at 1/74 of the FP32 rate
                              and the FP64 Gram-Schmidt passes are ALU-bound;
                              the FP32 basis takes the 32768-bead step from
                              ~66 to ~61 ms at the same iteration count and
                              accuracy */
};

/* Environment (read when a context is set up; defaults in brackets):
 *   FSD_OPERATOR_STREAMS=1   run an operator application on one stream
 *                            [2: the real-space sum beside the wave-space
 *                            chain on a second stream]
 *   FSD_RS_BLOCKS_PER_SM=k   persistent real-space blocks per SM while
 *                            overlapped [0: as many as fit]
 *   FSD_SPREAD_ATOMIC=1      FP32 spreading by vector atomic adds per bead
 *                            [grid-centric gather by 8^3 tiles]
 *   FSD_BATCH_THREADS=k      host threads of the batched launch phase [8]
 * Each choice changes speed only, not the arithmetic's result beyond the
 * order of FP32 sums. */

typedef struct {
  double a;              /* bead radius (1)                                        */
  double eta;            /* viscosity (1)                                          */
  double box;            /* side L of the periodic cube (required, > 0)            */
  double xi;             /* Ewald splitting (Sec. 3.2); <= 0: 0.5 / a, or in a box
                            too small for that cut-off 1.05 x the smallest xi with
                            R_c < L/2                                              */
  double xerr;           /* accuracy target of the parameter rules (1e-6)          */
  double rc;             /* real-space cut-off; <= 0: 2a + sqrt(-ln xerr)/xi       */
  int grid;              /* FFT points per side; 0: k_c L / pi with
                            k_c = 2 sqrt(-ln xerr) xi + 1 (Sec. 3.2), rounded up
                            to a 2,3,5-smooth multiple of 4 (a given grid need
                            only be even and 2,3,5-smooth)                         */
  int P;                 /* Gaussian support in grid points per side (even, 4..24);
                            0: from xerr (8 for 1e-4, 12 for 1e-6, 16 for 1e-8)    */
  double m_shape;        /* Gaussian shape factor; <= 0: 0.976 sqrt(pi P)          */
  double lub_cutoff;     /* lubrication cut-off r_lub (0: no near field)           */
  double precond_cutoff; /* r_p of the preconditioner (2.1 a, Sec. 2.2.2)          */
  double lub_hmin;       /* gap clamp of the pair functions (1e-3 a)               */
  double tol;            /* relative residual target (1e-6)                        */
  int restart;           /* GMRES restart length (30)                              */
  int max_iter;          /* Krylov iteration limit per solve (1000)                */
  int precision;         /* FSD_FP64 or FSD_MIXED                                  */
  int inner_restart;     /* mixed: FP32-operator GMRES iterations per refinement
                            sweep (60)                                             */
  double inner_tol;      /* mixed: floor of the inner relative tolerance; a sweep
                            aims at max(inner_tol, 0.3 tol / rel), rel the current
                            FP64 relative residual (1e-7: the FP32 operator's
                            relative error is ~1e-7, so at tol 1e-6 one sweep
                            usually suffices)                                      */
  int flags;             /* FSD_FLAG_*                                             */
  int tile;              /* real-space lanes per bead (4, 8, 16, 32); 0: from the
                            mean neighbour count                                   */
  double lanczos_tol;    /* fsd_brownian: a Lanczos square root stops when its
                            coefficients change by less than this, relative;
                            <= 0: 1e-7                                             */
  int lanczos_max_iter;  /* fsd_brownian: Lanczos step limit; <= 0: 60; at most
                            the Krylov basis length max(restart, inner_restart)   */
  double tilt;           /* Lees-Edwards offset of the box: the periodic image
                            across y sits at (x + tilt, y + L, z); lattice
                            e1 = (L,0,0), e2 = (tilt,L,0), e3 = (0,0,L).  Taken
                            modulo L into [-L/2, L/2) (0: the cube).  With a
                            non-zero tilt (or FSD_FLAG_LEES_EDWARDS) R_c and
                            the lubrication cut-off must stay below 0.447 L    */
  int nf_sampler;        /* fsd_brownian's near-field force: FSD_NF_PAIRWISE
                            (fsd_default_params: sum over lubrication pairs of
                            K_p^T psi_p, K_p the pair's dissipation-form
                            factor: exact covariance R_FU^nf, no iteration;
                            pair noise from Philox stream 5) or
                            FSD_NF_LANCZOS (0: the paper's preconditioned
                            Lanczos, Sec. 2.2; stops after lanczos_max_iter
                            steps, short of lanczos_tol on dense lubricated
                            suspensions)                                       */
  double rough_alpha;    /* surface roughness of the lubrication pairs (Sec. 4,
                            Eq. tan_fric): below the asperity height rough_h0
                            the sliding and rolling coefficients of the pair
                            model gain 6 pi eta a f(h) and 8 pi eta a^3 f(h),
                            f = rough_alpha (a/h0) (h0/h - 3 h/h0 + 2 h^2/h0^2)
                            (h the gap, clamped at lub_hmin): O(1/h) instead of
                            O(ln 1/h).  0: smooth spheres (default)            */
  double rough_h0;       /* asperity height h0 (> 0 when rough_alpha > 0)       */
} fsd_params;

typedef struct {
  int iters;          /* Krylov iterations (all levels)                     */
  int outer_iters;    /* outer iterations (restarts for FP64; refinement
                         steps for mixed)                                   */
  int matvec64;       /* FP64 saddle-operator applications                  */
  int matvec32;       /* FP32 saddle-operator applications                  */
  double rel_residual;/* true FP64 ||b - A x|| / ||b|| at exit              */
  double ms_total;    /* wall time of the call (ms)                         */
  int64_t n_pairs;    /* real-space neighbour pairs (directed)              */
  int64_t n_lub;      /* lubrication pairs (directed)                       */
  int grid;           /* FFT grid used                                      */
  int P;              /* Gaussian support used                              */
  double xi;          /* splitting used                                     */
  double rc;          /* real-space cut-off used                            */
  int64_t kernel_launches; /* CUDA kernels this call launched               */
} fsd_stats;

/* Defaults above (box must still be set). */
void fsd_default_params(fsd_params *p);

/* Create a context for one suspension (Algorithm 1 set-up).
 * n_beads >= 1; bead_pos [n_beads][3] (any periodic image: each aggregate is
 * unwrapped by the minimum image about its first bead); agg_id [n_beads] with
 * every id in 0..N-1 used at least once.  The body frame is the bead layout
 * given here (orientation quaternion = identity), centred on the bead
 * centroid X (equal bead masses, Sec. 2.3.1).  cuda_stream: a cudaStream_t or
 * NULL for a stream the context creates.  On failure *ctx is NULL. */
fsd_status fsd_setup(fsd_ctx **ctx, int64_t n_beads, const double *bead_pos,
                     const int32_t *agg_id, const fsd_params *p,
                     void *cuda_stream);

/* One saddle-point solve at the current configuration (Algorithm 1 steps 1
 * and 4).  agg_force_torque [N][6]: conservative force and torque about X
 * per aggregate, FF^P (NULL = 0).  Outputs: agg_velocity [N][6] = (U, Omega)
 * in the lab frame including U_inf(X), Omega_inf; agg_stresslet [N][9] =
 * S^H + S^C (Eq. stress_comp a, d) as a symmetric 3x3, row-major (NULL to
 * skip).  stats may be NULL. */
fsd_status fsd_solve(fsd_ctx *ctx, const double *agg_force_torque,
                     double shear_rate, double *agg_velocity,
                     double *agg_stresslet, fsd_stats *stats);

/* fsd_solve followed by the Euler-Maruyama rigid-body update (Sec. 2.4,
 * Eq. EM1-EM3): X += U dt; q <- normalise(q + dt/2 (0, Omega) q);
 * bead x = X + R(q) x_body.  agg_velocity may be NULL. */
fsd_status fsd_step(fsd_ctx *ctx, const double *agg_force_torque,
                    double shear_rate, double dt, double *agg_velocity,
                    fsd_stats *stats);

/* Current bead positions [n_beads][3] (unwrapped per aggregate) and
 * orientation quaternions [N][4] (w, x, y, z); either may be NULL. */
fsd_status fsd_get_beads(fsd_ctx *ctx, double *bead_pos, double *agg_quat);

/* Operator access (parity tests and users composing their own solvers).
 * Vectors use the solution layout: per bead 11 values (F: 3, L: 3, S: 5 in the
 * orthonormal basis {(xx-yy)/sqrt2, (2zz-xx-yy)/sqrt6, sqrt2 xy, sqrt2 xz,
 * sqrt2 yz}) in bead order, then per aggregate 6 values (U, Omega) in id order.
 * precision: FSD_FP64 or FSD_MIXED (= the FP32 operator). */

/* out[n_beads][11] = M_inf . in[n_beads][11]; part: 1 real space (incl. the
 * self term), 2 wave space, 3 both (Sec. 2.2, Eq. UBff split). */
fsd_status fsd_apply_mobility(fsd_ctx *ctx, const double *in, double *out,
                              int part, int precision);

/* y = A x, the saddle-point operator of Eq. spm_agg. */
fsd_status fsd_apply_saddle(fsd_ctx *ctx, const double *x, double *y,
                            int precision);

/* z = P^-1 r, the block-triangular preconditioner (Table 1, aggregates). */
fsd_status fsd_apply_precond(fsd_ctx *ctx, const double *r, double *z);

/* out[N][6] = RR_FU^nf . dU[N][6] (Sigma R^nf Sigma^T, Eq. FH_agg). */
fsd_status fsd_apply_lubrication(fsd_ctx *ctx, const double *dU, double *out,
                                 int precision);

/* Right-hand side of Eq. spm_agg (same layout as x). */
fsd_status fsd_rhs(fsd_ctx *ctx, const double *agg_force_torque,
                   double shear_rate, double *b);

/* Opt-in profiler: device time per kernel group, from CUDA events recorded
 * on the context's stream around each group (adds a few microseconds per
 * group launch; leave off for throughput runs).  Groups, in order:
 * realspace, spread, fft_green, interp, body_rows, precond, krylov,
 * neighbors, lub_assembly, misc. */
#define FSD_PROF_GROUPS 10
/* on != 0: reset the counters and start recording; 0: stop. */
fsd_status fsd_profile_enable(fsd_ctx *ctx, int on);
/* ms[g] = accumulated device milliseconds, count[g] = timed launches of
 * group g since the last enable; n >= FSD_PROF_GROUPS (either array may be
 * NULL).  Synchronises the context's stream. */
fsd_status fsd_profile_read(fsd_ctx *ctx, double *ms, int64_t *count, int n);
/* Name of group g (NULL when out of range). */
const char *fsd_profile_group_name(int g);

/* Wave-space mobility without any allocation (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. code whose device memory belongs to an allocator or pool it does not
 * own, a plug-in that must not grow the process's device footprint after
 * start-up, or a loop where an allocation and its implicit synchronisation
 * are not allowed).  Computes out = M_wave . in with the FP32 wave-space operator
 * of fsd_apply_mobility (part 2, precision FSD_MIXED): Gaussian spreading,
 * FFT with the Green's function, interpolation.  No context: the parameters
 * are given directly (m_shape <= 0 selects 0.976 sqrt(pi P)).
 *   bead_pos [n_beads][3], in [n_beads][11], out [n_beads][11]: DEVICE memory
 *   owned by the caller, layouts as for fsd_apply_mobility.
 *   Limits: n_beads <= 4096, grid <= 48 (even, 2,3,5-smooth), P even in
 *   4..24 and <= grid; larger requests return FSD_EINVAL before any GPU work.
 * Every intermediate lives in one 10 MiB file-scope device array that each
 * device loading the library holds until the process exits.  Each call looks
 * up that array's device address in the current device context
 * (cudaGetSymbolAddress; FSD_ECUDA if that fails).  All calls share the
 * array: calls whose GPU work overlaps race on it, so order them on one
 * stream (or with events).  Each call rewrites or zeroes everything it
 * reads.  Work is enqueued on cuda_stream (NULL: the default stream); out is
 * ready when that stream is.  The call may be captured into a CUDA graph
 * (cuda_stream capturing, in any capture mode): the graph then reads
 * bead_pos and in, and writes out, at each replay, with the parameters of
 * the captured call; its argument checks and the address lookup are host
 * queries made with the thread's capture mode relaxed for their duration.
 * An error already pending in the CUDA runtime
 * when the call starts is left in place and the call returns FSD_ECUDA
 * without doing anything. */
fsd_status fsd_apply_wave_noalloc(int64_t n_beads, const double *bead_pos,
                                  const double *in, double *out, double box,
                                  double xi, int grid, int P, double m_shape,
                                  double a, double eta, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent periodic suspensions (each with its own box,
 * beads, aggregates and parameters) advanced together.  The paper solves one
 * suspension per run; batching is this library's way to fill the GPU with
 * systems that are each too small to.  Each system gets its own context and
 * stream; each system's solve (or step) is one captured CUDA graph
 * (FSD_FLAG_GRAPH is forced on), and all systems' graphs are launched before
 * any is waited for, most expensive first, so they run concurrently.  Results
 * are those of fsd_solve / fsd_step on each system alone.  The streams share
 * the device's hardware work queues: the environment variable
 * CUDA_DEVICE_MAX_CONNECTIONS=32 (set before the process creates its CUDA
 * context; the default is 8) lets up to 32 systems' kernels run side by side
 * (measured on 64 systems: 438 -> 390 ms per step).
 * ------------------------------------------------------------------------- */
typedef struct fsd_batch fsd_batch;

/* n_sys >= 1 systems; bead_offsets [n_sys + 1] (host): system s owns beads
 * bead_offsets[s] .. bead_offsets[s+1]-1 of bead_pos [total][3] and agg_id
 * [total] (ids dense 0..N_s-1 within each system); params [n_sys] (host), each
 * as for fsd_setup (FSD_FLAG_AUTOTUNE tunes each system on its own).
 * cuda_stream: a stream that the batch's work is ordered after and that
 * waits for it (NULL: none).  On failure *batch is NULL and
 * fsd_batch_last_error(NULL) names the system. */
fsd_status fsd_setup_batch(fsd_batch **batch, int n_sys, const int64_t *bead_offsets,
                           const double *bead_pos, const int32_t *agg_id,
                           const fsd_params *params, void *cuda_stream);

/* n_sys, agg_offsets [n_sys + 1] (prefix sums of the aggregate counts: the
 * aggregate arrays below are concatenated in system order) and the
 * parameters each system uses; any pointer may be NULL. */
fsd_status fsd_batch_info(const fsd_batch *b, int *n_sys, int64_t *agg_offsets,
                          fsd_params *params);

/* fsd_solve on every system.  agg_force_torque [A][6] (NULL = 0),
 * shear_rates [n_sys] (host), agg_velocity [A][6], agg_stresslet [A][9]
 * (NULL to skip), stats [n_sys] (NULL to skip); A = agg_offsets[n_sys].
 * Returns when every system is done.  The status is the worst over the
 * systems (error > FSD_ENOCONV > FSD_EOVERLAP > FSD_OK);
 * fsd_batch_last_error names the system. */
fsd_status fsd_solve_batch(fsd_batch *b, const double *agg_force_torque,
                           const double *shear_rates, double *agg_velocity,
                           double *agg_stresslet, fsd_stats *stats);

/* fsd_step on every system (same dt). agg_velocity may be NULL. */
fsd_status fsd_step_batch(fsd_batch *b, const double *agg_force_torque,
                          const double *shear_rates, double dt,
                          double *agg_velocity, fsd_stats *stats);

/* Bead positions [total][3] and quaternions [A][4] of every system. */
fsd_status fsd_batch_get_beads(fsd_batch *b, double *bead_pos, double *agg_quat);

/* System s's context, owned by the batch (operator access, profiler, or
 * solving it alone); NULL when out of range. */
fsd_ctx *fsd_batch_system(fsd_batch *b, int s);

/* Message of the last error on b (NULL: of the last failed fsd_setup_batch). */
const char *fsd_batch_last_error(const fsd_batch *b);

void fsd_destroy_batch(fsd_batch *b);

/* Brownian forcing of the NEXT solve (Sec. 2.2 stochastic sampling, Eq. SP2,
 * Eq. UBff; Algorithm 1 step 3).  Samples, at the current configuration,
 *   far-field slip   u^B  = sqrt(2 kT/dt) (M_w^(1/2) psi_w + M_r^(1/2) psi_r)
 *   near-field force F^B  = sqrt(2 kT/dt) (R_FU^nf)^(1/2) psi_nf
 * with the wave part analytic (a random field scaled in k space, inverse FFT,
 * interpolation), the real-space and near-field square roots by Lanczos
 * iterations on the real-space operator (in the context's operator
 * precision) and the bead-level lubrication blocks (FP64).  The next
 * fsd_solve / fsd_step adds u^B to the bead rows (velocity, rotation and
 * strain) and -Sigma F^B to the body rows of Eq. spm_agg, then forgets them.
 * The Brownian drift and stresslet are not included.
 * Random inputs (host or device; NULL: drawn from Philox4x32-10 with key
 * (seed mod 2^32, seed / 2^32) and counter (index, stream * 256 + call,
 * step mod 2^32, step / 2^32); each call gives four normals by Box-Muller,
 * from the word pairs (0, 1) and (2, 3) with u = (word + 1) 2^-32:
 * sqrt(-2 ln u0) (cos, sin)(2 pi u1), then the same of u2, u3.  Stream 2:
 * psi_real of a bead, the first 11 normals of calls 0-2; stream 3: psi_nf,
 * the first 6 of calls 0-1; index = bead position in the setup arrays.
 * Stream 1: the wave field, drawn at the canonical point (kz, ky, kx) of
 * each Hermitian pair (the point itself when kx > 0; for kx = 0 the one of
 * (kz, ky) and ((n - kz) mod n, (n - ky) mod n) that comes first in (kz, ky)
 * order, the other holding its conjugate), index (kz n + ky)(n/2 + 1) + kx,
 * the six normals of calls 0-1 giving components 0, 1, 2 as
 * (normal 2c + i normal 2c+1) / sqrt 2):
 *   wave_field [3][n][n][n/2+1] complex (re, im) doubles, layout [c][kz][ky][kx]
 *     (k = 2 pi m / L, m_i = index, or index - n past n/2): standard complex
 *     Gaussians, Hermitian in the kx = 0 plane; Nyquist points and k = 0 are
 *     ignored;
 *   psi_real [n_beads][11], psi_nf [n_beads][6]: standard normals.
 * With nf_sampler = FSD_NF_PAIRWISE the near-field force is
 * sum_p K_p^T psi_p over the lubrication pairs p = (i < j, input order),
 * K_p (6 x 12) the pair's dissipation-form factor (K_p^T K_p = the pair's
 * 12x12 block of R_FU^nf), psi_p 6 normals from Philox with counter
 * (i, 5 * 256 + call, j, step mod 2^32), calls 0 and 1; psi_nf must then be
 * NULL.
 * Outputs (NULL to skip): slip [n_beads][11] = u^B, force_nf [n_beads][6] =
 * F^B.  stats: iters = real-space Lanczos steps, outer_iters = near-field
 * Lanczos steps (each stops when its coefficients change by less than
 * lanczos_tol relative, or after lanczos_max_iter steps), rel_residual = the
 * larger last relative change of the two. */
fsd_status fsd_brownian(fsd_ctx *ctx, double kT, double dt, uint64_t seed, uint64_t step,
                        const double *wave_field, const double *psi_real,
                        const double *psi_nf, double *slip, double *force_nf,
                        fsd_stats *stats);

/* Methods of fsd_drift. */
enum { FSD_DRIFT_RFD = 0, FSD_DRIFT_FIXMAN = 1 };

/* Brownian drift kT div(R_FU^-1) and Brownian stresslet S^B (Sec. 2.4; the
 * appendix on the drift), added to the velocity of the NEXT fsd_solve /
 * fsd_step (and so to its update), then forgotten.  A displacement of the
 * configuration by h v (v [N][6]) moves X by h v_t and rotates the lever
 * arms by the unit quaternion normalise(1, (h/2) v_w) (the Euler step of
 * Eq. EM2); each solve below has no background flow, and the stresslets
 * differenced are the hydrodynamic ones (S^ff - R_SU^nf Sigma^T U).
 *   FSD_DRIFT_RFD (Eq. rfd): U+- = the solve at x +- (eps/2) dq with body
 *     forcing dq; drift = kT (U+ - U-)/eps, S^B = kT (S+ - S-)/eps.
 *     param = eps (<= 0: a tol^(1/3), the error balance eps ~ tol^(1/3));
 *     dq [N][6] (host or device) or NULL: standard normals from Philox
 *     stream 4, index = aggregate id, calls 0 and 1, first 6 of the 8.
 *     Two solves; pending Brownian terms (fsd_brownian) stay pending; dt is
 *     not used.
 *   FSD_DRIFT_FIXMAN (modified Fixman midpoint): needs pending Brownian
 *     terms.  U0, S0 = the solve with them at x; x' = x + (dt/m) U0;
 *     U', S' = the solve with the same terms at x'; drift = (m/2)(U' - U0),
 *     S^B = -(m/2)(S' - S0).  param = m (<= 0: 100).  Two solves; the
 *     Brownian terms are spent: the next solve gets U0 + drift added instead.
 * The configuration, the warm-start vector and the flags are as before on
 * return; the solves run host-driven or as graphs like fsd_solve.  Outputs
 * (NULL to skip): drift [N][6], brownian_velocity [N][6] (Fixman: U0),
 * brownian_stresslet [N][9].  stats sum the two solves (rel_residual: the
 * larger).  FSD_ENOCONV from a solve is returned after the outputs are
 * written. */
fsd_status fsd_drift(fsd_ctx *ctx, int method, double kT, double dt, double param,
                     uint64_t seed, uint64_t step, const double *dq, double *drift,
                     double *brownian_velocity, double *brownian_stresslet,
                     fsd_stats *stats);

/* Hertz normal contact between beads of different aggregates at the current
 * configuration (Sec. 4: F_N = k_n delta^1.5 n, delta = 2a - r the overlap,
 * n the unit vector along the line of centres; the rod benchmark of
 * Sec. 3.3 uses normal contact between rods): each overlapping pair pushes
 * its two beads apart with kn delta^1.5; the bead forces are summed per
 * aggregate into a force and a torque about the centroid X.  Writes
 * agg_force_torque [N][6] (host or device; pass it to fsd_step / fsd_solve as
 * the applied force).  kn in units of force / length^1.5.  The neighbour
 * lists built here are reused by the next solve. */
fsd_status fsd_contact_forces(fsd_ctx *ctx, double kn, double *agg_force_torque);

/* Interparticle forces of Sec. 4 between beads of different aggregates. */
typedef struct {
  double kn;       /* Hertz normal contact k_n delta^1.5 (0: none)                 */
  double hamaker;  /* Hamaker constant A_H of the van der Waals attraction (0: none) */
  double zeta;     /* double-layer strength Z, energy per length: the repulsion is
                      (a^2/r) Z exp(-kappa (r - 2a)) (0: none)                      */
  double kappa;    /* inverse Debye length (> 0 when zeta != 0)                    */
  double h_c;      /* van der Waals regularisation: evaluated at gap h + h_c; under
                      overlap the attraction keeps its value at contact          */
  double r_cut;    /* DLVO cut-off on the centre distance; at most the real-space
                      cut-off R_c of the context (its neighbour list is used)     */
} fsd_pair_forces;

/* Hertz contact plus DLVO forces (Sec. 4, Eq. dlvo_potential, F = -grad V)
 * between beads of different aggregates at the current configuration: per
 * pair the central force f(r) n, f = k_n (2a - r)^1.5 [r < 2a] - dV/dr
 * [r < r_cut], with V = -(A_H/6) [2a^2/(r'^2 - 4a^2) + 2a^2/r'^2 +
 * ln(1 - 4a^2/r'^2)] (r' = max(r, 2a) + h_c in the attraction's derivative;
 * the sphere-sphere Hamaker form) + (a^2/r) Z exp(-kappa (r - 2a)).  The bead
 * forces are summed per aggregate into a force and a torque about the
 * centroid, written to agg_force_torque [N][6] (host or device), to be passed
 * to fsd_step / fsd_solve as the applied force.  FSD_EINVAL for r_cut above
 * R_c, a negative stiffness, or zeta != 0 with kappa <= 0. */
fsd_status fsd_interparticle_forces(fsd_ctx *ctx, const fsd_pair_forces *p,
                                    double *agg_force_torque);

/* Sets the Lees-Edwards offset of the box (see fsd_params.tilt; taken
 * modulo L).  fsd_get_params reports the current offset. */
fsd_status fsd_set_tilt(fsd_ctx *ctx, double tilt);

/* Measured fused multiply-add throughput of the current device (no
 * counterpart in the paper: the real-space pair sum and the FP64 operator
 * are bound by the FMA rate, so their rooflines need the rate of the GPU at
 * hand).  fp_bits 32 or 64; *flop_per_s = 2 x FMAs per second of a kernel of
 * independent FMA chains filling every SM (best of three ~2-5 ms launches,
 * CUDA events on cuda_stream; NULL: the default stream).  Synchronises
 * cuda_stream; allocates and frees a few bytes.  FSD_EINVAL for another
 * fp_bits or a NULL output, FSD_ECUDA on a CUDA error. */
fsd_status fsd_fma_throughput(int fp_bits, double *flop_per_s, void *cuda_stream);

/* Parameters actually used (after the defaulting rules). */
fsd_status fsd_get_params(const fsd_ctx *ctx, fsd_params *p);

/* Message of the last error on ctx (or of the last failed fsd_setup when ctx
 * is NULL).  Valid until the next call on the same context. */
const char *fsd_last_error(const fsd_ctx *ctx);

void fsd_destroy(fsd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FSD_H */
