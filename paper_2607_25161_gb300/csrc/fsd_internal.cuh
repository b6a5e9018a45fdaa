// Internal declarations of the FSD library: context, device buffers and the
// launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fsd.h"

namespace fsd {

constexpr double kPi = 3.14159265358979323846;
constexpr int LDB = 12;     // doubles per bead in a solution vector (11 + zero pad)
constexpr int NFUNC = 7;    // radial functions of the real-space table
// Polynomial coefficients per function per interval of the real-space radial
// table, per precision.  The functions are band-limited by K = 2 xi sqrt(46)
// and an interval is 1.6 / K long, so the Chebyshev fit's error relative to
// each function's largest value does not depend on xi: 6e-11 with 6
// coefficients (FP32 table), 1.5e-14 with 8 (FP64), 4e-9 with 5.
template <typename T>
constexpr int tab_coef() {
  return sizeof(T) == 4 ? 6 : 8;
}
// table values per interval: 8 per power (seven functions and a pad), plus
// 4 so that an FP32 interval spans an odd number of 16-byte units (bank
// spread when the lanes of a warp read different intervals)
template <typename T>
constexpr int tab_stride() {
  return tab_coef<T>() * 8 + 4;
}
constexpr int BLK = 36;     // 6x6 block

// ------------------------------------------------------------------ errors
struct CudaError {
  cudaError_t e;
  const char *what;
};

#define FSD_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess) throw ::fsd::CudaError{e__, #call};               \
  } while (0)

struct Invalid {
  std::string msg;
};

// ----------------------------------------------------------- device buffer
template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  void alloc(size_t count) {
    free();
    if (count == 0) count = 1;
    FSD_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void free() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DBuf() { free(); }
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
};

// ------------------------------------------------- per-precision operator
// Everything the FP32 or the FP64 operator needs beyond the shared geometry.
template <typename T>
struct OpData {
  DBuf<T> table;      // real-space radial table [nint][power][function padded to 8]
  T self_real[3];     // real-space self mobilities (translation, rotation, strain)
  DBuf<T> grid;       // spread densities, planar: [6][n^3]
  DBuf<T> spec;       // half spectra, planar: [6][n][n][n/2 + 1] complex
  DBuf<T> gout;       // velocity fields for interpolation, interleaved: [n^3][8] (6 used)
  DBuf<T> green;      // [m = kx^2+ky^2+kz^2][3]: (A fM^2, A fM fD, A fD^2)
  DBuf<T> twiddle;    // [n] complex: exp(-2 pi i t / n)
  DBuf<T> bval;       // lubrication BSR off-diagonal blocks [nnz][36]
  DBuf<T> bdiag;      // lubrication BSR diagonal blocks [Nt][36]
  DBuf<T> pos;        // wrapped positions [Nt][4] (x, y, z, 0)
  DBuf<T> lever;      // r_b = x_b - X_J [Nt][4]
  DBuf<T> packed;     // per bead (x, y, z, F, L, S6, 0) in the operator precision [Nt][16]
  DBuf<T> btab;       // Brownian wave-field scales [m = kx^2+ky^2+kz^2][2]: (c fM, c fD)
  DBuf<T> green_le;   // Lees-Edwards box: Green factors per wave vector [ky][kx][kz][3]
  double green_le_tilt = 0.0;  // box offset the table was built for (0: none)
};

// Kernel groups timed by the opt-in profiler (CUDA events on the stream).
enum ProfGroup {
  PG_REAL = 0,  // real-space pair sum
  PG_SPREAD,    // Gaussian spreading
  PG_FFT,       // FFT passes incl. the fused Green's function
  PG_INTERP,    // interpolation
  PG_BODY,      // aggregate rows: constraint gather + lubrication BSR
  PG_PRECOND,   // preconditioner apply
  PG_KRYLOV,    // Arnoldi dots / updates / scaling
  PG_NEIGHBOR,  // cell and neighbour lists
  PG_LUB,       // lubrication assembly + Schur LUs
  PG_MISC,      // rhs, outputs, integrator, permutations
  PG_COUNT
};

struct Ctx;
struct GraphCache;  // captured solve graphs of a context (graph.cu)

// Krylov statistics of one solve.
struct KStats {
  int iters = 0, m64 = 0, m32 = 0, outer = 0;
};

// What one captured step does (graph.cu).
struct GraphRun {
  int warm = 0;       // start from the previous solution
  int has_ft = 0;     // applied forces / torques staged in the graph's buffer
  int integrate = 0;  // advance the rigid bodies by dt after the solve
  int with_str = 0;   // write the stresslet
  int brown = 0;      // add the pending Brownian terms to the right-hand side
  int add_vel = 0;    // add the pending drift velocity to the velocity output
  int str_hydro = 0;  // stresslet output without the constraint part
  double shear = 0.0, dt = 0.0, brown_scale = 0.0;
};

struct ProfScope {
  Ctx *c;
  int g;
  cudaEvent_t e0 = nullptr;
  ProfScope(Ctx &cx, int grp);
  ~ProfScope();
};

struct Ctx {
  // ---- profiling and launch accounting
  bool prof = false;
  int64_t launches = 0;  // kernel launches issued by this context
  double prof_ms[PG_COUNT] = {};
  int64_t prof_n[PG_COUNT] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  // ---- parameters
  fsd_params prm{};
  double L = 0, a = 1, eta = 1, xi = 0.5, rc = 0, alpha = 0, h = 0;
  int n = 0, P = 8;
  double m_shape = 0;
  int Nt = 0, N = 0;
  int num_sms = 152;
  int64_t nunk = 0;  // padded length of a solution vector: LDB*Nt + 6*N
  // ---- real-space table geometry
  int tab_nint = 0;
  double tab_h = 0;
  // ---- stream
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // second stream: an operator application runs the real-space sum (ALU
  // bound) on it beside the wave-space chain (L2 / shared-memory bound)
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool overlap = false;        // use it (off while profiling)
  bool rs_overlapped = false;  // the real-space launch in progress is the overlapped one
  int rs_blocks_per_sm = 0;    // persistent real-space blocks per SM when overlapped (0: all
                               // that fit): on the 32768-bead step 63.6 ms (all) against
                               // 65.8 (two) and 65.4 (one stream)
  DBuf<double> yw;             // wave-space part of an overlapped application
  // grid-centric FP32 spreading: the grid in 8^3 tiles, per tile the beads
  // whose window reaches it (rebuilt when the positions change)
  bool spread_gather = true;
  bool tiles_valid = false;
  int tile_n = 0;                    // tiles per side
  DBuf<int> tile_count, tile_start, tile_cursor, tile_beads;
  // ---- geometry (internal order: beads grouped by aggregate, aggregates
  //      sorted spatially)
  std::vector<int> h_perm_bead;  // internal bead -> user bead
  std::vector<int> h_perm_body;  // internal body -> user id
  std::vector<int> h_body_start;
  int body_lanes = 32;  // lanes per aggregate in the aggregate-row kernels (4, 8, 16 or 32)
  DBuf<int> body_start, bead_body, perm_bead, perm_body;
  DBuf<double> X, q, rbody, pos64, lever64;
  // Lees-Edwards box: offset of the image across y (0: cube); wave-space
  // positions in sheared coordinates s = (x - (tilt/L) y, y, z), wrapped
  double tilt = 0.0;
  // device copy of tilt: with FSD_FLAG_LEES_EDWARDS the operator kernels read
  // the offset from it, so that a captured step graph follows the offset
  // (written on the stream whenever tilt changes)
  DBuf<double> tilt_dev;
  DBuf<double> wpos64;
  DBuf<float> wpos32;
  // ---- neighbour lists
  int cap = 0, lcap = 0, ncell = 1;
  DBuf<int> nbr, ncnt, lnbr, lcnt;
  DBuf<int> cell_count, cell_start, cell_beads, cell_cursor;
  DBuf<int> flags;  // [0] nbr overflow, [1] lub overflow, [2] overlap, [3] singular LU, [4] max count
  int *h_flags = nullptr;  // pinned
  // ---- lubrication BSR (rows = beads; diagonal separate)
  DBuf<int> brow, bcol;
  int nnz_cap = 0;
  // ---- preconditioner
  DBuf<double> schur;  // [N][36] LU factors
  DBuf<int> piv;       // [N][6]
  // ---- operators
  OpData<double> op64;
  OpData<float> op32;
  // ---- Krylov workspace
  int m = 30, m_in = 30;
  DBuf<double> V, Z, w, t1, t2, xsol, rhs, res, xprev, partial, hcol;
  // FP32 Krylov basis and preconditioned basis of the mixed solve's inner
  // GMRES with FSD_FLAG_FP32_KRYLOV ((m_in + 1) and m_in vectors); V (FP64)
  // serves the FP64 bases and the Lanczos square roots
  bool krylov32 = false;  // mixed with FSD_FLAG_FP32_KRYLOV: FP32 inner bases
  DBuf<float> V32, Z32;
  DBuf<double> kv, kz;  // FP64 copies of v_j and z_j for the FP32 basis
  DBuf<unsigned> cgs_ticket;  // blocks finished in the running Gram-Schmidt pass (0 between passes)
  double *h_pinned = nullptr;  // host pinned scratch (dots)
  bool have_prev = false;
  // ---- outputs / near field scratch
  DBuf<double> fnf, snf;  // per bead near-field force [Nt][6], stresslet [Nt][5]
  DBuf<double> pdiag;     // per bead preconditioner near-field diagonal block [Nt][36]
  DBuf<double> io_a, io_b;     // staging for host / permuted I/O
  std::string last_error;
  fsd_status last_warning = FSD_OK;
  int64_t n_pairs = 0, n_lub = 0;
  // ---- Brownian forcing of the next solve (brownian.cu)
  DBuf<double> bslip, bfnf, bwork, bwork2;  // slip u_w + u_r, near-field force (solution layout), scratch
  DBuf<double> bgain;               // per bead Cholesky factor L of the near-field diagonal block and L^-1
  bool brown_pending = false;       // the next solve adds them to its right-hand side
  bool geom_fresh = false;          // geometry prepared at the current positions (the next
                                    // solve may skip its own preparation)
  double brown_scale = 0.0;         // sqrt(2 kT / dt)
  // ---- Brownian drift (brownian.cu, api.cu)
  DBuf<double> vextra;              // [N][6] velocity added to the next solve's output
  bool vextra_pending = false;
  bool str_hydro = false;           // outputs write the hydrodynamic stresslet only
  DBuf<double> dsave, dwork, dxprev;  // saved X, q; drift vectors; saved previous solution
  DBuf<double> cwork;                 // contact forces: per bead [Nt][3], then [N][6]
  // ---- captured solve graphs
  GraphCache *gcache = nullptr;
  int64_t graph_pending = -1;
  double tuned_ms = 0.0;  // operator time measured by the autotuner (0: not tuned)
};

// ------------------------------------------------------ Lees-Edwards box
// Nearest image of a displacement in the sheared periodic box (lattice
// (L,0,0), (tilt,L,0), (0,0,L)): wrap y first, shifting x by the offset, then
// x and z.  tilt = 0 is the cube.
__device__ __forceinline__ void le_image(double &d0, double &d1, double &d2, double L, double tilt) {
  const double ny = rint(d1 / L);
  d0 -= ny * tilt;
  d1 -= ny * L;
  d0 -= L * rint(d0 / L);
  d2 -= L * rint(d2 / L);
}

// ------------------------------------------------- counter-based normals
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32 -> 64-bit multiplications with the Weyl key schedule; the Brownian
// sampler draws every random number from (counter, key), so any element can
// be generated independently and reproducibly.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Four standard normals for counter (index, stream * 256 + call, step) and
// key seed: Box-Muller on u_j = (x_j + 1) 2^-32.
__device__ inline void philox_normals4(uint64_t seed, uint64_t step, uint32_t stream, uint32_t call,
                                       uint32_t index, double z[4]) {
  uint32_t c[4] = {index, (stream << 8) | call, (uint32_t)step, (uint32_t)(step >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double s = 2.3283064365386963e-10;  // 2^-32
  const double u0 = ((double)c[0] + 1.0) * s, u1 = ((double)c[1] + 1.0) * s;
  const double u2 = ((double)c[2] + 1.0) * s, u3 = ((double)c[3] + 1.0) * s;
  const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
  double s0, c0, s1, c1;
  sincospi(2.0 * u1, &s0, &c0);
  sincospi(2.0 * u3, &s1, &c1);
  z[0] = r0 * c0;
  z[1] = r0 * s0;
  z[2] = r1 * c1;
  z[3] = r1 * s1;
}

// ------------------------------------------------------------ launchers
// realspace.cu
void build_real_table(Ctx &c);
void build_neighbors(Ctx &c);  // cell list + mobility and lubrication lists
template <typename T>
void launch_realspace(Ctx &c, const double *x, double *y, bool add_constraint,
                      bool self_only_real);
void launch_wrap_positions(Ctx &c);  // pos64 / op*.pos / levers from X, q, rbody
__global__ void k_exclusive_scan(int n, const int *__restrict__ in, int *out, int *cursor);
__global__ void __launch_bounds__(128) k_sort_cells(int ncells, const int *__restrict__ cell_start,
                                                    int *cell_beads);  // 128 threads: a warp per segment
// wavespace.cu: per-tile bead lists of the grid-centric spreading
void build_spread_tiles(Ctx &c);
// Lees-Edwards offset as the kernels take it: the host value and, with
// FSD_FLAG_LEES_EDWARDS, the device copy they read instead.
struct TauArg {
  double tau = 0.0;             // tilt / L (host value)
  const double *dev = nullptr;  // device tilt (overrides tau when set)
  double invL = 0.0;
};
__device__ __forceinline__ double tau_of(const TauArg &t) { return t.dev ? *t.dev * t.invL : t.tau; }
const double *tilt_dev_ptr(const Ctx &c);
TauArg tau_arg(const Ctx &c);
void sync_tilt(Ctx &c);
void refresh_le_tables(Ctx &c);
int realspace_group(const Ctx &c);   // lanes per bead of the pair sum

// wavespace.cu
void build_wave(Ctx &c);
template <typename T>
void launch_wavespace(Ctx &c, const double *x, double *y);  // y += M_w x

// nearfield.cu
void build_lubrication(Ctx &c);  // BSR blocks (both precisions) + Schur LU
template <typename T>
void launch_body_rows(Ctx &c, const double *x, double *y, bool with_lub);  // y2 = Sigma B^T x1 - RR x2
template <typename T>
void launch_lub_apply(Ctx &c, const double *dU, double *out);  // out = RR dU
void launch_precond(Ctx &c, const double *r, double *z);
// the same on column *col_dev of the bases V and Z (leading dimension ld),
// z also written to z2 (the captured Arnoldi step)
void launch_precond_col(Ctx &c, const double *V, double *Z, int64_t ld, const int *col_dev,
                        double *z2);
void launch_rhs(Ctx &c, const double *ft_internal, double shear, double *b);
void launch_outputs(Ctx &c, const double *x, double shear, double *vel_int,
                    double *str_int);
void launch_integrate(Ctx &c, const double *vel_int, double dt, double shear);
// Hertz contact: per-bead forces into fb_scratch [Nt][3], aggregate force and
// torque into ft_int [N][6] (internal order); needs the neighbour lists
void launch_contact(Ctx &c, const fsd_pair_forces &pf, double *fb_scratch, double *ft_int);
// pairwise near-field Brownian force (unscaled, solution layout) into f
void launch_nf_pairwise(Ctx &c, uint64_t seed, uint64_t step, double *f);
// brownian.cu: drift helpers
void launch_add_velocity(Ctx &c, double *vel_int);  // vel_int += vextra
void launch_dq_philox(Ctx &c, uint64_t seed, uint64_t step, double *user);  // [N][6], stream 4
void launch_scaled_diff(Ctx &c, const double *a, const double *b, double s, double *out, int64_t n);
void launch_axpy(Ctx &c, const double *x, double *y, int64_t n);  // y += x

// krylov.cu
void dot_multi(Ctx &c, const double *V, int64_t ld, int k, const double *w,
               double *out_dev);                   // out[j] = V_j . w, j < k
void axpy_multi(Ctx &c, double *w, const double *V, int64_t ld, int k,
                const double *coef_dev, double sign);  // w += sign * sum_j coef[j] V_j
void vec_scale_host(Ctx &c, double *y, const double *x, double s);  // y = s x
void cgs_pass(Ctx &c, int mode, const double *V, int64_t ld, int k, double *w,
              const double *coef_dev, double *out_dev);  // fused Gram-Schmidt pass
void cgs_pass_dev(Ctx &c, int mode, const double *V, int64_t ld, const int *k_dev, int k_add,
                  int kmax, double *w, const double *coef_dev,
                  double *out_dev);  // the same with k = *k_dev + k_add read on the device
void axpy_multi_dev(Ctx &c, double *w, const double *V, int64_t ld, const int *k_dev,
                    const double *coef_dev, double sign);
// the same over an FP32 basis (inner GMRES of the mixed solve): FP32 products
// and in-warp sums, FP64 w and cross-warp sums
void axpy_multi(Ctx &c, double *w, const float *V, int64_t ld, int k, const double *coef_dev,
                double sign);
void cgs_pass(Ctx &c, int mode, const float *V, int64_t ld, int k, double *w,
              const double *coef_dev, double *out_dev);
void cgs_pass_dev(Ctx &c, int mode, const float *V, int64_t ld, const int *k_dev, int k_add,
                  int kmax, double *w, const double *coef_dev, double *out_dev);
void axpy_multi_dev(Ctx &c, double *w, const float *V, int64_t ld, const int *k_dev,
                    const double *coef_dev, double sign);
void vec_scale_host(Ctx &c, float *y, const double *x, double s);  // y = (float)(s x)
void vec_widen(Ctx &c, double *y, const float *x);                 // y = (double) x
void vec_round_f32(Ctx &c, float *z32, double *z);  // z32 = (float) z, z = (double) z32
// Partial sums per dot product: a fixed count (not the SM count), so that the
// reduction order and hence every result is the same on any GPU; 608 is 4 per
// SM on a 152-SM part.
constexpr int kDotPartials = 608;
constexpr int kMaxBasis = 64;  // longest basis a Gram-Schmidt pass takes
int64_t cgs_partial_size(int64_t nunk, int kmax, int nsm);
void vec_axpby(Ctx &c, double *y, double a, const double *x, double b,
               int64_t n);                          // y = a x + b y
void norm2_dev(Ctx &c, const double *x, double *out_dev);

// api.cu (solver)
template <typename T>
void apply_saddle(Ctx &c, const double *x, double *y);
void k_bodies_in_launch(Ctx &c, const double *user, double *internal);  // [N][6] user -> internal order

// wavespace.cu (Brownian wave part): out (solution layout, bead rows) =
// M_w^(1/2) xi for the random field xi (field: complex [3][n][n][n/2+1] on the
// device, or null for the counter-based generator)
template <typename T>
void launch_brownian_wave(Ctx &c, const double *field, uint64_t seed, uint64_t step, double *out);

// brownian.cu
void brownian_sample(Ctx &c, double kT, double dt, uint64_t seed, uint64_t step,
                     const double *field_dev, const double *psi_r_dev, const double *psi_nf_dev,
                     int *iters_real, int *iters_nf,
                     double *change);  // fills bslip, bfnf; sets pending; change: last Lanczos step
void launch_brownian_rhs(Ctx &c, double *b);               // b += the pending Brownian terms
void brownian_outputs(Ctx &c, double *slip_user_dev, double *fnf_user_dev);  // scaled, user order

// graph.cu (device-resident solve)
void graph_launch(Ctx &c, const GraphRun &o);  // capture on first use of a key; launch on c.stream
double graph_finish(Ctx &c, KStats &st);       // wait; statistics; final relative residual
double *graph_ft_buffer(Ctx &c);               // device buffer [N][6] the graph reads forces from
void graph_cache_free(Ctx &c);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// count a kernel launch (every <<<>>> site is followed by this)
#define FSD_LAUNCHED(cx) (++(cx).launches)

void prof_collect(Ctx &c);  // fold finished event pairs into prof_ms

}  // namespace fsd
