// Device-resident solve of one time step (Algorithm 1 steps 4-5) as a single
// CUDA graph.  The restart cycles of the flexible GMRES, its Arnoldi steps and
// the sweeps of the FP64 iterative refinement are conditional WHILE / IF
// nodes; the Hessenberg least-squares problem (Givens rotations, triangular
// solve) runs in one-thread kernels on the device, so a whole solve needs no
// host round trip.  The arithmetic is the host-driven loop's, step for step:
// the same CGS2 passes, operator applications and update formulas.
//
// A graph is built per context and per launch key (precision, warm start,
// shear rate, presence of applied forces, integration step, and the buffer
// addresses and launch shapes that the geometry can change); a key change
// captures a new graph.
#include "fsd_internal.cuh"

#include <algorithm>
#include <climits>
#include <cstring>

namespace fsd {

constexpr int kMaxM = 60;  // longest restart the header allows

// Krylov state that lives in device memory for the whole solve.
struct GState {
  int j;          // Arnoldi index within the running cycle
  int total;      // Arnoldi steps in this solve
  int cyc_total;  // Arnoldi steps in the running GMRES call
  int cyc_max;    // limit of cyc_total
  int max_total;  // limit of total
  int m;          // restart length of the running GMRES
  int outer;      // refinement sweeps (mixed)
  int status;     // bit 0: NaN in the Krylov process
  int xnz;        // the iterate x is nonzero (its residual needs A x)
  int cont;       // the Arnoldi loop goes on
  int ky;         // length of the least-squares solution y
  int n_cycle, n_xnz, n_run;  // loop-body executions (launch accounting)
  int mv64, mv32;             // operator applications per precision
  double bnorm, tol, inner_tol, stoptol, beta, rel, scale, resid;
  double nrm;         // squared norm written by the reduction kernels
  double h[3 * 64];   // CGS outputs: first pass [64], second pass [64], ||w||^2
  double H[(kMaxM + 1) * kMaxM];
  double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
};

struct GraphKey {
  int mixed, warm, has_ft, integrate, with_str, group, lub, brown, add_vel, str_hydro, le;
  double shear, dt, brown_scale, tilt;
  const void *nbr, *lnbr, *bcol, *bval64, *bval32, *packed64, *packed32;
  int cap, lcap;
  int64_t nunk;
  bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // kernels captured per region, for the launch count of a run
  int64_t l_top = 0, l_cycle = 0, l_xnz = 0, l_run = 0, l_arn = 0;
};

struct GraphCache {
  DBuf<GState> state;
  GState *h_state = nullptr;  // pinned copy of the final state
  DBuf<double> vin, zf;       // fixed operand buffers of the Arnoldi step
  DBuf<double> ft;            // staged applied forces / torques [N][6] (user order)
  cudaStream_t cap_stream = nullptr;
  std::vector<GraphEntry> entries;  // most recent last
  bool warmed64 = false, warmed32 = false;
  ~GraphCache() {
    for (auto &e : entries) {
      if (e.exec) cudaGraphExecDestroy(e.exec);
      if (e.graph) cudaGraphDestroy(e.graph);
    }
    if (h_state) cudaFreeHost(h_state);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

void graph_cache_free(Ctx &c) {
  delete c.gcache;
  c.gcache = nullptr;
}

// ------------------------------------------------------------- kernels
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, bool v) {
  cudaGraphSetConditional(h, v ? 1u : 0u);
}

__global__ void k_g_reset(GState *s, int m, int cyc_max, int max_total, double tol,
                          double inner_tol, int xnz) {
  if (threadIdx.x | blockIdx.x) return;
  s->j = 0;
  s->total = 0;
  s->cyc_total = 0;
  s->cyc_max = cyc_max;
  s->max_total = max_total;
  s->m = m;
  s->outer = 0;
  s->status = 0;
  s->xnz = xnz;
  s->cont = 0;
  s->ky = 0;
  s->n_cycle = s->n_xnz = s->n_run = 0;
  s->mv64 = s->mv32 = 0;
  s->bnorm = 0.0;
  s->tol = tol;
  s->inner_tol = inner_tol;
  s->rel = 0.0;
}

// ||b|| from the reduction; with set != 0 arms the loop handle when b != 0.
__global__ void k_g_bnorm(GState *s, cudaGraphConditionalHandle h, int set) {
  if (threadIdx.x | blockIdx.x) return;
  const double bn = sqrt(fmax(0.0, s->nrm));
  s->bnorm = bn;
  if (!(bn == bn)) s->status |= 1;
  if (set) set_cond(h, bn > 0.0 && bn == bn);
}

// r = b - (x nonzero ? w : 0)
__global__ void k_g_residual(double *r, const double *__restrict__ b, const double *__restrict__ w,
                             const GState *s, int64_t n) {
  const bool sub = s->xnz != 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    r[i] = sub ? b[i] - w[i] : b[i];
}

__global__ void k_g_cycle_head(GState *s, cudaGraphConditionalHandle h_xnz) {
  if (threadIdx.x | blockIdx.x) return;
  s->n_cycle++;
  if (s->xnz) s->n_xnz++;
  set_cond(h_xnz, s->xnz != 0);
}

// Start of an FP64 restart cycle: residual norm, convergence test against the
// true residual, first Krylov vector scale, right-hand side of the small
// least-squares problem.
__global__ void k_g_cycle_begin(GState *s, cudaGraphConditionalHandle h_cycle,
                                cudaGraphConditionalHandle h_run) {
  if (threadIdx.x | blockIdx.x) return;
  const double beta = sqrt(fmax(0.0, s->nrm));
  if (s->xnz) s->mv64++;
  s->rel = beta / s->bnorm;
  if (!(beta == beta)) s->status |= 1;
  const bool stop = s->status != 0 || beta <= s->tol * s->bnorm || s->total >= s->max_total;
  set_cond(h_cycle, !stop);
  set_cond(h_run, !stop);
  if (stop) return;
  s->n_run++;
  s->beta = beta;
  s->scale = 1.0 / beta;
  s->g[0] = beta;
  for (int i = 1; i <= s->m; ++i) s->g[i] = 0.0;
  s->j = 0;
  s->cyc_total = 0;
  s->stoptol = s->tol * s->bnorm;
  s->resid = beta;
}

// Mixed path: relative residual of the FP64 refinement and the sweep test.
__global__ void k_g_outer_check(GState *s, cudaGraphConditionalHandle h_outer, int first) {
  if (threadIdx.x | blockIdx.x) return;
  const double rn = sqrt(fmax(0.0, s->nrm));
  if (!first) {
    s->mv64++;
    s->outer++;
  } else if (s->xnz) {
    s->mv64++;
  }
  if (s->bnorm == 0.0) {
    s->rel = 0.0;
    set_cond(h_outer, false);
    return;
  }
  s->rel = rn / s->bnorm;
  if (!(rn == rn)) s->status |= 1;
  const bool go = s->status == 0 && s->rel > s->tol && s->total < s->max_total && s->outer < 50;
  s->beta = rn;
  set_cond(h_outer, go);
}

// Mixed path: one FP32-operator GMRES cycle solving A d = r to a relative
// tolerance that only has to close the remaining gap to tol.
__global__ void k_g_inner_begin(GState *s, cudaGraphConditionalHandle h_arn) {
  if (threadIdx.x | blockIdx.x) return;
  const double rn = s->beta;
  const double itol = fmax(s->inner_tol, 0.3 * s->tol / s->rel);
  s->n_run++;
  s->stoptol = itol * rn;
  s->scale = 1.0 / rn;
  s->g[0] = rn;
  for (int i = 1; i <= s->m; ++i) s->g[i] = 0.0;
  s->j = 0;
  s->cyc_total = 0;
  s->resid = rn;
  set_cond(h_arn, true);
}

// y = scale * x (scale from the state; y in the basis precision B); the
// first thread arms a handle.
template <typename B>
__global__ void k_g_scale(B *y, const double *x, const GState *s, int64_t n,
                          cudaGraphConditionalHandle h, int arm) {
  if (arm && (threadIdx.x | blockIdx.x) == 0) set_cond(h, true);
  const double sc = s->scale;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = (B)(x[i] * sc);
}

// out = V_j (widened to FP64), with j read from the state
template <typename B>
__global__ void k_g_get_col(double *out, const B *__restrict__ V, int64_t ld, const GState *s,
                            int64_t n) {
  const B *v = V + (int64_t)s->j * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (double)v[i];
}

// Z_j = in; with an FP32 basis in is rounded to the stored value, so that the
// operator is applied to the vector that the update x += Z y uses
template <typename B>
__global__ void k_g_put_col(B *Z, int64_t ld, double *in, const GState *s, int64_t n) {
  B *z = Z + (int64_t)s->j * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const B v = (B)in[i];
    z[i] = v;
    if constexpr (sizeof(B) == 4) in[i] = (double)v;
  }
}

// Hessenberg column j from the two Gram-Schmidt passes, the earlier Givens
// rotations applied to it, a new rotation that zeroes h_{j+1,j}, and the
// stopping test of the Arnoldi loop.
__global__ void k_g_givens(GState *s, cudaGraphConditionalHandle h_arn, int is64) {
  if (threadIdx.x | blockIdx.x) return;
  const int j = s->j, m = s->m;
  double *H = s->H;
  for (int i = 0; i <= j; ++i) H[i * m + j] = s->h[i] + s->h[64 + i];
  const double hnext = sqrt(fmax(0.0, s->h[128]));
  if (is64)
    s->mv64++;
  else
    s->mv32++;
  if (!(hnext == hnext)) {
    s->status |= 1;
    s->cont = 0;
    set_cond(h_arn, false);
    return;
  }
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = s->cs[i] * a + s->sn[i] * b;
    H[(i + 1) * m + j] = -s->sn[i] * a + s->cs[i] * b;
  }
  const double a = H[j * m + j];
  const double den = hypot(a, hnext);
  s->cs[j] = den > 0 ? a / den : 1.0;
  s->sn[j] = den > 0 ? hnext / den : 0.0;
  H[j * m + j] = den;
  s->g[j + 1] = -s->sn[j] * s->g[j];
  s->g[j] = s->cs[j] * s->g[j];
  const double resid = fabs(s->g[j + 1]);
  s->resid = resid;
  s->j = j + 1;
  s->total++;
  s->cyc_total++;
  const bool stop = resid <= s->stoptol || hnext <= 1e-300 || s->j >= m ||
                    s->total >= s->max_total || s->cyc_total >= s->cyc_max;
  s->cont = stop ? 0 : 1;
  s->scale = stop ? 0.0 : 1.0 / hnext;
  set_cond(h_arn, !stop);
}

// V_j = w / h_{j,j-1} when the loop goes on
template <typename B>
__global__ void k_g_next_col(B *V, int64_t ld, const double *__restrict__ w, const GState *s,
                             int64_t n) {
  if (!s->cont) return;
  B *v = V + (int64_t)s->j * ld;
  const double sc = s->scale;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    v[i] = (B)(w[i] * sc);
}

// y = R^-1 g, R the rotated j x j upper triangle
__global__ void k_g_trisolve(GState *s) {
  if (threadIdx.x | blockIdx.x) return;
  const int jj = s->j, m = s->m;
  for (int i = jj - 1; i >= 0; --i) {
    double v = s->g[i];
    for (int k = i + 1; k < jj; ++k) v -= s->H[i * m + k] * s->y[k];
    s->y[i] = v / s->H[i * m + i];
  }
  s->ky = jj;
  s->xnz = 1;
}

__global__ void k_g_zero_if_b0(double *x, const GState *s, int64_t n) {
  if (s->bnorm != 0.0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = 0.0;
}

__global__ void k_g_nan_check(const double *__restrict__ x, int64_t n, int *flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (!(fabs(x[i]) <= 1e300)) atomicOr(flag, 1);
}

// ------------------------------------------------------------- capture
using Deps = std::vector<cudaGraphNode_t>;

static void cap_begin(Ctx &c, cudaGraph_t g, const Deps &d) {
  FSD_CUDA(cudaStreamBeginCaptureToGraph(c.stream, g, d.empty() ? nullptr : d.data(), nullptr,
                                         d.size(), cudaStreamCaptureModeThreadLocal));
}

static Deps cap_end(Ctx &c) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  FSD_CUDA(cudaStreamGetCaptureInfo(c.stream, &st, nullptr, nullptr, &deps, nullptr, &nd));
  Deps out(deps, deps + nd);
  cudaGraph_t g = nullptr;
  FSD_CUDA(cudaStreamEndCapture(c.stream, &g));
  return out;
}

// A conditional node after `deps` in g; deps becomes {node}; returns its body.
static cudaGraph_t add_cond(cudaGraph_t g, Deps &deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  FSD_CUDA(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
  deps.assign(1, node);
  return p.conditional.phGraph_out[0];
}

static cudaGraphConditionalHandle new_handle(cudaGraph_t g) {
  cudaGraphConditionalHandle h;
  FSD_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  return h;
}

static int vec_blocks(const Ctx &c, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)c.num_sms));
}

// Krylov bases by element type: FP64, or FP32 for the inner GMRES of a mixed
// solve with FSD_FLAG_FP32_KRYLOV.
static double *basis_v(Ctx &c, double) { return c.V.p; }
static float *basis_v(Ctx &c, float) { return c.V32.p; }
static double *basis_z(Ctx &c, double) { return c.Z.p; }
static float *basis_z(Ctx &c, float) { return c.Z32.p; }

// One Arnoldi step of the flexible GMRES on the operator of precision T with
// basis element type B: z_j = P^-1 v_j, w = A z_j, CGS2 against V_0..V_j,
// Givens update, v_{j+1}.
template <typename T, typename B>
static void arnoldi_step(Ctx &c, GState *s, cudaGraphConditionalHandle h_arn) {
  GraphCache &gc = *c.gcache;
  const int64_t ld = c.nunk, n = c.nunk;
  const int nb = vec_blocks(c, n);
  const int mm = sizeof(T) == 8 ? c.m : c.m_in;
  B *V = basis_v(c, B()), *Z = basis_z(c, B());
  if constexpr (sizeof(B) == 8) {
    // z_j = P^-1 v_j straight from and into the bases (column j read on the
    // device), and into the operator's fixed input buffer
    launch_precond_col(c, V, Z, ld, &s->j, gc.zf.p);
  } else {
    k_g_get_col<B><<<nb, 256, 0, c.stream>>>(gc.vin.p, V, ld, s, n);
    FSD_LAUNCHED(c);
    launch_precond(c, gc.vin.p, gc.zf.p);
    k_g_put_col<B><<<nb, 256, 0, c.stream>>>(Z, ld, gc.zf.p, s, n);
    FSD_LAUNCHED(c);
  }
  apply_saddle<T>(c, gc.zf.p, c.w.p);
  cgs_pass_dev(c, 0, V, ld, &s->j, 1, mm, c.w.p, nullptr, s->h);
  cgs_pass_dev(c, 1, V, ld, &s->j, 1, mm, c.w.p, s->h, s->h + 64);
  cgs_pass_dev(c, 2, V, ld, &s->j, 1, mm, c.w.p, s->h + 64, s->h + 128);
  k_g_givens<<<1, 32, 0, c.stream>>>(s, h_arn, sizeof(T) == 8 ? 1 : 0);
  FSD_LAUNCHED(c);
  k_g_next_col<B><<<nb, 256, 0, c.stream>>>(V, ld, c.w.p, s, n);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// x += Z y after a cycle (Z of element type B)
template <typename B>
static void cycle_update(Ctx &c, GState *s, double *x) {
  k_g_trisolve<<<1, 32, 0, c.stream>>>(s);
  FSD_LAUNCHED(c);
  axpy_multi_dev(c, x, basis_z(c, B()), c.nunk, &s->ky, s->y, 1.0);
}

// The captured solve of A x = b into c.xsol (b = c.rhs).  Appends to graph g
// after deps and returns the new tail.
static Deps capture_solve(Ctx &c, GraphEntry &e, cudaGraph_t g, Deps deps, bool warm) {
  GraphCache &gc = *c.gcache;
  GState *s = gc.state.p;
  const int64_t n = c.nunk;
  const int nb = vec_blocks(c, n);
  double *x = c.xsol.p, *b = c.rhs.p, *w = c.w.p;
  const bool mixed = c.prm.precision == FSD_MIXED;
  int64_t l0;
  // ---- set-up: x0, state, ||b||
  cap_begin(c, g, deps);
  l0 = c.launches;
  if (warm)
    FSD_CUDA(cudaMemcpyAsync(x, c.xprev.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  else
    FSD_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), c.stream));
  const int m = mixed ? c.m_in : c.m;
  k_g_reset<<<1, 32, 0, c.stream>>>(s, m, mixed ? c.m_in : INT_MAX, c.prm.max_iter, c.prm.tol,
                                     c.prm.inner_tol, warm ? 1 : 0);
  FSD_LAUNCHED(c);
  norm2_dev(c, b, &s->nrm);
  if (!mixed) {
    // ============ FP64: restarted FGMRES, true residual at every restart
    cudaGraphConditionalHandle h_cycle = new_handle(g);
    k_g_bnorm<<<1, 32, 0, c.stream>>>(s, h_cycle, 1);
    FSD_LAUNCHED(c);
    e.l_top += c.launches - l0;
    deps = cap_end(c);
    cudaGraph_t cyc = add_cond(g, deps, h_cycle, cudaGraphCondTypeWhile);
    {
      Deps d;
      cudaGraphConditionalHandle h_xnz = new_handle(cyc);
      cap_begin(c, cyc, d);
      l0 = c.launches;
      k_g_cycle_head<<<1, 32, 0, c.stream>>>(s, h_xnz);
      FSD_LAUNCHED(c);
      e.l_cycle += c.launches - l0;
      d = cap_end(c);
      cudaGraph_t xb = add_cond(cyc, d, h_xnz, cudaGraphCondTypeIf);
      {
        cap_begin(c, xb, {});
        l0 = c.launches;
        apply_saddle<double>(c, x, w);
        e.l_xnz += c.launches - l0;
        cap_end(c);
      }
      cudaGraphConditionalHandle h_run = new_handle(cyc);
      cap_begin(c, cyc, d);
      l0 = c.launches;
      k_g_residual<<<nb, 256, 0, c.stream>>>(c.V.p, b, w, s, n);
      FSD_LAUNCHED(c);
      norm2_dev(c, c.V.p, &s->nrm);
      k_g_cycle_begin<<<1, 32, 0, c.stream>>>(s, h_cycle, h_run);
      FSD_LAUNCHED(c);
      e.l_cycle += c.launches - l0;
      d = cap_end(c);
      cudaGraph_t run = add_cond(cyc, d, h_run, cudaGraphCondTypeIf);
      {
        Deps r;
        cudaGraphConditionalHandle h_arn = new_handle(run);
        cap_begin(c, run, r);
        l0 = c.launches;
        k_g_scale<double><<<nb, 256, 0, c.stream>>>(c.V.p, c.V.p, s, n, h_arn, 1);
        FSD_LAUNCHED(c);
        e.l_run += c.launches - l0;
        r = cap_end(c);
        cudaGraph_t arn = add_cond(run, r, h_arn, cudaGraphCondTypeWhile);
        {
          cap_begin(c, arn, {});
          l0 = c.launches;
          arnoldi_step<double, double>(c, s, h_arn);
          e.l_arn += c.launches - l0;
          cap_end(c);
        }
        cap_begin(c, run, r);
        l0 = c.launches;
        cycle_update<double>(c, s, x);
        e.l_run += c.launches - l0;
        cap_end(c);
      }
    }
  } else {
    // ============ mixed: FP64 iterative refinement, one FP32-operator
    //              FGMRES cycle per sweep
    k_g_bnorm<<<1, 32, 0, c.stream>>>(s, 0, 0);
    FSD_LAUNCHED(c);
    if (warm) apply_saddle<double>(c, x, w);
    k_g_residual<<<nb, 256, 0, c.stream>>>(c.res.p, b, w, s, n);
    FSD_LAUNCHED(c);
    norm2_dev(c, c.res.p, &s->nrm);
    cudaGraphConditionalHandle h_outer = new_handle(g);
    k_g_outer_check<<<1, 32, 0, c.stream>>>(s, h_outer, 1);
    FSD_LAUNCHED(c);
    e.l_top += c.launches - l0;
    deps = cap_end(c);
    cudaGraph_t outer = add_cond(g, deps, h_outer, cudaGraphCondTypeWhile);
    {
      Deps d;
      cudaGraphConditionalHandle h_arn = new_handle(outer);
      cap_begin(c, outer, d);
      l0 = c.launches;
      k_g_inner_begin<<<1, 32, 0, c.stream>>>(s, h_arn);
      FSD_LAUNCHED(c);
      if (c.krylov32)
        k_g_scale<float><<<nb, 256, 0, c.stream>>>(c.V32.p, c.res.p, s, n, 0, 0);
      else
        k_g_scale<double><<<nb, 256, 0, c.stream>>>(c.V.p, c.res.p, s, n, 0, 0);
      FSD_LAUNCHED(c);
      e.l_run += c.launches - l0;
      d = cap_end(c);
      cudaGraph_t arn = add_cond(outer, d, h_arn, cudaGraphCondTypeWhile);
      {
        cap_begin(c, arn, {});
        l0 = c.launches;
        if (c.krylov32)
          arnoldi_step<float, float>(c, s, h_arn);
        else
          arnoldi_step<float, double>(c, s, h_arn);
        e.l_arn += c.launches - l0;
        cap_end(c);
      }
      cap_begin(c, outer, d);
      l0 = c.launches;
      if (c.krylov32)
        cycle_update<float>(c, s, x);
      else
        cycle_update<double>(c, s, x);
      apply_saddle<double>(c, x, w);
      k_g_residual<<<nb, 256, 0, c.stream>>>(c.res.p, b, w, s, n);
      FSD_LAUNCHED(c);
      norm2_dev(c, c.res.p, &s->nrm);
      k_g_outer_check<<<1, 32, 0, c.stream>>>(s, h_outer, 0);
      FSD_LAUNCHED(c);
      e.l_run += c.launches - l0;
      cap_end(c);
    }
  }
  // ---- b == 0: x = 0
  cap_begin(c, g, deps);
  l0 = c.launches;
  k_g_zero_if_b0<<<nb, 256, 0, c.stream>>>(x, s, n);
  FSD_LAUNCHED(c);
  e.l_top += c.launches - l0;
  return cap_end(c);
}

static GraphKey make_key(Ctx &c, const GraphRun &o) {
  GraphKey k;
  std::memset(&k, 0, sizeof(k));
  k.mixed = c.prm.precision == FSD_MIXED;
  k.warm = o.warm;
  k.has_ft = o.has_ft;
  k.integrate = o.integrate;
  k.with_str = o.with_str;
  k.group = realspace_group(c);
  k.lub = c.n_lub > 0;
  k.shear = o.shear;
  k.dt = o.integrate ? o.dt : 0.0;
  k.brown = o.brown;
  k.brown_scale = o.brown ? o.brown_scale : 0.0;
  k.add_vel = o.add_vel;
  // a Lees-Edwards context's kernels read the offset from device memory: one
  // graph serves every offset
  k.le = tilt_dev_ptr(c) != nullptr;
  k.tilt = k.le ? 0.0 : c.tilt;
  k.str_hydro = o.str_hydro;
  k.nbr = c.nbr.p;
  k.lnbr = c.lnbr.p;
  k.bcol = c.bcol.p;
  k.bval64 = c.op64.bval.p;
  k.bval32 = c.op32.bval.p;
  k.packed64 = c.op64.packed.p;
  k.packed32 = c.op32.packed.p;
  k.cap = c.cap;
  k.lcap = c.lcap;
  k.nunk = c.nunk;
  return k;
}

static void ensure_cache(Ctx &c) {
  if (c.gcache) return;
  c.gcache = new GraphCache();
  GraphCache &gc = *c.gcache;
  gc.state.alloc(1);
  FSD_CUDA(cudaMemset(gc.state.p, 0, sizeof(GState)));
  FSD_CUDA(cudaMallocHost(&gc.h_state, sizeof(GState)));
  gc.vin.alloc(c.nunk);
  gc.zf.alloc(c.nunk);
  gc.ft.alloc(6 * (size_t)c.N);
  FSD_CUDA(cudaStreamCreateWithFlags(&gc.cap_stream, cudaStreamNonBlocking));
}

double *graph_ft_buffer(Ctx &c) {
  ensure_cache(c);
  return c.gcache->ft.p;
}

// Capture the whole step for key k (current launch shapes and buffers).
static GraphEntry &build_entry(Ctx &c, const GraphRun &o, const GraphKey &k) {
  GraphCache &gc = *c.gcache;
  if (gc.entries.size() >= 4) {
    GraphEntry &old = gc.entries.front();
    if (old.exec) cudaGraphExecDestroy(old.exec);
    if (old.graph) cudaGraphDestroy(old.graph);
    gc.entries.erase(gc.entries.begin());
  }
  gc.entries.emplace_back();
  GraphEntry &e = gc.entries.back();
  e.key = k;
  FSD_CUDA(cudaGraphCreate(&e.graph, 0));
  cudaStream_t user = c.stream;
  c.stream = gc.cap_stream;
  try {
    Deps deps;
    const int64_t l0 = c.launches;
    cap_begin(c, e.graph, deps);
    if (o.has_ft) {
      k_bodies_in_launch(c, gc.ft.p, c.t2.p);
    }
    launch_rhs(c, o.has_ft ? c.t2.p : nullptr, o.shear, c.rhs.p);
    if (o.brown) launch_brownian_rhs(c, c.rhs.p);
    e.l_top += c.launches - l0;
    deps = cap_end(c);
    deps = capture_solve(c, e, e.graph, deps, o.warm);
    cap_begin(c, e.graph, deps);
    const int64_t l1 = c.launches;
    FSD_CUDA(cudaMemcpyAsync(c.xprev.p, c.xsol.p, c.nunk * sizeof(double), cudaMemcpyDeviceToDevice,
                             c.stream));
    launch_outputs(c, c.xsol.p, o.shear, c.t1.p, o.with_str ? c.res.p : nullptr);
    if (o.add_vel) launch_add_velocity(c, c.t1.p);
    FSD_CUDA(cudaMemsetAsync(c.flags.p + 6, 0, sizeof(int), c.stream));
    k_g_nan_check<<<c.num_sms, 256, 0, c.stream>>>(c.t1.p, 6 * (int64_t)c.N, c.flags.p + 6);
    FSD_LAUNCHED(c);
    if (o.integrate) {
      launch_integrate(c, c.t1.p, o.dt, o.shear);
      launch_wrap_positions(c);
    }
    FSD_CUDA(cudaMemcpyAsync(c.h_flags, c.flags.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    FSD_CUDA(cudaMemcpyAsync(gc.h_state, gc.state.p, sizeof(GState), cudaMemcpyDeviceToHost, c.stream));
    e.l_top += c.launches - l1;
    cap_end(c);
    c.launches = l0;
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(c.stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c.stream, &g);
    }
    c.stream = user;
    cudaGraphDestroy(e.graph);
    gc.entries.pop_back();
    throw;
  }
  c.stream = user;
  FSD_CUDA(cudaGraphInstantiate(&e.exec, e.graph, 0));
  return e;
}

void graph_launch(Ctx &c, const GraphRun &o) {
  ensure_cache(c);
  GraphCache &gc = *c.gcache;
  // Lazily sized buffers and cached launch attributes of the operator
  // kernels are settled by one eager application per precision before the
  // key (which holds their addresses) is taken.
  const bool mixed = c.prm.precision == FSD_MIXED;
  if (!gc.warmed64 || (mixed && !gc.warmed32)) {
    apply_saddle<double>(c, c.xsol.p, c.w.p);
    if (mixed) apply_saddle<float>(c, c.xsol.p, c.w.p);
    FSD_CUDA(cudaStreamSynchronize(c.stream));
    gc.warmed64 = true;
    gc.warmed32 = gc.warmed32 || mixed;
  }
  const GraphKey k = make_key(c, o);
  GraphEntry *e = nullptr;
  for (auto &x : gc.entries)
    if (x.key == k) e = &x;
  if (!e) {
    // a new launch shape may meet a kernel attribute not yet set: settle it
    // outside the capture
    apply_saddle<double>(c, c.xsol.p, c.w.p);
    if (mixed) apply_saddle<float>(c, c.xsol.p, c.w.p);
    FSD_CUDA(cudaStreamSynchronize(c.stream));
    e = &build_entry(c, o, k);
  }
  FSD_CUDA(cudaGraphLaunch(e->exec, c.stream));
  c.graph_pending = e - gc.entries.data();
}

// Wait for the launched graph; fill the Krylov statistics; return the final
// relative residual.
double graph_finish(Ctx &c, KStats &st) {
  GraphCache &gc = *c.gcache;
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  const GraphEntry &e = gc.entries[c.graph_pending];
  const GState &s = *gc.h_state;
  if (s.status & 1) throw Invalid{"NaN in the Krylov process"};
  st.iters = s.total;
  st.m64 = s.mv64;
  st.m32 = s.mv32;
  st.outer = c.prm.precision == FSD_MIXED ? s.outer : 1;
  c.launches += e.l_top + (int64_t)s.n_cycle * e.l_cycle + (int64_t)s.n_xnz * e.l_xnz +
                (int64_t)s.n_run * e.l_run + (int64_t)s.total * e.l_arn;
  return s.rel;
}

}  // namespace fsd
