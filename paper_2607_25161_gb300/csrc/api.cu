// C ABI of the FSD library (include/fsd.h): set-up (Algorithm 1 step 1
// data), the saddle-point solve (step 4: GMRES with the block-triangular
// preconditioner of Table 1), the rigid-body step (step 5), and operator
// access.  Host orchestration only; every arithmetic step of the path runs in
// the CUDA kernels of realspace.cu, wavespace.cu, nearfield.cu, krylov.cu.
#include "fsd_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>

struct fsd_ctx {
  fsd::Ctx c;
};

// Independent suspensions solved together: one context (and stream) per
// system; every system's step is one captured graph, and all systems' graphs
// are in flight at once.
struct fsd_batch {
  std::vector<fsd_ctx *> sys;
  std::vector<int64_t> bead_off, agg_off;
  std::vector<int> order;  // launch order: most expensive system first
  cudaStream_t user = nullptr;
  cudaEvent_t ev_user = nullptr;
  std::vector<cudaEvent_t> ev_done;
  std::string last_error;
  int host_threads = 8;  // launch-phase threads
};

namespace fsd {

bool fft_size_ok(int n);
void vec_scale_host(Ctx &c, double *y, const double *x, double s);

static thread_local std::string g_setup_error;

static const char *kProfNames[PG_COUNT] = {"realspace", "spread", "fft_green", "interp",
                                           "body_rows", "precond", "krylov", "neighbors",
                                           "lub_assembly", "misc"};

static cudaEvent_t prof_event(Ctx &c) {
  if (!c.ev_pool.empty()) {
    cudaEvent_t e = c.ev_pool.back();
    c.ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

ProfScope::ProfScope(Ctx &cx, int grp) : c(&cx), g(grp) {
  if (!c->prof) return;
  e0 = prof_event(*c);
  if (e0) cudaEventRecord(e0, c->stream);
}

ProfScope::~ProfScope() {
  if (!c->prof || !e0) return;
  cudaEvent_t e1 = prof_event(*c);
  if (!e1) return;
  cudaEventRecord(e1, c->stream);
  c->ev_pending.push_back({g, {e0, e1}});
}

void prof_collect(Ctx &c) {
  for (auto &pr : c.ev_pending) {
    cudaEventSynchronize(pr.second.second);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.second.first, pr.second.second) == cudaSuccess) {
      c.prof_ms[pr.first] += ms;
      c.prof_n[pr.first] += 1;
    }
    c.ev_pool.push_back(pr.second.first);
    c.ev_pool.push_back(pr.second.second);
  }
  c.ev_pending.clear();
}

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ permutations
__global__ void k_beads_in(int Nt, const int *__restrict__ perm, const double *__restrict__ user,
                           double *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double *u = user + 11 * (size_t)perm[i];
  double *o = x + (size_t)i * LDB;
  for (int k = 0; k < 11; ++k) o[k] = u[k];
  o[11] = 0.0;
}
__global__ void k_beads_out(int Nt, const int *__restrict__ perm, const double *__restrict__ x,
                            double *user) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  double *u = user + 11 * (size_t)perm[i];
  const double *o = x + (size_t)i * LDB;
  for (int k = 0; k < 11; ++k) u[k] = o[k];
}
__global__ void k_bodies_in(int N, const int *__restrict__ perm, const double *__restrict__ user,
                            double *x, int w) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  for (int k = 0; k < w; ++k) x[(size_t)w * J + k] = user[(size_t)w * perm[J] + k];
}
__global__ void k_bodies_out(int N, const int *__restrict__ perm, const double *__restrict__ x,
                             double *user, int w) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  for (int k = 0; k < w; ++k) user[(size_t)w * perm[J] + k] = x[(size_t)w * J + k];
}
void k_bodies_in_launch(Ctx &c, const double *user, double *internal) {
  k_bodies_in<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, user, internal, 6);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}
__global__ void k_bead_pos_out(int Nt, const int *__restrict__ perm,
                               const int *__restrict__ bead_body, const double *__restrict__ X,
                               const double4 *__restrict__ lever, double *user) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const int J = bead_body[i];
  const double4 r = lever[i];
  double *u = user + 3 * (size_t)perm[i];
  u[0] = X[3 * J] + r.x;
  u[1] = X[3 * J + 1] + r.y;
  u[2] = X[3 * J + 2] + r.z;
}
__global__ void k_nan_check(const double *__restrict__ x, int64_t n, int *flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (!(fabs(x[i]) <= 1e300)) atomicOr(flag, 1);
}

// Host or device input of `bytes` -> a device pointer (staged in `buf` when host).
static const double *dev_in(Ctx &c, const double *p, size_t count, DBuf<double> &buf) {
  if (!p) return nullptr;
  if (is_device_ptr(p)) return p;
  if (buf.n < count) buf.alloc(count);
  FSD_CUDA(cudaMemcpyAsync(buf.p, p, count * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  return buf.p;
}

// ------------------------------------------------------------------ solver
template <typename T>
void apply_saddle(Ctx &c, const double *x, double *y) {
  if (!c.overlap || c.prof) {
    launch_realspace<T>(c, x, y, true, false);
    launch_wavespace<T>(c, x, y);
  } else {
    // the real-space sum on the second stream, the wave-space chain into yw
    // on this one; joined before the sum and the aggregate rows (in a
    // captured graph these are two parallel branches)
    const int64_t nb = (int64_t)LDB * c.Nt;
    FSD_CUDA(cudaEventRecord(c.ev_fork, c.stream));
    FSD_CUDA(cudaStreamWaitEvent(c.stream2, c.ev_fork, 0));
    cudaStream_t main = c.stream;
    c.stream = c.stream2;
    c.rs_overlapped = true;
    try {
      launch_realspace<T>(c, x, y, true, false);
    } catch (...) {
      c.stream = main;
      c.rs_overlapped = false;
      throw;
    }
    c.rs_overlapped = false;
    FSD_CUDA(cudaEventRecord(c.ev_join, c.stream2));
    c.stream = main;
    FSD_CUDA(cudaMemsetAsync(c.yw.p, 0, nb * sizeof(double), c.stream));
    launch_wavespace<T>(c, x, c.yw.p);
    FSD_CUDA(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
    launch_axpy(c, c.yw.p, y, nb);
  }
  launch_body_rows<T>(c, x, y, true);
}
template void apply_saddle<float>(Ctx &, const double *, double *);
template void apply_saddle<double>(Ctx &, const double *, double *);

static double host_norm(Ctx &c, const double *x) {
  double *d = c.hcol.p + 200;
  norm2_dev(c, x, d);
  FSD_CUDA(cudaMemcpyAsync(c.h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  return std::sqrt(std::max(0.0, c.h_pinned[0]));
}

// Krylov bases by element type: FP64, or FP32 for the inner GMRES of a mixed
// solve with FSD_FLAG_FP32_KRYLOV.
template <typename T> static T *krylov_v(Ctx &c);
template <> double *krylov_v<double>(Ctx &c) { return c.V.p; }
template <> float *krylov_v<float>(Ctx &c) { return c.V32.p; }
template <typename T> static T *krylov_z(Ctx &c);
template <> double *krylov_z<double>(Ctx &c) { return c.Z.p; }
template <> float *krylov_z<float>(Ctx &c) { return c.Z32.p; }

// Right-preconditioned restarted flexible GMRES (Z stores P^-1 v_j), CGS2
// Arnoldi, Givens rotations on the host.  The operator precision is T; the
// basis element type B is FP64 (Arnoldi in FP64), or FP32 for the inner solve
// of a mixed path with FSD_FLAG_FP32_KRYLOV (its basis vectors are widened to
// FP64 for the preconditioner, and the operator is applied to the FP32 value
// of z_j that the update x += Z y uses).  Solves A x = b from x (x_zero:
// x = 0).  Stops when the residual is below tol * bnorm (the true residual
// when true_check), or after max_iter iterations.  Returns the last residual
// / bnorm.
template <typename T, typename B>
static double gmres(Ctx &c, const double *b, double *x, double bnorm, double tol, int max_iter,
                    int m, bool x_zero, bool true_check, KStats &st) {
  constexpr bool f64 = sizeof(T) == 8;
  const int64_t ld = c.nunk;
  B *V = krylov_v<B>(c), *Z = krylov_z<B>(c);
  double *w = c.w.p;
  int total = 0;
  double rel = 1.0;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1);
  while (true) {
    const double *r = b;
    if (!x_zero) {
      // w = b - A x
      apply_saddle<T>(c, x, w);
      (f64 ? st.m64 : st.m32)++;
      vec_axpby(c, w, 1.0, b, -1.0, ld);
      r = w;
    }
    const double beta = host_norm(c, r);
    rel = beta / bnorm;
    if (!(beta == beta)) throw Invalid{"NaN in the Krylov residual"};
    if (beta <= tol * bnorm || total >= max_iter) return rel;
    vec_scale_host(c, V, r, 1.0 / beta);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    double resid = beta;
    for (; j < m && total < max_iter;) {
      if constexpr (sizeof(B) == 8) {
        double *vj = V + (int64_t)j * ld, *zj = Z + (int64_t)j * ld;
        launch_precond(c, vj, zj);
        apply_saddle<T>(c, zj, w);
      } else {
        vec_widen(c, c.kv.p, V + (int64_t)j * ld);
        launch_precond(c, c.kv.p, c.kz.p);
        vec_round_f32(c, Z + (int64_t)j * ld, c.kz.p);
        apply_saddle<T>(c, c.kz.p, w);
      }
      (f64 ? st.m64 : st.m32)++;
      double *h1 = c.hcol.p, *h2 = c.hcol.p + 64, *hn = c.hcol.p + 128;
      // classical Gram-Schmidt applied twice, three fused passes over V
      cgs_pass(c, 0, V, ld, j + 1, w, nullptr, h1);
      cgs_pass(c, 1, V, ld, j + 1, w, h1, h2);
      cgs_pass(c, 2, V, ld, j + 1, w, h2, hn);
      FSD_CUDA(cudaMemcpyAsync(c.h_pinned, c.hcol.p, 192 * sizeof(double),
                               cudaMemcpyDeviceToHost, c.stream));
      FSD_CUDA(cudaStreamSynchronize(c.stream));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = c.h_pinned[i] + c.h_pinned[64 + i];
      const double hnext = std::sqrt(std::max(0.0, c.h_pinned[128]));
      if (!(hnext == hnext)) throw Invalid{"NaN in the Arnoldi process"};
      // Givens
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[(size_t)j * m + j];
      double den = std::hypot(a, hnext);
      cs[j] = den > 0 ? a / den : 1.0;
      sn[j] = den > 0 ? hnext / den : 0.0;
      H[(size_t)j * m + j] = den;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      resid = std::fabs(g[j + 1]);
      ++j;
      ++total;
      ++st.iters;
      if (resid <= tol * bnorm || hnext <= 1e-300) break;
      if (j < m) vec_scale_host(c, V + (int64_t)j * ld, w, 1.0 / hnext);
    }
    // y = H^-1 g (upper triangular j x j); x += Z y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
      y[i] = s / H[(size_t)i * m + i];
    }
    if (x_zero) FSD_CUDA(cudaMemsetAsync(x, 0, ld * sizeof(double), c.stream));
    std::memcpy(c.h_pinned + 256, y.data(), j * sizeof(double));
    FSD_CUDA(cudaMemcpyAsync(c.hcol.p + 256, c.h_pinned + 256, j * sizeof(double),
                             cudaMemcpyHostToDevice, c.stream));
    axpy_multi(c, x, Z, ld, j, c.hcol.p + 256, 1.0);
    x_zero = false;
    rel = resid / bnorm;
    if (resid <= tol * bnorm && !true_check) {
      FSD_CUDA(cudaStreamSynchronize(c.stream));
      return rel;
    }
    if (total >= max_iter && !true_check) {
      FSD_CUDA(cudaStreamSynchronize(c.stream));
      return rel;
    }
  }
}

// Solve A x = b.  FP64: restarted GMRES on the FP64 operator.  Mixed: FP64
// iterative refinement; each correction from GMRES on the FP32 operator
// (FP64 Arnoldi, Hessenberg, Givens rotations and LU; FP32 Krylov bases with
// FSD_FLAG_FP32_KRYLOV), each residual from the FP64 operator.
static double solve_system(Ctx &c, const double *b, double *x, KStats &st, bool warm) {
  const int64_t ld = c.nunk;
  const double bnorm = host_norm(c, b);
  if (bnorm == 0.0) {
    FSD_CUDA(cudaMemsetAsync(x, 0, ld * sizeof(double), c.stream));
    return 0.0;
  }
  const double tol = c.prm.tol;
  if (c.prm.precision == FSD_FP64) {
    if (warm) FSD_CUDA(cudaMemcpyAsync(x, c.xprev.p, ld * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    double rel = gmres<double, double>(c, b, x, bnorm, tol, c.prm.max_iter, c.m, !warm, true, st);
    st.outer = 1;
    return rel;
  }
  double *r = c.res.p, *d = c.t1.p;
  if (warm) {
    FSD_CUDA(cudaMemcpyAsync(x, c.xprev.p, ld * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    apply_saddle<double>(c, x, c.w.p);
    st.m64++;
    FSD_CUDA(cudaMemcpyAsync(r, b, ld * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    vec_axpby(c, r, -1.0, c.w.p, 1.0, ld);
  } else {
    FSD_CUDA(cudaMemsetAsync(x, 0, ld * sizeof(double), c.stream));
    FSD_CUDA(cudaMemcpyAsync(r, b, ld * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  }
  double rel = host_norm(c, r) / bnorm;
  const int max_outer = 50;
  while (rel > tol && st.iters < c.prm.max_iter && st.outer < max_outer) {
    const double rn = rel * bnorm;
    // the correction only has to close the remaining gap to tol
    const double itol = std::max(c.prm.inner_tol, 0.3 * tol / rel);
    if (c.krylov32)
      gmres<float, float>(c, r, d, rn, itol, c.m_in, c.m_in, true, false, st);
    else
      gmres<float, double>(c, r, d, rn, itol, c.m_in, c.m_in, true, false, st);
    vec_axpby(c, x, 1.0, d, 1.0, ld);
    apply_saddle<double>(c, x, c.w.p);
    st.m64++;
    FSD_CUDA(cudaMemcpyAsync(r, b, ld * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    vec_axpby(c, r, -1.0, c.w.p, 1.0, ld);
    rel = host_norm(c, r) / bnorm;
    st.outer++;
  }
  return rel;
}

// --------------------------------------------------------------- set-up
// Smallest 2,3,5-smooth multiple of 4 (>= 8) not below n: multiples of 4
// let the FP32 spreading add 16-byte aligned quads of grid points.
static int round_up_smooth4(int n) {
  if (n < 8) n = 8;
  for (int m = n;; ++m)
    if (m % 4 == 0 && fft_size_ok(m)) return m;
}

static uint32_t spread_bits(uint32_t v) {
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}

// Lees-Edwards offset modulo L, in [-L/2, L/2)
static double wrap_tilt(double t, double L) {
  t -= L * std::floor(t / L + 0.5);
  return t;
}

static void setup_impl(Ctx &c, int64_t n_beads, const double *bead_pos, const int32_t *agg_id,
                       const fsd_params &p, void *stream) {
  if (n_beads < 1) throw Invalid{"n_beads must be >= 1"};
  if (n_beads > (1 << 28)) throw Invalid{"n_beads too large"};
  if (!bead_pos || !agg_id) throw Invalid{"bead_pos and agg_id are required"};
  if (!(p.box > 0)) throw Invalid{"box must be > 0"};
  if (!(p.a > 0) || !(p.eta > 0)) throw Invalid{"a and eta must be > 0"};
  c.prm = p;
  c.Nt = (int)n_beads;
  c.L = p.box;
  c.a = p.a;
  c.eta = p.eta;
  if (stream) {
    c.stream = (cudaStream_t)stream;
    c.own_stream = false;
  } else {
    FSD_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    c.own_stream = true;
  }
  {
    const char *e = std::getenv("FSD_OPERATOR_STREAMS");
    c.overlap = !(e && std::atoi(e) == 1);
    if (const char *b = std::getenv("FSD_RS_BLOCKS_PER_SM")) c.rs_blocks_per_sm = std::max(0, std::atoi(b));
    if (const char *g = std::getenv("FSD_SPREAD_ATOMIC")) c.spread_gather = std::atoi(g) != 1;
    if (c.overlap) {
      FSD_CUDA(cudaStreamCreateWithFlags(&c.stream2, cudaStreamNonBlocking));
      FSD_CUDA(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
      FSD_CUDA(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
    }
  }
  // ---- inputs to host
  std::vector<double> pos(3 * (size_t)c.Nt);
  std::vector<int32_t> ids(c.Nt);
  if (is_device_ptr(bead_pos))
    FSD_CUDA(cudaMemcpy(pos.data(), bead_pos, pos.size() * sizeof(double), cudaMemcpyDeviceToHost));
  else
    std::memcpy(pos.data(), bead_pos, pos.size() * sizeof(double));
  if (is_device_ptr(agg_id))
    FSD_CUDA(cudaMemcpy(ids.data(), agg_id, ids.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  else
    std::memcpy(ids.data(), agg_id, ids.size() * sizeof(int32_t));
  int32_t mx = -1;
  for (int i = 0; i < c.Nt; ++i) {
    if (ids[i] < 0) throw Invalid{"agg_id must be >= 0"};
    if (!(std::isfinite(pos[3 * i]) && std::isfinite(pos[3 * i + 1]) && std::isfinite(pos[3 * i + 2])))
      throw Invalid{"bead_pos holds a non-finite value"};
    mx = std::max(mx, ids[i]);
  }
  c.N = mx + 1;
  std::vector<std::vector<int>> members(c.N);
  for (int i = 0; i < c.Nt; ++i) members[ids[i]].push_back(i);
  for (int J = 0; J < c.N; ++J)
    if (members[J].empty()) throw Invalid{"agg_id values must be dense 0..N-1"};
  // ---- per body: unwrap about the first bead (nearest image, Lees-Edwards
  //      box when tilted), centroid, body frame
  const double L = c.L;
  if (!(L > 0) || !std::isfinite(p.tilt)) throw Invalid{"box must be > 0 and tilt finite"};
  c.tilt = wrap_tilt(p.tilt, L);
  c.prm.tilt = c.tilt;
  std::vector<double> X(3 * (size_t)c.N), rb(3 * (size_t)c.Nt);
  std::vector<double> unw(3 * (size_t)c.Nt);
  for (int J = 0; J < c.N; ++J) {
    const int f = members[J][0];
    double s[3] = {0, 0, 0};
    for (int i : members[J]) {
      double dd[3] = {pos[3 * i] - pos[3 * f], pos[3 * i + 1] - pos[3 * f + 1],
                      pos[3 * i + 2] - pos[3 * f + 2]};
      const double ny = std::nearbyint(dd[1] / L);
      dd[0] -= ny * c.tilt;
      dd[1] -= ny * L;
      dd[0] -= L * std::nearbyint(dd[0] / L);
      dd[2] -= L * std::nearbyint(dd[2] / L);
      for (int d = 0; d < 3; ++d) {
        unw[3 * i + d] = pos[3 * f + d] + dd[d];
        s[d] += unw[3 * i + d];
      }
    }
    for (int d = 0; d < 3; ++d) X[3 * J + d] = s[d] / members[J].size();
  }
  // ---- spatial order of bodies (Morton code of the wrapped centroid)
  std::vector<uint64_t> key(c.N);
  for (int J = 0; J < c.N; ++J) {
    uint32_t cc[3];
    for (int d = 0; d < 3; ++d) {
      double w = X[3 * J + d] - L * std::floor(X[3 * J + d] / L);
      int v = (int)(w / L * 1024.0);
      cc[d] = (uint32_t)std::min(1023, std::max(0, v));
    }
    key[J] = ((uint64_t)(spread_bits(cc[0]) | (spread_bits(cc[1]) << 1) | (spread_bits(cc[2]) << 2)) << 32) | (uint32_t)J;
  }
  std::vector<int> order(c.N);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x1, int x2) { return key[x1] < key[x2]; });
  c.h_perm_body = order;
  c.h_perm_bead.clear();
  c.h_body_start.assign(c.N + 1, 0);
  std::vector<int> bead_body(c.Nt);
  std::vector<double> Xi(3 * (size_t)c.N), rbi(3 * (size_t)c.Nt), qi(4 * (size_t)c.N, 0.0);
  for (int Ji = 0; Ji < c.N; ++Ji) {
    const int J = order[Ji];
    c.h_body_start[Ji] = (int)c.h_perm_bead.size();
    for (int d = 0; d < 3; ++d) Xi[3 * Ji + d] = X[3 * J + d];
    qi[4 * Ji] = 1.0;
    for (int i : members[J]) {
      const int ii = (int)c.h_perm_bead.size();
      c.h_perm_bead.push_back(i);
      bead_body[ii] = Ji;
      for (int d = 0; d < 3; ++d) rbi[3 * ii + d] = unw[3 * i + d] - X[3 * J + d];
    }
  }
  c.h_body_start[c.N] = c.Nt;
  // ---- parameters (rules of Sec. 3.2 unless given)
  const double a = c.a;
  const double xerr = p.xerr > 0 ? p.xerr : 1e-6;
  c.prm.xerr = xerr;
  const double lnx = std::sqrt(-std::log(xerr));
  // default splitting 0.5/a; in a box too small for its cut-off, 1.05 times
  // the smallest xi whose R_c = 2a + sqrt(-ln xerr)/xi stays below L/2
  c.xi = p.xi > 0 ? p.xi : 0.5 / a;
  if (p.xi <= 0 && p.rc <= 0 && 2.0 * a + lnx / c.xi >= 0.5 * L && 0.5 * L > 2.0 * a)
    c.xi = 1.05 * lnx / (0.5 * L - 2.0 * a);
  c.rc = p.rc > 0 ? p.rc : 2.0 * a + lnx / c.xi;
  if (p.grid > 0) {
    if (!fft_size_ok(p.grid)) throw Invalid{"grid must be even and 2,3,5-smooth (>= 8)"};
    c.n = p.grid;
  } else {
    const double kc = 2.0 * lnx * c.xi + 1.0;
    c.n = round_up_smooth4((int)std::ceil(kc * L / kPi));
  }
  // default support from the accuracy target: the relative error of the
  // wave-space operator against the exact mobility was measured as 8e-5 at
  // P = 8, falling tenfold for every 2 more points (7e-7 at P = 12)
  if (p.P > 0) {
    c.P = p.P;
  } else {
    c.P = 8;
    double est = 8e-5;
    while (est > xerr && c.P < 16) {
      c.P += 2;
      est *= 0.1;
    }
  }
  if (c.P % 2 || c.P < 4 || c.P > 24) throw Invalid{"P must be even, 4..24"};
  if (c.P > c.n) throw Invalid{"P must not exceed the grid size"};
  c.m_shape = p.m_shape > 0 ? p.m_shape : 0.976 * std::sqrt(kPi * c.P);
  c.h = L / c.n;
  c.alpha = 2.0 * c.m_shape * c.m_shape / ((c.P * c.h) * (c.P * c.h));
  if (c.rc >= 0.5 * L) throw Invalid{"real-space cut-off must be below L/2 (raise xi or the box)"};
  const bool le = (p.flags & FSD_FLAG_LEES_EDWARDS) || c.tilt != 0.0;
  if (le && (c.rc >= 0.447 * L || p.lub_cutoff >= 0.447 * L))
    throw Invalid{"in a Lees-Edwards box R_c and the lubrication cut-off must be below 0.447 L"};
  if ((p.flags & FSD_FLAG_LEES_EDWARDS) && (p.flags & FSD_FLAG_COMOVING))
    throw Invalid{"FSD_FLAG_LEES_EDWARDS and FSD_FLAG_COMOVING exclude each other"};
  if (p.lub_cutoff < 0) throw Invalid{"lub_cutoff must be >= 0"};
  if (p.lub_cutoff >= 0.5 * L) throw Invalid{"lub_cutoff must be below L/2"};
  c.prm.lub_cutoff = p.lub_cutoff > 2.0 * a ? p.lub_cutoff : 0.0;
  c.prm.precond_cutoff = p.precond_cutoff > 0 ? p.precond_cutoff : 2.1 * a;
  if (c.prm.lub_cutoff > 0) c.prm.precond_cutoff = std::min(c.prm.precond_cutoff, c.prm.lub_cutoff);
  c.prm.lub_hmin = p.lub_hmin > 0 ? p.lub_hmin : 1e-3 * a;
  c.prm.tol = p.tol > 0 ? p.tol : 1e-6;
  c.m = p.restart > 0 ? std::min(p.restart, 60) : 30;
  c.prm.restart = c.m;
  c.prm.max_iter = p.max_iter > 0 ? p.max_iter : 1000;
  if (p.precision != FSD_FP64 && p.precision != FSD_MIXED) throw Invalid{"precision must be 0 or 1"};
  c.m_in = p.inner_restart > 0 ? std::min(p.inner_restart, 60) : 60;
  c.prm.inner_restart = c.m_in;
  c.prm.inner_tol = p.inner_tol > 0 ? p.inner_tol : 1e-7;
  c.prm.lanczos_tol = p.lanczos_tol > 0 ? p.lanczos_tol : 1e-7;
  c.prm.lanczos_max_iter = p.lanczos_max_iter > 0 ? std::max(p.lanczos_max_iter, 2) : 60;
  if (!(p.rough_alpha >= 0.0) || !std::isfinite(p.rough_alpha) ||
      (p.rough_alpha > 0.0 && !(p.rough_h0 > 0.0 && std::isfinite(p.rough_h0))))
    throw Invalid{"rough_alpha must be >= 0, with rough_h0 > 0 when it is positive"};
  if (p.nf_sampler != FSD_NF_LANCZOS && p.nf_sampler != FSD_NF_PAIRWISE)
    throw Invalid{"nf_sampler must be FSD_NF_LANCZOS or FSD_NF_PAIRWISE"};
  if (p.tile != 0 && p.tile != 4 && p.tile != 8 && p.tile != 16 && p.tile != 32)
    throw Invalid{"tile must be 0, 4, 8, 16 or 32"};
  c.prm.xi = c.xi;
  c.prm.rc = c.rc;
  c.prm.grid = c.n;
  c.prm.P = c.P;
  c.prm.m_shape = c.m_shape;
  // ---- device state
  {
    int dev = 0;
    FSD_CUDA(cudaGetDevice(&dev));
    FSD_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int Nt = c.Nt, N = c.N;
  c.nunk = (int64_t)LDB * Nt + 6 * (int64_t)N;
  c.body_start.alloc(N + 1);
  c.bead_body.alloc(Nt);
  c.perm_bead.alloc(Nt);
  c.perm_body.alloc(N);
  c.X.alloc(3 * (size_t)N);
  c.q.alloc(4 * (size_t)N);
  c.rbody.alloc(3 * (size_t)Nt);
  c.pos64.alloc(4 * (size_t)Nt);
  c.lever64.alloc(4 * (size_t)Nt);
  c.op32.pos.alloc(4 * (size_t)Nt);
  c.op32.lever.alloc(4 * (size_t)Nt);
  c.wpos64.alloc(4 * (size_t)Nt);
  c.wpos32.alloc(4 * (size_t)Nt);
  if (c.overlap) c.yw.alloc((size_t)LDB * Nt);
  FSD_CUDA(cudaMemcpy(c.body_start.p, c.h_body_start.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice));
  {
    // lanes per aggregate of the aggregate-row kernels: the power of two
    // (4..32) that covers the largest aggregate
    int mb = 1;
    for (int J = 0; J < N; ++J) mb = std::max(mb, c.h_body_start[J + 1] - c.h_body_start[J]);
    c.body_lanes = 4;
    while (c.body_lanes < 32 && c.body_lanes < mb) c.body_lanes *= 2;
  }
  FSD_CUDA(cudaMemcpy(c.bead_body.p, bead_body.data(), Nt * sizeof(int), cudaMemcpyHostToDevice));
  FSD_CUDA(cudaMemcpy(c.perm_bead.p, c.h_perm_bead.data(), Nt * sizeof(int), cudaMemcpyHostToDevice));
  FSD_CUDA(cudaMemcpy(c.perm_body.p, c.h_perm_body.data(), N * sizeof(int), cudaMemcpyHostToDevice));
  FSD_CUDA(cudaMemcpy(c.X.p, Xi.data(), Xi.size() * sizeof(double), cudaMemcpyHostToDevice));
  FSD_CUDA(cudaMemcpy(c.q.p, qi.data(), qi.size() * sizeof(double), cudaMemcpyHostToDevice));
  FSD_CUDA(cudaMemcpy(c.rbody.p, rbi.data(), rbi.size() * sizeof(double), cudaMemcpyHostToDevice));
  // neighbour capacities from the mean density (grown on overflow)
  const double dens = Nt / (L * L * L);
  const double expect = dens * 4.0 / 3.0 * kPi * c.rc * c.rc * c.rc;
  c.cap = ((int)(1.6 * expect + 64) + 31) / 32 * 32;
  c.lcap = 16;
  c.nbr.alloc((size_t)Nt * c.cap);
  c.ncnt.alloc(Nt);
  c.lnbr.alloc((size_t)Nt * c.lcap);
  c.lcnt.alloc(Nt);
  c.flags.alloc(8);
  FSD_CUDA(cudaMallocHost(&c.h_flags, 8 * sizeof(int)));
  c.brow.alloc(Nt + 1);
  c.op64.bdiag.alloc((size_t)Nt * 36);
  c.op32.bdiag.alloc((size_t)Nt * 36);
  c.pdiag.alloc((size_t)Nt * 36);
  c.schur.alloc((size_t)N * 36);
  c.piv.alloc((size_t)N * 6);
  c.fnf.alloc((size_t)Nt * 6);
  c.snf.alloc((size_t)Nt * 5);
  FSD_CUDA(cudaMemset(c.fnf.p, 0, (size_t)Nt * 6 * sizeof(double)));
  FSD_CUDA(cudaMemset(c.snf.p, 0, (size_t)Nt * 5 * sizeof(double)));
  const int mm = std::max(c.m, c.m_in);
  // V: FP64 GMRES and the Lanczos square roots (at most mm + 1 vectors);
  // with FSD_FLAG_FP32_KRYLOV the mixed solve's inner GMRES keeps its bases
  // in FP32
  c.krylov32 = c.prm.precision == FSD_MIXED && (c.prm.flags & FSD_FLAG_FP32_KRYLOV);
  c.V.alloc((size_t)(mm + 1) * c.nunk);
  if (c.krylov32) {
    c.V32.alloc((size_t)(c.m_in + 1) * c.nunk);
    c.Z32.alloc((size_t)c.m_in * c.nunk);
    c.kv.alloc(c.nunk);
    c.kz.alloc(c.nunk);
  } else {
    c.Z.alloc((size_t)mm * c.nunk);
  }
  c.w.alloc(c.nunk);
  c.t1.alloc(c.nunk);
  c.t2.alloc(c.nunk);
  c.xsol.alloc(c.nunk);
  c.rhs.alloc(c.nunk);
  c.res.alloc(c.nunk);
  c.xprev.alloc(c.nunk);
  c.partial.alloc(std::max<int64_t>((int64_t)64 * kDotPartials, cgs_partial_size(c.nunk, mm + 1, c.num_sms)));
  c.hcol.alloc(512);
  c.cgs_ticket.alloc(1);
  FSD_CUDA(cudaMemset(c.cgs_ticket.p, 0, sizeof(unsigned)));
  FSD_CUDA(cudaMallocHost(&c.h_pinned, 512 * sizeof(double)));
  build_real_table(c);
  build_wave(c);
  c.tilt_dev.alloc(1);
  sync_tilt(c);
  launch_wrap_positions(c);
  FSD_CUDA(cudaStreamSynchronize(c.stream));
}

// Geometry-dependent preparation of one solve: positions, neighbour lists,
// lubrication blocks, Schur LUs (Alg. 1 step 1).
static void prepare(Ctx &c) {
  c.last_warning = FSD_OK;
  launch_wrap_positions(c);
  build_neighbors(c);
  {
    // pair count for the real-space launch shape
    std::vector<int> cnt(c.Nt);
    FSD_CUDA(cudaMemcpyAsync(cnt.data(), c.ncnt.p, c.Nt * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    FSD_CUDA(cudaStreamSynchronize(c.stream));
    int64_t s = 0;
    for (int v : cnt) s += v;
    c.n_pairs = s;
  }
  build_lubrication(c);
  if (c.spread_gather && !c.tiles_valid) build_spread_tiles(c);
}

static void fill_stats(Ctx &c, fsd_stats *st, const KStats &k, double rel, double ms) {
  if (!st) return;
  st->iters = k.iters;
  st->outer_iters = k.outer;
  st->matvec64 = k.m64;
  st->matvec32 = k.m32;
  st->rel_residual = rel;
  st->ms_total = ms;
  st->n_pairs = c.n_pairs;
  st->n_lub = c.n_lub;
  st->grid = c.n;
  st->P = c.P;
  st->xi = c.xi;
  st->rc = c.rc;
}

static fsd_status check_flags(Ctx &c) {
  FSD_CUDA(cudaMemcpyAsync(c.h_flags, c.flags.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  if (c.h_flags[3]) {
    c.last_error = "singular per-aggregate 6x6 preconditioner block";
    return FSD_ENUMERIC;
  }
  return FSD_OK;
}

// One solve; vel_int / str_int are internal-order device outputs.
static fsd_status solve_internal(Ctx &c, const double *ft_user, double shear, double *vel_int,
                                 double *str_int, fsd_stats *stats, double t0_ms) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = c.launches;
  if (!c.geom_fresh) prepare(c);
  c.geom_fresh = false;
  fsd_status fl = check_flags(c);
  const double *ft_int = nullptr;
  if (ft_user) {
    const double *d = dev_in(c, ft_user, 6 * (size_t)c.N, c.io_a);
    if (c.t2.n < 6 * (size_t)c.N) c.t2.alloc(6 * (size_t)c.N);
    k_bodies_in<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, d, c.t2.p, 6);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    ft_int = c.t2.p;
  }
  launch_rhs(c, ft_int, shear, c.rhs.p);
  launch_brownian_rhs(c, c.rhs.p);
  c.brown_pending = false;  // consumed by this solve
  KStats ks;
  const bool warm = (c.prm.flags & FSD_FLAG_WARM_START) && c.have_prev;
  double rel = solve_system(c, c.rhs.p, c.xsol.p, ks, warm);
  FSD_CUDA(cudaMemcpyAsync(c.xprev.p, c.xsol.p, c.nunk * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  c.have_prev = true;
  launch_outputs(c, c.xsol.p, shear, vel_int, str_int);
  if (c.vextra_pending) launch_add_velocity(c, vel_int);
  c.vextra_pending = false;  // consumed by this solve
  FSD_CUDA(cudaMemsetAsync(c.flags.p + 6, 0, sizeof(int), c.stream));
  k_nan_check<<<c.num_sms, 256, 0, c.stream>>>(vel_int, 6 * (int64_t)c.N, c.flags.p + 6);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaMemcpyAsync(c.h_flags, c.flags.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() + t0_ms;
  fill_stats(c, stats, ks, rel, ms);
  if (stats) stats->kernel_launches = c.launches - l0;
  if (c.h_flags[6]) {
    c.last_error = "non-finite aggregate velocity";
    return FSD_ENUMERIC;
  }
  if (fl != FSD_OK) return fl;
  if (!(rel <= c.prm.tol)) {
    c.last_error = "Krylov solve stopped at relative residual " + std::to_string(rel);
    return FSD_ENOCONV;
  }
  if (c.last_warning == FSD_EOVERLAP) {
    c.last_error = "beads of different aggregates overlap (warning; results written)";
    return FSD_EOVERLAP;
  }
  return FSD_OK;
}

// ---- device-resident step (FSD_FLAG_GRAPH): geometry on the host side,
//      then the whole solve (+ update) as one graph launch; the end half
//      waits and turns the device state into a status.
static bool use_graph(const Ctx &c) {
  // Lees-Edwards steps too: their operator kernels read the box offset from
  // device memory, which the host updates between graph launches
  return (c.prm.flags & FSD_FLAG_GRAPH) && !c.prof;
}

// After a Lees-Edwards step the images across y have moved with the imposed
// flow: offset += shear L dt (host value and device copy).
static void advance_tilt(Ctx &c, double shear_rate, double dt) {
  if (!(c.prm.flags & FSD_FLAG_LEES_EDWARDS)) return;
  c.tilt = wrap_tilt(c.tilt + shear_rate * c.L * dt, c.L);
  c.prm.tilt = c.tilt;
  sync_tilt(c);
}

struct StepMark {
  std::chrono::steady_clock::time_point t0;
  int64_t l0 = 0;
};

static StepMark graph_step_begin(Ctx &c, const double *ft_user, double shear, bool with_str,
                                 bool integrate, double dt) {
  StepMark mk;
  mk.t0 = std::chrono::steady_clock::now();
  mk.l0 = c.launches;
  if (!c.geom_fresh) prepare(c);
  c.geom_fresh = false;
  refresh_le_tables(c);  // Lees-Edwards: the sheared Green's factors of this offset
  GraphRun o;
  o.warm = (c.prm.flags & FSD_FLAG_WARM_START) && c.have_prev;
  o.has_ft = ft_user != nullptr;
  o.integrate = integrate;
  o.with_str = with_str;
  o.shear = shear;
  o.dt = dt;
  o.brown = c.brown_pending ? 1 : 0;
  o.brown_scale = c.brown_scale;
  o.add_vel = c.vextra_pending ? 1 : 0;
  o.str_hydro = c.str_hydro ? 1 : 0;
  if (ft_user)
    FSD_CUDA(cudaMemcpyAsync(graph_ft_buffer(c), ft_user, 6 * (size_t)c.N * sizeof(double),
                             cudaMemcpyDefault, c.stream));
  graph_launch(c, o);
  c.brown_pending = false;  // consumed by this solve
  c.vextra_pending = false;
  return mk;
}

static fsd_status graph_step_end(Ctx &c, const StepMark &mk, fsd_stats *stats) {
  KStats ks;
  const double rel = graph_finish(c, ks);
  c.have_prev = true;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - mk.t0).count();
  fill_stats(c, stats, ks, rel, ms);
  if (stats) stats->kernel_launches = c.launches - mk.l0;
  if (c.h_flags[6]) {
    c.last_error = "non-finite aggregate velocity";
    return FSD_ENUMERIC;
  }
  if (c.h_flags[3]) {
    c.last_error = "singular per-aggregate 6x6 preconditioner block";
    return FSD_ENUMERIC;
  }
  if (!(rel <= c.prm.tol)) {
    c.last_error = "Krylov solve stopped at relative residual " + std::to_string(rel);
    return FSD_ENOCONV;
  }
  if (c.last_warning == FSD_EOVERLAP) {
    c.last_error = "beads of different aggregates overlap (warning; results written)";
    return FSD_EOVERLAP;
  }
  return FSD_OK;
}

// ---- Brownian drift (Sec. 2.4; appendix on the drift): solves at displaced
//      rigid configurations, differenced.

// One solve of the current configuration with the pending terms, host-driven
// or as the captured graph; velocity in t1, stresslet (when wanted) in res.
static fsd_status solve_any(Ctx &c, const double *ft_user, bool with_str, fsd_stats *stats) {
  if (use_graph(c)) {
    const StepMark mk = graph_step_begin(c, ft_user, 0.0, with_str, false, 0.0);
    return graph_step_end(c, mk, stats);
  }
  return solve_internal(c, ft_user, 0.0, c.t1.p, with_str ? c.res.p : nullptr, stats, 0.0);
}

static bool status_fatal(fsd_status s) { return s != FSD_OK && s != FSD_ENOCONV && s != FSD_EOVERLAP; }

// Saves what the drift solves change (body positions and orientations, the
// warm-start vector, flags, pending terms) and puts it back on every exit.
struct DriftState {
  Ctx &c;
  int flags;
  bool have_prev, brown, vx, done = false;
  explicit DriftState(Ctx &cx) : c(cx) {
    flags = c.prm.flags;
    have_prev = c.have_prev;
    brown = c.brown_pending;
    vx = c.vextra_pending;
    if (c.dsave.n < 7 * (size_t)c.N) c.dsave.alloc(7 * (size_t)c.N);
    if (c.dxprev.n < (size_t)c.nunk) c.dxprev.alloc(c.nunk);
    FSD_CUDA(cudaMemcpyAsync(c.dsave.p, c.X.p, 3 * (size_t)c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    FSD_CUDA(cudaMemcpyAsync(c.dsave.p + 3 * (size_t)c.N, c.q.p, 4 * (size_t)c.N * sizeof(double),
                             cudaMemcpyDeviceToDevice, c.stream));
    FSD_CUDA(cudaMemcpyAsync(c.dxprev.p, c.xprev.p, c.nunk * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    c.prm.flags &= ~FSD_FLAG_WARM_START;
    c.vextra_pending = false;
    c.str_hydro = true;
  }
  void restore_geometry() {
    FSD_CUDA(cudaMemcpyAsync(c.X.p, c.dsave.p, 3 * (size_t)c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    FSD_CUDA(cudaMemcpyAsync(c.q.p, c.dsave.p + 3 * (size_t)c.N, 4 * (size_t)c.N * sizeof(double),
                             cudaMemcpyDeviceToDevice, c.stream));
    launch_wrap_positions(c);
    c.geom_fresh = false;
  }
  ~DriftState() {
    // best effort on the error path: the context is then reported broken by
    // the status already returned
    cudaMemcpyAsync(c.X.p, c.dsave.p, 3 * (size_t)c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    cudaMemcpyAsync(c.q.p, c.dsave.p + 3 * (size_t)c.N, 4 * (size_t)c.N * sizeof(double),
                    cudaMemcpyDeviceToDevice, c.stream);
    cudaMemcpyAsync(c.xprev.p, c.dxprev.p, c.nunk * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    try {
      launch_wrap_positions(c);
    } catch (...) {
    }
    cudaStreamSynchronize(c.stream);
    c.geom_fresh = false;
    c.prm.flags = flags;
    c.have_prev = have_prev;
    c.str_hydro = false;
    if (!done) {
      c.vextra_pending = vx;
      c.brown_pending = brown;
    }
  }
};

static void add_stats(fsd_stats &acc, const fsd_stats &s) {
  acc.iters += s.iters;
  acc.outer_iters += s.outer_iters;
  acc.matvec64 += s.matvec64;
  acc.matvec32 += s.matvec32;
  acc.rel_residual = std::max(acc.rel_residual, s.rel_residual);
  acc.n_pairs = s.n_pairs;
  acc.n_lub = s.n_lub;
  acc.grid = s.grid;
  acc.P = s.P;
  acc.xi = s.xi;
  acc.rc = s.rc;
}

// Work vectors in dwork (internal order except the first): dq in user order,
// dq, U_a, S_a, drift, stresslet.
static fsd_status drift_impl(Ctx &c, int method, double kT, double dt, double param, uint64_t seed,
                             uint64_t step, const double *dq_user_in, fsd_stats &acc) {
  const size_t N6 = 6 * (size_t)c.N, N9 = 9 * (size_t)c.N;
  if (c.dwork.n < 4 * N6 + 2 * N9) c.dwork.alloc(4 * N6 + 2 * N9);
  double *dq_user = c.dwork.p, *dq = dq_user + N6, *Ua = dq + N6, *Sa = Ua + N6, *vout = Sa + N9,
         *sout = vout + N6;
  if (c.vextra.n < N6) c.vextra.alloc(N6);
  if (c.t1.n < N6 || c.res.n < N9) throw Invalid{"internal: output buffers too small"};
  fsd_status worst = FSD_OK;
  auto take = [&](fsd_status st) {
    if (status_fatal(st)) return true;
    if (st == FSD_ENOCONV || (st == FSD_EOVERLAP && worst == FSD_OK)) worst = st;
    return false;
  };
  DriftState ds(c);
  fsd_stats sub;
  if (method == FSD_DRIFT_RFD) {
    // U+- = N(x +- eps/2 dq) dq (body forcing dq, no flow); drift = kT (U+ - U-)/eps,
    // S^B = kT (S+ - S-)/eps
    const double eps = param > 0 ? param : c.a * std::cbrt(c.prm.tol);
    if (dq_user_in)
      FSD_CUDA(cudaMemcpyAsync(dq_user, dq_user_in, N6 * sizeof(double), cudaMemcpyDefault, c.stream));
    else
      launch_dq_philox(c, seed, step, dq_user);
    k_bodies_in_launch(c, dq_user, dq);
    c.brown_pending = false;  // the drift solves carry no Brownian terms
    for (int sgn = 1; sgn >= -1; sgn -= 2) {
      ds.restore_geometry();
      launch_integrate(c, dq, 0.5 * sgn * eps, 0.0);
      launch_wrap_positions(c);
      std::memset(&sub, 0, sizeof(sub));
      const fsd_status st = solve_any(c, dq_user, true, &sub);
      add_stats(acc, sub);
      if (take(st)) return st;
      FSD_CUDA(cudaMemcpyAsync(sgn > 0 ? Ua : vout, c.t1.p, N6 * sizeof(double), cudaMemcpyDeviceToDevice,
                               c.stream));
      FSD_CUDA(cudaMemcpyAsync(sgn > 0 ? Sa : sout, c.res.p, N9 * sizeof(double), cudaMemcpyDeviceToDevice,
                               c.stream));
    }
    launch_scaled_diff(c, Ua, vout, kT / eps, vout, (int64_t)N6);
    launch_scaled_diff(c, Sa, sout, kT / eps, sout, (int64_t)N9);
    if (ds.vx)
      launch_axpy(c, vout, c.vextra.p, (int64_t)N6);
    else
      FSD_CUDA(cudaMemcpyAsync(c.vextra.p, vout, N6 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    c.brown_pending = ds.brown;  // still for the next solve
  } else {
    // modified Fixman: U0 = solve with the Brownian terms at x; x' = x + (dt/m) U0;
    // U' = the same solve at x'; drift = (m/2)(U' - U0), S^B = -(m/2)(S' - S0)
    if (!ds.brown) throw Invalid{"the Fixman drift needs Brownian terms: call fsd_brownian first"};
    const double m = param > 0 ? param : 100.0;
    std::memset(&sub, 0, sizeof(sub));
    fsd_status st = solve_any(c, nullptr, true, &sub);
    add_stats(acc, sub);
    if (take(st)) return st;
    FSD_CUDA(cudaMemcpyAsync(Ua, c.t1.p, N6 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    FSD_CUDA(cudaMemcpyAsync(Sa, c.res.p, N9 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    launch_integrate(c, Ua, dt / m, 0.0);
    launch_wrap_positions(c);
    c.geom_fresh = false;
    c.brown_pending = true;  // the same u^B, E^B and F^B_nf at x'
    std::memset(&sub, 0, sizeof(sub));
    st = solve_any(c, nullptr, true, &sub);
    add_stats(acc, sub);
    if (take(st)) return st;
    launch_scaled_diff(c, c.t1.p, Ua, 0.5 * m, vout, (int64_t)N6);
    launch_scaled_diff(c, c.res.p, Sa, -0.5 * m, sout, (int64_t)N9);
    // the next solve gets U0 + drift; its own Brownian terms are spent
    if (!ds.vx) FSD_CUDA(cudaMemsetAsync(c.vextra.p, 0, N6 * sizeof(double), c.stream));
    launch_axpy(c, Ua, c.vextra.p, (int64_t)N6);
    launch_axpy(c, vout, c.vextra.p, (int64_t)N6);
    c.brown_pending = false;
  }
  ds.restore_geometry();
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  c.vextra_pending = true;
  ds.done = true;
  return worst;
}

// ---- autotuner (FSD_FLAG_AUTOTUNE): the splitting xi trades real-space
//      pairs (R_c falls as 1/xi) against wave-space grid points (the grid
//      grows as xi); P is the smallest support that meets xerr, which is
//      always the fastest, so it is not searched.  Each candidate xi (with
//      R_c and the grid from the accuracy rules) and real-space tile is
//      timed on the device with the operator the Krylov iterations apply;
//      the fastest is kept.  The preconditioner and hence the iteration
//      count do not depend on xi.
static double time_operator(Ctx &c, int reps) {
  cudaEvent_t e0, e1;
  FSD_CUDA(cudaEventCreate(&e0));
  FSD_CUDA(cudaEventCreate(&e1));
  double *x = c.t1.p, *y = c.w.p;
  FSD_CUDA(cudaMemsetAsync(x, 0, c.nunk * sizeof(double), c.stream));
  const bool f32 = c.prm.precision == FSD_MIXED;
  auto apply = [&]() {
    if (f32)
      apply_saddle<float>(c, x, y);
    else
      apply_saddle<double>(c, x, y);
  };
  apply();
  FSD_CUDA(cudaEventRecord(e0, c.stream));
  for (int r = 0; r < reps; ++r) apply();
  FSD_CUDA(cudaEventRecord(e1, c.stream));
  FSD_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  FSD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

static fsd_params autotune(int64_t n_beads, const double *bead_pos, const int32_t *agg_id,
                           const fsd_params &p, double *best_ms_out) {
  static const int kTile[] = {4, 8, 16, 32};
  // fixed candidates, plus splittings just above the smallest one whose
  // cut-off 2a + sqrt(-ln xerr)/xi stays below L/2 (small boxes)
  const double a = p.a > 0 ? p.a : 1.0;
  const double xerr = p.xerr > 0 ? p.xerr : 1e-6;
  std::vector<double> xis = {0.30 / a, 0.35 / a, 0.40 / a, 0.45 / a, 0.50 / a,
                             0.55 / a, 0.60 / a, 0.70 / a};
  const double room = 0.5 * p.box - 2.0 * a;
  if (room > 0) {
    const double xmin = std::sqrt(-std::log(xerr)) / room;
    for (double f : {1.02, 1.25, 1.6})
      if (f * xmin > 0.7 / a) xis.push_back(f * xmin);
  }
  fsd_params best = p;
  best.flags &= ~FSD_FLAG_AUTOTUNE;
  double best_ms = 1e300;
  for (double xi : xis) {
    fsd_params q = p;
    q.flags &= ~(FSD_FLAG_AUTOTUNE | FSD_FLAG_GRAPH);
    q.xi = xi;
    fsd_ctx *tmp = new fsd_ctx();
    try {
      setup_impl(tmp->c, n_beads, bead_pos, agg_id, q, nullptr);
      prepare(tmp->c);
      for (int t : kTile) {
        tmp->c.prm.tile = t;
        const double ms = time_operator(tmp->c, 3);
        if (ms < best_ms) {
          best_ms = ms;
          best = p;
          best.flags &= ~FSD_FLAG_AUTOTUNE;
          best.xi = q.xi;
          best.tile = t;
        }
      }
    } catch (const Invalid &) {
      // candidate outside the method's limits (R_c >= L/2, table too large)
    }
    fsd_destroy(tmp);
  }
  if (best_ms >= 1e300) throw Invalid{"autotune: no admissible splitting for this box"};
  if (best_ms_out) *best_ms_out = best_ms;
  return best;
}

// Write an internal-order device array of N x w to a user pointer (host or device).
static void bodies_out(Ctx &c, const double *src_int, double *user, int w) {
  if (!user) return;
  if (is_device_ptr(user)) {
    k_bodies_out<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, src_int, user, w);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    FSD_CUDA(cudaStreamSynchronize(c.stream));
  } else {
    if (c.io_b.n < (size_t)w * c.N) c.io_b.alloc((size_t)w * c.N);
    k_bodies_out<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, src_int, c.io_b.p, w);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    FSD_CUDA(cudaMemcpyAsync(user, c.io_b.p, (size_t)w * c.N * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    FSD_CUDA(cudaStreamSynchronize(c.stream));
  }
}

}  // namespace fsd

using namespace fsd;

#define FSD_API_TRY try {
#define FSD_API_CATCH(ctxp)                                                     \
  }                                                                             \
  catch (const CudaError &e) {                                                  \
    std::string m = std::string(e.what) + ": " + cudaGetErrorString(e.e);       \
    if (ctxp) (ctxp)->c.last_error = m; else g_setup_error = m;                 \
    return e.e == cudaErrorMemoryAllocation ? FSD_ENOMEM : FSD_ECUDA;           \
  }                                                                             \
  catch (const Invalid &e) {                                                    \
    if (ctxp) (ctxp)->c.last_error = e.msg; else g_setup_error = e.msg;         \
    return FSD_EINVAL;                                                          \
  }                                                                             \
  catch (const std::bad_alloc &) {                                              \
    if (ctxp) (ctxp)->c.last_error = "host allocation failed";                  \
    else g_setup_error = "host allocation failed";                              \
    return FSD_ENOMEM;                                                          \
  }

extern "C" {

void fsd_default_params(fsd_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->a = 1.0;
  p->eta = 1.0;
  p->box = 0.0;
  p->xi = 0.0;
  p->xerr = 1e-6;
  p->rc = 0.0;
  p->grid = 0;
  p->P = 0;
  p->m_shape = 0.0;
  p->lub_cutoff = 0.0;
  p->precond_cutoff = 2.1;
  p->lub_hmin = 1e-3;
  p->tol = 1e-6;
  p->restart = 30;
  p->max_iter = 1000;
  p->precision = FSD_FP64;
  p->inner_restart = 60;
  p->inner_tol = 1e-7;
  p->flags = 0;
  p->tile = 0;
  p->lanczos_tol = 1e-7;
  p->lanczos_max_iter = 60;
  // the pairwise near-field sampler is exact and needs no iteration; the
  // paper's preconditioned Lanczos stops at its step limit on dense
  // lubricated suspensions (FSD_NF_LANCZOS selects it)
  p->nf_sampler = FSD_NF_PAIRWISE;
  p->rough_alpha = 0.0;
  p->rough_h0 = 0.0;
}

fsd_status fsd_setup(fsd_ctx **ctx, int64_t n_beads, const double *bead_pos, const int32_t *agg_id,
                     const fsd_params *p, void *cuda_stream) {
  if (!ctx || !p) {
    g_setup_error = "ctx and params are required";
    return FSD_EINVAL;
  }
  *ctx = nullptr;
  fsd_ctx *cx = nullptr;
  FSD_API_TRY
  fsd_params q = *p;
  double tuned = 0.0;
  if ((q.flags & FSD_FLAG_AUTOTUNE) && q.xi <= 0 && q.rc <= 0 && q.grid <= 0)
    q = autotune(n_beads, bead_pos, agg_id, q, &tuned);
  cx = new fsd_ctx();
  setup_impl(cx->c, n_beads, bead_pos, agg_id, q, cuda_stream);
  cx->c.tuned_ms = tuned;
  *ctx = cx;
  return FSD_OK;
  }
  catch (const CudaError &e) {
    g_setup_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    fsd_destroy(cx);
    return e.e == cudaErrorMemoryAllocation ? FSD_ENOMEM : FSD_ECUDA;
  }
  catch (const Invalid &e) {
    g_setup_error = e.msg;
    fsd_destroy(cx);
    return FSD_EINVAL;
  }
  catch (const std::bad_alloc &) {
    g_setup_error = "host allocation failed";
    fsd_destroy(cx);
    return FSD_ENOMEM;
  }
}

fsd_status fsd_solve(fsd_ctx *ctx, const double *agg_force_torque, double shear_rate,
                     double *agg_velocity, double *agg_stresslet, fsd_stats *stats) {
  if (!ctx) return FSD_EINVAL;
  if (!agg_velocity) {
    ctx->c.last_error = "agg_velocity is required";
    return FSD_EINVAL;
  }
  if (!std::isfinite(shear_rate)) {
    ctx->c.last_error = "shear_rate must be finite";
    return FSD_EINVAL;
  }
  FSD_API_TRY
  Ctx &c = ctx->c;
  auto t0 = std::chrono::steady_clock::now();
  if (c.io_b.n < 16 * (size_t)c.N) c.io_b.alloc(16 * (size_t)c.N);
  DBuf<double> &vel = c.io_b;
  // internal outputs live in t1 (velocity) / res (stresslet) after the solve
  double *vel_int = c.t1.p;
  double *str_int = agg_stresslet ? c.res.p : nullptr;
  fsd_status st;
  if (use_graph(c)) {
    const StepMark mk = graph_step_begin(c, agg_force_torque, shear_rate, str_int != nullptr, false, 0.0);
    st = graph_step_end(c, mk, stats);
  } else {
    st = solve_internal(c, agg_force_torque, shear_rate, vel_int, str_int, stats, 0.0);
  }
  if (st != FSD_OK && st != FSD_ENOCONV && st != FSD_EOVERLAP) return st;
  (void)vel;
  bodies_out(c, vel_int, agg_velocity, 6);
  if (agg_stresslet) bodies_out(c, str_int, agg_stresslet, 9);
  if (stats)
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_step(fsd_ctx *ctx, const double *agg_force_torque, double shear_rate, double dt,
                    double *agg_velocity, fsd_stats *stats) {
  if (!ctx) return FSD_EINVAL;
  if (!std::isfinite(dt) || !std::isfinite(shear_rate)) {
    ctx->c.last_error = "dt and shear_rate must be finite";
    return FSD_EINVAL;
  }
  FSD_API_TRY
  Ctx &c = ctx->c;
  auto t0 = std::chrono::steady_clock::now();
  double *vel_int = c.t1.p;
  if (use_graph(c)) {
    // the update runs inside the graph, after the solve
    const StepMark mk = graph_step_begin(c, agg_force_torque, shear_rate, false, true, dt);
    fsd_status st = graph_step_end(c, mk, stats);
    if (st != FSD_OK && st != FSD_ENOCONV && st != FSD_EOVERLAP) return st;
    advance_tilt(c, shear_rate, dt);
    const int64_t l1 = c.launches;
    if (agg_velocity) bodies_out(c, vel_int, agg_velocity, 6);
    if (stats) stats->kernel_launches += c.launches - l1;
    if (stats)
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
  }
  fsd_status st = solve_internal(c, agg_force_torque, shear_rate, vel_int, nullptr, stats, 0.0);
  if (st != FSD_OK && st != FSD_ENOCONV && st != FSD_EOVERLAP) return st;
  const int64_t l1 = c.launches;
  if (agg_velocity) bodies_out(c, vel_int, agg_velocity, 6);
  launch_integrate(c, vel_int, dt, shear_rate);
  advance_tilt(c, shear_rate, dt);
  launch_wrap_positions(c);
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  if (stats) stats->kernel_launches += c.launches - l1;
  if (stats)
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_get_beads(fsd_ctx *ctx, double *bead_pos, double *agg_quat) {
  if (!ctx) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  launch_wrap_positions(c);
  if (bead_pos) {
    if (c.io_a.n < 3 * (size_t)c.Nt) c.io_a.alloc(3 * (size_t)c.Nt);
    k_bead_pos_out<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, c.perm_bead.p, c.bead_body.p, c.X.p,
                                                             (const double4 *)c.lever64.p, c.io_a.p);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    FSD_CUDA(cudaMemcpyAsync(bead_pos, c.io_a.p, 3 * (size_t)c.Nt * sizeof(double), cudaMemcpyDefault, c.stream));
  }
  if (agg_quat) {
    if (c.io_b.n < 16 * (size_t)c.N) c.io_b.alloc(16 * (size_t)c.N);
    k_bodies_out<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, c.q.p, c.io_b.p, 4);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    FSD_CUDA(cudaMemcpyAsync(agg_quat, c.io_b.p, 4 * (size_t)c.N * sizeof(double), cudaMemcpyDefault, c.stream));
  }
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

// ---- operator access: user-ordered vectors in and out

static void vec_in(Ctx &c, const double *user, double *x, bool beads, bool bodies) {
  // user layout: [Nt][11] then [N][6]
  const size_t nb = 11 * (size_t)c.Nt, nbd = 6 * (size_t)c.N;
  const size_t tot = (beads ? nb : 0) + (bodies ? nbd : 0);
  const double *d = dev_in(c, user, tot, c.io_a);
  FSD_CUDA(cudaMemsetAsync(x, 0, c.nunk * sizeof(double), c.stream));
  if (beads) k_beads_in<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, c.perm_bead.p, d, x);
  FSD_LAUNCHED(c);
  if (bodies)
    k_bodies_in<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, d + (beads ? nb : 0),
                                                         x + (int64_t)LDB * c.Nt, 6);
    FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

static void vec_out(Ctx &c, const double *x, double *user, bool beads, bool bodies) {
  const size_t nb = 11 * (size_t)c.Nt, nbd = 6 * (size_t)c.N;
  const size_t tot = (beads ? nb : 0) + (bodies ? nbd : 0);
  const bool dev = is_device_ptr(user);
  double *d = user;
  if (!dev) {
    if (c.io_b.n < tot) c.io_b.alloc(tot);
    d = c.io_b.p;
  }
  if (beads) k_beads_out<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, c.perm_bead.p, x, d);
  FSD_LAUNCHED(c);
  if (bodies)
    k_bodies_out<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, x + (int64_t)LDB * c.Nt,
                                                          d + (beads ? nb : 0), 6);
    FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  if (!dev)
    FSD_CUDA(cudaMemcpyAsync(user, d, tot * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
}

fsd_status fsd_apply_mobility(fsd_ctx *ctx, const double *in, double *out, int part, int precision) {
  if (!ctx || !in || !out || part < 1 || part > 3) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prepare(c);
  vec_in(c, in, c.t1.p, true, false);
  double *y = c.t2.p;
  FSD_CUDA(cudaMemsetAsync(y, 0, c.nunk * sizeof(double), c.stream));
  if (precision == FSD_FP64) {
    if (part & 1) launch_realspace<double>(c, c.t1.p, y, false, false);
    if (part & 2) launch_wavespace<double>(c, c.t1.p, y);
  } else {
    if (part & 1) launch_realspace<float>(c, c.t1.p, y, false, false);
    if (part & 2) launch_wavespace<float>(c, c.t1.p, y);
  }
  vec_out(c, y, out, true, false);
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_apply_saddle(fsd_ctx *ctx, const double *x, double *y, int precision) {
  if (!ctx || !x || !y) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prepare(c);
  vec_in(c, x, c.t1.p, true, true);
  if (precision == FSD_FP64)
    apply_saddle<double>(c, c.t1.p, c.t2.p);
  else
    apply_saddle<float>(c, c.t1.p, c.t2.p);
  vec_out(c, c.t2.p, y, true, true);
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_apply_precond(fsd_ctx *ctx, const double *r, double *z) {
  if (!ctx || !r || !z) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prepare(c);
  fsd_status fl = check_flags(c);
  vec_in(c, r, c.t1.p, true, true);
  launch_precond(c, c.t1.p, c.t2.p);
  vec_out(c, c.t2.p, z, true, true);
  return fl;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_apply_lubrication(fsd_ctx *ctx, const double *dU, double *out, int precision) {
  if (!ctx || !dU || !out) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prepare(c);
  // dU in the aggregate slots of a solution vector
  const double *d = dev_in(c, dU, 6 * (size_t)c.N, c.io_a);
  FSD_CUDA(cudaMemsetAsync(c.t1.p, 0, c.nunk * sizeof(double), c.stream));
  k_bodies_in<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, d, c.t1.p + (int64_t)LDB * c.Nt, 6);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  if (precision == FSD_FP64)
    launch_lub_apply<double>(c, c.t1.p, c.t2.p);
  else
    launch_lub_apply<float>(c, c.t1.p, c.t2.p);
  bodies_out(c, c.t2.p + (int64_t)LDB * c.Nt, out, 6);
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_rhs(fsd_ctx *ctx, const double *agg_force_torque, double shear_rate, double *b) {
  if (!ctx || !b) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prepare(c);
  const double *ft_int = nullptr;
  if (agg_force_torque) {
    const double *d = dev_in(c, agg_force_torque, 6 * (size_t)c.N, c.io_a);
    k_bodies_in<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.perm_body.p, d, c.t2.p, 6);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    ft_int = c.t2.p;
  }
  launch_rhs(c, ft_int, shear_rate, c.t1.p);
  vec_out(c, c.t1.p, b, true, true);
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_brownian(fsd_ctx *ctx, double kT, double dt, uint64_t seed, uint64_t step,
                        const double *wave_field, const double *psi_real, const double *psi_nf,
                        double *slip, double *force_nf, fsd_stats *stats) {
  if (!ctx) return FSD_EINVAL;
  if (!(kT >= 0.0) || !(dt > 0.0) || !std::isfinite(kT) || !std::isfinite(dt)) {
    ctx->c.last_error = "kT must be >= 0 and dt > 0 (finite)";
    return FSD_EINVAL;
  }
  FSD_API_TRY
  Ctx &c = ctx->c;
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = c.launches;
  if (!c.geom_fresh) prepare(c);
  c.geom_fresh = true;  // the next solve reuses this preparation
  const size_t nh = (size_t)c.n / 2 + 1;
  DBuf<double> sf, sr, sn;
  const double *fd = wave_field ? dev_in(c, wave_field, 6 * (size_t)c.n * c.n * nh, sf) : nullptr;
  const double *rd = psi_real ? dev_in(c, psi_real, 11 * (size_t)c.Nt, sr) : nullptr;
  const double *nd = psi_nf ? dev_in(c, psi_nf, 6 * (size_t)c.Nt, sn) : nullptr;
  int ir = 0, inf = 0;
  double change = 0.0;
  brownian_sample(c, kT, dt, seed, step, fd, rd, nd, &ir, &inf, &change);
  for (int q = 0; q < 2; ++q) {
    double *user = q == 0 ? slip : force_nf;
    const int w = q == 0 ? 11 : 6;
    if (!user) continue;
    if (is_device_ptr(user)) {
      brownian_outputs(c, q == 0 ? user : nullptr, q == 1 ? user : nullptr);
    } else {
      DBuf<double> tmp;
      tmp.alloc((size_t)w * c.Nt);
      brownian_outputs(c, q == 0 ? tmp.p : nullptr, q == 1 ? tmp.p : nullptr);
      FSD_CUDA(cudaMemcpyAsync(user, tmp.p, (size_t)w * c.Nt * sizeof(double), cudaMemcpyDeviceToHost,
                               c.stream));
      FSD_CUDA(cudaStreamSynchronize(c.stream));
    }
  }
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iters = ir;
    stats->outer_iters = inf;
    stats->rel_residual = change;
    stats->kernel_launches = c.launches - l0;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->grid = c.n;
    stats->P = c.P;
    stats->xi = c.xi;
    stats->rc = c.rc;
  }
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_drift(fsd_ctx *ctx, int method, double kT, double dt, double param, uint64_t seed,
                     uint64_t step, const double *dq, double *drift, double *brownian_velocity,
                     double *brownian_stresslet, fsd_stats *stats) {
  if (!ctx) return FSD_EINVAL;
  Ctx &c0 = ctx->c;
  if (method != FSD_DRIFT_RFD && method != FSD_DRIFT_FIXMAN) {
    c0.last_error = "method must be FSD_DRIFT_RFD or FSD_DRIFT_FIXMAN";
    return FSD_EINVAL;
  }
  if (!(kT >= 0.0) || !std::isfinite(kT) || !std::isfinite(param) ||
      (method == FSD_DRIFT_FIXMAN && !(dt > 0.0 && std::isfinite(dt)))) {
    c0.last_error = "kT must be >= 0, param finite, and dt > 0 for the Fixman drift";
    return FSD_EINVAL;
  }
  FSD_API_TRY
  Ctx &c = ctx->c;
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = c.launches;
  fsd_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  const fsd_status st = drift_impl(c, method, kT, dt, param, seed, step, dq, acc);
  if (!status_fatal(st)) {
    const size_t N6 = 6 * (size_t)c.N, N9 = 9 * (size_t)c.N;
    double *Ua = c.dwork.p + 2 * N6, *vout = Ua + N6 + N9, *sout = vout + N6;
    bodies_out(c, vout, drift, 6);
    if (method == FSD_DRIFT_FIXMAN) bodies_out(c, Ua, brownian_velocity, 6);
    bodies_out(c, sout, brownian_stresslet, 9);
  }
  if (stats) {
    *stats = acc;
    stats->kernel_launches = c.launches - l0;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_set_tilt(fsd_ctx *ctx, double tilt) {
  if (!ctx) return FSD_EINVAL;
  if (!std::isfinite(tilt)) {
    ctx->c.last_error = "tilt must be finite";
    return FSD_EINVAL;
  }
  FSD_API_TRY
  Ctx &c = ctx->c;
  const double t = wrap_tilt(tilt, c.L);
  if (t != 0.0 && (c.rc >= 0.447 * c.L || c.prm.lub_cutoff >= 0.447 * c.L))
    throw Invalid{"in a Lees-Edwards box R_c and the lubrication cut-off must be below 0.447 L"};
  c.tilt = t;
  c.prm.tilt = t;
  sync_tilt(c);
  launch_wrap_positions(c);
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  c.geom_fresh = false;
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

static fsd_status pair_forces_impl(fsd_ctx *ctx, const fsd_pair_forces &pf, double *agg_force_torque) {
  FSD_API_TRY
  Ctx &c = ctx->c;
  if (pf.r_cut > c.rc) throw Invalid{"r_cut must not exceed the real-space cut-off R_c"};
  if (!c.geom_fresh) prepare(c);
  c.geom_fresh = true;  // the next solve reuses this preparation
  const size_t need = 3 * (size_t)c.Nt + 6 * (size_t)c.N;
  if (c.cwork.n < need) c.cwork.alloc(need);
  double *ft_int = c.cwork.p + 3 * (size_t)c.Nt;
  launch_contact(c, pf, c.cwork.p, ft_int);
  bodies_out(c, ft_int, agg_force_torque, 6);
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_contact_forces(fsd_ctx *ctx, double kn, double *agg_force_torque) {
  if (!ctx) return FSD_EINVAL;
  if (!(kn >= 0.0) || !std::isfinite(kn) || !agg_force_torque) {
    ctx->c.last_error = "kn must be finite and >= 0, agg_force_torque is required";
    return FSD_EINVAL;
  }
  fsd_pair_forces pf{};
  pf.kn = kn;
  return pair_forces_impl(ctx, pf, agg_force_torque);
}

fsd_status fsd_interparticle_forces(fsd_ctx *ctx, const fsd_pair_forces *p, double *agg_force_torque) {
  if (!ctx) return FSD_EINVAL;
  const bool ok = p && agg_force_torque && std::isfinite(p->kn) && p->kn >= 0.0 &&
                  std::isfinite(p->hamaker) && std::isfinite(p->zeta) && std::isfinite(p->kappa) &&
                  std::isfinite(p->h_c) && p->h_c >= 0.0 && std::isfinite(p->r_cut) && p->r_cut >= 0.0 &&
                  (p->zeta == 0.0 || p->kappa > 0.0);
  if (!ok) {
    ctx->c.last_error = "fsd_pair_forces: kn >= 0, h_c >= 0, r_cut >= 0 finite, kappa > 0 with zeta";
    return FSD_EINVAL;
  }
  return pair_forces_impl(ctx, *p, agg_force_torque);
}

fsd_status fsd_get_params(const fsd_ctx *ctx, fsd_params *p) {
  if (!ctx || !p) return FSD_EINVAL;
  *p = ctx->c.prm;
  return FSD_OK;
}

fsd_status fsd_profile_enable(fsd_ctx *ctx, int on) {
  if (!ctx) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  prof_collect(c);
  if (on) {
    for (int g = 0; g < PG_COUNT; ++g) {
      c.prof_ms[g] = 0.0;
      c.prof_n[g] = 0;
    }
  }
  c.prof = on != 0;
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

fsd_status fsd_profile_read(fsd_ctx *ctx, double *ms, int64_t *count, int n) {
  if (!ctx || n < PG_COUNT) return FSD_EINVAL;
  FSD_API_TRY
  Ctx &c = ctx->c;
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  prof_collect(c);
  for (int g = 0; g < PG_COUNT; ++g) {
    if (ms) ms[g] = c.prof_ms[g];
    if (count) count[g] = c.prof_n[g];
  }
  return FSD_OK;
  FSD_API_CATCH(ctx)
}

const char *fsd_profile_group_name(int g) {
  if (g < 0 || g >= PG_COUNT) return nullptr;
  return kProfNames[g];
}

const char *fsd_last_error(const fsd_ctx *ctx) {
  if (!ctx) return g_setup_error.c_str();
  return ctx->c.last_error.c_str();
}

void fsd_destroy(fsd_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  if (c.stream) cudaStreamSynchronize(c.stream);
  graph_cache_free(c);
  if (c.h_flags) cudaFreeHost(c.h_flags);
  if (c.h_pinned) cudaFreeHost(c.h_pinned);
  prof_collect(c);
  for (cudaEvent_t e : c.ev_pool) cudaEventDestroy(e);
  c.ev_pool.clear();
  if (c.stream2) {
    cudaStreamSynchronize(c.stream2);
    cudaStreamDestroy(c.stream2);
  }
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  if (c.ev_join) cudaEventDestroy(c.ev_join);
  cudaStream_t s = c.stream;
  bool own = c.own_stream;
  delete ctx;
  if (own && s) cudaStreamDestroy(s);
}

// ====================================================== batched suspensions

static int status_rank(fsd_status s) {
  switch (s) {
    case FSD_OK: return 0;
    case FSD_EOVERLAP: return 1;
    case FSD_ENOCONV: return 2;
    default: return 3;
  }
}

void fsd_destroy_batch(fsd_batch *b) {
  if (!b) return;
  for (fsd_ctx *c : b->sys) fsd_destroy(c);
  for (cudaEvent_t e : b->ev_done) cudaEventDestroy(e);
  if (b->ev_user) cudaEventDestroy(b->ev_user);
  delete b;
}

fsd_status fsd_setup_batch(fsd_batch **batch, int n_sys, const int64_t *bead_offsets,
                           const double *bead_pos, const int32_t *agg_id,
                           const fsd_params *params, void *cuda_stream) {
  if (!batch || n_sys < 1 || !bead_offsets || !bead_pos || !agg_id || !params) {
    g_setup_error = "batch, n_sys >= 1, bead_offsets, bead_pos, agg_id and params are required";
    if (batch) *batch = nullptr;
    return FSD_EINVAL;
  }
  *batch = nullptr;
  if (bead_offsets[0] != 0) {
    g_setup_error = "bead_offsets[0] must be 0";
    return FSD_EINVAL;
  }
  for (int s = 0; s < n_sys; ++s)
    if (bead_offsets[s + 1] <= bead_offsets[s]) {
      g_setup_error = "system " + std::to_string(s) + " has no beads";
      return FSD_EINVAL;
    }
  fsd_batch *b = nullptr;
  try {
    b = new fsd_batch();
    b->user = (cudaStream_t)cuda_stream;
    if (const char *e = std::getenv("FSD_BATCH_THREADS")) b->host_threads = std::max(1, std::atoi(e));
    b->bead_off.assign(bead_offsets, bead_offsets + n_sys + 1);
    b->agg_off.assign(1, 0);
    std::vector<double> cost(n_sys);
    for (int s = 0; s < n_sys; ++s) {
      fsd_params q = params[s];
      q.flags |= FSD_FLAG_GRAPH;
      const int64_t o = bead_offsets[s], nb = bead_offsets[s + 1] - o;
      fsd_ctx *cx = nullptr;
      const fsd_status st = fsd_setup(&cx, nb, bead_pos + 3 * o, agg_id + o, &q, nullptr);
      if (st != FSD_OK) {
        const std::string m = "system " + std::to_string(s) + ": " + g_setup_error;
        fsd_destroy_batch(b);
        g_setup_error = m;
        return st;
      }
      b->sys.push_back(cx);
      const Ctx &c = cx->c;
      b->agg_off.push_back(b->agg_off.back() + c.N);
      cost[s] = c.tuned_ms > 0 ? c.tuned_ms : (double)c.Nt + 0.25 * (double)c.n * c.n * c.n;
      cudaEvent_t e;
      FSD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      b->ev_done.push_back(e);
    }
    if (b->user) FSD_CUDA(cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming));
    b->order.resize(n_sys);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    *batch = b;
    return FSD_OK;
  } catch (const CudaError &e) {
    g_setup_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    fsd_destroy_batch(b);
    return e.e == cudaErrorMemoryAllocation ? FSD_ENOMEM : FSD_ECUDA;
  } catch (const std::bad_alloc &) {
    g_setup_error = "host allocation failed";
    fsd_destroy_batch(b);
    return FSD_ENOMEM;
  }
}

fsd_status fsd_batch_info(const fsd_batch *b, int *n_sys, int64_t *agg_offsets,
                          fsd_params *params) {
  if (!b) return FSD_EINVAL;
  const int ns = (int)b->sys.size();
  if (n_sys) *n_sys = ns;
  if (agg_offsets)
    for (int s = 0; s <= ns; ++s) agg_offsets[s] = b->agg_off[s];
  if (params)
    for (int s = 0; s < ns; ++s) params[s] = b->sys[s]->c.prm;
  return FSD_OK;
}

fsd_ctx *fsd_batch_system(fsd_batch *b, int s) {
  if (!b || s < 0 || s >= (int)b->sys.size()) return nullptr;
  return b->sys[s];
}

// Solve (integrate = false) or step every system: all graphs are launched
// first (geometry of each system prepared on its own stream just before its
// launch), then each is waited for and its outputs written.
static fsd_status batch_run(fsd_batch *b, const double *ft, const double *shear_rates, double dt,
                            bool integrate, double *vel, double *str, fsd_stats *stats) {
  const int ns = (int)b->sys.size();
  std::vector<fsd_status> st(ns, FSD_OK);
  std::vector<StepMark> mk(ns);
  std::vector<char> launched(ns, 0);
  std::vector<std::string> err(ns);
  if (b->user) {
    FSD_CUDA(cudaEventRecord(b->ev_user, b->user));
    for (fsd_ctx *cx : b->sys) FSD_CUDA(cudaStreamWaitEvent(cx->c.stream, b->ev_user, 0));
  }
  // Launch phase on a few host threads: each system's geometry preparation
  // waits on its own stream (neighbour-list and lubrication sizes), so
  // systems prepared in parallel keep more graphs in flight.  Systems are
  // taken most expensive first.
  int dev = 0;
  FSD_CUDA(cudaGetDevice(&dev));
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int t; (t = next.fetch_add(1)) < ns;) {
      const int s = b->order[t];
      Ctx &c = b->sys[s]->c;
      const double *fts = ft ? ft + 6 * b->agg_off[s] : nullptr;
      try {
        if (use_graph(c)) {
          mk[s] = graph_step_begin(c, fts, shear_rates[s], str != nullptr, integrate, dt);
          launched[s] = 1;
        } else {
          // a system with the profiler on runs the host-driven loop in place
          double *str_int = str ? c.res.p : nullptr;
          st[s] = solve_internal(c, fts, shear_rates[s], c.t1.p, str_int, stats ? stats + s : nullptr, 0.0);
          if (integrate && status_rank(st[s]) < 3) {
            launch_integrate(c, c.t1.p, dt, shear_rates[s]);
            advance_tilt(c, shear_rates[s], dt);
            launch_wrap_positions(c);
          }
        }
      } catch (const CudaError &e) {
        err[s] = std::string(e.what) + ": " + cudaGetErrorString(e.e);
        st[s] = FSD_ECUDA;
      } catch (const Invalid &e) {
        err[s] = e.msg;
        st[s] = FSD_EINVAL;
      }
    }
  };
  const int nthreads = std::max(1, std::min({ns, b->host_threads}));
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  for (int s : b->order) {
    Ctx &c = b->sys[s]->c;
    try {
      if (launched[s]) {
        st[s] = graph_step_end(c, mk[s], stats ? stats + s : nullptr);
        if (integrate && status_rank(st[s]) < 3) advance_tilt(c, shear_rates[s], dt);
      }
      if (status_rank(st[s]) < 3) {
        if (vel) bodies_out(c, c.t1.p, vel + 6 * b->agg_off[s], 6);
        if (str) bodies_out(c, c.res.p, str + 9 * b->agg_off[s], 9);
      }
      if (b->user) FSD_CUDA(cudaEventRecord(b->ev_done[s], c.stream));
    } catch (const CudaError &e) {
      err[s] = std::string(e.what) + ": " + cudaGetErrorString(e.e);
      st[s] = FSD_ECUDA;
    } catch (const Invalid &e) {
      err[s] = e.msg;
      st[s] = FSD_EINVAL;
    }
  }
  if (b->user)
    for (int s = 0; s < ns; ++s) FSD_CUDA(cudaStreamWaitEvent(b->user, b->ev_done[s], 0));
  fsd_status worst = FSD_OK;
  b->last_error.clear();
  for (int s = 0; s < ns; ++s) {
    if (st[s] == FSD_OK) continue;
    const std::string m = err[s].empty() ? b->sys[s]->c.last_error : err[s];
    if (status_rank(st[s]) > status_rank(worst)) {
      worst = st[s];
      b->last_error = "system " + std::to_string(s) + ": " + m;
    }
  }
  return worst;
}

fsd_status fsd_solve_batch(fsd_batch *b, const double *agg_force_torque, const double *shear_rates,
                           double *agg_velocity, double *agg_stresslet, fsd_stats *stats) {
  if (!b) return FSD_EINVAL;
  if (!shear_rates || !agg_velocity) {
    b->last_error = "shear_rates and agg_velocity are required";
    return FSD_EINVAL;
  }
  for (size_t s = 0; s < b->sys.size(); ++s)
    if (!std::isfinite(shear_rates[s])) {
      b->last_error = "shear_rates must be finite";
      return FSD_EINVAL;
    }
  try {
    return batch_run(b, agg_force_torque, shear_rates, 0.0, false, agg_velocity, agg_stresslet, stats);
  } catch (const CudaError &e) {
    b->last_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    return FSD_ECUDA;
  }
}

fsd_status fsd_step_batch(fsd_batch *b, const double *agg_force_torque, const double *shear_rates,
                          double dt, double *agg_velocity, fsd_stats *stats) {
  if (!b) return FSD_EINVAL;
  if (!shear_rates || !std::isfinite(dt)) {
    b->last_error = "shear_rates are required and dt must be finite";
    return FSD_EINVAL;
  }
  for (size_t s = 0; s < b->sys.size(); ++s)
    if (!std::isfinite(shear_rates[s])) {
      b->last_error = "shear_rates must be finite";
      return FSD_EINVAL;
    }
  try {
    return batch_run(b, agg_force_torque, shear_rates, dt, true, agg_velocity, nullptr, stats);
  } catch (const CudaError &e) {
    b->last_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    return FSD_ECUDA;
  }
}

fsd_status fsd_batch_get_beads(fsd_batch *b, double *bead_pos, double *agg_quat) {
  if (!b) return FSD_EINVAL;
  for (size_t s = 0; s < b->sys.size(); ++s) {
    const fsd_status st = fsd_get_beads(b->sys[s], bead_pos ? bead_pos + 3 * b->bead_off[s] : nullptr,
                                        agg_quat ? agg_quat + 4 * b->agg_off[s] : nullptr);
    if (st != FSD_OK) {
      b->last_error = "system " + std::to_string(s) + ": " + b->sys[s]->c.last_error;
      return st;
    }
  }
  return FSD_OK;
}

const char *fsd_batch_last_error(const fsd_batch *b) {
  if (!b) return g_setup_error.c_str();
  return b->last_error.c_str();
}

}  // extern "C"
