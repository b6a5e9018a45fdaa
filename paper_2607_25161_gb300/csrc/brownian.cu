// Brownian forcing of the saddle-point solve (Sec. 2.2 "stochastic
// sampling", Eq. SP2, Eq. UBff; Algorithm 1 step 3):
//   far-field slip      u^B  = sqrt(2 kT/dt) (M_w^(1/2) psi_w + M_r^(1/2) psi_r)
//   near-field force    F^B  = sqrt(2 kT/dt) (R_FU^nf)^(1/2) psi_nf
// The wave part is analytic (wavespace.cu: a random field scaled in k space,
// inverse FFT, interpolation); the real-space square root comes from Lanczos
// iterations (Krylov approximation of f(A) b, f = sqrt) on the library's
// real-space operator.  The near-field force comes either from the exact
// pairwise sampler (the default: F = sum over lubrication pairs of the pair
// model's dissipation factor applied to pair noise, k_nf_pairwise in
// nearfield.cu; covariance exactly R_FU^nf) or from the paper's Lanczos
// iteration on the bead-level lubrication blocks.  The next
// solve adds u^B to the bead rows (all 11 components) and -Sigma F^B to the
// body rows of its right-hand side.
//
// Random numbers: given by the caller, or drawn from Philox4x32-10 with the
// counter layout (index, stream * 256 + call, step): stream 1 the wave field
// (wavespace.cu), stream 2 psi_r (11 per bead), stream 3 psi_nf (6 per bead,
// Lanczos near-field sampler), stream 4 the drift's random body vectors
// (indexed by body), stream 5 the pairwise near-field sampler's pair noise
// (nearfield.cu, a four-word counter holding both beads of the pair); the
// index of a bead is its position in the caller's bead array.
#include "fsd_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace fsd {

// ---------------------------------------------------------------- kernels
// y = R_FU^nf x, bead rows, R the bead-level near-field FU blocks (BSR,
// diagonal separate); components 6..11 of y are zero.
__global__ void k_bsr_bead(int Nt, const int *__restrict__ brow, const int *__restrict__ bcol,
                           const double *__restrict__ bval, const double *__restrict__ bdiag,
                           const double *__restrict__ x, double *y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Nt) return;
  double g[6];
  const double *xb = x + (size_t)b * LDB;
  const double *D = bdiag + (size_t)b * 36;
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) s += D[6 * a + q] * xb[q];
    g[a] = s;
  }
  for (int k = brow[b]; k < brow[b + 1]; ++k) {
    const double *xc = x + (size_t)bcol[k] * LDB;
    const double *Bk = bval + (size_t)k * 36;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) s += Bk[6 * a + q] * xc[q];
      g[a] += s;
    }
  }
  double *yb = y + (size_t)b * LDB;
#pragma unroll
  for (int a = 0; a < 6; ++a) yb[a] = g[a];
#pragma unroll
  for (int a = 6; a < LDB; ++a) yb[a] = 0.0;
}

// Per bead: Cholesky factor L of the near-field diagonal block D (6x6,
// symmetric positive semidefinite), regularised as D + 1e-6 (tr D / 6) I so
// that null directions (which carry no near-field coupling) stay
// invertible, and G = L^-1 (forward substitution).  A bead without
// near-field pairs (tr D = 0) gets L = G = I.  Row-major 6x6 each.
__global__ void k_block_chol(int Nt, const double *__restrict__ bdiag, double *Lm, double *Gm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Nt) return;
  const double *D = bdiag + (size_t)b * 36;
  double A[6][6], L[6][6], G[6][6];
  double tr = 0.0;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      A[i][j] = 0.5 * (D[6 * i + j] + D[6 * j + i]);
      L[i][j] = G[i][j] = 0.0;
    }
    tr += A[i][i];
  }
  if (tr > 0.0) {
    const double reg = 1e-6 * tr / 6.0;
    for (int i = 0; i < 6; ++i) A[i][i] += reg;
    for (int j = 0; j < 6; ++j) {
      double s = A[j][j];
      for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
      L[j][j] = sqrt(s > 0.0 ? s : reg);
      for (int i = j + 1; i < 6; ++i) {
        double t = A[i][j];
        for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
        L[i][j] = t / L[j][j];
      }
    }
    for (int c = 0; c < 6; ++c)
      for (int i = c; i < 6; ++i) {
        double t = i == c ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) t -= L[i][k] * G[k][c];
        G[i][c] = t / L[i][i];
      }
  } else {
    for (int i = 0; i < 6; ++i) L[i][i] = G[i][i] = 1.0;
  }
  double *lo = Lm + (size_t)b * 36, *go = Gm + (size_t)b * 36;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      lo[6 * i + j] = L[i][j];
      go[6 * i + j] = G[i][j];
    }
}

// y_b = B_b x_b, or B_b^T x_b with tr (6x6 per bead, components 0..5;
// 6..11 zero).  May run in place: every input of a bead is read before its
// output is written.
__global__ void k_block_apply(int Nt, const double *__restrict__ Bm, int tr, const double *x,
                              double *y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Nt) return;
  const double *B = Bm + (size_t)b * 36;
  const double *xb = x + (size_t)b * LDB;
  double o[6];
  for (int a = 0; a < 6; ++a) {
    double s = 0.0;
    for (int q = 0; q < 6; ++q) s += (tr ? B[6 * q + a] : B[6 * a + q]) * xb[q];
    o[a] = s;
  }
  double *yb = y + (size_t)b * LDB;
  for (int a = 0; a < 6; ++a) yb[a] = o[a];
  for (int a = 6; a < LDB; ++a) yb[a] = 0.0;
}

// caller's psi [Nt][w] (bead order of the caller) -> solution layout
__global__ void k_psi_in(int Nt, const int *__restrict__ perm, const double *__restrict__ user, int w,
                         double *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double *u = user + (size_t)perm[i] * w;
  double *o = x + (size_t)i * LDB;
  for (int k = 0; k < LDB; ++k) o[k] = k < w ? u[k] : 0.0;
}

// psi from Philox: bead i draws with the index of its caller position
__global__ void k_psi_philox(int Nt, const int *__restrict__ perm, uint64_t seed, uint64_t step,
                             uint32_t stream, int w, double *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  double z[12];
  const int calls = (w + 3) / 4;
  for (int q = 0; q < calls; ++q) philox_normals4(seed, step, stream, (uint32_t)q, (uint32_t)perm[i], z + 4 * q);
  double *o = x + (size_t)i * LDB;
  for (int k = 0; k < LDB; ++k) o[k] = k < w ? z[k] : 0.0;
}

// user[perm[i]][k] = s x[i][k], k < w
__global__ void k_brown_out(int Nt, const int *__restrict__ perm, const double *__restrict__ x, int w,
                            double s, double *user) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double *v = x + (size_t)i * LDB;
  double *u = user + (size_t)perm[i] * w;
  for (int k = 0; k < w; ++k) u[k] = s * v[k];
}

// bead rows of b += s u^B (velocity, rotation, strain)
__global__ void k_brown_rhs_bead(int Nt, const double *__restrict__ slip, double s, double *b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Nt * LDB) return;
  if (e % LDB < 11) b[e] += s * slip[e];
}

// body rows of b -= s Sigma F^B: per body the summed force and the torque
// about X (L_b + r_b x F_b)
__global__ void k_brown_rhs_body(int N, const int *__restrict__ body_start,
                                 const double4 *__restrict__ lever, const double *__restrict__ fnf,
                                 double s, double *b, int64_t off) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = body_start[J]; i < body_start[J + 1]; ++i) {
    const double *f = fnf + (size_t)i * LDB;
    const double4 r = lever[i];
    acc[0] += f[0];
    acc[1] += f[1];
    acc[2] += f[2];
    acc[3] += f[3] + r.y * f[2] - r.z * f[1];
    acc[4] += f[4] + r.z * f[0] - r.x * f[2];
    acc[5] += f[5] + r.x * f[1] - r.y * f[0];
  }
  double *o = b + off + 6 * (size_t)J;
  for (int a = 0; a < 6; ++a) o[a] -= s * acc[a];
}

// ------------------------------------------------------------- Lanczos
// ||b|| f(T) e_1, f = sqrt, for the symmetric tridiagonal T (diagonal al,
// off-diagonal be): implicit QR steps with the Wilkinson shift (Golub & Van
// Loan, the implicit symmetric QR step) diagonalise T = Z diag(lam) Z^T with
// Z the product of the Givens rotations G_1 G_2 ...; only the first row of Z
// is kept during the sweep, and Z y is formed at the end by applying the
// recorded rotations to y in reverse.
struct Rot {
  int k;
  double c, s;
};
static std::vector<double> sqrt_coeffs(int m, const std::vector<double> &al,
                                       const std::vector<double> &be, double bnorm) {
  std::vector<double> d(al.begin(), al.begin() + m), e(std::max(m, 1), 0.0);
  for (int i = 0; i + 1 < m; ++i) e[i] = be[i];
  std::vector<double> z0(m, 0.0);
  if (m > 0) z0[0] = 1.0;
  std::vector<Rot> rots;
  rots.reserve((size_t)4 * m * m + 16);
  int q = m - 1, guard = 0;
  while (q > 0 && guard < 60 * m) {
    for (int i = 0; i < q; ++i)
      if (std::fabs(e[i]) <= 1e-16 * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    while (q > 0 && e[q - 1] == 0.0) --q;
    if (q == 0) break;
    int p = q - 1;
    while (p > 0 && e[p - 1] != 0.0) --p;
    ++guard;
    const double a = d[q - 1], b = e[q - 1], c = d[q];
    const double dl = 0.5 * (a - c);
    const double mu = c - b * b / (dl + (dl >= 0.0 ? 1.0 : -1.0) * std::hypot(dl, b));
    double x = d[p] - mu, z = e[p];
    for (int k = p; k < q; ++k) {
      const double r = std::hypot(x, z);
      const double cs = r > 0 ? x / r : 1.0, sn = r > 0 ? z / r : 0.0;
      if (k > p) e[k - 1] = r;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = cs * cs * dk + 2.0 * cs * sn * ek + sn * sn * dk1;
      d[k + 1] = sn * sn * dk - 2.0 * cs * sn * ek + cs * cs * dk1;
      e[k] = cs * sn * (dk1 - dk) + (cs * cs - sn * sn) * ek;
      if (k + 1 < q) {
        z = sn * e[k + 1];
        e[k + 1] = cs * e[k + 1];
        x = e[k];
      }
      const double a0 = z0[k], a1 = z0[k + 1];
      z0[k] = cs * a0 + sn * a1;
      z0[k + 1] = -sn * a0 + cs * a1;
      rots.push_back({k, cs, sn});
    }
  }
  std::vector<double> y(m);
  for (int k = 0; k < m; ++k) y[k] = std::sqrt(std::max(0.0, d[k])) * z0[k];
  for (size_t j = rots.size(); j-- > 0;) {
    const Rot &g = rots[j];
    const double a0 = y[g.k], a1 = y[g.k + 1];
    y[g.k] = g.c * a0 - g.s * a1;
    y[g.k + 1] = g.s * a0 + g.c * a1;
  }
  for (double &v : y) v *= bnorm;
  return y;
}

static double dev_norm(Ctx &c, const double *x) {
  double *d = c.hcol.p + 200;
  norm2_dev(c, x, d);
  FSD_CUDA(cudaMemcpyAsync(c.h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  return std::sqrt(std::max(0.0, c.h_pinned[0]));
}

// out = A^(1/2) b by Lanczos with full re-orthogonalisation: V_m T_m^(1/2)
// (||b|| e_1), stopped when the coefficients change by less than tol
// (relative).  apply(x, y) sets y = A x (bead rows; body rows must stay 0).
template <class Apply>
static int lanczos_sqrt(Ctx &c, Apply apply, const double *b, double *out, double tol, int maxit,
                        double *change) {
  const int64_t ld = c.nunk, n = c.nunk;
  double *V = c.V.p, *w = c.w.p;
  const double bnorm = dev_norm(c, b);
  FSD_CUDA(cudaMemsetAsync(out, 0, n * sizeof(double), c.stream));
  if (change) *change = 0.0;
  if (!(bnorm > 0.0)) return 0;
  vec_scale_host(c, V, b, 1.0 / bnorm);
  std::vector<double> al, be, cf, prev;
  double *h1 = c.hcol.p, *hn = c.hcol.p + 128;
  int m = 0;
  for (int j = 0; j < maxit; ++j) {
    apply(V + (int64_t)j * ld, w);
    FSD_CUDA(cudaMemsetAsync(w + (int64_t)LDB * c.Nt, 0, 6 * (size_t)c.N * sizeof(double), c.stream));
    cgs_pass(c, 0, V, ld, j + 1, w, nullptr, h1);
    cgs_pass(c, 2, V, ld, j + 1, w, h1, hn);
    FSD_CUDA(cudaMemcpyAsync(c.h_pinned, c.hcol.p, 192 * sizeof(double), cudaMemcpyDeviceToHost,
                             c.stream));
    FSD_CUDA(cudaStreamSynchronize(c.stream));
    al.push_back(c.h_pinned[j]);
    const double beta = std::sqrt(std::max(0.0, c.h_pinned[128]));
    if (!(beta == beta)) throw Invalid{"NaN in the Lanczos process"};
    m = j + 1;
    cf = sqrt_coeffs(m, al, be, bnorm);
    double dn = 0.0, cn = 0.0;
    for (int i = 0; i < m; ++i) {
      const double d = cf[i] - (i < (int)prev.size() ? prev[i] : 0.0);
      dn += d * d;
      cn += cf[i] * cf[i];
    }
    prev = cf;
    if (change) *change = j > 0 && cn > 0 ? std::sqrt(dn / cn) : 1.0;
    if (j > 0 && dn <= tol * tol * cn) break;
    if (beta <= 1e-14 * bnorm || j + 1 == maxit) break;
    be.push_back(beta);
    vec_scale_host(c, V + (int64_t)(j + 1) * ld, w, 1.0 / beta);
  }
  std::memcpy(c.h_pinned + 256, cf.data(), m * sizeof(double));
  FSD_CUDA(cudaMemcpyAsync(c.hcol.p + 256, c.h_pinned + 256, m * sizeof(double),
                           cudaMemcpyHostToDevice, c.stream));
  axpy_multi(c, out, V, ld, m, c.hcol.p + 256, 1.0);
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  return m;
}

// ------------------------------------------------------------- sampling
void brownian_sample(Ctx &c, double kT, double dt, uint64_t seed, uint64_t step,
                     const double *field_dev, const double *psi_r_dev, const double *psi_nf_dev,
                     int *iters_real, int *iters_nf, double *change) {
  if (!(kT >= 0.0) || !(dt > 0.0)) throw Invalid{"kT must be >= 0 and dt > 0"};
  const int64_t n = c.nunk;
  if (c.bslip.n < (size_t)n) c.bslip.alloc(n);
  if (c.bfnf.n < (size_t)n) c.bfnf.alloc(n);
  if (c.bwork.n < (size_t)n) c.bwork.alloc(n);
  const bool f32 = c.prm.precision == FSD_MIXED;
  const int maxit = std::min(std::max(c.m, c.m_in), c.prm.lanczos_max_iter);
  const double tol = c.prm.lanczos_tol;
  // wave part: u_w = M_w^(1/2) psi_w
  if (f32)
    launch_brownian_wave<float>(c, field_dev, seed, step, c.bslip.p);
  else
    launch_brownian_wave<double>(c, field_dev, seed, step, c.bslip.p);
  // real-space part: u_r = M_r^(1/2) psi_r (Lanczos on the real-space operator)
  FSD_CUDA(cudaMemsetAsync(c.bwork.p, 0, n * sizeof(double), c.stream));
  if (psi_r_dev)
    k_psi_in<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, psi_r_dev, 11, c.bwork.p);
  else
    k_psi_philox<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, seed, step, 2u, 11,
                                                           c.bwork.p);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  auto real_op = [&](const double *x, double *y) {
    if (f32)
      launch_realspace<float>(c, x, y, false, false);
    else
      launch_realspace<double>(c, x, y, false, false);
  };
  double ch_r = 0.0, ch_n = 0.0;
  const int ir = lanczos_sqrt(c, real_op, c.bwork.p, c.t2.p, tol, maxit, &ch_r);
  vec_axpby(c, c.bslip.p, 1.0, c.t2.p, 1.0, n);
  // near-field part: F^B = R_FU^(1/2) psi_nf (Lanczos on the bead-level blocks)
  int inf = 0;
  if (c.n_lub > 0 && c.prm.nf_sampler == FSD_NF_PAIRWISE) {
    // exact in distribution, no Krylov iteration: sum over pairs of
    // K_p^T psi_p, K_p the pair's dissipation-form factor (the pair noise
    // drawn here, Philox stream 5)
    if (psi_nf_dev) throw Invalid{"the pairwise near-field sampler draws its own pair noise: psi_nf must be NULL"};
    launch_nf_pairwise(c, seed, step, c.bfnf.p);
  } else if (c.n_lub > 0) {
    FSD_CUDA(cudaMemsetAsync(c.bwork.p, 0, n * sizeof(double), c.stream));
    if (psi_nf_dev)
      k_psi_in<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, psi_nf_dev, 6, c.bwork.p);
    else
      k_psi_philox<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, seed, step, 3u, 6,
                                                             c.bwork.p);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    // preconditioned sampling: with L L^T the bead's regularised diagonal
    // block and G = L^-1, F = L (G R G^T)^(1/2) psi has covariance R
    // (L G = I) and the Lanczos iteration runs on G R G^T, whose diagonal
    // blocks are (nearly) the identity
    if (c.bgain.n < (size_t)c.Nt * 72) c.bgain.alloc((size_t)c.Nt * 72);
    double *Lb = c.bgain.p, *G = c.bgain.p + (size_t)c.Nt * 36;
    k_block_chol<<<ceil_div(c.Nt, 64), 64, 0, c.stream>>>(c.Nt, c.op64.bdiag.p, Lb, G);
    FSD_LAUNCHED(c);
    if (c.bwork2.n < (size_t)n) c.bwork2.alloc(n);
    double *tmp = c.bwork2.p;
    FSD_CUDA(cudaMemsetAsync(tmp, 0, n * sizeof(double), c.stream));
    auto nf_op = [&](const double *x, double *y) {
      k_block_apply<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, G, 1, x, tmp);
      FSD_LAUNCHED(c);
      k_bsr_bead<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.brow.p, c.bcol.p, c.op64.bval.p,
                                                            c.op64.bdiag.p, tmp, y);
      FSD_LAUNCHED(c);
      k_block_apply<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, G, 0, y, y);
      FSD_LAUNCHED(c);
      FSD_CUDA(cudaGetLastError());
    };
    inf = lanczos_sqrt(c, nf_op, c.bwork.p, c.t2.p, tol, maxit, &ch_n);
    k_block_apply<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, Lb, 0, c.t2.p, c.bfnf.p);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  } else {
    FSD_CUDA(cudaMemsetAsync(c.bfnf.p, 0, n * sizeof(double), c.stream));
  }
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  c.brown_scale = std::sqrt(2.0 * kT / dt);
  c.brown_pending = true;
  if (iters_real) *iters_real = ir;
  if (iters_nf) *iters_nf = inf;
  if (change) *change = std::max(ch_r, ch_n);
}

void launch_brownian_rhs(Ctx &c, double *b) {
  if (!c.brown_pending) return;
  ProfScope ps(c, PG_MISC);
  k_brown_rhs_bead<<<ceil_div((int64_t)c.Nt * LDB, 256), 256, 0, c.stream>>>(c.Nt, c.bslip.p,
                                                                           c.brown_scale, b);
  FSD_LAUNCHED(c);
  k_brown_rhs_body<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(
      c.N, c.body_start.p, (const double4 *)c.lever64.p, c.bfnf.p, c.brown_scale, b,
      (int64_t)LDB * c.Nt);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void brownian_outputs(Ctx &c, double *slip_user_dev, double *fnf_user_dev) {
  if (slip_user_dev) {
    k_brown_out<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, c.bslip.p, 11,
                                                           c.brown_scale, slip_user_dev);
    FSD_LAUNCHED(c);
  }
  if (fnf_user_dev) {
    k_brown_out<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, c.perm_bead.p, c.bfnf.p, 6,
                                                           c.brown_scale, fnf_user_dev);
    FSD_LAUNCHED(c);
  }
  FSD_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------- drift helpers
// Random body vector dq of the random finite differences (appendix on the
// Brownian drift, Eq. rfd): Philox stream 4, index = user body id, calls 0
// and 1 give 8 normals of which the first 6 are used.
__global__ void k_dq_philox(int N, uint64_t seed, uint64_t step, double *user) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  double z[8];
  philox_normals4(seed, step, 4u, 0u, (uint32_t)J, z);
  philox_normals4(seed, step, 4u, 1u, (uint32_t)J, z + 4);
  for (int k = 0; k < 6; ++k) user[6 * (size_t)J + k] = z[k];
}

__global__ void k_scaled_diff(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                              double s, double *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = s * (a[i] - b[i]);
}

__global__ void k_axpy1(int64_t n, const double *__restrict__ x, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

static int small_grid(const Ctx &c, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4 * (int64_t)c.num_sms));
}

void launch_dq_philox(Ctx &c, uint64_t seed, uint64_t step, double *user) {
  k_dq_philox<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, seed, step, user);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_scaled_diff(Ctx &c, const double *a, const double *b, double s, double *out, int64_t n) {
  k_scaled_diff<<<small_grid(c, n), 256, 0, c.stream>>>(n, a, b, s, out);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_axpy(Ctx &c, const double *x, double *y, int64_t n) {
  k_axpy1<<<small_grid(c, n), 256, 0, c.stream>>>(n, x, y);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_add_velocity(Ctx &c, double *vel_int) { launch_axpy(c, c.vextra.p, vel_int, 6 * (int64_t)c.N); }

}  // namespace fsd
