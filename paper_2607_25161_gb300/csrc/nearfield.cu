// Near-field lubrication (BSR of 6x6 bead blocks over inter-body pairs,
// Alg. 1 step 1), the rigid-body constraint Sigma / Sigma^T (Eq. gc,
// Eq. sigma), the block-triangular preconditioner with one 6x6 LU per
// aggregate (Table 1; Alg. 1 step 1), the right-hand side of Eq. spm_agg,
// the outputs (Eq. stress_comp a, d) and the rigid-body integrator
// (Eq. EM1-EM3).
//
// Pair resistance (per inter-body pair i, j; n from i to j, gap h = r - 2a,
// eps = max(h, hmin)/a, cut-off eps_c = r_lub/a - 2):
//   relative surface velocity  s = (du_j - du_i) + (r/2) n x (dw_i + dw_j) + r E.n
//   relative rotation          t = dw_i - dw_j
//   dissipation s.G.s + t.Gt.t,  G = A nn + B (I - nn),  Gt = D (I - nn)
//   A = 6 pi eta a [q(eps) - q(eps_c)],  q(e) = 1/(4e) + (9/40) ln(1/e)
//   B = 6 pi eta a (1/6) ln(eps_c/eps),  D = 8 pi eta a^3 (1/10) ln(eps_c/eps)
// (leading equal-sphere lubrication terms, shifted to vanish at the cut-off).
#include "fsd_internal.cuh"

#include <algorithm>

namespace fsd {

struct PairCoef {
  double A, B, D;
};

// Gap clamp and surface roughness of the pair model.
struct LubModel {
  double hmin = 1e-3;          // the gap is clamped below at hmin
  double alpha = 0.0, h0 = 0.0;  // roughness (Sec. 4, Eq. tan_fric); alpha 0: smooth
};

static LubModel lub_model(const Ctx &c) {
  LubModel m;
  m.hmin = c.prm.lub_hmin;
  m.alpha = c.prm.rough_alpha;
  m.h0 = c.prm.rough_h0;
  return m;
}

__device__ __forceinline__ PairCoef lub_coef(double r, double a, double eta, double rcut,
                                            LubModel m) {
  const double ec = rcut / a - 2.0;
  double e = (r - 2.0 * a) / a;
  const double emin = m.hmin / a;
  if (e < emin) e = emin;
  const double qe = 0.25 / e + 0.225 * log(1.0 / e);
  const double qc = 0.25 / ec + 0.225 * log(1.0 / ec);
  PairCoef p;
  p.A = 6.0 * kPi * eta * a * (qe - qc);
  p.B = kPi * eta * a * log(ec / e);
  p.D = 0.8 * kPi * eta * a * a * a * log(ec / e);
  if (p.A < 0) p.A = 0;
  if (p.B < 0) p.B = 0;
  if (p.D < 0) p.D = 0;
  // rough surfaces: below the asperity height the sliding and rolling
  // resistances grow as 1/h (f vanishes at h0 and is added to the
  // normalised tangential coefficients)
  const double h = e * a;
  if (m.alpha > 0.0 && m.h0 > 0.0 && h < m.h0) {
    const double t = h / m.h0;
    const double f = m.alpha * (a / m.h0) * (1.0 / t - 3.0 * t + 2.0 * t * t);
    p.B += 6.0 * kPi * eta * a * f;
    p.D += 8.0 * kPi * eta * a * a * a * f;
  }
  return p;
}

// 6x6 blocks of one pair as seen from row i (n from i to j):
//   R_ii = [[G, -(rB/2) N], [(rB/2) N, (r^2 B/4 + D)(I - nn)]]
//   R_ij = [[-G, -(rB/2) N], [-(rB/2) N, (r^2 B/4 - D)(I - nn)]]
// with N v = n x v.
__device__ __forceinline__ void pair_blocks(const double n[3], double r, PairCoef p,
                                            double *Rii, double *Rij) {
  double G[9], Nm[9], Pt[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double nn = n[a] * n[b];
      double id = a == b ? 1.0 : 0.0;
      G[3 * a + b] = p.A * nn + p.B * (id - nn);
      Pt[3 * a + b] = id - nn;
    }
  Nm[0] = 0;
  Nm[1] = -n[2];
  Nm[2] = n[1];
  Nm[3] = n[2];
  Nm[4] = 0;
  Nm[5] = -n[0];
  Nm[6] = -n[1];
  Nm[7] = n[0];
  Nm[8] = 0;
  const double hb = 0.5 * r * p.B;
  const double cp = 0.25 * r * r * p.B + p.D, cm = 0.25 * r * r * p.B - p.D;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Rii[6 * a + b] = G[3 * a + b];
      Rii[6 * a + b + 3] = -hb * Nm[3 * a + b];
      Rii[6 * (a + 3) + b] = hb * Nm[3 * a + b];
      Rii[6 * (a + 3) + b + 3] = cp * Pt[3 * a + b];
      Rij[6 * a + b] = -G[3 * a + b];
      Rij[6 * a + b + 3] = -hb * Nm[3 * a + b];
      Rij[6 * (a + 3) + b] = -hb * Nm[3 * a + b];
      Rij[6 * (a + 3) + b + 3] = cm * Pt[3 * a + b];
    }
}

__device__ __forceinline__ void min_image(double &d0, double &d1, double &d2, double L,
                                          double tilt) {
  le_image(d0, d1, d2, L, tilt);
}

// Thread per bead row: off-diagonal blocks in CSR order, the diagonal block,
// and the preconditioner's diagonal block (pairs closer than r_p only).
__global__ void k_lub_assemble(int Nt, const double4 *__restrict__ pos,
                               const int *__restrict__ lnbr, const int *__restrict__ lcnt,
                               int lcap, const int *__restrict__ brow, int *bcol, double *bval64,
                               float *bval32, double *bdiag64, float *bdiag32, double *pdiag,
                               double L, double tilt, double a, double eta, double rcut,
                               double rp, LubModel lm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  double Dg[36], Pg[36];
  for (int k = 0; k < 36; ++k) Dg[k] = Pg[k] = 0.0;
  const double4 pi = pos[i];
  const int cnt = lcnt[i];
  for (int k = 0; k < cnt; ++k) {
    const int j = lnbr[(size_t)i * lcap + k];
    const double4 pj = pos[j];
    double d0 = pj.x - pi.x, d1 = pj.y - pi.y, d2 = pj.z - pi.z;
    min_image(d0, d1, d2, L, tilt);
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double n[3] = {d0 / r, d1 / r, d2 / r};
    PairCoef p = lub_coef(r, a, eta, rcut, lm);
    double Rii[36], Rij[36];
    pair_blocks(n, r, p, Rii, Rij);
    const int slot = brow[i] + k;
    bcol[slot] = j;
    for (int e = 0; e < 36; ++e) {
      bval64[(size_t)slot * 36 + e] = Rij[e];
      bval32[(size_t)slot * 36 + e] = (float)Rij[e];
      Dg[e] += Rii[e];
      if (r < rp) Pg[e] += Rii[e];
    }
  }
  for (int e = 0; e < 36; ++e) {
    bdiag64[(size_t)i * 36 + e] = Dg[e];
    bdiag32[(size_t)i * 36 + e] = (float)Dg[e];
    pdiag[(size_t)i * 36 + e] = Pg[e];
  }
}

// Sigma M Sigma^T for the bead lever r: Sigma = [[I, 0], [[r]x, I]].
__device__ __forceinline__ void sigma_congruence(const double *M, const double r[3], double *out) {
  double S[36] = {};
  for (int a = 0; a < 6; ++a) S[6 * a + a] = 1.0;
  // lower-left [r]x: ([r]x)_ab v_b = (r x v)_a
  S[6 * 3 + 1] = -r[2];
  S[6 * 3 + 2] = r[1];
  S[6 * 4 + 0] = r[2];
  S[6 * 4 + 2] = -r[0];
  S[6 * 5 + 0] = -r[1];
  S[6 * 5 + 1] = r[0];
  double T[36];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double s = 0;
      for (int k = 0; k < 6; ++k) s += S[6 * a + k] * M[6 * k + b];
      T[6 * a + b] = s;
    }
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double s = 0;
      for (int k = 0; k < 6; ++k) s += T[6 * a + k] * S[6 * b + k];
      out[6 * a + b] += s;
    }
}

// Thread per aggregate: B_J = sum_b Sigma_b (zeta0 I + R~_bb) Sigma_b^T,
// LU with partial pivoting, stored in place.
__global__ void k_schur_lu(int N, const int *__restrict__ body_start,
                           const double4 *__restrict__ lever, const double *__restrict__ pdiag,
                           double zeta0, double *schur, int *piv, int *flags) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  double Bm[36] = {};
  for (int b = body_start[J]; b < body_start[J + 1]; ++b) {
    double M[36];
    for (int e = 0; e < 36; ++e) M[e] = pdiag[(size_t)b * 36 + e];
    for (int a = 0; a < 6; ++a) M[6 * a + a] += zeta0;
    const double4 rv = lever[b];
    const double r[3] = {rv.x, rv.y, rv.z};
    sigma_congruence(M, r, Bm);
  }
  int pv[6];
  double scale = 0;
  for (int e = 0; e < 36; ++e) scale = fmax(scale, fabs(Bm[e]));
  for (int k = 0; k < 6; ++k) {
    int p = k;
    double best = fabs(Bm[6 * k + k]);
    for (int rr = k + 1; rr < 6; ++rr)
      if (fabs(Bm[6 * rr + k]) > best) {
        best = fabs(Bm[6 * rr + k]);
        p = rr;
      }
    pv[k] = p;
    if (best <= 1e-14 * scale || !(best == best)) {
      atomicOr(&flags[3], 1);
      Bm[6 * k + k] = (best == best && scale > 0) ? 1e-14 * scale : 1.0;
      p = k;
      pv[k] = k;
    }
    if (p != k)
      for (int cc = 0; cc < 6; ++cc) {
        double t = Bm[6 * k + cc];
        Bm[6 * k + cc] = Bm[6 * p + cc];
        Bm[6 * p + cc] = t;
      }
    for (int rr = k + 1; rr < 6; ++rr) {
      double f = Bm[6 * rr + k] / Bm[6 * k + k];
      Bm[6 * rr + k] = f;
      for (int cc = k + 1; cc < 6; ++cc) Bm[6 * rr + cc] -= f * Bm[6 * k + cc];
    }
  }
  for (int e = 0; e < 36; ++e) schur[(size_t)J * 36 + e] = Bm[e];
  for (int k = 0; k < 6; ++k) piv[J * 6 + k] = pv[k];
}

__device__ __forceinline__ void lu_solve6(const double *LU, const int *pv, double *v) {
  for (int k = 0; k < 6; ++k) {
    int p = pv[k];
    if (p != k) {
      double t = v[k];
      v[k] = v[p];
      v[p] = t;
    }
  }
  for (int a = 1; a < 6; ++a)
    for (int k = 0; k < a; ++k) v[a] -= LU[6 * a + k] * v[k];
  for (int a = 5; a >= 0; --a) {
    for (int k = a + 1; k < 6; ++k) v[a] -= LU[6 * a + k] * v[k];
    v[a] /= LU[6 * a + a];
  }
}

// Preconditioner (Table 1, aggregates; M_inf^-1 ~ zeta0 I):
//   y2 = r2 - zeta0 Sigma B^T r1;  z2 = -B_J^-1 y2;  z1 = zeta0 (r1 - B Sigma^T z2)
// LPA lanes per aggregate (a power of two covering its beads): the lanes sum
// Sigma B^T r1 over the aggregate's beads, reduce within their group, each
// solve the 6x6 LU system (the same numbers in every lane of the group), and
// then write the bead rows z1 of their beads from z2 held in registers.
// With col_dev non-null, r and z are column *col_dev of bases with leading
// dimension ld (the captured Arnoldi step, whose column index lives on the
// device), and z is also written to z2.
template <int LPA>
__global__ void __launch_bounds__(256) k_precond(int N, const int *__restrict__ body_start,
                                                 const double4 *__restrict__ lever,
                                                 const double *__restrict__ r, double *z,
                                                 const double *__restrict__ schur,
                                                 const int *__restrict__ piv, double zeta0,
                                                 int64_t off, const int *col_dev, int64_t ld,
                                                 double *z2) {
  if (col_dev) {
    const int64_t o = (int64_t)*col_dev * ld;
    r += o;
    z += o;
  }
  const int J = (blockIdx.x * blockDim.x + threadIdx.x) / LPA;
  const int sub = threadIdx.x & (LPA - 1);
  const bool active = J < N;
  const int b0 = active ? body_start[J] : 0, b1 = active ? body_start[J + 1] : 0;
  double g[6] = {0, 0, 0, 0, 0, 0};
  for (int b = b0 + sub; b < b1; b += LPA) {
    const double *rb = r + (size_t)b * LDB;
    const double4 rv = lever[b];
    g[0] += rb[0];
    g[1] += rb[1];
    g[2] += rb[2];
    g[3] += rb[3] + rv.y * rb[2] - rv.z * rb[1];
    g[4] += rb[4] + rv.z * rb[0] - rv.x * rb[2];
    g[5] += rb[5] + rv.x * rb[1] - rv.y * rb[0];
  }
#pragma unroll
  for (int o = LPA / 2; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
  if (!active) return;
  double v[6];
  for (int k = 0; k < 6; ++k) v[k] = r[off + 6 * (size_t)J + k] - zeta0 * g[k];
  lu_solve6(schur + (size_t)J * 36, piv + 6 * J, v);
  // u = z2 = -v
  if (sub == 0)
    for (int k = 0; k < 6; ++k) {
      z[off + 6 * (size_t)J + k] = -v[k];
      if (z2) z2[off + 6 * (size_t)J + k] = -v[k];
    }
  for (int b = b0 + sub; b < b1; b += LPA) {
    const double4 rv = lever[b];
    const double *ri = r + (size_t)b * LDB;
    double zo[LDB];
    zo[0] = zeta0 * (ri[0] + (v[0] + v[4] * rv.z - v[5] * rv.y));
    zo[1] = zeta0 * (ri[1] + (v[1] + v[5] * rv.x - v[3] * rv.z));
    zo[2] = zeta0 * (ri[2] + (v[2] + v[3] * rv.y - v[4] * rv.x));
    zo[3] = zeta0 * (ri[3] + v[3]);
    zo[4] = zeta0 * (ri[4] + v[4]);
    zo[5] = zeta0 * (ri[5] + v[5]);
    for (int k = 6; k < 11; ++k) zo[k] = zeta0 * ri[k];
    zo[11] = 0.0;
    double *zi = z + (size_t)b * LDB;
    for (int k = 0; k < LDB; ++k) zi[k] = zo[k];
    if (z2) {
      double *zj = z2 + (size_t)b * LDB;
      for (int k = 0; k < LDB; ++k) zj[k] = zo[k];
    }
  }
}

// -------------------------------------------------- aggregate rows (matvec)
template <typename T>
struct LV;
template <>
struct LV<double> {
  using type = double4;
};
template <>
struct LV<float> {
  using type = float4;
};

// LPA lanes per aggregate (a power of two covering its beads): y2_J =
// Sigma B^T x1 - [Sigma R Sigma^T x2]_J, the BSR row of every bead evaluated
// with its neighbours' rigid velocities formed on the fly from x2 (constraint
// scatter fused into the SpMV).
template <typename T, int LPA>
__global__ void __launch_bounds__(256) k_body_rows(
    int N, const int *__restrict__ body_start, const int *__restrict__ bead_body,
    const typename LV<T>::type *__restrict__ lever, const double *__restrict__ x, double *y,
    const int *__restrict__ brow, const int *__restrict__ bcol, const T *__restrict__ bval,
    const T *__restrict__ bdiag, int with_lub, int64_t off, T sgn_bead, T sgn_lub) {
  const int J = (blockIdx.x * blockDim.x + threadIdx.x) / LPA;
  const int sub = threadIdx.x & (LPA - 1);
  const bool active = J < N;
  const int b0 = active ? body_start[J] : 0, b1 = active ? body_start[J + 1] : 0;
  T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int b = b0 + sub; b < b1; b += LPA) {
    const double *xb = x + (size_t)b * LDB;
    const auto rv = lever[b];
    const T F0 = (T)xb[0], F1 = (T)xb[1], F2 = (T)xb[2];
    T f[6] = {F0, F1, F2, (T)xb[3], (T)xb[4], (T)xb[5]};
    if (with_lub) {
      T v[6];
      {
        const double *u = x + off + 6 * (size_t)bead_body[b];
        const T u0 = (T)u[0], u1 = (T)u[1], u2 = (T)u[2], w0 = (T)u[3], w1 = (T)u[4], w2 = (T)u[5];
        v[0] = u0 + w1 * rv.z - w2 * rv.y;
        v[1] = u1 + w2 * rv.x - w0 * rv.z;
        v[2] = u2 + w0 * rv.y - w1 * rv.x;
        v[3] = w0;
        v[4] = w1;
        v[5] = w2;
      }
      T g[6];
      const T *D = bdiag + (size_t)b * 36;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) s += D[6 * a + c] * v[c];
        g[a] = s;
      }
      for (int k = brow[b]; k < brow[b + 1]; ++k) {
        const int cidx = bcol[k];
        const double *u = x + off + 6 * (size_t)bead_body[cidx];
        const auto rc = lever[cidx];
        const T u0 = (T)u[0], u1 = (T)u[1], u2 = (T)u[2], w0 = (T)u[3], w1 = (T)u[4], w2 = (T)u[5];
        T vc[6];
        vc[0] = u0 + w1 * rc.z - w2 * rc.y;
        vc[1] = u1 + w2 * rc.x - w0 * rc.z;
        vc[2] = u2 + w0 * rc.y - w1 * rc.x;
        vc[3] = w0;
        vc[4] = w1;
        vc[5] = w2;
        const T *Bk = bval + (size_t)k * 36;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          T s = T(0);
#pragma unroll
          for (int c = 0; c < 6; ++c) s += Bk[6 * a + c] * vc[c];
          g[a] += s;
        }
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) f[a] = sgn_bead * f[a] + sgn_lub * g[a];
    } else {
#pragma unroll
      for (int a = 0; a < 6; ++a) f[a] = sgn_bead * f[a];
    }
    // Sigma: (f_F, f_L + r x f_F)
    acc[0] += f[0];
    acc[1] += f[1];
    acc[2] += f[2];
    acc[3] += f[3] + rv.y * f[2] - rv.z * f[1];
    acc[4] += f[4] + rv.z * f[0] - rv.x * f[2];
    acc[5] += f[5] + rv.x * f[1] - rv.y * f[0];
  }
#pragma unroll
  for (int o = LPA / 2; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (active && sub == 0) {
    double *yr = y + off + 6 * (size_t)J;
    for (int k = 0; k < 6; ++k) yr[k] = (double)acc[k];
  }
}

// --------------------------------------- near-field bead forces and stresslets
// Thread per bead: near-field force / torque / stresslet from the pair forms
// at body velocities dU (may be NULL = 0) and strain E (6 comps: xx yy zz xy xz yz).
//   du_b = dU_J + dOm_J x r_b - E r_b,   dw_b = dOm_J
//   F_i  = G s,  torque_i = (r/2) n x (G s) - D (I-nn)(dw_i - dw_j),
//   S_i  = (r/2) sym(G s (x) n)  (5 basis coordinates)
__global__ void k_nf_bead(int Nt, const double4 *__restrict__ pos,
                          const double4 *__restrict__ lever, const int *__restrict__ bead_body,
                          const int *__restrict__ lnbr, const int *__restrict__ lcnt, int lcap,
                          const double *__restrict__ dU, double e00, double e11, double e22,
                          double e01, double e02, double e12, double *fnf, double *snf, double L,
                          double tilt, double a, double eta, double rcut, LubModel lm,
                          const double *__restrict__ tilt_dev) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  if (tilt_dev) tilt = *tilt_dev;  // Lees-Edwards steps: the offset in device memory
  const double E[9] = {e00, e01, e02, e01, e11, e12, e02, e12, e22};
  auto bead_vel = [&](int b, double *du, double *dw) {
    const double4 rv = lever[b];
    const double r[3] = {rv.x, rv.y, rv.z};
    double U[6] = {0, 0, 0, 0, 0, 0};
    if (dU)
      for (int k = 0; k < 6; ++k) U[k] = dU[6 * (size_t)bead_body[b] + k];
    du[0] = U[0] + U[4] * r[2] - U[5] * r[1];
    du[1] = U[1] + U[5] * r[0] - U[3] * r[2];
    du[2] = U[2] + U[3] * r[1] - U[4] * r[0];
    for (int a2 = 0; a2 < 3; ++a2) du[a2] -= E[3 * a2] * r[0] + E[3 * a2 + 1] * r[1] + E[3 * a2 + 2] * r[2];
    dw[0] = U[3];
    dw[1] = U[4];
    dw[2] = U[5];
  };
  double dui[3], dwi[3];
  bead_vel(i, dui, dwi);
  double F[6] = {0, 0, 0, 0, 0, 0};
  double Sm[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
  const double4 pi = pos[i];
  for (int k = 0; k < lcnt[i]; ++k) {
    const int j = lnbr[(size_t)i * lcap + k];
    const double4 pj = pos[j];
    double d0 = pj.x - pi.x, d1 = pj.y - pi.y, d2 = pj.z - pi.z;
    min_image(d0, d1, d2, L, tilt);
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double n[3] = {d0 / r, d1 / r, d2 / r};
    PairCoef p = lub_coef(r, a, eta, rcut, lm);
    double duj[3], dwj[3];
    bead_vel(j, duj, dwj);
    double sw[3] = {dwi[0] + dwj[0], dwi[1] + dwj[1], dwi[2] + dwj[2]};
    double s[3];
    s[0] = duj[0] - dui[0] + 0.5 * r * (n[1] * sw[2] - n[2] * sw[1]) +
           r * (E[0] * n[0] + E[1] * n[1] + E[2] * n[2]);
    s[1] = duj[1] - dui[1] + 0.5 * r * (n[2] * sw[0] - n[0] * sw[2]) +
           r * (E[3] * n[0] + E[4] * n[1] + E[5] * n[2]);
    s[2] = duj[2] - dui[2] + 0.5 * r * (n[0] * sw[1] - n[1] * sw[0]) +
           r * (E[6] * n[0] + E[7] * n[1] + E[8] * n[2]);
    const double ns = n[0] * s[0] + n[1] * s[1] + n[2] * s[2];
    double Gs[3];
    for (int a2 = 0; a2 < 3; ++a2) Gs[a2] = p.A * ns * n[a2] + p.B * (s[a2] - ns * n[a2]);
    double t[3] = {dwi[0] - dwj[0], dwi[1] - dwj[1], dwi[2] - dwj[2]};
    const double nt = n[0] * t[0] + n[1] * t[1] + n[2] * t[2];
    F[0] += Gs[0];
    F[1] += Gs[1];
    F[2] += Gs[2];
    F[3] += 0.5 * r * (n[1] * Gs[2] - n[2] * Gs[1]) - p.D * (t[0] - nt * n[0]);
    F[4] += 0.5 * r * (n[2] * Gs[0] - n[0] * Gs[2]) - p.D * (t[1] - nt * n[1]);
    F[5] += 0.5 * r * (n[0] * Gs[1] - n[1] * Gs[0]) - p.D * (t[2] - nt * n[2]);
    const double hr = 0.5 * r;
    Sm[0] += hr * Gs[0] * n[0];
    Sm[1] += hr * Gs[1] * n[1];
    Sm[2] += hr * Gs[2] * n[2];
    Sm[3] += hr * 0.5 * (Gs[0] * n[1] + Gs[1] * n[0]);
    Sm[4] += hr * 0.5 * (Gs[0] * n[2] + Gs[2] * n[0]);
    Sm[5] += hr * 0.5 * (Gs[1] * n[2] + Gs[2] * n[1]);
  }
  for (int k = 0; k < 6; ++k) fnf[(size_t)i * 6 + k] = F[k];
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637, s2 = 1.41421356237309504880;
  snf[(size_t)i * 5 + 0] = r2i * (Sm[0] - Sm[1]);
  snf[(size_t)i * 5 + 1] = r6i * (2.0 * Sm[2] - Sm[0] - Sm[1]);
  snf[(size_t)i * 5 + 2] = s2 * Sm[3];
  snf[(size_t)i * 5 + 3] = s2 * Sm[4];
  snf[(size_t)i * 5 + 4] = s2 * Sm[5];
}

// ---------------------------------------------------------------- RHS
// Bead rows: (E r_b, 0, e5).  Aggregate rows: -(FT_J + sum_b Sigma_b f0_b),
// f0 the near-field bead forces with every body moving with the ambient flow
// at its centroid (dU = 0).
__global__ void k_rhs_bead(int Nt, const double4 *__restrict__ lever, double e00, double e11,
                           double e22, double e01, double e02, double e12, double *b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double4 rv = lever[i];
  double *bi = b + (size_t)i * LDB;
  bi[0] = e00 * rv.x + e01 * rv.y + e02 * rv.z;
  bi[1] = e01 * rv.x + e11 * rv.y + e12 * rv.z;
  bi[2] = e02 * rv.x + e12 * rv.y + e22 * rv.z;
  bi[3] = bi[4] = bi[5] = 0.0;
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637, s2 = 1.41421356237309504880;
  bi[6] = r2i * (e00 - e11);
  bi[7] = r6i * (2.0 * e22 - e00 - e11);
  bi[8] = s2 * e01;
  bi[9] = s2 * e02;
  bi[10] = s2 * e12;
  bi[11] = 0.0;
}

__global__ void k_rhs_body(int N, const int *__restrict__ body_start,
                           const double4 *__restrict__ lever, const double *__restrict__ fnf,
                           const double *__restrict__ ft, double *b, int64_t off, int have_nf) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  double g[6] = {0, 0, 0, 0, 0, 0};
  if (have_nf)
    for (int bb = body_start[J]; bb < body_start[J + 1]; ++bb) {
      const double *f = fnf + (size_t)bb * 6;
      const double4 rv = lever[bb];
      g[0] += f[0];
      g[1] += f[1];
      g[2] += f[2];
      g[3] += f[3] + rv.y * f[2] - rv.z * f[1];
      g[4] += f[4] + rv.z * f[0] - rv.x * f[2];
      g[5] += f[5] + rv.x * f[1] - rv.y * f[0];
    }
  for (int k = 0; k < 6; ++k) b[off + 6 * (size_t)J + k] = -((ft ? ft[6 * (size_t)J + k] : 0.0) + g[k]);
}

// ---------------------------------------------------------------- outputs
// Thread per aggregate: lab-frame velocity and S^H + S^C (S^H alone when
// with_constraint is 0).
__global__ void k_outputs(int N, const int *__restrict__ body_start,
                          const double4 *__restrict__ lever, const double *__restrict__ X,
                          const double *__restrict__ x, const double *__restrict__ fnf,
                          const double *__restrict__ snf, int have_nf, double gamma,
                          double *vel, double *str, int64_t off, int with_constraint) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  const double *u = x + off + 6 * (size_t)J;
  double *v = vel + 6 * (size_t)J;
  v[0] = u[0] + gamma * X[3 * J + 1];
  v[1] = u[1];
  v[2] = u[2];
  v[3] = u[3];
  v[4] = u[4];
  v[5] = u[5] - 0.5 * gamma;
  if (!str) return;
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637;
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = body_start[J]; b < body_start[J + 1]; ++b) {
    const double *xb = x + (size_t)b * LDB;
    double s5[5];
    for (int k = 0; k < 5; ++k) s5[k] = xb[6 + k] + (have_nf ? snf[(size_t)b * 5 + k] : 0.0);
    const double Sxx = r2i * s5[0] - r6i * s5[1], Syy = -r2i * s5[0] - r6i * s5[1],
                 Szz = 2.0 * r6i * s5[1];
    const double Sxy = r2i * s5[2], Sxz = r2i * s5[3], Syz = r2i * s5[4];
    double F[3] = {xb[0], xb[1], xb[2]};
    if (have_nf)
      for (int k = 0; k < 3; ++k) F[k] += fnf[(size_t)b * 6 + k];
    const double4 rv = lever[b];
    const double r[3] = {rv.x, rv.y, rv.z};
    const double Sh[9] = {Sxx, Sxy, Sxz, Sxy, Syy, Syz, Sxz, Syz, Szz};
    for (int p = 0; p < 3; ++p)
      for (int qq = 0; qq < 3; ++qq)
        S[3 * p + qq] += Sh[3 * p + qq] + (with_constraint ? 0.5 * (r[p] * F[qq] + F[p] * r[qq]) : 0.0);
  }
  for (int k = 0; k < 9; ++k) str[9 * (size_t)J + k] = S[k];
}

// ---------------------------------------------------------------- integrator
__global__ void k_integrate(int N, const double *__restrict__ vel, double dt, double *X,
                            double *q, double affine_gamma) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  const double *u = vel + 6 * (size_t)J;
  // affine_gamma != 0: disturbance motion only (U - U_inf, Omega - Omega_inf)
  const double ux = u[0] - affine_gamma * X[3 * J + 1];
  X[3 * J] += ux * dt;
  X[3 * J + 1] += u[1] * dt;
  X[3 * J + 2] += u[2] * dt;
  double *qq = q + 4 * (size_t)J;
  const double w = qq[0], x = qq[1], y = qq[2], z = qq[3];
  const double o0 = u[3], o1 = u[4], o2 = u[5] + 0.5 * affine_gamma;
  // (0, Omega) (x) q
  const double dw = -(o0 * x + o1 * y + o2 * z);
  const double dx = o0 * w + (o1 * z - o2 * y);
  const double dy = o1 * w + (o2 * x - o0 * z);
  const double dz = o2 * w + (o0 * y - o1 * x);
  double nw = w + 0.5 * dt * dw, nx = x + 0.5 * dt * dx, ny = y + 0.5 * dt * dy,
         nz = z + 0.5 * dt * dz;
  const double inv = 1.0 / sqrt(nw * nw + nx * nx + ny * ny + nz * nz);
  qq[0] = nw * inv;
  qq[1] = nx * inv;
  qq[2] = ny * inv;
  qq[3] = nz * inv;
}

// ------------------------------------------------------------ Hertz contact
// Normal contact between beads of different aggregates (Sec. 4: F_N =
// k_n delta^1.5 n, delta = 2a - r, n along the line of centres; the rod
// benchmark of Sec. 3.3): bead i receives kn delta^1.5 (x_i - x_j)/r from
// each such neighbour j.  The mobility neighbour list (r < R_c, R_c > 2a)
// holds every pair that can touch.
// Central force between two beads of different aggregates at distance r
// (positive: repulsive): Hertz k_n delta^1.5 under overlap, and the DLVO
// force -dV/dr (Sec. 4) within r_cut.  The van der Waals part is the
// derivative of the sphere-sphere Hamaker energy
//   -(A_H/6) [2a^2/(r^2 - 4a^2) + 2a^2/r^2 + ln((r^2 - 4a^2)/r^2)]
// taken at r' = max(r, 2a) + h_c (gap shifted by h_c, held at its contact
// value under overlap); the double layer (a^2/r) Z exp(-kappa (r - 2a)).
__device__ __forceinline__ double pair_force_scalar(double r, double a, const fsd_pair_forces &pf) {
  double f = 0.0;
  const double two_a = 2.0 * a;
  if (pf.kn > 0.0 && r < two_a) {
    const double delta = two_a - r;
    f += pf.kn * delta * sqrt(delta);
  }
  if (r < pf.r_cut) {
    if (pf.hamaker != 0.0) {
      const double rv = fmax(r, two_a) + pf.h_c;
      const double s2 = two_a * two_a, q = rv * rv - s2, a2 = a * a;
      const double dv = -4.0 * a2 * rv / (q * q) - 4.0 * a2 / (rv * rv * rv) + 2.0 * rv / q - 2.0 / rv;
      f += pf.hamaker / 6.0 * dv;  // -(dV/dr) with V = -(A_H/6)(...)
    }
    if (pf.zeta != 0.0) {
      const double e = exp(-pf.kappa * (r - two_a));
      f += a * a * pf.zeta * e * (1.0 / (r * r) + pf.kappa / r);
    }
  }
  return f;
}

__global__ void k_contact_bead(int Nt, const double4 *__restrict__ pos, const int *__restrict__ nbr,
                               const int *__restrict__ ncnt, int cap,
                               const int *__restrict__ bead_body, double L, double tilt,
                               double a, fsd_pair_forces pf, double *fb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double4 p = pos[i];
  const int bi = bead_body[i];
  const double reach = fmax(2.0 * a, pf.r_cut);
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  const int n = ncnt[i];
  for (int k = 0; k < n; ++k) {
    const int j = nbr[(size_t)i * cap + k];
    if (bead_body[j] == bi) continue;
    const double4 q = pos[j];
    double d0 = p.x - q.x, d1 = p.y - q.y, d2 = p.z - q.z;
    le_image(d0, d1, d2, L, tilt);
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (r2 >= reach * reach || r2 == 0.0) continue;
    const double r = sqrt(r2);
    const double s = pair_force_scalar(r, a, pf) / r;
    f0 += s * d0;
    f1 += s * d1;
    f2 += s * d2;
  }
  fb[3 * (size_t)i] = f0;
  fb[3 * (size_t)i + 1] = f1;
  fb[3 * (size_t)i + 2] = f2;
}

// Aggregate force and torque about the centroid: F_J = sum_b F_b,
// T_J = sum_b r_b x F_b.
__global__ void k_contact_body(int N, const int *__restrict__ body_start,
                               const double4 *__restrict__ lever, const double *__restrict__ fb,
                               double *ft) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  double o[6] = {0, 0, 0, 0, 0, 0};
  for (int b = body_start[J]; b < body_start[J + 1]; ++b) {
    const double f0 = fb[3 * (size_t)b], f1 = fb[3 * (size_t)b + 1], f2 = fb[3 * (size_t)b + 2];
    const double4 r = lever[b];
    o[0] += f0;
    o[1] += f1;
    o[2] += f2;
    o[3] += r.y * f2 - r.z * f1;
    o[4] += r.z * f0 - r.x * f2;
    o[5] += r.x * f1 - r.y * f0;
  }
  for (int k = 0; k < 6; ++k) ft[6 * (size_t)J + k] = o[k];
}

// --------------------------------------- pairwise near-field Brownian force
// The near-field resistance is a sum over pairs of the pair model's
// dissipation form, R_FU^nf = sum_p K_p^T K_p with
// K_p = [G^(1/2) Ls; Gt^(1/2) Lt] (6 x 12): s = (du_j - du_i) +
// (r/2) n x (dw_i + dw_j) and t = dw_i - dw_j are the pair's relative surface
// velocity and rotation, G = A nn + B (I - nn), Gt = D (I - nn).  So
// F = -sum_p K_p^T eta_p with 6 independent normals per pair has covariance
// exactly R_FU^nf (the sign of a centred Gaussian changes nothing; this one
// makes the force on bead i +g_s): with g_s = G^(1/2) eta_s and
// g_t = Gt^(1/2) eta_t, force_i = g_s, torque_i = (r/2) n x g_s - g_t,
// force_j = -g_s, torque_j = (r/2) n x g_s + g_t.  Thread per bead; each pair is taken once,
// by its bead of smaller input index; the pair noise from Philox with
// counter (i, 5 * 256 + call, j, step mod 2^32) in input order.
__global__ void k_nf_pairwise(int Nt, const double4 *__restrict__ pos, const int *__restrict__ lnbr,
                              const int *__restrict__ lcnt, int lcap, const int *__restrict__ perm,
                              double L, double tilt, double a, double eta, double rcut, LubModel lm,
                              uint64_t seed, uint64_t step, double *f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const int iu = perm[i];
  const double4 pi = pos[i];
  const int cnt = lcnt[i];
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int k = 0; k < cnt; ++k) {
    const int j = lnbr[(size_t)i * lcap + k];
    const int ju = perm[j];
    if (ju < iu) continue;  // the pair belongs to its bead of smaller input index
    const double4 pj = pos[j];
    double d0 = pj.x - pi.x, d1 = pj.y - pi.y, d2 = pj.z - pi.z;
    min_image(d0, d1, d2, L, tilt);
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double n[3] = {d0 / r, d1 / r, d2 / r};
    const PairCoef pc = lub_coef(r, a, eta, rcut, lm);
    double z[8];
    for (int call = 0; call < 2; ++call) {
      uint32_t cw[4] = {(uint32_t)iu, (5u << 8) | (uint32_t)call, (uint32_t)ju, (uint32_t)step};
      philox4x32_10(cw, k0, k1);
      const double sc = 2.3283064365386963e-10;  // 2^-32
      const double u0 = ((double)cw[0] + 1.0) * sc, u1 = ((double)cw[1] + 1.0) * sc;
      const double u2 = ((double)cw[2] + 1.0) * sc, u3 = ((double)cw[3] + 1.0) * sc;
      const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
      double s0, c0, s1, c1;
      sincospi(2.0 * u1, &s0, &c0);
      sincospi(2.0 * u3, &s1, &c1);
      z[4 * call] = r0 * c0;
      z[4 * call + 1] = r0 * s0;
      z[4 * call + 2] = r1 * c1;
      z[4 * call + 3] = r1 * s1;
    }
    const double sA = sqrt(pc.A), sB = sqrt(pc.B), sD = sqrt(pc.D);
    const double ns = n[0] * z[0] + n[1] * z[1] + n[2] * z[2];
    const double nt = n[0] * z[3] + n[1] * z[4] + n[2] * z[5];
    double gs[3], gt[3];
    for (int e = 0; e < 3; ++e) {
      gs[e] = sA * ns * n[e] + sB * (z[e] - ns * n[e]);
      gt[e] = sD * (z[3 + e] - nt * n[e]);
    }
    const double h = 0.5 * r;
    const double cx[3] = {h * (n[1] * gs[2] - n[2] * gs[1]), h * (n[2] * gs[0] - n[0] * gs[2]),
                          h * (n[0] * gs[1] - n[1] * gs[0])};
    for (int e = 0; e < 3; ++e) {
      atomicAdd(&f[(size_t)i * LDB + e], gs[e]);
      atomicAdd(&f[(size_t)i * LDB + 3 + e], cx[e] - gt[e]);
      atomicAdd(&f[(size_t)j * LDB + e], -gs[e]);
      atomicAdd(&f[(size_t)j * LDB + 3 + e], cx[e] + gt[e]);
    }
  }
}

// ============================================================ host side

static void strain6(double shear, double *e) {
  // E_inf = gamma/2 (xy + yx): xx yy zz xy xz yz
  e[0] = e[1] = e[2] = e[4] = e[5] = 0.0;
  e[3] = 0.5 * shear;
}

void build_lubrication(Ctx &c) {
  ProfScope ps(c, PG_LUB);
  const int Nt = c.Nt;
  // CSR rows from the lubrication neighbour counts
  std::vector<int> cnt(Nt);
  FSD_CUDA(cudaMemcpyAsync(cnt.data(), c.lcnt.p, Nt * sizeof(int), cudaMemcpyDeviceToHost,
                           c.stream));
  FSD_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int> row(Nt + 1, 0);
  for (int i = 0; i < Nt; ++i) row[i + 1] = row[i] + cnt[i];
  const int nnz = row[Nt];
  c.n_lub = nnz;
  if (nnz > c.nnz_cap || !c.bcol.p) {
    c.nnz_cap = std::max(nnz + nnz / 4 + 64, 64);
    c.bcol.alloc(c.nnz_cap);
    c.op64.bval.alloc((size_t)c.nnz_cap * 36);
    c.op32.bval.alloc((size_t)c.nnz_cap * 36);
  }
  FSD_CUDA(cudaMemcpyAsync(c.brow.p, row.data(), (Nt + 1) * sizeof(int), cudaMemcpyHostToDevice,
                           c.stream));
  const double rl = c.prm.lub_cutoff > 2.0 * c.a ? c.prm.lub_cutoff : 2.0 * c.a;
  k_lub_assemble<<<ceil_div(Nt, 128), 128, 0, c.stream>>>(
      Nt, (const double4 *)c.pos64.p, c.lnbr.p, c.lcnt.p, c.lcap, c.brow.p, c.bcol.p,
      c.op64.bval.p, c.op32.bval.p, c.op64.bdiag.p, c.op32.bdiag.p, c.pdiag.p, c.L, c.tilt, c.a, c.eta, rl,
      c.prm.precond_cutoff, lub_model(c));
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  const double zeta0 = 6.0 * kPi * c.eta * c.a;
  k_schur_lu<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.body_start.p,
                                                      (const double4 *)c.lever64.p, c.pdiag.p,
                                                      zeta0, c.schur.p, c.piv.p, c.flags.p);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

template <typename T>
static const typename LV<T>::type *lever_ptr(Ctx &c);
template <>
const double4 *lever_ptr<double>(Ctx &c) {
  return (const double4 *)c.lever64.p;
}
template <>
const float4 *lever_ptr<float>(Ctx &c) {
  return (const float4 *)c.op32.lever.p;
}
template <typename T>
static OpData<T> &opx(Ctx &c);
template <>
OpData<double> &opx<double>(Ctx &c) {
  return c.op64;
}
template <>
OpData<float> &opx<float>(Ctx &c) {
  return c.op32;
}

template <typename T>
static void body_rows_launch(Ctx &c, const double *x, double *y, int lub, T sgn_bead, T sgn_lub) {
  OpData<T> &op = opx<T>(c);
  const int64_t off = (int64_t)LDB * c.Nt;
#define FSD_BODY_ROWS(LPA)                                                                      \
  k_body_rows<T, LPA><<<ceil_div((int64_t)c.N * LPA, 256), 256, 0, c.stream>>>(                \
      c.N, c.body_start.p, c.bead_body.p, lever_ptr<T>(c), x, y, c.brow.p, c.bcol.p, op.bval.p, \
      op.bdiag.p, lub, off, sgn_bead, sgn_lub)
  switch (c.body_lanes) {
    case 4: FSD_BODY_ROWS(4); break;
    case 8: FSD_BODY_ROWS(8); break;
    case 16: FSD_BODY_ROWS(16); break;
    default: FSD_BODY_ROWS(32); break;
  }
#undef FSD_BODY_ROWS
}

template <typename T>
void launch_body_rows(Ctx &c, const double *x, double *y, bool with_lub) {
  ProfScope ps(c, PG_BODY);
  const bool lub = with_lub && c.n_lub > 0;
  body_rows_launch<T>(c, x, y, lub ? 1 : 0, T(1), T(-1));
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// out = RR dU (aggregate rows only; the bead part of x is ignored).
template <typename T>
void launch_lub_apply(Ctx &c, const double *x, double *y) {
  ProfScope ps(c, PG_BODY);
  body_rows_launch<T>(c, x, y, c.n_lub > 0 ? 1 : 0, T(0), T(1));
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

static void precond_launch(Ctx &c, const double *r, double *z, const int *col_dev, int64_t ld,
                           double *z2) {
  ProfScope ps(c, PG_PRECOND);
  const int64_t off = (int64_t)LDB * c.Nt;
  const double zeta0 = 6.0 * kPi * c.eta * c.a;
#define FSD_PRECOND(LPA)                                                                  \
  k_precond<LPA><<<ceil_div((int64_t)c.N * LPA, 256), 256, 0, c.stream>>>(                \
      c.N, c.body_start.p, (const double4 *)c.lever64.p, r, z, c.schur.p, c.piv.p, zeta0, off, \
      col_dev, ld, z2)
  switch (c.body_lanes) {
    case 4: FSD_PRECOND(4); break;
    case 8: FSD_PRECOND(8); break;
    case 16: FSD_PRECOND(16); break;
    default: FSD_PRECOND(32); break;
  }
#undef FSD_PRECOND
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_precond(Ctx &c, const double *r, double *z) { precond_launch(c, r, z, nullptr, 0, nullptr); }

void launch_precond_col(Ctx &c, const double *V, double *Z, int64_t ld, const int *col_dev,
                        double *z2) {
  precond_launch(c, V, Z, col_dev, ld, z2);
}

void launch_rhs(Ctx &c, const double *ft_int, double shear, double *b) {
  ProfScope ps(c, PG_MISC);
  double e[6];
  strain6(shear, e);
  const int64_t off = (int64_t)LDB * c.Nt;
  k_rhs_bead<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, (const double4 *)c.lever64.p, e[0],
                                                       e[1], e[2], e[3], e[4], e[5], b);
  FSD_LAUNCHED(c);
  const bool nf = c.n_lub > 0;
  if (nf) {
    const double rl = c.prm.lub_cutoff;
    k_nf_bead<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(
        c.Nt, (const double4 *)c.pos64.p, (const double4 *)c.lever64.p, c.bead_body.p, c.lnbr.p,
        c.lcnt.p, c.lcap, nullptr, e[0], e[1], e[2], e[3], e[4], e[5], c.fnf.p, c.snf.p, c.L, c.tilt, c.a,
        c.eta, rl, lub_model(c), tilt_dev_ptr(c));
    FSD_LAUNCHED(c);
  }
  k_rhs_body<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.body_start.p,
                                                      (const double4 *)c.lever64.p, c.fnf.p,
                                                      ft_int, b, off, nf ? 1 : 0);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_outputs(Ctx &c, const double *x, double shear, double *vel_int, double *str_int) {
  ProfScope ps(c, PG_MISC);
  double e[6];
  strain6(shear, e);
  const int64_t off = (int64_t)LDB * c.Nt;
  const bool nf = c.n_lub > 0;
  if (nf) {
    k_nf_bead<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(
        c.Nt, (const double4 *)c.pos64.p, (const double4 *)c.lever64.p, c.bead_body.p, c.lnbr.p,
        c.lcnt.p, c.lcap, x + off, e[0], e[1], e[2], e[3], e[4], e[5], c.fnf.p, c.snf.p, c.L, c.tilt, c.a,
        c.eta, c.prm.lub_cutoff, lub_model(c), tilt_dev_ptr(c));
    FSD_LAUNCHED(c);
  }
  k_outputs<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.body_start.p,
                                                     (const double4 *)c.lever64.p, c.X.p, x,
                                                     c.fnf.p, c.snf.p, nf ? 1 : 0, shear, vel_int,
                                                     str_int, off, c.str_hydro ? 0 : 1);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_integrate(Ctx &c, const double *vel_int, double dt, double shear) {
  ProfScope ps(c, PG_MISC);
  const double ag = (c.prm.flags & FSD_FLAG_COMOVING) ? shear : 0.0;
  k_integrate<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, vel_int, dt, c.X.p, c.q.p, ag);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_contact(Ctx &c, const fsd_pair_forces &pf, double *fb_scratch, double *ft_int) {
  ProfScope ps(c, PG_MISC);
  k_contact_bead<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(
      c.Nt, (const double4 *)c.pos64.p, c.nbr.p, c.ncnt.p, c.cap, c.bead_body.p, c.L, c.tilt, c.a, pf,
      fb_scratch);
  FSD_LAUNCHED(c);
  k_contact_body<<<ceil_div(c.N, 128), 128, 0, c.stream>>>(c.N, c.body_start.p,
                                                          (const double4 *)c.lever64.p, fb_scratch, ft_int);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_nf_pairwise(Ctx &c, uint64_t seed, uint64_t step, double *f) {
  FSD_CUDA(cudaMemsetAsync(f, 0, (size_t)c.nunk * sizeof(double), c.stream));
  k_nf_pairwise<<<ceil_div(c.Nt, 64), 64, 0, c.stream>>>(
      c.Nt, (const double4 *)c.pos64.p, c.lnbr.p, c.lcnt.p, c.lcap, c.perm_bead.p, c.L, c.tilt, c.a,
      c.eta, c.prm.lub_cutoff, lub_model(c), seed, step, f);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

template void launch_body_rows<float>(Ctx &, const double *, double *, bool);
template void launch_body_rows<double>(Ctx &, const double *, double *, bool);
template void launch_lub_apply<float>(Ctx &, const double *, double *);
template void launch_lub_apply<double>(Ctx &, const double *, double *);

}  // namespace fsd
