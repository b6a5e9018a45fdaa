// Real-space part of the PSE mobility (Sec. 2.2; the real-space Ewald sum of
// Sec. 3.2): neighbour lists over a cell list, the radial table of the
// wave-part scalar functions, and the warp-cooperative FTS pair sum.
//
// Every 11x11 pair block is built from derivatives of one radial scalar per
// (source, read-out) kind pair, Phi with FT  -W(k) f_s(ka) f_t(ka)/(eta k^4):
//   monopole factor f_M = j0(ka), dipole factor f_D = 3 j1(ka)/(ka).
// Real part = free kernel (closed form for r >= 2a: Faxen operators on the
// biharmonic r/(8 pi eta)) minus the wave part (H-filtered, tabulated).
#include "fsd_internal.cuh"

#include <climits>
#include <mutex>

#include <algorithm>

namespace fsd {

// ============================================================ host tables

static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// j_n(z) / z^n: power series below z = 4, upward recurrence above (stable
// for z > n; n <= 4 here).
static double jn_over_zn(int n, double z) {
  if (z < 4.0) {
    double df = 1.0;
    for (int m = 1; m <= 2 * n + 1; m += 2) df *= m;
    double term = 1.0 / df, acc = term, z2 = z * z;
    for (int k = 1; k < 80; ++k) {
      term *= -z2 / (2.0 * k * (2.0 * n + 2.0 * k + 1.0));
      acc += term;
      if (std::fabs(term) < 1e-19 * std::fabs(acc)) break;
    }
    return acc;
  }
  double s = std::sin(z), c = std::cos(z);
  double jm = s / z;
  if (n == 0) return jm;
  double jc = s / (z * z) - c / z;
  for (int k = 1; k < n; ++k) {
    double jn = (2.0 * k + 1.0) / z * jc - jm;
    jm = jc;
    jc = jn;
  }
  return jc / std::pow(z, n);
}

static double fM(double z) { return jn_over_zn(0, z); }
static double fD(double z) { return 3.0 * jn_over_zn(1, z); }

// function f: 0 MM n1, 1 MM n2, 2 MD n2, 3 MD n3, 4 DD n2, 5 DD n3, 6 DD n4
static const int kFuncKind[NFUNC] = {0, 0, 1, 1, 2, 2, 2};
static const int kFuncOrder[NFUNC] = {1, 2, 2, 3, 2, 3, 4};

struct WaveQuad {
  std::vector<double> k, w, g[3];  // g[kind] = w * H * f_s f_t
  double eta;
};

static WaveQuad make_quad(double xi, double a, double eta, int nq) {
  WaveQuad q;
  q.eta = eta;
  double K = 2.0 * xi * std::sqrt(46.0);
  std::vector<double> t, w;
  gauss_legendre(nq, t, w);
  q.k.resize(nq);
  q.w.resize(nq);
  for (int kind = 0; kind < 3; ++kind) q.g[kind].resize(nq);
  for (int i = 0; i < nq; ++i) {
    double k = 0.5 * K * (t[i] + 1.0);
    double wk = 0.5 * K * w[i];
    double x = k * k / (4.0 * xi * xi);
    double H = (1.0 + x) * std::exp(-x);
    double m = fM(k * a), d = fD(k * a);
    q.k[i] = k;
    q.w[i] = wk;
    q.g[0][i] = wk * H * m * m;
    q.g[1][i] = wk * H * m * d;
    q.g[2][i] = wk * H * d * d;
  }
  return q;
}

// Phi_n of the wave part:
//   (-1)^(n+1)/(2 pi^2 eta) int_0^K H f_s f_t k^(2n-2) j_n(kr)/(kr)^n dk
static double wave_phi(const WaveQuad &q, int f, double r) {
  int kind = kFuncKind[f], n = kFuncOrder[f];
  double acc = 0.0;
  for (size_t i = 0; i < q.k.size(); ++i) {
    double k = q.k[i];
    acc += q.g[kind][i] * std::pow(k, 2 * n - 2) * jn_over_zn(n, k * r);
  }
  double sign = (n % 2 == 1) ? 1.0 : -1.0;  // (-1)^(n+1)
  return sign * acc / (2.0 * kPi * kPi * q.eta);
}

// Chebyshev fit of the seven wave-part functions on nint intervals of
// length ht with NC coefficients each, stored as monomials in t in [-1, 1]:
// layout [interval][power p][function, padded to 8], stride values per
// interval.
static std::vector<double> fit_table(const WaveQuad &q, int nint, double ht, int NC, int stride) {
  std::vector<double> tab((size_t)nint * stride, 0.0);
  std::vector<double> tk(NC), v(NC), cc(NC);
  for (int k = 0; k < NC; ++k) tk[k] = std::cos(kPi * (k + 0.5) / NC);
  // Chebyshev T_j(t) as monomials: cheb[j][p]
  std::vector<std::vector<double>> cheb(NC, std::vector<double>(NC, 0.0));
  cheb[0][0] = 1.0;
  if (NC > 1) cheb[1][1] = 1.0;
  for (int j = 2; j < NC; ++j)
    for (int p = 0; p < NC; ++p)
      cheb[j][p] = (p > 0 ? 2.0 * cheb[j - 1][p - 1] : 0.0) - cheb[j - 2][p];
  for (int iv = 0; iv < nint; ++iv) {
    double r0 = iv * ht;
    for (int f = 0; f < NFUNC; ++f) {
      for (int k = 0; k < NC; ++k) v[k] = wave_phi(q, f, r0 + 0.5 * (tk[k] + 1.0) * ht);
      for (int j = 0; j < NC; ++j) {
        double s = 0.0;
        for (int k = 0; k < NC; ++k) s += v[k] * std::cos(j * kPi * (k + 0.5) / NC);
        cc[j] = (j == 0 ? 1.0 : 2.0) * s / NC;
      }
      for (int p = 0; p < NC; ++p) {
        double s = 0.0;
        for (int j = 0; j < NC; ++j) s += cc[j] * cheb[j][p];
        tab[(size_t)iv * stride + (size_t)p * 8 + f] = s;
      }
    }
  }
  return tab;
}

void build_real_table(Ctx &c) {
  double K = 2.0 * c.xi * std::sqrt(46.0);
  double ht = std::min(1.6 / K, 0.25);
  int nint = (int)std::ceil(c.rc / ht) + 2;
  c.tab_h = ht;
  c.tab_nint = nint;
  WaveQuad q = make_quad(c.xi, c.a, c.eta, 400);
  const std::vector<double> tab = fit_table(q, nint, ht, tab_coef<double>(), tab_stride<double>());
  const std::vector<double> tab32 = fit_table(q, nint, ht, tab_coef<float>(), tab_stride<float>());
  // real-space self terms: isolated-sphere self mobilities minus the wave
  // part at r = 0 (translation 2 Phi1_MM, rotation -5/2 Phi2_DD, strain -3 Phi2_DD)
  double mt = 1.0 / (6.0 * kPi * c.eta * c.a);
  double mr = 1.0 / (8.0 * kPi * c.eta * c.a * c.a * c.a);
  double ms = 3.0 / (20.0 * kPi * c.eta * c.a * c.a * c.a);
  double w1 = wave_phi(q, 0, 0.0), w2 = wave_phi(q, 4, 0.0);
  double self[3] = {mt - 2.0 * w1, mr + 2.5 * w2, ms + 3.0 * w2};
  c.op64.table.alloc(tab.size());
  FSD_CUDA(cudaMemcpy(c.op64.table.p, tab.data(), tab.size() * sizeof(double),
                      cudaMemcpyHostToDevice));
  std::vector<float> tabf(tab32.begin(), tab32.end());
  c.op32.table.alloc(tabf.size());
  FSD_CUDA(cudaMemcpy(c.op32.table.p, tabf.data(), tabf.size() * sizeof(float),
                      cudaMemcpyHostToDevice));
  for (int i = 0; i < 3; ++i) {
    c.op64.self_real[i] = self[i];
    c.op32.self_real[i] = (float)self[i];
  }
}

// ====================================================== positions / levers

__device__ __forceinline__ void quat_rot(const double *q, const double *v, double *o) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double R00 = 1 - 2 * (y * y + z * z), R01 = 2 * (x * y - w * z), R02 = 2 * (x * z + w * y);
  double R10 = 2 * (x * y + w * z), R11 = 1 - 2 * (x * x + z * z), R12 = 2 * (y * z - w * x);
  double R20 = 2 * (x * z - w * y), R21 = 2 * (y * z + w * x), R22 = 1 - 2 * (x * x + y * y);
  o[0] = R00 * v[0] + R01 * v[1] + R02 * v[2];
  o[1] = R10 * v[0] + R11 * v[1] + R12 * v[2];
  o[2] = R20 * v[0] + R21 * v[1] + R22 * v[2];
}

__device__ __forceinline__ double wrap_box(double x, double L) {
  x -= L * floor(x / L);
  if (x >= L) x -= L;
  if (x < 0) x = 0;
  return x;
}

// Bead positions from the rigid-body state, wrapped into the periodic box:
// in a Lees-Edwards box (offset tilt) a bead wrapped across y moves by the
// offset along x.  wpos holds the wave-space (sheared) coordinates
// s = (x - (tilt/L) y, y, z) wrapped into [0, L): the box is a plain cube in
// them, so spreading and interpolation run on a regular grid (equal to pos
// for tilt 0).
__global__ void k_wrap_positions(int Nt, double L, double tilt, const int *__restrict__ bead_body,
                                 const double *__restrict__ X, const double *__restrict__ q,
                                 const double *__restrict__ rbody, double4 *pos64,
                                 double4 *lever64, float4 *pos32, float4 *lever32,
                                 double4 *wpos64, float4 *wpos32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  int J = bead_body[i];
  double rb[3] = {rbody[3 * i], rbody[3 * i + 1], rbody[3 * i + 2]};
  double lv[3];
  quat_rot(q + 4 * J, rb, lv);
  double x = X[3 * J] + lv[0], y = X[3 * J + 1] + lv[1], z = X[3 * J + 2] + lv[2];
  const double ny = floor(y / L);
  y -= ny * L;
  x -= ny * tilt;
  x = wrap_box(x, L);
  y = wrap_box(y, L);
  z = wrap_box(z, L);
  const double sx = tilt != 0.0 ? wrap_box(x - (tilt / L) * y, L) : x;
  pos64[i] = make_double4(x, y, z, 0.0);
  lever64[i] = make_double4(lv[0], lv[1], lv[2], 0.0);
  pos32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
  lever32[i] = make_float4((float)lv[0], (float)lv[1], (float)lv[2], 0.f);
  wpos64[i] = make_double4(sx, y, z, 0.0);
  wpos32[i] = make_float4((float)sx, (float)y, (float)z, 0.f);
}

__global__ void k_set_scalar(double *p, double v) { *p = v; }

// Device copy of the box offset (read by the operator kernels of a
// Lees-Edwards context); never called inside a stream capture.
void sync_tilt(Ctx &c) {
  if (!c.tilt_dev.p) return;
  k_set_scalar<<<1, 1, 0, c.stream>>>(c.tilt_dev.p, c.tilt);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void launch_wrap_positions(Ctx &c) {
  c.tiles_valid = false;  // the spreading tiles follow the positions
  k_wrap_positions<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(
      c.Nt, c.L, c.tilt, c.bead_body.p, c.X.p, c.q.p, c.rbody.p, (double4 *)c.pos64.p,
      (double4 *)c.lever64.p, (float4 *)c.op32.pos.p, (float4 *)c.op32.lever.p,
      (double4 *)c.wpos64.p, (float4 *)c.wpos32.p);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// ========================================================= neighbour lists

__device__ __forceinline__ int cell_of(double x, double L, int nc) {
  int ci = (int)(x / L * nc);
  return ci < 0 ? 0 : (ci >= nc ? nc - 1 : ci);
}

__global__ void k_cell_count(int Nt, const double4 *__restrict__ pos, double L, int nc,
                             int *cell_count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  double4 p = pos[i];
  int id = (cell_of(p.x, L, nc) * nc + cell_of(p.y, L, nc)) * nc + cell_of(p.z, L, nc);
  atomicAdd(&cell_count[id], 1);
}

// single-block exclusive scan (n up to a few million; serial chunks + block scan)
__global__ void k_exclusive_scan(int n, const int *__restrict__ in, int *out, int *cursor) {
  __shared__ int sums[1024];
  int t = threadIdx.x;
  int per = (n + blockDim.x - 1) / blockDim.x;
  int b = t * per, e = min(n, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  sums[t] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int v = (t >= off) ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int run = sums[t] - s;
  for (int i = b; i < e; ++i) {
    out[i] = run;
    if (cursor) cursor[i] = run;
    run += in[i];
  }
  if (t == blockDim.x - 1) out[n] = sums[t];
}

__global__ void k_cell_fill(int Nt, const double4 *__restrict__ pos, double L, int nc,
                            int *cursor, int *cell_beads) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  double4 p = pos[i];
  int id = (cell_of(p.x, L, nc) * nc + cell_of(p.y, L, nc)) * nc + cell_of(p.z, L, nc);
  int slot = atomicAdd(&cursor[id], 1);
  cell_beads[slot] = i;
}

// Sort each cell's bead indices (one thread per cell): with the cells
// visited in a fixed order, every neighbour row, and so every pair sum, then
// runs in an order that does not depend on the atomic fill.
// Sort each segment [start[c], start[c + 1]) of `items` ascending (the
// atomically filled cell and tile lists, so that every later sum runs in a
// fixed order).  One warp per segment: a bitonic sort in shared memory for
// segments of up to kSortMax items (padded to a power of two with INT_MAX),
// an insertion sort by one lane beyond that.
constexpr int kSortMax = 512;

__global__ void __launch_bounds__(128) k_sort_cells(int ncells, const int *__restrict__ cell_start,
                                                    int *cell_beads) {
  __shared__ int buf[4][kSortMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cidx = blockIdx.x * 4 + warp;
  if (cidx >= ncells) return;
  const int b = cell_start[cidx], e = cell_start[cidx + 1], len = e - b;
  if (len <= 1) return;
  if (len > kSortMax) {
    if (lane == 0)
      for (int s = b + 1; s < e; ++s) {
        int v = cell_beads[s], k = s;
        while (k > b && cell_beads[k - 1] > v) {
          cell_beads[k] = cell_beads[k - 1];
          --k;
        }
        cell_beads[k] = v;
      }
    return;
  }
  int p2 = 2;
  while (p2 < len) p2 <<= 1;
  int *a = buf[warp];
  for (int i = lane; i < p2; i += 32) a[i] = i < len ? cell_beads[b + i] : INT_MAX;
  __syncwarp();
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < p2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const int x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if (up ? x > y : x < y) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
  for (int i = lane; i < len; i += 32) cell_beads[b + i] = a[i];
}

// One thread per bead: mobility neighbours (r < rc, any body, j != i) and
// lubrication neighbours (r < rlub, different body).  Each candidate's
// nearest-image distance is first taken in FP32 from the FP32 positions; only
// a candidate whose squared distance lies within m2 of a cut-off is measured
// again in FP64, so every decision is the FP64 one (m2 bounds the FP32
// rounding of the positions and of the image shift many times over; an
// image chosen differently in FP32 has a component near L/2, beyond every
// cut-off either way).  FP64 arithmetic runs at 1/74 of the FP32 rate on
// this part, and the FP64 test with its three divisions by L was the cost.
__global__ void k_neighbors(int Nt, const double4 *__restrict__ pos,
                            const float4 *__restrict__ pos32,
                            const double4 *__restrict__ spos, double L, double tilt, int nc,
                            const int *__restrict__ cell_start,
                            const int *__restrict__ cell_beads,
                            const int *__restrict__ bead_body, double rc2, double rl2,
                            double ov2, float m2, int cap, int lcap, int *nbr, int *ncnt,
                            int *lnbr, int *lcnt, int *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const double4 p = pos[i];
  const float4 pf = pos32[i];
  const double4 sp = spos[i];
  int bi = bead_body[i];
  int cx = cell_of(sp.x, L, nc), cy = cell_of(sp.y, L, nc), cz = cell_of(sp.z, L, nc);
  int cnt = 0, lc = 0;
  int span = nc >= 3 ? 1 : 0;
  int *row = nbr + (size_t)i * cap;
  int *lrow = lnbr + (size_t)i * lcap;
  const float Lf = (float)L, invLf = 1.f / Lf, tiltf = (float)tilt;
  const float rc2f = (float)rc2, rl2f = (float)rl2, ov2f = (float)ov2;
  const float hi = fmaxf(rc2f, fmaxf(rl2f, ov2f)) + m2;
  for (int dx = -span; dx <= span; ++dx)
    for (int dy = -span; dy <= span; ++dy)
      for (int dz = -span; dz <= span; ++dz) {
        int ax = (cx + dx + nc) % nc, ay = (cy + dy + nc) % nc, az = (cz + dz + nc) % nc;
        int id = (ax * nc + ay) * nc + az;
        for (int s = cell_start[id]; s < cell_start[id + 1]; ++s) {
          int j = cell_beads[s];
          if (j == i) continue;
          const float4 qf = pos32[j];
          float e0 = qf.x - pf.x, e1 = qf.y - pf.y, e2 = qf.z - pf.z;
          {
            const float ny = rintf(e1 * invLf);
            e0 -= ny * tiltf;
            e1 -= ny * Lf;
            e0 -= Lf * rintf(e0 * invLf);
            e2 -= Lf * rintf(e2 * invLf);
          }
          const float r2f = e0 * e0 + e1 * e1 + e2 * e2;
          if (r2f >= hi) continue;
          double r2 = (double)r2f;
          if (fabsf(r2f - rc2f) < m2 || fabsf(r2f - rl2f) < m2 || fabsf(r2f - ov2f) < m2) {
            const double4 q = pos[j];
            double d0 = q.x - p.x, d1 = q.y - p.y, d2 = q.z - p.z;
            le_image(d0, d1, d2, L, tilt);
            r2 = d0 * d0 + d1 * d1 + d2 * d2;
          }
          if (r2 < rc2) {
            if (cnt < cap) row[cnt] = j;
            ++cnt;
          }
          if (bead_body[j] != bi) {
            if (r2 < ov2) atomicOr(&flags[2], 1);
            if (r2 < rl2) {
              if (lc < lcap) lrow[lc] = j;
              ++lc;
            }
          }
        }
      }
  const int m = min(cnt, cap);
  ncnt[i] = m;
  lcnt[i] = min(lc, lcap);
  if (cnt > cap) atomicOr(&flags[0], 1);
  if (lc > lcap) atomicOr(&flags[1], 1);
  atomicMax(&flags[4], cnt);
  atomicMax(&flags[5], lc);
}

// Within each block of 32 consecutive neighbours of a bead (the pairs one
// warp step of the real-space sum takes together) order by distance: the
// lanes then read the radial table at neighbouring intervals, which fall in
// distinct shared-memory banks, instead of at random ones; the set of pairs
// in each block, and so the warp's global loads, stays the same.  One warp per
// bead, a bitonic sort of (r^2, index) across the lanes per block (ties by
// index, so the order is deterministic).
__global__ void __launch_bounds__(256) k_nbr_order(int Nt, const float4 *__restrict__ pos32,
                                                   float L, float tilt, int *nbr,
                                                   const int *__restrict__ ncnt, int cap) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Nt) return;
  const float4 pf = pos32[i];
  const float invL = 1.f / L;
  const int m = ncnt[i];
  int *row = nbr + (size_t)i * cap;
  for (int b0 = 0; b0 < m; b0 += 32) {
    const int q = b0 + lane;
    float key = INFINITY;
    int idx = INT_MAX;
    if (q < m) {
      idx = row[q];
      const float4 qf = pos32[idx];
      float e0 = qf.x - pf.x, e1 = qf.y - pf.y, e2 = qf.z - pf.z;
      const float ny = rintf(e1 * invL);
      e0 -= ny * tilt;
      e1 -= ny * L;
      e0 -= L * rintf(e0 * invL);
      e2 -= L * rintf(e2 * invL);
      key = e0 * e0 + e1 * e1 + e2 * e2;
    }
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, key, j);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, j);
        const bool other_less = ok < key || (ok == key && oi < idx);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        // the lower lane of an ascending pair keeps the smaller element
        if (lower == up ? other_less : !other_less) {
          key = ok;
          idx = oi;
        }
      }
    if (q < m) row[q] = idx;
  }
}

void build_neighbors(Ctx &c) {
  ProfScope ps(c, PG_NEIGHBOR);
  // cells in sheared coordinates: a pair at distance r differs by up to
  // r sqrt(1 + (tilt/L)^2) in s_x, so the cells widen by that factor
  const double shear_f = std::sqrt(1.0 + (c.tilt / c.L) * (c.tilt / c.L));
  int nc = (int)std::floor(c.L / (shear_f * std::max(c.rc, c.prm.lub_cutoff)));
  if (nc < 3) nc = 1;
  if (nc > 128) nc = 128;
  int ncells = nc * nc * nc;
  if (c.ncell != nc || !c.cell_count.p) {
    c.ncell = nc;
    c.cell_count.alloc(ncells);
    c.cell_start.alloc(ncells + 1);
    c.cell_cursor.alloc(ncells);
    c.cell_beads.alloc(c.Nt);
  }
  const double4 *pos = (const double4 *)c.pos64.p;
  const double4 *spos = (const double4 *)c.wpos64.p;
  for (int attempt = 0; attempt < 4; ++attempt) {
    FSD_CUDA(cudaMemsetAsync(c.cell_count.p, 0, ncells * sizeof(int), c.stream));
    FSD_CUDA(cudaMemsetAsync(c.flags.p, 0, 8 * sizeof(int), c.stream));
    k_cell_count<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, spos, c.L, nc, c.cell_count.p);
    FSD_LAUNCHED(c);
    k_exclusive_scan<<<1, 1024, 0, c.stream>>>(ncells, c.cell_count.p, c.cell_start.p,
                                               c.cell_cursor.p);
    FSD_LAUNCHED(c);
    k_cell_fill<<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, spos, c.L, nc, c.cell_cursor.p,
                                                           c.cell_beads.p);
    FSD_LAUNCHED(c);
    k_sort_cells<<<ceil_div(ncells, 4), 128, 0, c.stream>>>(ncells, c.cell_start.p,
                                                             c.cell_beads.p);
    FSD_LAUNCHED(c);
    double rl = c.prm.lub_cutoff > 2.0 * c.a ? c.prm.lub_cutoff : 0.0;
    double ov = 2.0 * c.a * (1.0 - 1e-6);
    // margin of the FP32 pre-test on r^2: the FP32 positions and the image
    // shift are within a few 1e-7 L of the FP64 ones, so the FP32 r^2 is off
    // by at most ~2e-6 L r_max (five times below the margin)
    const float m2 = (float)(1e-5 * c.L * std::max({c.rc, rl, ov}) + 1e-12);
    k_neighbors<<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(
        c.Nt, pos, (const float4 *)c.op32.pos.p, spos, c.L, c.tilt, nc, c.cell_start.p,
        c.cell_beads.p, c.bead_body.p, c.rc * c.rc, rl * rl, ov * ov, m2, c.cap, c.lcap, c.nbr.p,
        c.ncnt.p, c.lnbr.p, c.lcnt.p, c.flags.p);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    FSD_CUDA(cudaMemcpyAsync(c.h_flags, c.flags.p, 8 * sizeof(int), cudaMemcpyDeviceToHost,
                             c.stream));
    FSD_CUDA(cudaStreamSynchronize(c.stream));
    bool redo = false;
    if (c.h_flags[0]) {
      c.cap = ((c.h_flags[4] + 32) / 32 + 1) * 32;
      c.nbr.alloc((size_t)c.Nt * c.cap);
      redo = true;
    }
    if (c.h_flags[1]) {
      c.lcap = ((c.h_flags[5] + 8) / 8 + 1) * 8;
      c.lnbr.alloc((size_t)c.Nt * c.lcap);
      redo = true;
    }
    if (!redo) break;
  }
  k_nbr_order<<<ceil_div((int64_t)c.Nt * 32, 256), 256, 0, c.stream>>>(
      c.Nt, (const float4 *)c.op32.pos.p, (float)c.L, (float)c.tilt, c.nbr.p, c.ncnt.p, c.cap);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  if (c.h_flags[2]) c.last_warning = FSD_EOVERLAP;
}

// ============================================================ pair sum

template <typename T>
struct RS;
template <>
struct RS<float> {
  using V4 = float4;
};
template <>
struct RS<double> {
  using V4 = double4;
};

template <typename T>
__device__ __forceinline__ T rint_t(T x);
template <>
__device__ __forceinline__ float rint_t<float>(float x) { return rintf(x); }
template <>
__device__ __forceinline__ double rint_t<double>(double x) { return rint(x); }

template <typename T>
__device__ __forceinline__ T sqrt_t(T x);
template <>
__device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }

// Accumulate the action of one FTS pair block (given its seven radial
// scalars) on the source moments (F, L, S) into (u, omega, e6).
//   ph = {Phi1_MM, Phi2_MM, Phi2_MD, Phi3_MD, Phi2_DD, Phi3_DD, Phi4_DD}
//   x  = x_target - x_source.
// e6 = (exx, eyy, ezz, exy, exz, eyz) without its isotropic part.
template <typename T>
__device__ __forceinline__ void pair_apply(const T x0, const T x1, const T x2, const T r2,
                                           const T *ph, const T *F, const T *Lm, const T *S6,
                                           T *acc) {
  const T p1 = ph[0], p2 = ph[1], q2 = ph[2], q3 = ph[3], s2 = ph[4], s3 = ph[5], s4 = ph[6];
  const T xF = x0 * F[0] + x1 * F[1] + x2 * F[2];
  const T xL = x0 * Lm[0] + x1 * Lm[1] + x2 * Lm[2];
  const T Sx0 = S6[0] * x0 + S6[3] * x1 + S6[4] * x2;
  const T Sx1 = S6[3] * x0 + S6[1] * x1 + S6[5] * x2;
  const T Sx2 = S6[4] * x0 + S6[5] * x1 + S6[2] * x2;
  const T xSx = x0 * Sx0 + x1 * Sx1 + x2 * Sx2;
  const T cxL0 = x1 * Lm[2] - x2 * Lm[1], cxL1 = x2 * Lm[0] - x0 * Lm[2],
          cxL2 = x0 * Lm[1] - x1 * Lm[0];
  const T cxF0 = x1 * F[2] - x2 * F[1], cxF1 = x2 * F[0] - x0 * F[2], cxF2 = x0 * F[1] - x1 * F[0];
  const T cxS0 = x1 * Sx2 - x2 * Sx1, cxS1 = x2 * Sx0 - x0 * Sx2, cxS2 = x0 * Sx1 - x1 * Sx0;
  const T g = r2 * q3 + T(5) * q2;           // grad lap Phi_MD = g x
  const T cUS = -(r2 * q3 + T(3) * q2);
  const T al = r2 * s4 + T(7) * s3;          // grad grad lap Phi_DD = al xx + be I
  const T be = r2 * s3 + T(5) * s2;
  const T ta = al * r2 + T(3) * be;          // lap^2 Phi_DD
  const T cUF = r2 * p2 + T(2) * p1;
  const T hg = T(0.5) * g;
  // velocity
  const T cu = q3 * xSx - p2 * xF;
  acc[0] += cUF * F[0] + cu * x0 + hg * cxL0 + cUS * Sx0;
  acc[1] += cUF * F[1] + cu * x1 + hg * cxL1 + cUS * Sx1;
  acc[2] += cUF * F[2] + cu * x2 + hg * cxL2 + cUS * Sx2;
  // rotation
  const T qa = T(0.25) * al * xL, qb = T(0.25) * (be - ta), ha = T(0.5) * al;
  acc[3] += hg * cxF0 + qa * x0 + qb * Lm[0] - ha * cxS0;
  acc[4] += hg * cxF1 + qa * x1 + qb * Lm[1] - ha * cxS1;
  acc[5] += hg * cxF2 + qa * x2 + qb * Lm[2] - ha * cxS2;
  // strain: sym(x (x) v) + A2 xx + A6 S, v = A1 F + (al/2)(x x L) + A5 Sx
  const T A1 = -cUS, A2 = s4 * xSx - q3 * xF, A5 = T(4) * s3 - al, A6 = T(2) * s2 - be;
  const T v0 = A1 * F[0] + ha * cxL0 + A5 * Sx0;
  const T v1 = A1 * F[1] + ha * cxL1 + A5 * Sx1;
  const T v2 = A1 * F[2] + ha * cxL2 + A5 * Sx2;
  acc[6] += x0 * v0 + A2 * x0 * x0 + A6 * S6[0];
  acc[7] += x1 * v1 + A2 * x1 * x1 + A6 * S6[1];
  acc[8] += x2 * v2 + A2 * x2 * x2 + A6 * S6[2];
  acc[9] += T(0.5) * (x0 * v1 + v0 * x1) + A2 * x0 * x1 + A6 * S6[3];
  acc[10] += T(0.5) * (x0 * v2 + v0 * x2) + A2 * x0 * x2 + A6 * S6[4];
  acc[11] += T(0.5) * (x1 * v2 + v1 * x2) + A2 * x1 * x2 + A6 * S6[5];
}

// Free-space radial scalars (r >= 2a), Faxen on the biharmonic:
// Phi = (r + 2 c a^2 / r)/(8 pi eta), c = 1/3 (MM), 4/15 (MD), 1/5 (DD).
template <typename T>
__device__ __forceinline__ void free_phi(const T inv, const T a2, const T c8, T *ph) {
  const T i2 = inv * inv, i3 = i2 * inv, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
  ph[0] = c8 * (inv - T(2.0 / 3.0) * a2 * i3);
  ph[1] = c8 * (-i3 + T(2) * a2 * i5);
  ph[2] = c8 * (-i3 + T(1.6) * a2 * i5);
  ph[3] = c8 * (T(3) * i5 - T(8) * a2 * i7);
  ph[4] = c8 * (-i3 + T(1.2) * a2 * i5);
  ph[5] = c8 * (T(3) * i5 - T(6) * a2 * i7);
  ph[6] = c8 * (T(-15) * i7 + T(42) * a2 * i9);
}

// Wave-part radial functions from the Chebyshev-fitted table (monomials in
// t in [-1, 1] per interval), all seven functions per Horner step.
template <typename T>
__device__ __forceinline__ void wave_table(const T *tab, int nint, T inv_h, T r, T *w);
template <>
__device__ __forceinline__ void wave_table<float>(const float *tab, int nint, float inv_h, float r,
                                                  float *w) {
  const float s = r * inv_h;
  int iv = (int)s;
  iv = iv < 0 ? 0 : (iv >= nint ? nint - 1 : iv);
  const float t = 2.f * (s - (float)iv) - 1.f;
  constexpr int NC = tab_coef<float>();
  const float4 *c = (const float4 *)(tab + (size_t)iv * tab_stride<float>());
  float4 lo = c[2 * (NC - 1)], hi = c[2 * (NC - 1) + 1];
  float v0 = lo.x, v1 = lo.y, v2 = lo.z, v3 = lo.w, v4 = hi.x, v5 = hi.y, v6 = hi.z;
#pragma unroll
  for (int p = NC - 2; p >= 0; --p) {
    lo = c[2 * p];
    hi = c[2 * p + 1];
    v0 = v0 * t + lo.x; v1 = v1 * t + lo.y; v2 = v2 * t + lo.z; v3 = v3 * t + lo.w;
    v4 = v4 * t + hi.x; v5 = v5 * t + hi.y; v6 = v6 * t + hi.z;
  }
  w[0] = v0; w[1] = v1; w[2] = v2; w[3] = v3; w[4] = v4; w[5] = v5; w[6] = v6;
}
template <>
__device__ __forceinline__ void wave_table<double>(const double *tab, int nint, double inv_h,
                                                   double r, double *w) {
  const double s = r * inv_h;
  int iv = (int)s;
  iv = iv < 0 ? 0 : (iv >= nint ? nint - 1 : iv);
  const double t = 2.0 * (s - (double)iv) - 1.0;
  constexpr int NC = tab_coef<double>();
  const double2 *c = (const double2 *)(tab + (size_t)iv * tab_stride<double>());
  double v[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 a = c[4 * (NC - 1) + q];
    v[2 * q] = a.x;
    v[2 * q + 1] = a.y;
  }
#pragma unroll
  for (int p = NC - 2; p >= 0; --p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 a = c[4 * p + q];
      v[2 * q] = v[2 * q] * t + a.x;
      v[2 * q + 1] = v[2 * q + 1] * t + a.y;
    }
#pragma unroll
  for (int f = 0; f < NFUNC; ++f) w[f] = v[f];
}

template <typename T>
__device__ __forceinline__ void load_moments(const double *__restrict__ x, int j, T *F, T *Lm,
                                             T *S6) {
  const double2 *p = (const double2 *)(x + (size_t)j * LDB);
  double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3), e = __ldg(p + 4);
  double s4 = __ldg(x + (size_t)j * LDB + 10);
  F[0] = (T)a.x;
  F[1] = (T)a.y;
  F[2] = (T)b.x;
  Lm[0] = (T)b.y;
  Lm[1] = (T)c.x;
  Lm[2] = (T)c.y;
  const T s0 = (T)d.x, s1 = (T)d.y, s2 = (T)e.x, s3 = (T)e.y, s5 = (T)s4;
  const T r2i = T(0.70710678118654752440), r6i = T(0.40824829046386301637);
  S6[0] = r2i * s0 - r6i * s1;
  S6[1] = -r2i * s0 - r6i * s1;
  S6[2] = T(2) * r6i * s1;
  S6[3] = r2i * s2;
  S6[4] = r2i * s3;
  S6[5] = r2i * s5;
}

// Per-matvec packing of the source beads in the operator precision:
// (x, y, z, F0 | F1, F2, L0, L1 | L2, Sxx, Syy, Szz | Sxy, Sxz, Syz, 0)
// so that one neighbour costs four 16-byte loads (FP32) in the pair loop.
template <typename T>
__global__ void k_pack_sources(int Nt, const double4 *__restrict__ pos,
                               const double *__restrict__ x, T *packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  T F[3], Lm[3], S6[6];
  load_moments<T>(x, i, F, Lm, S6);
  const double4 p = pos[i];
  T *o = packed + (size_t)i * 16;
  o[0] = (T)p.x;
  o[1] = (T)p.y;
  o[2] = (T)p.z;
  o[3] = F[0];
  o[4] = F[1];
  o[5] = F[2];
  o[6] = Lm[0];
  o[7] = Lm[1];
  o[8] = Lm[2];
  o[9] = S6[0];
  o[10] = S6[1];
  o[11] = S6[2];
  o[12] = S6[3];
  o[13] = S6[4];
  o[14] = S6[5];
  o[15] = T(0);
}

template <typename T>
__device__ __forceinline__ void load_packed(const T *__restrict__ packed, int j, T *pj, T *F,
                                            T *Lm, T *S6);
template <>
__device__ __forceinline__ void load_packed<float>(const float *__restrict__ packed, int j,
                                                   float *pj, float *F, float *Lm, float *S6) {
  const float4 *q = (const float4 *)(packed + (size_t)j * 16);
  const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  pj[0] = a.x; pj[1] = a.y; pj[2] = a.z;
  F[0] = a.w; F[1] = b.x; F[2] = b.y;
  Lm[0] = b.z; Lm[1] = b.w; Lm[2] = c.x;
  S6[0] = c.y; S6[1] = c.z; S6[2] = c.w; S6[3] = d.x; S6[4] = d.y; S6[5] = d.z;
}
template <>
__device__ __forceinline__ void load_packed<double>(const double *__restrict__ packed, int j,
                                                    double *pj, double *F, double *Lm,
                                                    double *S6) {
  const double2 *q = (const double2 *)(packed + (size_t)j * 16);
  const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  const double2 e = __ldg(q + 4), f = __ldg(q + 5), g = __ldg(q + 6), h = __ldg(q + 7);
  pj[0] = a.x; pj[1] = a.y; pj[2] = b.x;
  F[0] = b.y; F[1] = c.x; F[2] = c.y;
  Lm[0] = d.x; Lm[1] = d.y; Lm[2] = e.x;
  S6[0] = e.y; S6[1] = f.x; S6[2] = f.y; S6[3] = g.x; S6[4] = g.y; S6[5] = h.x;
}

// G lanes per target bead; the group sums its neighbours, reduces with warp
// shuffles and its first lane writes the bead row:
//   y_i = sum_j M_r(x_i - x_j) x_j + M_self,r x_i [+ (dU + dOm x r_i, dOm, 0)]
template <typename T, int G>
__global__ void __launch_bounds__(256, 4) k_realspace(
    int Nt, const T *__restrict__ packed, const int *__restrict__ nbr,
    const int *__restrict__ ncnt, int cap, const double *__restrict__ x, double *__restrict__ y,
    const T *__restrict__ tab_g, int nint, T inv_h, T L, T tilt, T a, T c8, T self_t, T self_r,
    T self_s, int add_constraint, const int *__restrict__ bead_body,
    const double4 *__restrict__ lever, int Nt_off, const double *__restrict__ tilt_dev) {
  if (tilt_dev) tilt = (T)*tilt_dev;  // Lees-Edwards steps: the offset in device memory
  // the radial table is staged once per (persistent) CTA in shared memory
  extern __shared__ __align__(16) unsigned char tab_raw[];
  T *tab = (T *)tab_raw;
  {
    const int nv = nint * tab_stride<T>() * (int)sizeof(T) / 16;
    const uint4 *src = (const uint4 *)tab_g;
    uint4 *dst = (uint4 *)tab_raw;
    for (int q = threadIdx.x; q < nv; q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const int groups_per_block = blockDim.x / G;
  const int lane = threadIdx.x % G;
  for (int gbase = blockIdx.x * groups_per_block; gbase < Nt; gbase += gridDim.x * groups_per_block) {
  const int gid = gbase + threadIdx.x / G;
  const bool active = gid < Nt;
  const int i = active ? gid : Nt - 1;
  T acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(0);
  const T *pio = packed + (size_t)i * 16;
  const T pi0 = pio[0], pi1 = pio[1], pi2 = pio[2];
  const int cnt = active ? ncnt[i] : 0;
  const int *row = nbr + (size_t)i * cap;
  const T a2 = a * a, two_a = T(2) * a;
  const T invL = T(1) / L;
#pragma unroll 2
  for (int k = lane; k < cnt; k += G) {
    const int j = __ldg(row + k);
    T pj[3], F[3], Lm[3], S6[6];
    load_packed<T>(packed, j, pj, F, Lm, S6);
    T d0 = pi0 - pj[0], d1 = pi1 - pj[1], d2 = pi2 - pj[2];
    {
      // Lees-Edwards image: across y the box is offset by tilt along x
      const T ny = rint_t<T>(d1 * invL);
      d0 -= ny * tilt;
      d1 -= L * ny;
    }
    d0 -= L * rint_t<T>(d0 * invL);
    d2 -= L * rint_t<T>(d2 * invL);
    const T r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const T r = sqrt_t<T>(r2);
    T wv[NFUNC];
    wave_table<T>(tab, nint, inv_h, r, wv);
    T ph[NFUNC];
    if (r >= two_a * T(1 - 1e-6)) {
      free_phi<T>(T(1) / r, a2, c8, ph);
#pragma unroll
      for (int f = 0; f < NFUNC; ++f) ph[f] -= wv[f];
      pair_apply<T>(d0, d1, d2, r2, ph, F, Lm, S6, acc);
    } else {
      // overlapping beads of different bodies: the free kernel is taken at
      // separation 2a along the true direction; the wave part at the true x
      const T sc = two_a / r;
      free_phi<T>(T(1) / two_a, a2, c8, ph);
      pair_apply<T>(d0 * sc, d1 * sc, d2 * sc, two_a * two_a, ph, F, Lm, S6, acc);
#pragma unroll
      for (int f = 0; f < NFUNC; ++f) ph[f] = -wv[f];
      pair_apply<T>(d0, d1, d2, r2, ph, F, Lm, S6, acc);
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off, G);
  if (!active || lane != 0) continue;
  // self term and rigid-body constraint rows
  double xi_[11];
  const double *xr = x + (size_t)i * LDB;
#pragma unroll
  for (int k = 0; k < 11; ++k) xi_[k] = xr[k];
  double o[12];
  o[0] = (double)acc[0] + (double)self_t * xi_[0];
  o[1] = (double)acc[1] + (double)self_t * xi_[1];
  o[2] = (double)acc[2] + (double)self_t * xi_[2];
  o[3] = (double)acc[3] + (double)self_r * xi_[3];
  o[4] = (double)acc[4] + (double)self_r * xi_[4];
  o[5] = (double)acc[5] + (double)self_r * xi_[5];
  const double exx = acc[6], eyy = acc[7], ezz = acc[8], exy = acc[9], exz = acc[10],
               eyz = acc[11];
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637, s2 = 1.41421356237309504880;
  o[6] = r2i * (exx - eyy) + (double)self_s * xi_[6];
  o[7] = r6i * (2.0 * ezz - exx - eyy) + (double)self_s * xi_[7];
  o[8] = s2 * exy + (double)self_s * xi_[8];
  o[9] = s2 * exz + (double)self_s * xi_[9];
  o[10] = s2 * eyz + (double)self_s * xi_[10];
  o[11] = 0.0;
  if (add_constraint) {
    const int J = bead_body[i];
    const double *u = x + Nt_off + 6 * (size_t)J;
    const double4 rv = lever[i];
    o[0] += u[0] + (u[4] * rv.z - u[5] * rv.y);
    o[1] += u[1] + (u[5] * rv.x - u[3] * rv.z);
    o[2] += u[2] + (u[3] * rv.y - u[4] * rv.x);
    o[3] += u[3];
    o[4] += u[4];
    o[5] += u[5];
  }
  double2 *yo = (double2 *)(y + (size_t)i * LDB);
#pragma unroll
  for (int k = 0; k < 6; ++k) yo[k] = make_double2(o[2 * k], o[2 * k + 1]);
  }
}

template <typename T>
static const typename RS<T>::V4 *pos_ptr(Ctx &c);
template <>
const double4 *pos_ptr<double>(Ctx &c) {
  return (const double4 *)c.pos64.p;
}
template <>
const float4 *pos_ptr<float>(Ctx &c) {
  return (const float4 *)c.op32.pos.p;
}

template <typename T>
static OpData<T> &opdata(Ctx &c);
template <>
OpData<double> &opdata<double>(Ctx &c) {
  return c.op64;
}
template <>
OpData<float> &opdata<float>(Ctx &c) {
  return c.op32;
}

// Lanes that share one bead's neighbour list, from the mean neighbour count
// (a tile shape the caller may fix with fsd_params.tile).  On the 32768-bead
// benchmark (168 neighbours per bead) 16 lanes beat 32: 0.122 against 0.133
// ms per application, fewer idle lanes at the end of each list and a shorter
// reduction.
int realspace_group(const Ctx &c) {
  const int t = c.prm.tile;
  if (t == 4 || t == 8 || t == 16 || t == 32) return t;
  const double avg = (double)c.n_pairs / std::max(1, c.Nt);
  return avg > 256 ? 32 : (avg > 40 ? 16 : (avg > 16 ? 8 : 4));
}

// Resident blocks per SM of k_realspace<T, GG> at `smem` bytes of dynamic
// shared memory.  The kernel's shared-memory limit is only ever raised (to
// the largest table any context has used): contexts with different tables
// share the kernel, and a lower limit would fail the larger ones' launches.
// Thread-safe: contexts may run on several host threads.
template <typename T, int GG>
static int realspace_occupancy(size_t smem, int threads) {
  static std::mutex mu;
  static std::vector<std::pair<size_t, int>> seen;
  static size_t limit = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (smem > limit) {
    FSD_CUDA(cudaFuncSetAttribute(k_realspace<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max<size_t>(smem, 48 * 1024)));
    limit = smem;
  }
  for (auto &e : seen)
    if (e.first == smem) return e.second;
  int occ = 0;
  FSD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_realspace<T, GG>, threads, smem));
  seen.emplace_back(smem, occ);
  return occ;
}

template <typename T>
void launch_realspace(Ctx &c, const double *x, double *y, bool add_constraint, bool) {
  ProfScope ps(c, PG_REAL);
  OpData<T> &op = opdata<T>(c);
  const int threads = 256;
  if (op.packed.n < (size_t)c.Nt * 16) op.packed.alloc((size_t)c.Nt * 16);
  k_pack_sources<T><<<ceil_div(c.Nt, 256), 256, 0, c.stream>>>(c.Nt, (const double4 *)c.pos64.p, x,
                                                              op.packed.p);
  FSD_LAUNCHED(c);
  const int G = realspace_group(c);
  const size_t smem = (size_t)c.tab_nint * tab_stride<T>() * sizeof(T);
  if (smem > 200 * 1024) throw Invalid{"real-space table too large (reduce rc or raise xi)"};
  const T inv_h = (T)(1.0 / c.tab_h);
  const T c8 = (T)(1.0 / (8.0 * kPi * c.eta));
#define FSD_RS_LAUNCH(GG)                                                                    \
  {                                                                                          \
    int per_sm = realspace_occupancy<T, GG>(smem, threads);                                  \
    if (c.rs_overlapped && c.rs_blocks_per_sm > 0) per_sm = std::min(per_sm, c.rs_blocks_per_sm); \
    k_realspace<T, GG><<<std::min<int64_t>(ceil_div((int64_t)c.Nt * GG, threads),             \
                                           (int64_t)std::max(1, per_sm) * c.num_sms),       \
                         threads, smem, c.stream>>>(                                         \
        c.Nt, op.packed.p, c.nbr.p, c.ncnt.p, c.cap, x, y, op.table.p, c.tab_nint, inv_h,    \
        (T)c.L, (T)c.tilt, (T)c.a, c8, op.self_real[0], op.self_real[1], op.self_real[2],  \
        add_constraint ? 1 : 0, c.bead_body.p, (const double4 *)c.lever64.p,                 \
        (int)(LDB * (int64_t)c.Nt), tilt_dev_ptr(c));                                        \
  }
  switch (G) {
    case 32: FSD_RS_LAUNCH(32); FSD_LAUNCHED(c); break;
    case 16: FSD_RS_LAUNCH(16); FSD_LAUNCHED(c); break;
    case 8: FSD_RS_LAUNCH(8); FSD_LAUNCHED(c); break;
    default: FSD_RS_LAUNCH(4); FSD_LAUNCHED(c); break;
  }
#undef FSD_RS_LAUNCH
  FSD_CUDA(cudaGetLastError());
}

template void launch_realspace<float>(Ctx &, const double *, double *, bool, bool);
template void launch_realspace<double>(Ctx &, const double *, double *, bool, bool);

}  // namespace fsd
