// Wave-space part of the PSE mobility (Sec. 2.2, Eq. UBff split; Sec. 3.2
// grid rule): Gaussian spreading of the force and force-dipole densities, a
// hand-written shared-memory mixed-radix 3D FFT with the Green's function
// scaling fused into the z pass, and interpolation of the velocity and
// velocity gradient.
//
// Spreading.  FP32 (the Krylov operator): grid-centric, k_spread_gather.
// The grid is cut into 8^3 tiles; k_tile_bin lists, per tile, the beads
// whose P^3 window reaches it (rebuilt on the device when positions
// change), and one block per tile sums its beads' window contributions for
// each (y, z) row in registers and stores the six planar fields [6][n^3]
// once (no atomics, no zeroing pass).  FP64, and FP32 with
// FSD_SPREAD_ATOMIC=1: bead-centric k_spread / k_spread_v4 (warp-wide and
// 16-byte vector atomic adds into zeroed fields).
//
// FFT.  The forward pass turns the six real fields into half spectra
// [6][n][n][n/2 + 1] (complex, planar per component).  FP32 planes that fit
// in shared memory run fused x + y kernels (k_fft_xy_fwd / k_fft_xy_inv, one
// 1024-thread block per (component, z) plane, radix-16 / 9 / 8 register
// DFTs) and the inverse writes planar velocity fields [6][n^3]; larger
// grids and FP64 take separate x and y passes (the same radix-16 / 9 / 8
// plans) and interleaved velocity fields [n^3][8].  k_fft_z_green does the z transforms with the
// Green's function applied between forward and inverse.
//   comps 0..2  monopole density g_F = sum_j F_j W(x - x_j)
//   comps 3..5  dipole density   g_D = sum_j 2 alpha W(x - x_j) D_j (x - x_j),
//                D = S + A, A y = (1/2) L x y
// Spectral kernel (Hasimoto split, Gaussian window W_hat = exp(-k^2/(4 alpha))
// removed twice):
//   u_hat = A(k) (I - kk) [fM g_F_hat + fD g_D_hat],
//   A(k) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2) + k^2/(2 alpha)) / (eta k^2),
// read-outs: velocity from fM u_hat, rotation / strain from grad (fD u_hat)
// (k_interp_v4 for FP32 planar fields on grids that are multiples of 4,
// k_interp for other FP32 planar fields, k_interp_rows for interleaved
// fields: FP64 and the large FP32 grids).
#include "fsd_internal.cuh"

#include <algorithm>
#include <mutex>

namespace fsd {

template <typename T>
struct Cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cscale(Cx<T> a, T s) {
  return {a.x * s, a.y * s};
}
// multiply by i * sg (sg = +-1)
template <typename T>
__device__ __forceinline__ Cx<T> cmul_i(Cx<T> a, T sg) {
  return {-sg * a.y, sg * a.x};
}

constexpr int kMaxStages = 12;

// Division by a runtime constant d for numerators below 2^31 without an
// integer divide: q = (umulhi(x, m) + x) >> s with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, s = l (Granlund-Montgomery round-up
// method; d = 1 gives m = s = 0).
struct FastDiv {
  uint32_t d, m, s;
};

static FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 0u, 0u};
  if (d <= 1) return f;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  f.s = l;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv &f) {
  return (__umulhi(x, f.m) + x) >> f.s;
}

struct FftStage {
  int R, Ns, toff;   // radix, size of the sub-transforms already done, twiddle offset
  FastDiv nb, ns;    // divisions by n / R and by Ns
};

struct FftPlan {
  int n, nst, ntw;
  FastDiv fn, fnh;   // divisions by n and by n/2 + 1
  FftStage st[kMaxStages];
};

// Stages 16^a 9^b 8^c 4^d 2^e 3^f 5^g with big_radix (the largest register
// DFTs first: fewer passes through shared memory, and fewer twiddle products,
// which is what an FP64 transform spends its time on where FP64 runs at 1/74
// of the FP32 rate), else 4^d 2^e 3^f 5^g; per stage the twiddles
// exp(-2 pi i r k / (Ns R)), r = 1..R-1, k < Ns, stored contiguously
// (complex) from toff.
static FftPlan make_plan(int n, std::vector<double> *tw, bool big_radix) {
  FftPlan p{};
  p.n = n;
  p.fn = make_fastdiv(n);
  p.fnh = make_fastdiv(n / 2 + 1);
  int m = n, k = 0;
  std::vector<int> radices;
  if (big_radix)
    for (int f : {16, 9, 8})
      while (m % f == 0) {
        radices.push_back(f);
        m /= f;
      }
  while (m % 4 == 0) {
    radices.push_back(4);
    m /= 4;
  }
  for (int f : {2, 3, 5})
    while (m % f == 0) {
      radices.push_back(f);
      m /= f;
    }
  int Ns = 1, off = 0;
  if (tw) tw->clear();
  for (int R : radices) {
    FftStage &s = p.st[k++];
    s.R = R;
    s.Ns = Ns;
    s.toff = off;
    s.nb = make_fastdiv(n / R);
    s.ns = make_fastdiv(Ns);
    for (int r = 1; r < R; ++r)
      for (int kk = 0; kk < Ns; ++kk) {
        const double ang = -2.0 * kPi * r * kk / ((double)Ns * R);
        if (tw) {
          tw->push_back(std::cos(ang));
          tw->push_back(std::sin(ang));
        }
      }
    off += (R - 1) * Ns;
    Ns *= R;
  }
  p.nst = k;
  p.ntw = off;
  return p;
}

bool fft_size_ok(int n) {
  if (n < 8 || n % 2) return false;
  int m = n;
  for (int f : {2, 3, 5})
    while (m % f == 0) m /= f;
  return m == 1;
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void dft_two_level(Cx<T> *v, T sg);

// Small DFT of size R in registers, sign sg (-1 forward, +1 inverse).
template <typename T, int R>
__device__ __forceinline__ void dft_small(Cx<T> *v, T sg) {
  if constexpr (R == 16) {
    dft_two_level<T, 4, 4>(v, sg);
  } else if constexpr (R == 9) {
    dft_two_level<T, 3, 3>(v, sg);
  } else if constexpr (R == 8) {
    dft_two_level<T, 2, 4>(v, sg);
  } else if (R == 2) {
    Cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 3) {
    const T h = T(0.86602540378443864676);
    Cx<T> t1 = cadd(v[1], v[2]);
    Cx<T> t2 = {v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y};
    Cx<T> t3 = cmul_i(cscale(csub(v[1], v[2]), h), sg);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  } else if (R == 4) {
    Cx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    Cx<T> c = cadd(v[1], v[3]), d = cmul_i(csub(v[1], v[3]), sg);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  } else if (R == 5) {
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
    const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);
    Cx<T> a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    Cx<T> a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    Cx<T> x0 = v[0];
    Cx<T> r1 = {x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
    Cx<T> r2 = {x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
    Cx<T> i1 = cmul_i(Cx<T>{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y}, sg);
    Cx<T> i2 = cmul_i(Cx<T>{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y}, sg);
    v[0] = {x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
    v[1] = cadd(r1, i1);
    v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2);
    v[3] = csub(r2, i2);
  }
}

// exp(sg 2 pi i m / R) for R in {8, 9, 16}; m is a compile-time constant
// after unrolling, so the table reads fold away.
template <typename T, int R>
__device__ __forceinline__ Cx<T> root_of_unity(int m, T sg) {
  constexpr double c16[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440,
                              0.38268343236508977173, 0.0, -0.38268343236508977173,
                              -0.70710678118654752440, -0.92387953251128675613, -1.0,
                              -0.92387953251128675613, -0.70710678118654752440,
                              -0.38268343236508977173, 0.0, 0.38268343236508977173,
                              0.70710678118654752440, 0.92387953251128675613};
  constexpr double s16[16] = {0.0, 0.38268343236508977173, 0.70710678118654752440,
                              0.92387953251128675613, 1.0, 0.92387953251128675613,
                              0.70710678118654752440, 0.38268343236508977173, 0.0,
                              -0.38268343236508977173, -0.70710678118654752440,
                              -0.92387953251128675613, -1.0, -0.92387953251128675613,
                              -0.70710678118654752440, -0.38268343236508977173};
  constexpr double c9[9] = {1.0, 0.76604444311897803520, 0.17364817766693034885, -0.5,
                            -0.93969262078590838405, -0.93969262078590838405, -0.5,
                            0.17364817766693034885, 0.76604444311897803520};
  constexpr double s9[9] = {0.0, 0.64278760968653932632, 0.98480775301220805936,
                            0.86602540378443864676, 0.34202014332566873304,
                            -0.34202014332566873304, -0.86602540378443864676,
                            -0.98480775301220805936, -0.64278760968653932632};
  m %= R;
  if (R == 9) return {T(c9[m]), sg * T(s9[m])};
  const int q = m * (16 / R);  // R = 8 or 16
  return {T(c16[q]), sg * T(s16[q])};
}

template <typename T, int R>
__device__ __forceinline__ void dft_small(Cx<T> *v, T sg);

// DFT of size R1 R2 in registers (Cooley-Tukey): with n = R2 n1 + n2 and
// k = k1 + R1 k2, X_k = sum_n2 w_R^(n2 k1) w_R2^(n2 k2) [DFT_R1 over n1 of
// x_(R2 n1 + n2)]_k1.
template <typename T, int R1, int R2>
__device__ __forceinline__ void dft_two_level(Cx<T> *v, T sg) {
  constexpr int R = R1 * R2;
  Cx<T> y[R];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    Cx<T> t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
    dft_small<T, R1>(t, sg);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = cmul(t[k1], root_of_unity<T, R>(n2 * k1, sg));
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    Cx<T> t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    dft_small<T, R2>(t, sg);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
  }
}

// Line buffers in shared memory store element i of a line at i + i/16: a
// radix-16 stage writes with a stride of 16 elements, which the padding
// spreads over distinct banks.  fft_ls(n) is the padded line length.
__host__ __device__ __forceinline__ int fft_ls(int n) { return n + (n - 1) / 16 + 1; }
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// One Stockham stage of radix R over nl lines stored with stride ls:
//   for butterfly j < n/R, k = j mod Ns, g = j div Ns:
//   v_r = in[j + r n/R] w_(r,k),  DFT_R,  out[g Ns R + k + r Ns] = v_r.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const Cx<T> *in, Cx<T> *out, int nl, int n, int ls,
                                               const FftStage &st, const Cx<T> *tws, T sg) {
  const int nb = n / R;
  const int Ns = st.Ns;
  const int total = nl * nb;
  const Cx<T> *tw = tws + st.toff;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = (int)fdiv((uint32_t)b, st.nb);
    const int j = b - line * nb;
    const int g = (int)fdiv((uint32_t)j, st.ns);
    const int k = j - g * Ns;
    const Cx<T> *src = in + line * ls;
    Cx<T> v[R];
    v[0] = src[fpad(j)];
    if (Ns == 1) {  // first stage: every twiddle is 1
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = src[fpad(j + r * nb)];
    } else {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        Cx<T> w = tw[(r - 1) * Ns + k];
        w.y *= -sg;  // tables hold the forward twiddles
        v[r] = cmul(src[fpad(j + r * nb)], w);
      }
    }
    dft_small<T, R>(v, sg);
    Cx<T> *dst = out + line * ls;
    const int d0 = g * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[fpad(d0 + r * Ns)] = v[r];
  }
}

// Full transform of nl lines: data starts in A; returns the buffer holding
// the result (A or B).
template <typename T>
__device__ Cx<T> *fft_lines(Cx<T> *A, Cx<T> *B, int nl, int n, int ls, const FftPlan &plan,
                            const Cx<T> *tws, T sg) {
  Cx<T> *in = A, *out = B;
  for (int s = 0; s < plan.nst; ++s) {
    const FftStage &st = plan.st[s];
    if (st.R == 16)
      stockham_stage<T, 16>(in, out, nl, n, ls, st, tws, sg);
    else if (st.R == 9)
      stockham_stage<T, 9>(in, out, nl, n, ls, st, tws, sg);
    else if (st.R == 8)
      stockham_stage<T, 8>(in, out, nl, n, ls, st, tws, sg);
    else if (st.R == 4)
      stockham_stage<T, 4>(in, out, nl, n, ls, st, tws, sg);
    else if (st.R == 2)
      stockham_stage<T, 2>(in, out, nl, n, ls, st, tws, sg);
    else if (st.R == 3)
      stockham_stage<T, 3>(in, out, nl, n, ls, st, tws, sg);
    else
      stockham_stage<T, 5>(in, out, nl, n, ls, st, tws, sg);
    __syncthreads();
    Cx<T> *t = in;
    in = out;
    out = t;
  }
  return in;
}

// The 144-point transform (radix 16 then 9) on lines of stride kLS144 = 153
// (= 9 mod 16): the first stage reads the lines in natural order and writes
// padded order (element i at i + i/16), the second reads padded order and
// writes natural order back into A.  Every access is a fixed offset from the
// butterfly's base address (no per-element index arithmetic), and neither
// stage has shared-memory bank conflicts: in natural order the lanes of a
// half-warp read 16 consecutive elements of one or two lines, 153 apart; the
// padding spreads the first stage's stride-16 writes and the second stage's
// stride-16 reads.  tw2: the second stage's twiddles exp(-2 pi i r j / 144),
// [r - 1][j], r < 9, j < 16.
constexpr int kLS144 = 153;

template <typename T>
__device__ __forceinline__ void fft144_lines(Cx<T> *A, Cx<T> *B, int nl, const Cx<T> *tw2, T sg) {
  for (int b = threadIdx.x; b < nl * 9; b += blockDim.x) {
    const int line = b / 9, j = b - line * 9;
    const Cx<T> *src = A + line * kLS144 + j;
    Cx<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = src[9 * r];
    dft_small<T, 16>(v, sg);
    Cx<T> *dst = B + line * kLS144 + 17 * j;
#pragma unroll
    for (int r = 0; r < 16; ++r) dst[r] = v[r];
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nl * 16; b += blockDim.x) {
    const int line = b >> 4, j = b & 15;
    const Cx<T> *src = B + line * kLS144 + j;
    Cx<T> v[9];
    v[0] = src[0];
#pragma unroll
    for (int r = 1; r < 9; ++r) {
      Cx<T> w = tw2[(r - 1) * 16 + j];
      w.y *= -sg;  // tables hold the forward twiddles
      v[r] = cmul(src[17 * r], w);
    }
    dft_small<T, 9>(v, sg);
    Cx<T> *dst = A + line * kLS144 + j;
#pragma unroll
    for (int r = 0; r < 9; ++r) dst[16 * r] = v[r];
  }
  __syncthreads();
}

// Plans served by fft144_lines: n = 144 as 16 x 9 with lines of stride 153.
__host__ __device__ __forceinline__ bool is_fft144(const FftPlan &p) {
  return p.n == 144 && p.nst == 2 && p.st[0].R == 16 && p.st[1].R == 9 && fft_ls(144) == kLS144;
}

template <typename T>
__device__ __forceinline__ void load_twiddles(Cx<T> *tw_s, const T *__restrict__ tw, int ntw) {
  for (int t = threadIdx.x; t < ntw; t += blockDim.x) tw_s[t] = {tw[2 * t], tw[2 * t + 1]};
}

// ---------------------------------------------------------------- x passes
// Forward: for each row (z, y) and pair p < 3, z = g_p + i g_{p+3}; after the
// DFT the two half spectra are A_k = (Z_k + conj Z_{n-k})/2 and
// B_k = (Z_k - conj Z_{n-k})/(2i), written to spec[p] and spec[p + 3].
template <typename T>
__device__ __forceinline__ void load6(const T *q, T *v);
template <>
__device__ __forceinline__ void load6<float>(const float *q, float *v) {
  const float4 a = *(const float4 *)q;
  const float2 b = *(const float2 *)(q + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
template <>
__device__ __forceinline__ void load6<double>(const double *q, double *v) {
  const double2 a = *(const double2 *)q, b = *(const double2 *)(q + 2),
                c = *(const double2 *)(q + 4);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
template <typename T>
__device__ __forceinline__ void store6(T *q, const T *v);
template <>
__device__ __forceinline__ void store6<float>(float *q, const float *v) {
  *(float4 *)q = make_float4(v[0], v[1], v[2], v[3]);
  *(float2 *)(q + 4) = make_float2(v[4], v[5]);
}
template <>
__device__ __forceinline__ void store6<double>(double *q, const double *v) {
  *(double2 *)q = make_double2(v[0], v[1]);
  *(double2 *)(q + 2) = make_double2(v[2], v[3]);
  *(double2 *)(q + 4) = make_double2(v[4], v[5]);
}

template <typename T>
__global__ void k_fft_x_fwd(const T *__restrict__ grid, Cx<T> *spec, FftPlan plan,
                            const T *__restrict__ tw, int NL) {
  // grid: planar [6][n^3]
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1;
  const int NLL = 3 * NL;
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + NLL * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int64_t nrows = (int64_t)n * n;  // rows (z, y)
  const int64_t row0 = (int64_t)blockIdx.x * NL;
  {
    const int64_t n3 = nrows * n;
    const int total = NL * n;
    for (int e0 = threadIdx.x; e0 < total; e0 += 2 * blockDim.x) {
      T v[2][6];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e0 + u * blockDim.x;
        const int l = (int)fdiv((uint32_t)e, plan.fn), xx = e - l * n;
        const int64_t row = row0 + l;
        const bool ok = e < total && row < nrows;
        const int64_t o = row * n + xx;
#pragma unroll
        for (int c = 0; c < 6; ++c) v[u][c] = ok ? grid[c * n3 + o] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= total) continue;
        const int l = (int)fdiv((uint32_t)e, plan.fn), xx = e - l * n;
#pragma unroll
        for (int p = 0; p < 3; ++p) A[(l * 3 + p) * ls + fpad(xx)] = {v[u][p], v[u][p + 3]};
      }
    }
  }
  __syncthreads();
  Cx<T> *Z = fft_lines<T>(A, B, NLL, n, ls, plan, tw_s, T(-1));
  const int64_t cs = nrows * nh;
  for (int e = threadIdx.x; e < NLL * nh; e += blockDim.x) {
    const int lp = (int)fdiv((uint32_t)e, plan.fnh), k = e - lp * nh;
    const int l = lp / 3, p = lp - 3 * l;
    const int64_t row = row0 + l;
    if (row >= nrows) continue;
    const Cx<T> zk = Z[lp * ls + fpad(k)];
    const Cx<T> zm = Z[lp * ls + fpad(k == 0 ? 0 : n - k)];
    // (Z_k - conj Z_{n-k}) / (2i): (p + iq)/(2i) = (q - ip)/2
    spec[p * cs + row * nh + k] = {T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
    spec[(p + 3) * cs + row * nh + k] = {T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
  }
}

// Inverse: Z_k = A_k + i B_k (k <= n/2), conj(A_{n-k}) + i conj(B_{n-k})
// beyond; the inverse DFT gives a + i b, stored as comps p and p + 3.
template <typename T>
__global__ void k_fft_x_inv(T *grid, const Cx<T> *__restrict__ spec, FftPlan plan,
                            const T *__restrict__ tw, int NL) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1;
  const int NLL = 3 * NL;
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + NLL * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int64_t nrows = (int64_t)n * n;
  const int64_t row0 = (int64_t)blockIdx.x * NL;
  const int64_t cs = nrows * nh;
  {
    constexpr int U = 4;
    const int total = NLL * n;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
      Cx<T> a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        const int lp = (int)fdiv((uint32_t)e, plan.fn), k = e - lp * n;
        const int l = lp / 3, p = lp - 3 * l;
        const int64_t row = row0 + l;
        const int kk = k <= n / 2 ? k : n - k;
        if (e < total && row < nrows) {
          a[u] = spec[p * cs + row * nh + kk];
          b[u] = spec[(p + 3) * cs + row * nh + kk];
        } else {
          a[u] = {T(0), T(0)};
          b[u] = {T(0), T(0)};
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= total) continue;
        const int lp = (int)fdiv((uint32_t)e, plan.fn), k = e - lp * n;
        // k <= n/2: a + i b;  beyond: conj(a) + i conj(b) of the mirrored bin
        A[lp * ls + fpad(k)] = k <= n / 2 ? Cx<T>{a[u].x - b[u].y, a[u].y + b[u].x}
                                    : Cx<T>{a[u].x + b[u].y, -a[u].y + b[u].x};
      }
    }
  }
  __syncthreads();
  Cx<T> *Z = fft_lines<T>(A, B, NLL, n, ls, plan, tw_s, T(1));
  for (int e = threadIdx.x; e < NL * n; e += blockDim.x) {
    const int l = (int)fdiv((uint32_t)e, plan.fn), xx = e - l * n;
    const int64_t row = row0 + l;
    if (row >= nrows) continue;
    T v[6];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const Cx<T> z = Z[(l * 3 + p) * ls + fpad(xx)];
      v[p] = z.x;
      v[p + 3] = z.y;
    }
    store6<T>(grid + (row * n + xx) * 8, v);
  }
}

// ---------------------------------------------------------------- y pass
// Lines along y for fixed (comp, z), a tile of TX = 2^LTX consecutive kx.
template <typename T>
__global__ void k_fft_y(Cx<T> *spec, FftPlan plan, const T *__restrict__ tw, int LTX, T sg) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1;
  const int TX = 1 << LTX;
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + TX * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int ntile = (nh + TX - 1) >> LTX;
  const int cz = blockIdx.x / ntile;  // comp * n + z
  const int tile = blockIdx.x - cz * ntile;
  const int kx0 = tile << LTX;
  Cx<T> *base = spec + (int64_t)cz * n * nh;  // rows of nh complex
  {
    constexpr int U = 8;
    const int total = n << LTX;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
      Cx<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        const int yy = e >> LTX, t = e & (TX - 1);
        const int kx = kx0 + t;
        v[u] = (e < total && kx < nh) ? base[(int64_t)yy * nh + kx] : Cx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) A[(e & (TX - 1)) * ls + fpad(e >> LTX)] = v[u];
      }
    }
  }
  __syncthreads();
  Cx<T> *Z = fft_lines<T>(A, B, TX, n, ls, plan, tw_s, sg);
  for (int e = threadIdx.x; e < (n << LTX); e += blockDim.x) {
    const int yy = e >> LTX, t = e & (TX - 1);
    const int kx = kx0 + t;
    if (kx < nh) base[(int64_t)yy * nh + kx] = Z[t * ls + fpad(yy)];
  }
}

// ------------------------------------------------ fused x + y passes (FP32)
// One block per (component, z) plane, both transforms in shared memory
// (FP32 planes up to n = 160 fit next to their ping-pong copy).
// Forward: rows y = 2r and 2r + 1 of the real plane form the complex line
// z_r = g_2r + i g_2r+1; after the x DFT the half spectra of the two rows are
// A_k = (Z_k + conj Z_{n-k})/2 and B_k = (Z_k - conj Z_{n-k})/(2i), k <= n/2.
// They are transposed into nh = n/2 + 1 lines along y, transformed, and
// written as spec[comp][z][y][kx].
template <typename T, bool S144>
__global__ void __launch_bounds__(1024) k_fft_xy_fwd(const T *__restrict__ grid, Cx<T> *spec,
                                                    FftPlan plan, const T *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1, nr = n / 2;
  // element i of a line: natural order for the 144-point path, padded else
  auto P = [](int i) { return S144 ? i : fpad(i); };
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;  // nh lines of ls
  Cx<T> *B = A + nh * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int64_t cz = blockIdx.x;  // comp * n + z
  const T *g = grid + cz * n * n;
  {
    // eight loads in flight per thread: the plane load is latency-bound
    constexpr int U = 8;
    const int total = nr * n;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
      T va[U], vb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        const int r = (int)fdiv((uint32_t)e, plan.fn), x = e - r * n;
        va[u] = e < total ? g[(2 * r) * n + x] : T(0);
        vb[u] = e < total ? g[(2 * r + 1) * n + x] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= total) continue;
        const int r = (int)fdiv((uint32_t)e, plan.fn), x = e - r * n;
        A[r * ls + P(x)] = {va[u], vb[u]};
      }
    }
  }
  __syncthreads();
  Cx<T> *Z, *Y;
  if constexpr (S144) {
    fft144_lines<T>(A, B, nr, tw_s + plan.st[1].toff, T(-1));
    Z = A;
    Y = B;
  } else {
    Z = fft_lines<T>(A, B, nr, n, ls, plan, tw_s, T(-1));
    Y = (Z == A) ? B : A;
  }
  for (int e = threadIdx.x; e < nr * nh; e += blockDim.x) {
    const int r = (int)fdiv((uint32_t)e, plan.fnh), k = e - r * nh;
    const Cx<T> zk = Z[r * ls + P(k)];
    const Cx<T> zm = Z[r * ls + P(k == 0 ? 0 : n - k)];
    Y[k * ls + P(2 * r)] = {T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
    Y[k * ls + P(2 * r + 1)] = {T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
  }
  __syncthreads();
  Cx<T> *R;
  if constexpr (S144) {
    fft144_lines<T>(Y, Z, nh, tw_s + plan.st[1].toff, T(-1));
    R = Y;
  } else {
    R = fft_lines<T>(Y, Z, nh, n, ls, plan, tw_s, T(-1));
  }
  Cx<T> *out = spec + cz * n * nh;
  for (int e = threadIdx.x; e < n * nh; e += blockDim.x) {
    const int y = (int)fdiv((uint32_t)e, plan.fnh), k = e - y * nh;
    out[e] = R[k * ls + P(y)];
  }
}

// Inverse of k_fft_xy_fwd: the y lines are transformed back, rows 2r and
// 2r + 1 are packed as Z_k = A_k + i B_k (k <= n/2; conj(A_{n-k}) +
// i conj(B_{n-k}) beyond), and the inverse x DFT gives the two real rows as
// its real and imaginary parts, written to a planar field [comp][z][y][x].
template <typename T, bool S144>
__global__ void __launch_bounds__(1024) k_fft_xy_inv(T *field, const Cx<T> *__restrict__ spec,
                                                    FftPlan plan, const T *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1, nr = n / 2;
  auto P = [](int i) { return S144 ? i : fpad(i); };
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + nh * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int64_t cz = blockIdx.x;
  const Cx<T> *in = spec + cz * n * nh;
  {
    constexpr int U = 8;
    const int total = n * nh;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
      Cx<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < total ? in[e] : Cx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= total) continue;
        const int y = (int)fdiv((uint32_t)e, plan.fnh), k = e - y * nh;
        A[k * ls + P(y)] = v[u];
      }
    }
  }
  __syncthreads();
  Cx<T> *Y, *Z;
  if constexpr (S144) {
    fft144_lines<T>(A, B, nh, tw_s + plan.st[1].toff, T(1));
    Y = A;
    Z = B;
  } else {
    Y = fft_lines<T>(A, B, nh, n, ls, plan, tw_s, T(1));
    Z = (Y == A) ? B : A;
  }
  for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
    const int r = (int)fdiv((uint32_t)e, plan.fn), k = e - r * n;
    const int kk = k <= n / 2 ? k : n - k;
    const Cx<T> a = Y[kk * ls + P(2 * r)], b = Y[kk * ls + P(2 * r + 1)];
    Z[r * ls + P(k)] = k <= n / 2 ? Cx<T>{a.x - b.y, a.y + b.x} : Cx<T>{a.x + b.y, -a.y + b.x};
  }
  __syncthreads();
  Cx<T> *X;
  if constexpr (S144) {
    fft144_lines<T>(Z, Y, nr, tw_s + plan.st[1].toff, T(1));
    X = Z;
  } else {
    X = fft_lines<T>(Z, Y, nr, n, ls, plan, tw_s, T(1));
  }
  T *o = field + cz * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int y = (int)fdiv((uint32_t)e, plan.fn), x = e - y * n;
    const Cx<T> v = X[(y >> 1) * ls + P(x)];
    o[e] = (y & 1) ? v.y : v.x;
  }
}

// ------------------------------------------------------- z pass + Green
// Lines along z for fixed y, TX = 2^LTX consecutive kx, all six components:
// forward DFT, Green's function, inverse DFT.
// Green's function factors for the Lees-Edwards box (tau = tilt / L):
// A(k) f_s(ka) f_t(ka) with A = (1 + k^2/(4 xi^2)) e^(-k^2/(4 xi^2)) e^(k_s^2/(2 alpha))
// / (eta k^2 n^3), k the physical and k_s the sheared-grid wave vector
// (the same expression the cubic table holds, with k_s = k there).
struct GreenLE {
  double tau = 0.0, ks2 = 0.0, xi = 0.0, alpha = 0.0, a = 0.0, eta = 0.0, inv_n3 = 0.0;
  int on = 0;                   // sheared box: the tabulated factors and the physical k
  const double *dev = nullptr;  // device tilt (overrides tau when set)
  double invL = 0.0;
  double isv = 0.0;  // 1 / sqrt(V): the Brownian wave-field scale
};

__device__ __forceinline__ void green_le(const GreenLE &g, double mp, double ms, double &t1,
                                         double &t2, double &t3) {
  const double k2 = g.ks2 * mp;
  const double e = -k2 / (4.0 * g.xi * g.xi) + g.ks2 * ms / (2.0 * g.alpha);
  const double A = (1.0 + k2 / (4.0 * g.xi * g.xi)) * exp(e) / (g.eta * k2) * g.inv_n3;
  const double z = sqrt(k2) * g.a;
  const double fm = z < 1e-3 ? 1.0 - z * z / 6.0 + z * z * z * z / 120.0 : sin(z) / z;
  const double fd = z < 1e-2 ? 1.0 - z * z / 10.0 + z * z * z * z / 280.0
                             : 3.0 * (sin(z) - z * cos(z)) / (z * z * z);
  t1 = A * fm * fm;
  t2 = A * fm * fd;
  t3 = A * fd * fd;
}

// z index of the q-th row a z-pass block visits: on the 144-point path the
// rows of each group of 16 are visited in 4 x 4 transposed order (q = 4a + b
// -> z = 4b + a), so that the 4 kx columns x 4 rows of a half-warp's
// shared-memory accesses (lines 153 = 9 mod 16 elements apart) fall in 16
// distinct banks; the sheared Green's table is stored in the same visiting
// order.  The map is its own inverse.
template <bool S144>
__host__ __device__ __forceinline__ int zorder(int q) {
  if constexpr (S144)
    return (q & ~15) | ((q & 3) << 2) | ((q >> 2) & 3);
  else
    return q;
}

// Lees-Edwards Green factors for every half-spectrum point, laid out as the
// z pass visits them: [ky index][kx][kz in visiting order (zorder)][3].
template <typename T>
__global__ void k_green_le_table(int n, GreenLE le, T *gle, int s144) {
  const int nh = n / 2 + 1;
  const int64_t total = (int64_t)n * nh * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int zq = (int)(e % n);
    const int zz = s144 ? zorder<true>(zq) : zq;
    const int kx = (int)((e / n) % nh);
    const int yy = (int)(e / ((int64_t)n * nh));
    const int ky = yy <= n / 2 ? yy : yy - n, kz = zz <= n / 2 ? zz : zz - n;
    const int m = kx * kx + ky * ky + kz * kz;
    double g1 = 0.0, g2 = 0.0, g3 = 0.0;
    if (m > 0) {
      const double kyp = (double)ky - le.tau * (double)kx;
      const double mp = (double)kx * kx + kyp * kyp + (double)kz * kz;
      green_le(le, mp, (double)m, g1, g2, g3);
    }
    gle[3 * e] = (T)g1;
    gle[3 * e + 1] = (T)g2;
    gle[3 * e + 2] = (T)g3;
  }
}

template <typename T, bool S144>
__global__ void k_fft_z_green(Cx<T> *spec, FftPlan plan, const T *__restrict__ tw,
                              const T *__restrict__ green, int LTX, GreenLE le,
                              const T *__restrict__ gle) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1;
  const int TX = 1 << LTX;
  const int NLn = 6 * TX;
  auto P = [](int i) { return S144 ? i : fpad(i); };
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + NLn * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int ntile = (nh + TX - 1) >> LTX;
  const int yy = blockIdx.x / ntile;
  const int tile = blockIdx.x - yy * ntile;
  const int kx0 = tile << LTX;
  Cx<T> *g = spec;
  const int64_t zstride = (int64_t)n * nh, cstride = (int64_t)n * zstride;
  {
    constexpr int U = 8;
    const int total = NLn * n;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
      Cx<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        const int t = e & (TX - 1), rest = e >> LTX;
        const int comp = (int)fdiv((uint32_t)rest, plan.fn), zz = zorder<S144>(rest - comp * n);
        const int kx = kx0 + t;
        v[u] = (e < total && kx < nh) ? g[comp * cstride + zz * zstride + (int64_t)yy * nh + kx]
                                      : Cx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= total) continue;
        const int t = e & (TX - 1), rest = e >> LTX;
        const int comp = (int)fdiv((uint32_t)rest, plan.fn), zz = zorder<S144>(rest - comp * n);
        A[(comp * TX + t) * ls + P(zz)] = v[u];
      }
    }
  }
  __syncthreads();
  Cx<T> *Z;
  if constexpr (S144) {
    fft144_lines<T>(A, B, NLn, tw_s + plan.st[1].toff, T(-1));
    Z = A;
  } else {
    Z = fft_lines<T>(A, B, NLn, n, ls, plan, tw_s, T(-1));
  }
  // Green's function, one (kx, ky, kz) per thread iteration
  const int ky = yy <= n / 2 ? yy : yy - n;
  const double le_tau = le.dev ? *le.dev * le.invL : le.tau;
  for (int e = threadIdx.x; e < (n << LTX); e += blockDim.x) {
    const int t = e & (TX - 1), zq = e >> LTX, zz = zorder<S144>(zq);
    const int kx = kx0 + t;
    const int kz = zz <= n / 2 ? zz : zz - n;
    const int m = kx * kx + ky * ky + kz * kz;
    Cx<T> gF[3], gD[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gF[d] = Z[(d * TX + t) * ls + P(zz)];
      gD[d] = Z[((d + 3) * TX + t) * ls + P(zz)];
    }
    Cx<T> oM[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    Cx<T> oD[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    if (m > 0 && kx < nh) {
      T t1, t2, t3, kk[3], im;
      if (!le.on) {
        t1 = green[3 * m];
        t2 = green[3 * m + 1];
        t3 = green[3 * m + 2];
        kk[0] = (T)kx;
        kk[1] = (T)ky;
        kk[2] = (T)kz;
        im = T(1) / (T)m;
      } else {
        // Lees-Edwards box: the grid index k_s = (kx, ky, kz) is the wave
        // vector of the sheared coordinates; the physical one is
        // (kx, ky - tau kx, kz) (in 2 pi / L).  The window factor stays on
        // |k_s|^2; H(k), 1/k^2, the form factors and the projection take
        // the physical k (evaluated here in FP64)
        const double kyp = (double)ky - le_tau * (double)kx;
        const double mp = (double)kx * kx + kyp * kyp + (double)kz * kz;
        // factors of this box offset, tabulated once per offset
        const T *gq = gle + 3 * (((size_t)yy * nh + kx) * n + zq);
        t1 = gq[0];
        t2 = gq[1];
        t3 = gq[2];
        kk[0] = (T)kx;
        kk[1] = (T)kyp;
        kk[2] = (T)kz;
        im = (T)(1.0 / mp);
      }
      Cx<T> sF = {T(0), T(0)}, sD = {T(0), T(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        sF.x += kk[d] * gF[d].x;
        sF.y += kk[d] * gF[d].y;
        sD.x += kk[d] * gD[d].x;
        sD.y += kk[d] * gD[d].y;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Cx<T> pF = {gF[d].x - kk[d] * sF.x * im, gF[d].y - kk[d] * sF.y * im};
        const Cx<T> pD = {gD[d].x - kk[d] * sD.x * im, gD[d].y - kk[d] * sD.y * im};
        oM[d] = {t1 * pF.x + t2 * pD.x, t1 * pF.y + t2 * pD.y};
        oD[d] = {t2 * pF.x + t3 * pD.x, t2 * pF.y + t3 * pD.y};
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Z[(d * TX + t) * ls + P(zz)] = oM[d];
      Z[((d + 3) * TX + t) * ls + P(zz)] = oD[d];
    }
  }
  __syncthreads();
  Cx<T> *O = Z;
  Cx<T> *other = (Z == A) ? B : A;
  Cx<T> *R;
  if constexpr (S144) {
    fft144_lines<T>(O, other, NLn, tw_s + plan.st[1].toff, T(1));
    R = O;
  } else {
    R = fft_lines<T>(O, other, NLn, n, ls, plan, tw_s, T(1));
  }
  for (int e = threadIdx.x; e < NLn * n; e += blockDim.x) {
    const int t = e & (TX - 1), rest = e >> LTX;
    const int comp = (int)fdiv((uint32_t)rest, plan.fn), zz = zorder<S144>(rest - comp * n);
    const int kx = kx0 + t;
    if (kx < nh) g[comp * cstride + zz * zstride + (int64_t)yy * nh + kx] = R[(comp * TX + t) * ls + P(zz)];
  }
}

// ----------------------------------------------- Brownian z pass (PSE)
// Lines along z for fixed ky, TX = 2^LTX consecutive kx: the random field
// xi(k) (three complex components; from `field`, or from Philox stream 1 at
// the canonical point of a Hermitian pair), projected by (I - k k) and scaled
// by btab = (c fM, c fD), gives the velocity field (components 0-2) and the
// dipole read-out field (3-5) in k space; the inverse z transform leaves them
// in the state the operator's z pass leaves its output in.  Nyquist points
// and k = 0 carry no noise.
template <typename T>
__global__ void k_brown_z(Cx<T> *spec, FftPlan plan, const T *__restrict__ tw,
                          const T *__restrict__ btab, const double *__restrict__ field,
                          uint64_t seed, uint64_t step, int LTX, GreenLE le) {
  extern __shared__ unsigned char smem_raw[];
  const int n = plan.n, ls = fft_ls(n), nh = n / 2 + 1;
  const int TX = 1 << LTX;
  const int NLn = 6 * TX;
  Cx<T> *tw_s = (Cx<T> *)smem_raw;
  Cx<T> *A = tw_s + plan.ntw;
  Cx<T> *B = A + NLn * ls;
  load_twiddles(tw_s, tw, plan.ntw);
  const int ntile = (nh + TX - 1) >> LTX;
  const int yy = blockIdx.x / ntile;
  const int tile = blockIdx.x - yy * ntile;
  const int kx0 = tile << LTX;
  const int ky = yy <= n / 2 ? yy : yy - n;
  for (int e = threadIdx.x; e < (n << LTX); e += blockDim.x) {
    const int t = e & (TX - 1), zz = e >> LTX;
    const int kx = kx0 + t;
    const int kz = zz <= n / 2 ? zz : zz - n;
    Cx<T> oM[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    Cx<T> oD[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    const bool nyq = kx == n / 2 || yy == n / 2 || zz == n / 2;
    if (kx < nh && !nyq && (kx | yy | zz) != 0) {
      double xr[3], xim[3];
      if (field) {
        const int64_t cs = (int64_t)n * n * nh;
        const int64_t o = ((int64_t)zz * n + yy) * nh + kx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xr[c] = field[2 * (c * cs + o)];
          xim[c] = field[2 * (c * cs + o) + 1];
        }
      } else {
        int cz = zz, cy = yy;
        bool conj = false;
        if (kx == 0) {
          const int mz = (n - zz) % n, my = (n - yy) % n;
          if (mz < zz || (mz == zz && my < yy)) {
            cz = mz;
            cy = my;
            conj = true;
          }
        }
        const uint32_t idx = (uint32_t)(((int64_t)cz * n + cy) * nh + kx);
        double z0[4], z1[4];
        philox_normals4(seed, step, 1u, 0u, idx, z0);
        philox_normals4(seed, step, 1u, 1u, idx, z1);
        const double s = 0.70710678118654752440;
        xr[0] = s * z0[0]; xim[0] = s * z0[1];
        xr[1] = s * z0[2]; xim[1] = s * z0[3];
        xr[2] = s * z1[0]; xim[2] = s * z1[1];
        if (conj)
#pragma unroll
          for (int c = 0; c < 3; ++c) xim[c] = -xim[c];
      }
      // physical wave vector (the grid's in a cube; (kx, ky - tau kx, kz) in a
      // Lees-Edwards box, whose window factor stays on the grid index)
      const double ms = (double)kx * kx + (double)ky * ky + (double)kz * kz;
      const double kyp = (double)ky - le.tau * (double)kx;
      const double kk[3] = {(double)kx, kyp, (double)kz};
      const double m = kk[0] * kk[0] + kk[1] * kk[1] + kk[2] * kk[2];
      double pr = 0.0, pi = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pr += kk[c] * xr[c];
        pi += kk[c] * xim[c];
      }
      T bm, bd;
      if (le.tau == 0.0) {
        const int mi = (int)ms;
        bm = btab[2 * mi];
        bd = btab[2 * mi + 1];
      } else {
        const double k2 = le.ks2 * m;
        const double H = (1.0 + k2 / (4.0 * le.xi * le.xi)) * exp(-k2 / (4.0 * le.xi * le.xi));
        const double sc = sqrt(H / (le.eta * k2)) * exp(le.ks2 * ms / (4.0 * le.alpha)) * le.isv;
        const double z = sqrt(k2) * le.a;
        const double fm = z < 1e-3 ? 1.0 - z * z / 6.0 + z * z * z * z / 120.0 : sin(z) / z;
        const double fd = z < 1e-2 ? 1.0 - z * z / 10.0 + z * z * z * z / 280.0
                                   : 3.0 * (sin(z) - z * cos(z)) / (z * z * z);
        bm = (T)(sc * fm);
        bd = (T)(sc * fd);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T vr = (T)(xr[c] - kk[c] * pr / m), vi = (T)(xim[c] - kk[c] * pi / m);
        oM[c] = {bm * vr, bm * vi};
        oD[c] = {bd * vr, bd * vi};
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      A[(d * TX + t) * ls + fpad(zz)] = oM[d];
      A[((d + 3) * TX + t) * ls + fpad(zz)] = oD[d];
    }
  }
  __syncthreads();
  Cx<T> *R = fft_lines<T>(A, B, NLn, n, ls, plan, tw_s, T(1));
  const int64_t zstride = (int64_t)n * nh, cstride = (int64_t)n * zstride;
  for (int e = threadIdx.x; e < NLn * n; e += blockDim.x) {
    const int t = e & (TX - 1), rest = e >> LTX;
    const int comp = (int)fdiv((uint32_t)rest, plan.fn), zz = rest - comp * n;
    const int kx = kx0 + t;
    if (kx < nh) spec[comp * cstride + zz * zstride + (int64_t)yy * nh + kx] = R[(comp * TX + t) * ls + fpad(zz)];
  }
}

// ------------------------------------------------------------ spreading
template <typename T>
struct V4Of;
template <>
struct V4Of<float> {
  using type = float4;
};
template <>
struct V4Of<double> {
  using type = double4;
};

template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T floor_t(T x);
template <>
__device__ __forceinline__ float floor_t<float>(float x) { return floorf(x); }
template <>
__device__ __forceinline__ double floor_t<double>(double x) { return floor(x); }

constexpr int kMaxP = 24;

// One warp per bead: 1D Gaussian factors in shared memory, then the P^3
// points split over the lanes with atomic accumulation into the six fields.
template <typename T>
__global__ void __launch_bounds__(256) k_spread(int Nt, const typename V4Of<T>::type *__restrict__ pos,
                                                const double *__restrict__ x, T *grid, int n, int P,
                                                T h, T alpha, T cnorm, TauArg ta_) {
  const T tau = (T)tau_of(ta_);
  __shared__ T sw[8][3][kMaxP], sy[8][3][kMaxP];
  __shared__ int si[8][3][kMaxP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= Nt) return;
  const auto p = pos[i];
  const T pc[3] = {p.x, p.y, p.z};
  for (int e = lane; e < 3 * P; e += 32) {
    int d = e / P, k = e - d * P;
    int g0 = (int)floor_t<T>(pc[d] / h) - P / 2 + 1;
    int g = g0 + k;
    T yv = T(g) * h - pc[d];
    sw[warp][d][k] = exp_t<T>(-alpha * yv * yv);
    sy[warp][d][k] = yv;
    si[warp][d][k] = ((g % n) + n) % n;
  }
  __syncwarp();
  const double *xr = x + (size_t)i * LDB;
  const T F0 = (T)xr[0], F1 = (T)xr[1], F2 = (T)xr[2];
  const T L0 = (T)xr[3], L1 = (T)xr[4], L2 = (T)xr[5];
  const T r2i = T(0.70710678118654752440), r6i = T(0.40824829046386301637);
  const T s0 = (T)xr[6], s1 = (T)xr[7], s2 = (T)xr[8], s3 = (T)xr[9], s4 = (T)xr[10];
  const T Sxx = r2i * s0 - r6i * s1, Syy = -r2i * s0 - r6i * s1, Szz = T(2) * r6i * s1;
  const T Sxy = r2i * s2, Sxz = r2i * s3, Syz = r2i * s4;
  // D = S + A with A y = (1/2) L x y; in a Lees-Edwards box the window is a
  // Gaussian of the sheared coordinates, whose x-gradient is the s-gradient
  // transformed by A^-T: column 0 of D takes -tau column 1
  const T D01 = Sxy - T(0.5) * L2, D11 = Syy, D21 = Syz + T(0.5) * L0;
  const T D00 = Sxx - tau * D01, D02 = Sxz + T(0.5) * L1;
  const T D10 = Sxy + T(0.5) * L2 - tau * D11, D12 = Syz - T(0.5) * L0;
  const T D20 = Sxz - T(0.5) * L1 - tau * D21, D22 = Szz;
  const int P3 = P * P * P;
  const T ta = T(2) * alpha;
  for (int t = lane; t < P3; t += 32) {
    const int ix = t % P, iy = (t / P) % P, iz = t / (P * P);
    const T W = cnorm * sw[warp][0][ix] * sw[warp][1][iy] * sw[warp][2][iz];
    const T y0 = sy[warp][0][ix], y1 = sy[warp][1][iy], y2 = sy[warp][2][iz];
    const T Wd = ta * W;
    T *q = grid + (((int64_t)si[warp][2][iz] * n + si[warp][1][iy]) * n + si[warp][0][ix]);
    const int64_t n3 = (int64_t)n * n * n;
    atomicAdd(q, W * F0);
    atomicAdd(q + n3, W * F1);
    atomicAdd(q + 2 * n3, W * F2);
    atomicAdd(q + 3 * n3, Wd * (D00 * y0 + D01 * y1 + D02 * y2));
    atomicAdd(q + 4 * n3, Wd * (D10 * y0 + D11 * y1 + D12 * y2));
    atomicAdd(q + 5 * n3, Wd * (D20 * y0 + D21 * y1 + D22 * y2));
  }
}

// FP32 spreading with 16-byte vector reductions (grids whose side n is a
// multiple of 4): the same sums as k_spread, but each lane owns an aligned
// quad of four x points of one grid row and adds its six components with
// one red.global.add.v4.f32 each, so a bead issues a quarter of the atomic
// operations.  The bead's x window [g0, g0 + P) is covered by the aligned
// quads from a0 = 4 floor(g0 / 4); slots outside the window carry weight 0.
constexpr int kMaxQ = (kMaxP + 6) / 4;

__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__global__ void __launch_bounds__(256) k_spread_v4(int Nt, const float4 *__restrict__ pos,
                                                   const double *__restrict__ x, float *grid, int n,
                                                   int P, float h, float alpha, float cnorm, TauArg ta_) {
  const float tau = (float)tau_of(ta_);
  __shared__ float sw[8][2][kMaxP], sy[8][2][kMaxP];
  __shared__ int si[8][2][kMaxP];
  __shared__ float sxw[8][4 * kMaxQ], sxy[8][4 * kMaxQ];
  __shared__ int sxq[8][kMaxQ];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= Nt) return;
  const float4 p = pos[i];
  const int g0x = (int)floorf(p.x / h) - P / 2 + 1;
  const int a0 = g0x >= 0 ? (g0x & ~3) : -((-g0x + 3) & ~3);  // 4 floor(g0x / 4)
  const int nq = (g0x - a0 + P + 3) >> 2;                      // quads covering the window
  for (int e = lane; e < 2 * P; e += 32) {
    const int d = e / P, k = e - d * P;
    const float pc = d == 0 ? p.y : p.z;
    const int g = (int)floorf(pc / h) - P / 2 + 1 + k;
    const float yv = float(g) * h - pc;
    sw[warp][d][k] = expf(-alpha * yv * yv);
    sy[warp][d][k] = yv;
    si[warp][d][k] = ((g % n) + n) % n;
  }
  for (int sl = lane; sl < 4 * nq; sl += 32) {
    const int g = a0 + sl, k = g - g0x;
    const float yv = float(g) * h - p.x;
    sxw[warp][sl] = (k >= 0 && k < P) ? expf(-alpha * yv * yv) : 0.f;
    sxy[warp][sl] = yv;
  }
  for (int q = lane; q < nq; q += 32) sxq[warp][q] = (((a0 + 4 * q) % n) + n) % n;
  __syncwarp();
  const double *xr = x + (size_t)i * LDB;
  const float F0 = (float)xr[0], F1 = (float)xr[1], F2 = (float)xr[2];
  const float L0 = (float)xr[3], L1 = (float)xr[4], L2 = (float)xr[5];
  const float r2i = 0.70710678118654752440f, r6i = 0.40824829046386301637f;
  const float s0 = (float)xr[6], s1 = (float)xr[7], s2 = (float)xr[8], s3 = (float)xr[9],
              s4 = (float)xr[10];
  const float Sxx = r2i * s0 - r6i * s1, Syy = -r2i * s0 - r6i * s1, Szz = 2.f * r6i * s1;
  const float Sxy = r2i * s2, Sxz = r2i * s3, Syz = r2i * s4;
  const float D01 = Sxy - 0.5f * L2, D11 = Syy, D21 = Syz + 0.5f * L0;
  const float D00 = Sxx - tau * D01, D02 = Sxz + 0.5f * L1;
  const float D10 = Sxy + 0.5f * L2 - tau * D11, D12 = Syz - 0.5f * L0;
  const float D20 = Sxz - 0.5f * L1 - tau * D21, D22 = Szz;
  const float ta = 2.f * alpha;
  const int64_t n3 = (int64_t)n * n * n;
  const int T = P * P * nq;
  for (int t = lane; t < T; t += 32) {
    const int q = t % nq, r = t / nq;
    const int iy = r % P, iz = r / P;
    const float wyz = cnorm * sw[warp][0][iy] * sw[warp][1][iz];
    const float y1 = sy[warp][0][iy], y2 = sy[warp][1][iz];
    const float b0 = D01 * y1 + D02 * y2, b1 = D11 * y1 + D12 * y2, b2 = D21 * y1 + D22 * y2;
    float W[4], d0[4], d1[4], d2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float w = wyz * sxw[warp][4 * q + j];
      const float y0 = sxy[warp][4 * q + j];
      const float wd = ta * w;
      W[j] = w;
      d0[j] = wd * (D00 * y0 + b0);
      d1[j] = wd * (D10 * y0 + b1);
      d2[j] = wd * (D20 * y0 + b2);
    }
    float *g = grid + (((int64_t)si[warp][1][iz] * n + si[warp][0][iy]) * n + sxq[warp][q]);
    red_add_v4(g, W[0] * F0, W[1] * F0, W[2] * F0, W[3] * F0);
    red_add_v4(g + n3, W[0] * F1, W[1] * F1, W[2] * F1, W[3] * F1);
    red_add_v4(g + 2 * n3, W[0] * F2, W[1] * F2, W[2] * F2, W[3] * F2);
    red_add_v4(g + 3 * n3, d0[0], d0[1], d0[2], d0[3]);
    red_add_v4(g + 4 * n3, d1[0], d1[1], d1[2], d1[3]);
    red_add_v4(g + 5 * n3, d2[0], d2[1], d2[2], d2[3]);
  }
}

// One warp per bead: u = h^3 sum W u_M, G_ab = h^3 sum 2 alpha W y_b u_D,a;
// omega = (1/2) curl, e = sym G projected; added to the bead row of y.
// PL: the six fields are planar [6][n^3] (from the fused FFT) instead of
// interleaved [n^3][8].
template <typename T, bool PL>
__global__ void __launch_bounds__(256) k_interp(int Nt, const typename V4Of<T>::type *__restrict__ pos,
                                                const T *__restrict__ grid, double *y, int n, int P,
                                                T h, T alpha, T cnorm_h3, TauArg ta_) {
  const double tau = tau_of(ta_);
  __shared__ T sw[8][3][kMaxP], sy[8][3][kMaxP];
  __shared__ int si[8][3][kMaxP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= Nt) return;
  const auto p = pos[i];
  const T pc[3] = {p.x, p.y, p.z};
  for (int e = lane; e < 3 * P; e += 32) {
    int d = e / P, k = e - d * P;
    int g0 = (int)floor_t<T>(pc[d] / h) - P / 2 + 1;
    int g = g0 + k;
    T yv = T(g) * h - pc[d];
    sw[warp][d][k] = exp_t<T>(-alpha * yv * yv);
    sy[warp][d][k] = yv;
    si[warp][d][k] = ((g % n) + n) % n;
  }
  __syncwarp();
  const int P3 = P * P * P;
  const T ta = T(2) * alpha;
  T acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(0);
  for (int t = lane; t < P3; t += 32) {
    const int ix = t % P, iy = (t / P) % P, iz = t / (P * P);
    const T W = sw[warp][0][ix] * sw[warp][1][iy] * sw[warp][2][iz];
    const T y0 = sy[warp][0][ix], y1 = sy[warp][1][iy], y2 = sy[warp][2][iz];
    T g6[6];
    const int64_t gi = ((int64_t)si[warp][2][iz] * n + si[warp][1][iy]) * n + si[warp][0][ix];
    if (PL) {
      const int64_t n3 = (int64_t)n * n * n;
#pragma unroll
      for (int c = 0; c < 6; ++c) g6[c] = grid[c * n3 + gi];
    } else {
      load6<T>(grid + (gi << 3), g6);
    }
    const T u0 = g6[0], u1 = g6[1], u2 = g6[2], d0 = g6[3], d1 = g6[4], d2 = g6[5];
    acc[0] += W * u0;
    acc[1] += W * u1;
    acc[2] += W * u2;
    T Wd = ta * W;
    T w0 = Wd * y0, w1 = Wd * y1, w2 = Wd * y2;
    acc[3] += d0 * w0;  // G_00
    acc[4] += d0 * w1;  // G_01
    acc[5] += d0 * w2;  // G_02
    acc[6] += d1 * w0;  // G_10
    acc[7] += d1 * w1;  // G_11
    acc[8] += d1 * w2;  // G_12
    acc[9] += d2 * w0;  // G_20
    acc[10] += d2 * w1; // G_21
    acc[11] += d2 * w2; // G_22
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  if (lane != 0) return;
  double a_[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) a_[k] = (double)acc[k] * (double)cnorm_h3;
  // Lees-Edwards box: d/dy = d/ds_y - tau d/ds_x on the sheared window
  const double G00 = a_[3], G01 = a_[4] - tau * a_[3], G02 = a_[5], G10 = a_[6],
               G11 = a_[7] - tau * a_[6], G12 = a_[8], G20 = a_[9], G21 = a_[10] - tau * a_[9],
               G22 = a_[11];
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637,
               s2 = 1.41421356237309504880;
  double *yr = y + (size_t)i * LDB;
  yr[0] += a_[0];
  yr[1] += a_[1];
  yr[2] += a_[2];
  yr[3] += 0.5 * (G21 - G12);
  yr[4] += 0.5 * (G02 - G20);
  yr[5] += 0.5 * (G10 - G01);
  yr[6] += r2i * (G00 - G11);
  yr[7] += r6i * (2.0 * G22 - G00 - G11);
  yr[8] += s2 * 0.5 * (G01 + G10);
  yr[9] += s2 * 0.5 * (G02 + G20);
  yr[10] += s2 * 0.5 * (G12 + G21);
}

// The sums of k_interp from interleaved fields [n^3][8], factored by grid
// row: each lane takes whole (y, z) rows of the window and first sums the
// row along x (the six fields weighted by w_x, the three dipole fields also
// by w_x (x - p_x)), then adds the row's sums with its y and z factors.
// Ten products per window point instead of eighteen: the FP64 operator,
// whose arithmetic runs at 1/74 of the FP32 rate, spends its interpolation
// there.
template <typename T>
__global__ void __launch_bounds__(256) k_interp_rows(int Nt, const typename V4Of<T>::type *__restrict__ pos,
                                                     const T *__restrict__ grid, double *y, int n,
                                                     int P, T h, T alpha, T cnorm_h3, TauArg ta_,
                                                     FastDiv fp) {
  const double tau = tau_of(ta_);
  __shared__ T sw[8][3][kMaxP], sy[8][3][kMaxP], swx[8][kMaxP];
  __shared__ int si[8][3][kMaxP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= Nt) return;
  const auto p = pos[i];
  const T pc[3] = {p.x, p.y, p.z};
  for (int e = lane; e < 3 * P; e += 32) {
    int d = e / P, k = e - d * P;
    int g0 = (int)floor_t<T>(pc[d] / h) - P / 2 + 1;
    int g = g0 + k;
    T yv = T(g) * h - pc[d];
    const T w = exp_t<T>(-alpha * yv * yv);
    sw[warp][d][k] = w;
    sy[warp][d][k] = yv;
    si[warp][d][k] = ((g % n) + n) % n;
    if (d == 0) swx[warp][k] = w * yv;
  }
  __syncwarp();
  const T ta = T(2) * alpha;
  T acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(0);
  for (int r = lane; r < P * P; r += 32) {
    const int iz = (int)fdiv((uint32_t)r, fp), iy = r - iz * P;
    const T* row = grid + (((int64_t)si[warp][2][iz] * n + si[warp][1][iy]) * n << 3);
    T S[6], Tx[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) S[c] = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) Tx[a] = T(0);
    for (int ix = 0; ix < P; ++ix) {
      T g6[6];
      load6<T>(row + ((int64_t)si[warp][0][ix] << 3), g6);
      const T w = sw[warp][0][ix], wy = swx[warp][ix];
#pragma unroll
      for (int c = 0; c < 6; ++c) S[c] += w * g6[c];
#pragma unroll
      for (int a = 0; a < 3; ++a) Tx[a] += wy * g6[3 + a];
    }
    const T wyz = sw[warp][1][iy] * sw[warp][2][iz];
    const T tw = ta * wyz, t1 = tw * sy[warp][1][iy], t2 = tw * sy[warp][2][iz];
    acc[0] += wyz * S[0];
    acc[1] += wyz * S[1];
    acc[2] += wyz * S[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[3 + 3 * a] += tw * Tx[a];     // G_a0
      acc[4 + 3 * a] += t1 * S[3 + a];  // G_a1
      acc[5 + 3 * a] += t2 * S[3 + a];  // G_a2
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  if (lane != 0) return;
  double a_[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) a_[k] = (double)acc[k] * (double)cnorm_h3;
  // Lees-Edwards box: d/dy = d/ds_y - tau d/ds_x on the sheared window
  const double G00 = a_[3], G01 = a_[4] - tau * a_[3], G02 = a_[5], G10 = a_[6],
               G11 = a_[7] - tau * a_[6], G12 = a_[8], G20 = a_[9], G21 = a_[10] - tau * a_[9],
               G22 = a_[11];
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637,
               s2 = 1.41421356237309504880;
  double *yr = y + (size_t)i * LDB;
  yr[0] += a_[0];
  yr[1] += a_[1];
  yr[2] += a_[2];
  yr[3] += 0.5 * (G21 - G12);
  yr[4] += 0.5 * (G02 - G20);
  yr[5] += 0.5 * (G10 - G01);
  yr[6] += r2i * (G00 - G11);
  yr[7] += r6i * (2.0 * G22 - G00 - G11);
  yr[8] += s2 * 0.5 * (G01 + G10);
  yr[9] += s2 * 0.5 * (G02 + G20);
  yr[10] += s2 * 0.5 * (G12 + G21);
}

// FP32 interpolation from planar fields [6][n^3] (n a multiple of 4): the
// sums of k_interp, with each lane reading an aligned quad of four x points
// of one grid row per field (six 16-byte loads); slots outside the bead's x
// window carry weight 0 (the quads of k_spread_v4).  The warp's items are
// (quad, y row, z row) with a fixed quad count NQ = (P + 7) / 4 per row
// (lanes past the bead's own quad count skip), so that the item index splits
// with two multiply-shift divisions; the window tables hold (w, offset)
// pairs and the rows' grid offsets, and the factor 2 alpha of the dipole
// read-out is applied once per bead.
__global__ void __launch_bounds__(256, 4) k_interp_v4(int Nt, const float4 *__restrict__ pos,
                                                   const float *__restrict__ field, double *y, int n,
                                                   int P, float h, float alpha, float cnorm_h3,
                                                   TauArg ta_, FastDiv fq, FastDiv fp) {
  const double tau = tau_of(ta_);
  __shared__ float2 swy[8][2][kMaxP];  // (w, offset) of the y and z window rows
  __shared__ int srow[8][2][kMaxP];    // grid offsets of the rows: y n, z n^2
  __shared__ __align__(16) float sxw[8][4 * kMaxQ], sxy[8][4 * kMaxQ];
  __shared__ int sxq[8][kMaxQ];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= Nt) return;
  const float4 p = pos[i];
  const int g0x = (int)floorf(p.x / h) - P / 2 + 1;
  const int a0 = g0x >= 0 ? (g0x & ~3) : -((-g0x + 3) & ~3);
  const int nq = (g0x - a0 + P + 3) >> 2;
  const int NQ = (int)fq.d;
  for (int e = lane; e < 2 * P; e += 32) {
    const int d = e / P, k = e - d * P;
    const float pc = d == 0 ? p.y : p.z;
    const int g = (int)floorf(pc / h) - P / 2 + 1 + k;
    const float yv = float(g) * h - pc;
    swy[warp][d][k] = make_float2(expf(-alpha * yv * yv), yv);
    const int gi = ((g % n) + n) % n;
    srow[warp][d][k] = d == 0 ? gi * n : gi * n * n;
  }
  for (int sl = lane; sl < 4 * NQ; sl += 32) {
    const int g = a0 + sl, k = g - g0x;
    const float yv = float(g) * h - p.x;
    sxw[warp][sl] = (k >= 0 && k < P) ? expf(-alpha * yv * yv) : 0.f;
    sxy[warp][sl] = yv;
  }
  for (int q = lane; q < NQ; q += 32) sxq[warp][q] = (((a0 + 4 * q) % n) + n) % n;
  __syncwarp();
  const int64_t n3 = (int64_t)n * n * n;
  float acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = 0.f;
  const int T = P * P * NQ;
#pragma unroll 2
  for (int t = lane; t < T; t += 32) {
    const int r = (int)fdiv((uint32_t)t, fq), q = t - r * NQ;
    if (q >= nq) continue;
    const int iz = (int)fdiv((uint32_t)r, fp), iy = r - iz * P;
    const float2 wy = swy[warp][0][iy], wz = swy[warp][1][iz];
    const float wyz = wy.x * wz.x, y1 = wy.y, y2 = wz.y;
    const float *g = field + (srow[warp][1][iz] + srow[warp][0][iy] + sxq[warp][q]);
    float4 f[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) f[c] = __ldg((const float4 *)(g + c * n3));
    const float4 xw = *(const float4 *)&sxw[warp][4 * q], xy = *(const float4 *)&sxy[warp][4 * q];
    const float W[4] = {wyz * xw.x, wyz * xw.y, wyz * xw.z, wyz * xw.w};
    const float WY[4] = {W[0] * xy.x, W[1] * xy.y, W[2] * xy.z, W[3] * xy.w};
#pragma unroll
    for (int c = 0; c < 3; ++c)
      acc[c] += W[0] * f[c].x + W[1] * f[c].y + W[2] * f[c].z + W[3] * f[c].w;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 d = f[3 + a];
      const float s = W[0] * d.x + W[1] * d.y + W[2] * d.z + W[3] * d.w;
      acc[3 + 3 * a] += WY[0] * d.x + WY[1] * d.y + WY[2] * d.z + WY[3] * d.w;  // G_a0
      acc[4 + 3 * a] += s * y1;                                                // G_a1
      acc[5 + 3 * a] += s * y2;                                                // G_a2
    }
  }
  {
    const float ta = 2.f * alpha;
#pragma unroll
    for (int k = 3; k < 12; ++k) acc[k] *= ta;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  if (lane != 0) return;
  double a_[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) a_[k] = (double)acc[k] * (double)cnorm_h3;
  // Lees-Edwards box: d/dy = d/ds_y - tau d/ds_x on the sheared window
  const double G00 = a_[3], G01 = a_[4] - tau * a_[3], G02 = a_[5], G10 = a_[6],
               G11 = a_[7] - tau * a_[6], G12 = a_[8], G20 = a_[9], G21 = a_[10] - tau * a_[9],
               G22 = a_[11];
  const double r2i = 0.70710678118654752440, r6i = 0.40824829046386301637,
               s2 = 1.41421356237309504880;
  double *yr = y + (size_t)i * LDB;
  yr[0] += a_[0];
  yr[1] += a_[1];
  yr[2] += a_[2];
  yr[3] += 0.5 * (G21 - G12);
  yr[4] += 0.5 * (G02 - G20);
  yr[5] += 0.5 * (G10 - G01);
  yr[6] += r2i * (G00 - G11);
  yr[7] += r6i * (2.0 * G22 - G00 - G11);
  yr[8] += s2 * 0.5 * (G01 + G10);
  yr[9] += s2 * 0.5 * (G02 + G20);
  yr[10] += s2 * 0.5 * (G12 + G21);
}

// ------------------------------------------- grid-centric FP32 spreading
// The same sums as k_spread_v4, organised by grid point instead of by bead:
// the grid is cut into 8^3 tiles and each tile keeps the list of beads whose
// P^3 window reaches it (built once per geometry).  One block of 64 threads
// per tile, one thread per (y, z) row of the tile summing, in registers, the
// contributions of the tile's beads to its 8 points: no atomics, and every
// grid point is written exactly once (no zeroing pass).
constexpr int kTS = 8;      // tile side
constexpr int kTCH = 32;    // beads per shared-memory chunk

// distinct tiles (per axis) covered by the window of a bead at coordinate p
__device__ __forceinline__ int window_tiles(float p, float h, int P, int n, int t[5]) {
  const int g0 = (int)floorf(p / h) - P / 2 + 1;
  int cnt = 0;
  for (int k = 0; k < P; ++k) {
    const int g = ((g0 + k) % n + n) % n;
    const int tt = g / kTS;
    bool seen = false;
    for (int q = 0; q < cnt; ++q) seen |= t[q] == tt;
    if (!seen && cnt < 5) t[cnt++] = tt;
  }
  return cnt;
}

template <bool FILL>
__global__ void k_tile_bin(int Nt, const float4 *__restrict__ pos, float h, int P, int n, int nt,
                           int *count_or_cursor, int *tile_beads, int64_t cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt) return;
  const float4 p = pos[i];
  int tx[5], ty[5], tz[5];
  const int cx = window_tiles(p.x, h, P, n, tx), cy = window_tiles(p.y, h, P, n, ty),
            cz = window_tiles(p.z, h, P, n, tz);
  for (int a = 0; a < cz; ++a)
    for (int b = 0; b < cy; ++b)
      for (int d = 0; d < cx; ++d) {
        const int id = (tz[a] * nt + ty[b]) * nt + tx[d];
        const int slot = atomicAdd(&count_or_cursor[id], 1);
        if (FILL && slot < cap) tile_beads[slot] = i;
      }
}

// Per chunk of kTCH beads the block stages, per bead: the x-window factors w
// and their products with the offset, w (g h - p), for the tile's 8 x
// points (the dipole term's x factor); (w, offset) pairs for its 8 y and 8 z
// points; the twelve scaled moments; and 8-bit masks of the tile's y and z
// rows its window reaches.  Each thread then iterates over exactly the
// beads whose window covers its (y, z) row (a bit mask over the chunk, from
// sixteen warp ballots), so a warp runs the largest count among its rows
// instead of every bead listed for the tile.
__global__ void __launch_bounds__(64, 12) k_spread_gather(int n, int nt, int P, float h, float alpha,
                                                      float cnorm, TauArg ta_,
                                                      const float4 *__restrict__ pos,
                                                      const double *__restrict__ x,
                                                      const int *__restrict__ tile_start,
                                                      const int *__restrict__ tile_beads,
                                                      float *grid) {
  const float tau = (float)tau_of(ta_);
  // records padded to an odd number of 16-byte units (bank spread when the
  // lanes of a warp read different beads)
  __shared__ __align__(16) float swx[kTCH][20];      // w[8], w * offset[8], pad
  __shared__ __align__(16) float2 syz[kTCH][2][9];   // (w, offset) of y[8] and z[8], pad
  __shared__ __align__(16) float sm[kTCH][12];
  __shared__ unsigned scov[2][kTCH];  // y and z rows of the tile each bead's window reaches
  const int tile = blockIdx.x;
  const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
  const int x0 = tx * kTS, y0 = ty * kTS, z0 = tz * kTS;
  const int iy = threadIdx.x & 7, iz = threadIdx.x >> 3;
  float acc[6][kTS];
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int k = 0; k < kTS; ++k) acc[c][k] = 0.f;
  const int b0 = tile_start[tile], b1 = tile_start[tile + 1];
  const float ta = 2.f * alpha;
  for (int cb = b0; cb < b1; cb += kTCH) {
    const int nc = min(kTCH, b1 - cb);
    __syncthreads();
    // 1D window factors and offsets of each bead at this tile's coordinates:
    // one (bead, axis) pair per task, its window start from one division; the
    // y and z rows the window reaches as bit masks
    for (int e = threadIdx.x; e < nc * 3; e += blockDim.x) {
      const int bi = e / 3, d = e - bi * 3;
      const float4 p = pos[tile_beads[cb + bi]];
      const float pc = d == 0 ? p.x : (d == 1 ? p.y : p.z);
      const int g0 = (int)floorf(pc / h) - P / 2 + 1;
      const int gb = d == 0 ? x0 : (d == 1 ? y0 : z0);
      unsigned cov = 0;
#pragma unroll 1
      for (int k = 0; k < kTS; ++k) {
        const int gt = gb + k;
        float w = 0.f, yv = 0.f;
        if (gt < n) {
          // slot of this grid index in the window (g0 is within one box of gt)
          int off = gt - g0;
          if (off < 0) off += n;
          if (off >= n) off -= n;
          if (off < P) {
            yv = float(g0 + off) * h - pc;
            w = expf(-alpha * yv * yv);
          }
        }
        cov |= (w != 0.f ? 1u : 0u) << k;
        if (d == 0) {
          swx[bi][k] = w;
          swx[bi][kTS + k] = w * yv;
        } else {
          syz[bi][d - 1][k] = make_float2(w, yv);
        }
      }
      if (d > 0) scov[d - 1][bi] = cov;
    }
    // moments: F and the dipole D (= S + antisym(L); column 0 takes -tau
    // column 1 in a Lees-Edwards box), with the window norm and 2 alpha
    for (int bi = threadIdx.x; bi < nc; bi += blockDim.x) {
      const double *xr = x + (size_t)tile_beads[cb + bi] * LDB;
      const float F0 = (float)xr[0], F1 = (float)xr[1], F2 = (float)xr[2];
      const float L0 = (float)xr[3], L1 = (float)xr[4], L2 = (float)xr[5];
      const float r2i = 0.70710678118654752440f, r6i = 0.40824829046386301637f;
      const float s0 = (float)xr[6], s1 = (float)xr[7], s2 = (float)xr[8], s3 = (float)xr[9],
                  s4 = (float)xr[10];
      const float Sxx = r2i * s0 - r6i * s1, Syy = -r2i * s0 - r6i * s1, Szz = 2.f * r6i * s1;
      const float Sxy = r2i * s2, Sxz = r2i * s3, Syz = r2i * s4;
      const float D01 = Sxy - 0.5f * L2, D11 = Syy, D21 = Syz + 0.5f * L0;
      const float D00 = Sxx - tau * D01, D02 = Sxz + 0.5f * L1;
      const float D10 = Sxy + 0.5f * L2 - tau * D11, D12 = Syz - 0.5f * L0;
      const float D20 = Sxz - 0.5f * L1 - tau * D21, D22 = Szz;
      const float cd = ta * cnorm;
      float *m = sm[bi];
      m[0] = cnorm * F0;
      m[1] = cnorm * F1;
      m[2] = cnorm * F2;
      m[3] = cd * D00;
      m[4] = cd * D01;
      m[5] = cd * D02;
      m[6] = cd * D10;
      m[7] = cd * D11;
      m[8] = cd * D12;
      m[9] = cd * D20;
      m[10] = cd * D21;
      m[11] = cd * D22;
    }
    __syncthreads();
    // the beads whose window covers this thread's (y, z) row, as a bit mask
    // over the chunk: per y row and per z row a ballot across the lanes
    // (lane b of each warp stands for bead b of the chunk)
    unsigned mask;
    {
      const int lane = threadIdx.x & 31;
      const unsigned yc = lane < nc ? scov[0][lane] : 0u, zc = lane < nc ? scov[1][lane] : 0u;
      unsigned my = 0, mz = 0;
#pragma unroll
      for (int k = 0; k < kTS; ++k) {
        const unsigned by = __ballot_sync(0xffffffffu, (yc >> k) & 1u);
        const unsigned bz = __ballot_sync(0xffffffffu, (zc >> k) & 1u);
        if (k == iy) my = by;
        if (k == iz) mz = bz;
      }
      mask = my & mz;
    }
    while (mask) {
      const int bi = __ffs(mask) - 1;
      mask &= mask - 1;
      const float2 py = syz[bi][0][iy], pz = syz[bi][1][iz];
      const float wyz = py.x * pz.x, yy = py.y, yz = pz.y;
      const float4 m0 = *(const float4 *)&sm[bi][0], m1 = *(const float4 *)&sm[bi][4],
                   m2 = *(const float4 *)&sm[bi][8];
      const float f0 = m0.x * wyz, f1 = m0.y * wyz, f2 = m0.z * wyz;
      const float a0 = m0.w * wyz, a1 = m1.z * wyz, a2 = m2.y * wyz;
      const float c0 = (m1.x * yy + m1.y * yz) * wyz, c1 = (m1.w * yy + m2.x * yz) * wyz,
                  c2 = (m2.z * yy + m2.w * yz) * wyz;
      const float4 wa = *(const float4 *)&swx[bi][0], wb = *(const float4 *)&swx[bi][4];
      const float4 pa = *(const float4 *)&swx[bi][8], pb = *(const float4 *)&swx[bi][12];
      const float wx[kTS] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
      const float px[kTS] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
#pragma unroll
      for (int k = 0; k < kTS; ++k) {
        acc[0][k] += f0 * wx[k];
        acc[1][k] += f1 * wx[k];
        acc[2][k] += f2 * wx[k];
        acc[3][k] += a0 * px[k] + c0 * wx[k];
        acc[4][k] += a1 * px[k] + c1 * wx[k];
        acc[5][k] += a2 * px[k] + c2 * wx[k];
      }
    }
  }
  const int yg = y0 + iy, zg = z0 + iz;
  if (yg >= n || zg >= n) return;
  const int64_t n3 = (int64_t)n * n * n;
  float *row = grid + ((int64_t)zg * n + yg) * n + x0;
  if (x0 + kTS <= n && (n & 3) == 0) {  // 16-byte aligned rows
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 *r4 = (float4 *)(row + c * n3);
      r4[0] = make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
      r4[1] = make_float4(acc[c][4], acc[c][5], acc[c][6], acc[c][7]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int k = 0; k < kTS; ++k)
        if (x0 + k < n) row[c * n3 + k] = acc[c][k];
  }
}

// ------------------------------------------------------------ host side

static double j0h(double z) {
  if (z < 1e-3) return 1.0 - z * z / 6.0 + z * z * z * z / 120.0;
  return std::sin(z) / z;
}
static double fDh(double z) {
  if (z < 1e-2) return 1.0 - z * z / 10.0 + z * z * z * z / 280.0;
  return 3.0 * (std::sin(z) - z * std::cos(z)) / (z * z * z);
}

template <typename T>
static void upload(DBuf<T> &buf, const std::vector<double> &v) {
  std::vector<T> tv(v.begin(), v.end());
  buf.alloc(tv.size());
  FSD_CUDA(cudaMemcpy(buf.p, tv.data(), tv.size() * sizeof(T), cudaMemcpyHostToDevice));
}

void build_wave(Ctx &c) {
  const int n = c.n;
  const size_t gsize = (size_t)6 * n * n * n;
  const size_t osize = (size_t)8 * n * n * n;
  const size_t ssize = (size_t)6 * n * n * (n + 2);
  c.op64.grid.alloc(gsize);
  c.op32.grid.alloc(gsize);
  c.op64.gout.alloc(osize);
  c.op32.gout.alloc(osize);
  c.op64.spec.alloc(ssize);
  c.op32.spec.alloc(ssize);
  // per-stage twiddle tables of the plan
  std::vector<double> tw;
  make_plan(n, &tw, true);
  upload(c.op64.twiddle, tw);
  upload(c.op32.twiddle, tw);
  // Green table by m = kx^2 + ky^2 + kz^2
  const int hm = n / 2;
  const int mmax = 3 * hm * hm;
  std::vector<double> gr(3 * (size_t)(mmax + 1), 0.0);
  const double n3 = (double)n * n * n;
  for (int m = 1; m <= mmax; ++m) {
    double k = 2.0 * kPi * std::sqrt((double)m) / c.L;
    double k2 = k * k;
    double e = -k2 / (4.0 * c.xi * c.xi) + k2 / (2.0 * c.alpha);
    double A = (1.0 + k2 / (4.0 * c.xi * c.xi)) * std::exp(e) / (c.eta * k2) / n3;
    double fm = j0h(k * c.a), fd = fDh(k * c.a);
    gr[3 * m] = A * fm * fm;
    gr[3 * m + 1] = A * fm * fd;
    gr[3 * m + 2] = A * fd * fd;
  }
  upload(c.op64.green, gr);
  upload(c.op32.green, gr);
  // Brownian wave-field scales (Sec. 2.2, Eq. UBff): the random field xi(k)
  // becomes f(k) sqrt(H(k)/(eta k^2)) / (sqrt(V) W^(k)) (I - k k) xi(k), the
  // analytic square root of the wave part once the interpolation's Gaussian
  // W^(k) = exp(-k^2/(4 alpha)) is divided out
  std::vector<double> bt(2 * (size_t)(mmax + 1), 0.0);
  const double isv = 1.0 / std::sqrt(c.L * c.L * c.L);
  for (int m = 1; m <= mmax; ++m) {
    double k = 2.0 * kPi * std::sqrt((double)m) / c.L;
    double k2 = k * k;
    double H = (1.0 + k2 / (4.0 * c.xi * c.xi)) * std::exp(-k2 / (4.0 * c.xi * c.xi));
    double sc = std::sqrt(H / (c.eta * k2)) * std::exp(k2 / (4.0 * c.alpha)) * isv;
    bt[2 * m] = sc * j0h(k * c.a);
    bt[2 * m + 1] = sc * fDh(k * c.a);
  }
  upload(c.op64.btab, bt);
  upload(c.op32.btab, bt);
}

template <typename T>
static OpData<T> &opd(Ctx &c);
template <>
OpData<double> &opd<double>(Ctx &c) {
  return c.op64;
}
template <>
OpData<float> &opd<float>(Ctx &c) {
  return c.op32;
}
template <typename T>
static const typename V4Of<T>::type *posp(Ctx &c);
// wave-space bead positions: the sheared coordinates of a Lees-Edwards box
// (the ordinary wrapped positions for tilt 0)
template <>
const double4 *posp<double>(Ctx &c) {
  return (const double4 *)c.wpos64.p;
}
template <>
const float4 *posp<float>(Ctx &c) {
  return (const float4 *)c.wpos32.p;
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, size);
// thread-safe (contexts may run on several host threads).
template <typename T>
static void set_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void *, size_t>> done;
  std::lock_guard<std::mutex> lock(mu);
  for (auto &d : done)
    if (d.first == fn && d.second >= bytes) return;
  FSD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done.push_back({fn, bytes});
}

// Largest log2 line count <= want whose two line buffers (lines_per_unit
// lines each of the padded length) and the twiddles fit one block's shared
// memory; large grids (FP64 above n ~ 270) take fewer lines per block.
template <typename T>
static int fit_log2_lines(int want, int lines_per_unit, int n, int ntw) {
  for (int l = want; l >= 0; --l) {
    const size_t b = (size_t)(ntw + 2 * (size_t)lines_per_unit * (1 << l) * fft_ls(n)) * sizeof(Cx<T>);
    if (b <= (size_t)227 * 1024) return l;
  }
  throw Invalid{"FFT grid too large for one line per block in shared memory"};
}

// Inverse y and x transforms of the six fields held in spec (after the z
// pass), then interpolation: y += h^3 sum W (fields) per bead.
template <typename T>
static void wave_tail(Ctx &c, OpData<T> &op, const FftPlan &plan, Cx<T> *spec, double *y) {
  const int n = c.n, P = c.P;
  const T h = (T)c.h, alpha = (T)c.alpha;
  const double cn = std::pow(c.alpha / kPi, 1.5);
  const int nh = n / 2 + 1;
  const int threads = 256;
  const int ntw = plan.ntw;
  const size_t sm_xy = (size_t)(ntw + 2 * nh * fft_ls(n)) * sizeof(Cx<T>);
  const bool fused = sizeof(T) == 4 && sm_xy <= (size_t)227 * 1024;
  const int LTXy = fit_log2_lines<T>(sizeof(T) == 8 ? 3 : 4, 1, n, ntw);
  const int TXy = 1 << LTXy;
  const size_t smy = (size_t)(ntw + 2 * TXy * fft_ls(n)) * sizeof(Cx<T>);
  const int blocks_y = 6 * n * ceil_div(nh, TXy);
  {
  ProfScope ps(c, PG_FFT);
  if (fused) {
    if (is_fft144(plan)) {
      set_smem<T>((const void *)k_fft_xy_inv<T, true>, sm_xy);
      k_fft_xy_inv<T, true><<<6 * n, 1024, sm_xy, c.stream>>>(op.gout.p, spec, plan, op.twiddle.p);
    } else {
      set_smem<T>((const void *)k_fft_xy_inv<T, false>, sm_xy);
      k_fft_xy_inv<T, false><<<6 * n, 1024, sm_xy, c.stream>>>(op.gout.p, spec, plan, op.twiddle.p);
    }
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  } else {
    // the Brownian wave sample can reach this before any forward pass has
    // raised the kernel's shared-memory limit
    set_smem<T>((const void *)k_fft_y<T>, smy);
    k_fft_y<T><<<blocks_y, threads, smy, c.stream>>>(spec, plan, op.twiddle.p, LTXy, T(1));
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    const int NL = 1 << fit_log2_lines<T>(2, 3, n, ntw);
    size_t sm = (size_t)(ntw + 2 * 3 * NL * fft_ls(n)) * sizeof(Cx<T>);
    set_smem<T>((const void *)k_fft_x_inv<T>, sm);
    int blocks = ceil_div((int64_t)n * n, NL);
    k_fft_x_inv<T><<<blocks, threads, sm, c.stream>>>(op.gout.p, spec, plan, op.twiddle.p, NL);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  }
  }
  ProfScope ps2(c, PG_INTERP);
  const double h3 = c.h * c.h * c.h;
  const bool planar = sizeof(T) == 4 &&
                      (size_t)(make_plan(n, nullptr, true).ntw + 2 * (n / 2 + 1) * fft_ls(n)) * sizeof(Cx<T>) <=
                          (size_t)227 * 1024;
  if (planar && n % 4 == 0)
    k_interp_v4<<<ceil_div(c.Nt, 8), 256, 0, c.stream>>>(c.Nt, (const float4 *)c.wpos32.p,
                                                         (const float *)op.gout.p, y, n, P,
                                                         (float)h, (float)alpha, (float)(cn * h3),
                                                         tau_arg(c), make_fastdiv((P + 7) / 4),
                                                         make_fastdiv(P));
  else if (planar)
    k_interp<T, true><<<ceil_div(c.Nt, 8), 256, 0, c.stream>>>(c.Nt, posp<T>(c), op.gout.p, y, n, P,
                                                              h, alpha, (T)(cn * h3), tau_arg(c));
  else
    k_interp_rows<T><<<ceil_div(c.Nt, 8), 256, 0, c.stream>>>(c.Nt, posp<T>(c), op.gout.p, y, n,
                                                              P, h, alpha, (T)(cn * h3),
                                                              tau_arg(c), make_fastdiv(P));
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}


// Per-tile bead lists of the grid-centric spreading, from the FP32
// wave-space positions: count, scan, fill, then each list sorted (a fixed
// summation order).  Device-only (no host round trip).
void build_spread_tiles(Ctx &c) {
  const int n = c.n, nt = ceil_div(n, kTS);
  const int ntiles = nt * nt * nt;
  // a window of P consecutive grid indices meets at most ceil(P/8) + 1
  // aligned tiles, one more when it wraps past a partial last tile
  const int per_axis = ceil_div(c.P, kTS) + 2;
  const size_t cap = (size_t)c.Nt * per_axis * per_axis * per_axis;
  if (c.tile_n != nt || !c.tile_count.p) {
    c.tile_n = nt;
    c.tile_count.alloc(ntiles);
    c.tile_start.alloc(ntiles + 1);
    c.tile_cursor.alloc(ntiles);
  }
  if (c.tile_beads.n < cap) c.tile_beads.alloc(cap);
  const float h = (float)c.h;
  FSD_CUDA(cudaMemsetAsync(c.tile_count.p, 0, ntiles * sizeof(int), c.stream));
  k_tile_bin<false><<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, (const float4 *)c.wpos32.p, h, c.P, n,
                                                              nt, c.tile_count.p, nullptr, 0);
  FSD_LAUNCHED(c);
  k_exclusive_scan<<<1, 1024, 0, c.stream>>>(ntiles, c.tile_count.p, c.tile_start.p, c.tile_cursor.p);
  FSD_LAUNCHED(c);
  k_tile_bin<true><<<ceil_div(c.Nt, 128), 128, 0, c.stream>>>(c.Nt, (const float4 *)c.wpos32.p, h, c.P, n,
                                                             nt, c.tile_cursor.p, c.tile_beads.p,
                                                             (int64_t)c.tile_beads.n);
  FSD_LAUNCHED(c);
  k_sort_cells<<<ceil_div(ntiles, 4), 128, 0, c.stream>>>(ntiles, c.tile_start.p, c.tile_beads.p);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  c.tiles_valid = true;
}

const double *tilt_dev_ptr(const Ctx &c) {
  return (c.prm.flags & FSD_FLAG_LEES_EDWARDS) && c.tilt_dev.p ? c.tilt_dev.p : nullptr;
}

TauArg tau_arg(const Ctx &c) {
  TauArg t;
  t.tau = c.tilt / c.L;
  t.dev = tilt_dev_ptr(c);
  t.invL = 1.0 / c.L;
  return t;
}

// Sheared-lattice Green's function factors of the current offset (built on
// the stream; a captured step graph reads them through the same pointer).
__global__ void k_narrow(float *out, const double *__restrict__ in, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (float)in[i];
}

// The sheared Green's factors of the current box offset (once per offset).
// They are evaluated in FP64 in either precision, so the FP32 table is the
// FP64 one rounded (bit for bit what an FP32 evaluation stored before).
template <typename T>
static void refresh_le_table(Ctx &c, OpData<T> &op) {
  if (op.green_le_tilt == c.tilt && op.green_le.p) return;
  const int n = c.n, nh = n / 2 + 1;
  const size_t cnt = (size_t)3 * n * nh * n;
  if (op.green_le.n < cnt) op.green_le.alloc(cnt);
  if constexpr (sizeof(T) == 4) {
    OpData<double> &o64 = opd<double>(c);
    refresh_le_table<double>(c, o64);
    k_narrow<<<4 * c.num_sms, 256, 0, c.stream>>>(op.green_le.p, o64.green_le.p, (int64_t)cnt);
  } else {
    GreenLE le;
    le.on = 1;
    le.tau = c.tilt / c.L;
    le.ks2 = (2.0 * kPi / c.L) * (2.0 * kPi / c.L);
    le.xi = c.xi;
    le.alpha = c.alpha;
    le.a = c.a;
    le.eta = c.eta;
    le.inv_n3 = 1.0 / ((double)n * n * n);
    k_green_le_table<T><<<4 * c.num_sms, 256, 0, c.stream>>>(
        n, le, op.green_le.p, is_fft144(make_plan(n, nullptr, true)) ? 1 : 0);
  }
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  op.green_le_tilt = c.tilt;
}

void refresh_le_tables(Ctx &c) {
  if (!tilt_dev_ptr(c)) return;
  refresh_le_table<double>(c, opd<double>(c));
  if (c.prm.precision == FSD_MIXED) refresh_le_table<float>(c, opd<float>(c));
}

template <typename T>
void launch_wavespace(Ctx &c, const double *x, double *y) {
  OpData<T> &op = opd<T>(c);
  const int n = c.n, P = c.P;
  const T h = (T)c.h, alpha = (T)c.alpha;
  const double cn = std::pow(c.alpha / kPi, 1.5);
  const size_t gbytes = (size_t)6 * n * n * n * sizeof(T);
  {
  ProfScope ps(c, PG_SPREAD);
  if (sizeof(T) == 4 && c.spread_gather) {
    if (!c.tiles_valid) build_spread_tiles(c);
    const int nt = c.tile_n;
    k_spread_gather<<<nt * nt * nt, 64, 0, c.stream>>>(n, nt, P, (float)h, (float)alpha, (float)cn,
                                                       tau_arg(c), (const float4 *)c.wpos32.p,
                                                       x, c.tile_start.p, c.tile_beads.p,
                                                       (float *)op.grid.p);
  } else {
  FSD_CUDA(cudaMemsetAsync(op.grid.p, 0, gbytes, c.stream));
  if (sizeof(T) == 4 && n % 4 == 0)
    k_spread_v4<<<ceil_div(c.Nt, 8), 256, 0, c.stream>>>(c.Nt, (const float4 *)c.wpos32.p, x,
                                                         (float *)op.grid.p, n, P, (float)h,
                                                         (float)alpha, (float)cn,
                                                         tau_arg(c));
  else
    k_spread<T><<<ceil_div(c.Nt, 8), 256, 0, c.stream>>>(c.Nt, posp<T>(c), x, op.grid.p, n, P, h,
                                                        alpha, (T)cn, tau_arg(c));
  }
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
  }
  const FftPlan plan = make_plan(n, nullptr, true);
  Cx<T> *spec = (Cx<T> *)op.spec.p;
  {
  ProfScope ps(c, PG_FFT);
  const int nh = n / 2 + 1;
  const int threads = 256;
  const int ntw = plan.ntw;
  // FP32 planes that fit in shared memory with their ping-pong copy take the
  // fused x + y kernels (interpolation then reads planar fields); otherwise
  // separate x and y passes (interleaved fields).
  const size_t sm_xy = (size_t)(ntw + 2 * nh * fft_ls(n)) * sizeof(Cx<T>);
  const bool fused = sizeof(T) == 4 && sm_xy <= (size_t)227 * 1024;
  const int LTXy = fit_log2_lines<T>(sizeof(T) == 8 ? 3 : 4, 1, n, ntw);
  const int TXy = 1 << LTXy;
  const size_t smy = (size_t)(ntw + 2 * TXy * fft_ls(n)) * sizeof(Cx<T>);
  const int blocks_y = 6 * n * ceil_div(nh, TXy);
  if (fused) {
    if (is_fft144(plan)) {
      set_smem<T>((const void *)k_fft_xy_fwd<T, true>, sm_xy);
      k_fft_xy_fwd<T, true><<<6 * n, 1024, sm_xy, c.stream>>>(op.grid.p, spec, plan, op.twiddle.p);
    } else {
      set_smem<T>((const void *)k_fft_xy_fwd<T, false>, sm_xy);
      k_fft_xy_fwd<T, false><<<6 * n, 1024, sm_xy, c.stream>>>(op.grid.p, spec, plan, op.twiddle.p);
    }
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  } else {
    const int NL = 1 << fit_log2_lines<T>(2, 3, n, ntw);
    size_t sm = (size_t)(ntw + 2 * 3 * NL * fft_ls(n)) * sizeof(Cx<T>);
    set_smem<T>((const void *)k_fft_x_fwd<T>, sm);
    int blocks = ceil_div((int64_t)n * n, NL);
    k_fft_x_fwd<T><<<blocks, threads, sm, c.stream>>>(op.grid.p, spec, plan, op.twiddle.p, NL);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
    set_smem<T>((const void *)k_fft_y<T>, smy);
    k_fft_y<T><<<blocks_y, threads, smy, c.stream>>>(spec, plan, op.twiddle.p, LTXy, T(-1));
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  }
  {
    // four kx columns: 6 x 4 lines keep 4 CTAs per SM (FP32)
    const int LTX = fit_log2_lines<T>(2, 6, n, ntw);
    const int TX = 1 << LTX;
    size_t sm = (size_t)(ntw + 2 * 6 * TX * fft_ls(n)) * sizeof(Cx<T>);
    const bool s144 = is_fft144(plan);
    set_smem<T>(s144 ? (const void *)k_fft_z_green<T, true> : (const void *)k_fft_z_green<T, false>,
                sm);
    int blocks = n * ceil_div(nh, TX);
    GreenLE le;
    if (c.tilt != 0.0 || tilt_dev_ptr(c)) {
      le.on = 1;
      le.tau = c.tilt / c.L;
      le.dev = tilt_dev_ptr(c);
      le.invL = 1.0 / c.L;
      le.ks2 = (2.0 * kPi / c.L) * (2.0 * kPi / c.L);
      le.xi = c.xi;
      le.alpha = c.alpha;
      le.a = c.a;
      le.eta = c.eta;
      le.inv_n3 = 1.0 / ((double)n * n * n);
      refresh_le_table<T>(c, op);  // once per box offset
    }
    if (s144)
      k_fft_z_green<T, true><<<blocks, threads, sm, c.stream>>>(spec, plan, op.twiddle.p,
                                                                op.green.p, LTX, le, op.green_le.p);
    else
      k_fft_z_green<T, false><<<blocks, threads, sm, c.stream>>>(spec, plan, op.twiddle.p,
                                                                 op.green.p, LTX, le, op.green_le.p);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  }
  }
  wave_tail<T>(c, op, plan, spec, y);
}

template void launch_wavespace<float>(Ctx &, const double *, double *);
template void launch_wavespace<double>(Ctx &, const double *, double *);

template <typename T>
void launch_brownian_wave(Ctx &c, const double *field, uint64_t seed, uint64_t step, double *out) {
  OpData<T> &op = opd<T>(c);
  const int n = c.n, nh = n / 2 + 1;
  const FftPlan plan = make_plan(n, nullptr, true);
  Cx<T> *spec = (Cx<T> *)op.spec.p;
  {
    ProfScope ps(c, PG_FFT);
    const int LTX = fit_log2_lines<T>(2, 6, n, plan.ntw);
    const int TX = 1 << LTX;
    const size_t sm = (size_t)(plan.ntw + 2 * 6 * TX * fft_ls(n)) * sizeof(Cx<T>);
    set_smem<T>((const void *)k_brown_z<T>, sm);
    GreenLE le;
    if (c.tilt != 0.0) {
      le.tau = c.tilt / c.L;
      le.ks2 = (2.0 * kPi / c.L) * (2.0 * kPi / c.L);
      le.xi = c.xi;
      le.alpha = c.alpha;
      le.a = c.a;
      le.eta = c.eta;
      le.isv = 1.0 / std::sqrt(c.L * c.L * c.L);
    }
    k_brown_z<T><<<n * ceil_div(nh, TX), 256, sm, c.stream>>>(spec, plan, op.twiddle.p, op.btab.p,
                                                               field, seed, step, LTX, le);
    FSD_LAUNCHED(c);
    FSD_CUDA(cudaGetLastError());
  }
  FSD_CUDA(cudaMemsetAsync(out, 0, (size_t)c.nunk * sizeof(double), c.stream));
  wave_tail<T>(c, op, plan, spec, out);
}
template void launch_brownian_wave<float>(Ctx &, const double *, uint64_t, uint64_t, double *);
template void launch_brownian_wave<double>(Ctx &, const double *, uint64_t, uint64_t, double *);

}  // namespace fsd

// ==================================================================
// Wave-space mobility without any allocation.
//
// Some callers cannot allocate device memory at all: applications whose
// device memory is owned by an allocator or pool they do not control (a host
// framework that reserved it up front), plug-ins that must not change the
// process's device footprint after start-up, or real-time loops where an
// allocation (and the implicit synchronisation cudaMalloc / cudaFree can
// cause) is not allowed.  For them fsd_apply_wave_noalloc applies the FP32
// wave-space operator with every intermediate (density grids, half spectra,
// velocity grid, Green's table, twiddles, staged bead data) placed in one
// file-scope device array of fixed size.  The array exists on every device
// that loads this library and stays there until the process exits.  All
// calls share it: two calls whose GPU work overlaps race on it, so a caller
// must order them (one stream, or events).  Each call rewrites the parts it
// reads before reading them and zeroes the density grids and the staged
// output before accumulating into them.  Host code cannot use the array's
// name as a device address: each call looks the address up in the current
// device context (cudaGetSymbolAddress), so a device reset or another
// context on the same device never leaves a stale address behind.
namespace fsd {
namespace {

constexpr int kNaMaxGrid = 48;     // largest FFT grid per side
constexpr int kNaMaxBeads = 4096;  // largest bead count
constexpr size_t kNaBytes = 10u << 20;

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct NaLayout {
  size_t grid, spec, gout, green, tw, pos, x, y, end;
};

size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }

NaLayout na_layout(int n, int nb) {
  NaLayout l{};
  size_t o = 0;
  l.grid = o;
  o += na_round((size_t)6 * n * n * n * sizeof(float));
  l.spec = o;
  o += na_round((size_t)6 * n * n * (n / 2 + 1) * 2 * sizeof(float));
  l.gout = o;
  o += na_round((size_t)8 * n * n * n * sizeof(float));
  l.green = o;
  o += na_round((size_t)3 * (3 * (n / 2) * (n / 2) + 1) * sizeof(float));
  l.tw = o;
  o += na_round((size_t)2 * n * sizeof(float));
  l.pos = o;
  o += na_round((size_t)4 * nb * sizeof(float));
  l.x = o;
  o += na_round((size_t)LDB * nb * sizeof(double));
  l.y = o;
  o += na_round((size_t)LDB * nb * sizeof(double));
  l.end = o;
  return l;
}

// FFT plan built without any host container (same stages as make_plan).
FftPlan na_plan(int n) {
  FftPlan p{};
  p.n = n;
  p.fn = make_fastdiv(n);
  p.fnh = make_fastdiv(n / 2 + 1);
  int m = n, k = 0, Ns = 1, off = 0;
  int rad[kMaxStages];
  int nr = 0;
  while (m % 4 == 0) {
    rad[nr++] = 4;
    m /= 4;
  }
  for (int f : {2, 3, 5})
    while (m % f == 0) {
      rad[nr++] = f;
      m /= f;
    }
  for (int i = 0; i < nr; ++i) {
    FftStage &s = p.st[k++];
    s.R = rad[i];
    s.Ns = Ns;
    s.toff = off;
    s.nb = make_fastdiv(n / rad[i]);
    s.ns = make_fastdiv(Ns);
    off += (rad[i] - 1) * Ns;
    Ns *= rad[i];
  }
  p.nst = k;
  p.ntw = off;
  return p;
}

// Twiddles of the plan and the Green's table (same formulas as build_wave).
__global__ void k_na_tables(FftPlan plan, float *tw, float *green, int mmax, double L, double xi,
                            double alpha, double a, double eta) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  for (int t = t0; t < plan.ntw; t += stride) {
    int s = 0;
    while (s + 1 < plan.nst && plan.st[s + 1].toff <= t) ++s;
    const int u = t - plan.st[s].toff;
    const int r = 1 + u / plan.st[s].Ns, kk = u % plan.st[s].Ns;
    const double ang = -2.0 * kPi * r * kk / ((double)plan.st[s].Ns * plan.st[s].R);
    tw[2 * t] = (float)cos(ang);
    tw[2 * t + 1] = (float)sin(ang);
  }
  const double n3 = (double)plan.n * plan.n * plan.n;
  for (int m = t0; m <= mmax; m += stride) {
    if (m == 0) {
      green[0] = green[1] = green[2] = 0.f;
      continue;
    }
    const double k = 2.0 * kPi * sqrt((double)m) / L, k2 = k * k;
    const double e = -k2 / (4.0 * xi * xi) + k2 / (2.0 * alpha);
    const double A = (1.0 + k2 / (4.0 * xi * xi)) * exp(e) / (eta * k2) / n3;
    const double z = k * a;
    const double fm = z < 1e-3 ? 1.0 - z * z / 6.0 + z * z * z * z / 120.0 : sin(z) / z;
    const double fd = z < 1e-2 ? 1.0 - z * z / 10.0 + z * z * z * z / 280.0
                               : 3.0 * (sin(z) - z * cos(z)) / (z * z * z);
    green[3 * m] = (float)(A * fm * fm);
    green[3 * m + 1] = (float)(A * fm * fd);
    green[3 * m + 2] = (float)(A * fd * fd);
  }
}

// Bead positions (wrapped into [0, L)) and moments into the staged layout;
// the staged output rows are zeroed (interpolation accumulates into them).
__global__ void k_na_stage_in(int nb, const double *__restrict__ pos, const double *__restrict__ in,
                              double L, float4 *pos4, double *x, double *y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  float p[3];
  for (int d = 0; d < 3; ++d) {
    double v = pos[3 * (size_t)i + d];
    v -= L * floor(v / L);
    if (v >= L) v -= L;
    if (v < 0) v = 0;
    p[d] = (float)v;
  }
  pos4[i] = make_float4(p[0], p[1], p[2], 0.f);
  for (int k = 0; k < 11; ++k) x[(size_t)i * LDB + k] = in[(size_t)i * 11 + k];
  x[(size_t)i * LDB + 11] = 0.0;
  for (int k = 0; k < LDB; ++k) y[(size_t)i * LDB + k] = 0.0;
}

__global__ void k_na_stage_out(int nb, const double *__restrict__ y, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  for (int k = 0; k < 11; ++k) out[(size_t)i * 11 + k] = y[(size_t)i * LDB + k];
}

}  // namespace
}  // namespace fsd

extern "C" fsd_status fsd_apply_wave_noalloc(int64_t n_beads, const double *bead_pos,
                                             const double *in, double *out, double box,
                                             double xi, int grid, int P, double m_shape,
                                             double a, double eta, void *cuda_stream) {
  using namespace fsd;
  // The error and pointer queries and the symbol lookup below queue no GPU
  // work, but a stream capture begun in global or thread-local mode forbids
  // this thread runtime calls it counts as potentially unsafe.  They run with
  // the thread's capture mode relaxed; the caller's mode is put back on
  // every return.
  struct RelaxCapture {
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    RelaxCapture() { cudaThreadExchangeStreamCaptureMode(&mode); }
    ~RelaxCapture() { cudaThreadExchangeStreamCaptureMode(&mode); }
  } relax_capture;
  // an error left pending by the caller's earlier work is not this call's:
  // leave it in place for the caller and do nothing
  if (cudaPeekAtLastError() != cudaSuccess) return FSD_ECUDA;
  if (n_beads < 1 || n_beads > kNaMaxBeads) return FSD_EINVAL;
  if (!bead_pos || !in || !out || !(box > 0) || !(xi > 0) || !(a > 0) || !(eta > 0)) return FSD_EINVAL;
  if (!fft_size_ok(grid) || grid > kNaMaxGrid) return FSD_EINVAL;
  if (P % 2 || P < 4 || P > 24 || P > grid) return FSD_EINVAL;
  for (const void *p : {(const void *)bead_pos, (const void *)in, (const void *)out}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return FSD_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return FSD_EINVAL;
  }
  const int n = grid;
  const int nb = (int)n_beads;
  const NaLayout lay = na_layout(n, nb);
  if (lay.end > kNaBytes) return FSD_EINVAL;
  // the array's device address in the current context (the host-side name
  // of a __device__ array is not a device pointer)
  unsigned char *base = nullptr;
  {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FSD_ECUDA;
    }
    base = (unsigned char *)p;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float *gridp = (float *)(base + lay.grid);
  Cx<float> *spec = (Cx<float> *)(base + lay.spec);
  float *gout = (float *)(base + lay.gout);
  float *green = (float *)(base + lay.green);
  float *tw = (float *)(base + lay.tw);
  float4 *pos4 = (float4 *)(base + lay.pos);
  double *x = (double *)(base + lay.x);
  double *y = (double *)(base + lay.y);
  const double L = box, h = L / n;
  const double ms = m_shape > 0 ? m_shape : 0.976 * std::sqrt(kPi * P);
  const double alpha = 2.0 * ms * ms / ((P * h) * (P * h));
  const FftPlan plan = na_plan(n);
  const int hm = n / 2, mmax = 3 * hm * hm;
  const int nh = n / 2 + 1;
  const int threads = 256;
  k_na_tables<<<8, 256, 0, st>>>(plan, tw, green, mmax, L, xi, alpha, a, eta);
  k_na_stage_in<<<(nb + 127) / 128, 128, 0, st>>>(nb, bead_pos, in, L, pos4, x, y);
  if (cudaMemsetAsync(gridp, 0, (size_t)6 * n * n * n * sizeof(float), st) != cudaSuccess)
    return FSD_ECUDA;
  const double cn = std::pow(alpha / kPi, 1.5);
  k_spread<float><<<(nb + 7) / 8, 256, 0, st>>>(nb, pos4, x, gridp, n, P, (float)h, (float)alpha,
                                               (float)cn, TauArg());
  const int ntw = plan.ntw;
  k_fft_x_fwd<float><<<(n * n + 3) / 4, threads, (ntw + 2 * 3 * 4 * fft_ls(n)) * sizeof(Cx<float>),
                       st>>>(gridp, spec, plan, tw, 4);
  const int blocks_y = 6 * n * ((nh + 15) / 16);
  const size_t smy = (size_t)(ntw + 2 * 16 * fft_ls(n)) * sizeof(Cx<float>);
  k_fft_y<float><<<blocks_y, threads, smy, st>>>(spec, plan, tw, 4, -1.f);
  k_fft_z_green<float, false><<<n * ((nh + 3) / 4), threads,
                         (ntw + 2 * 6 * 4 * fft_ls(n)) * sizeof(Cx<float>), st>>>(spec, plan, tw,
                                                                                green, 2, GreenLE(),
                                                                                nullptr);
  k_fft_y<float><<<blocks_y, threads, smy, st>>>(spec, plan, tw, 4, 1.f);
  k_fft_x_inv<float><<<(n * n + 3) / 4, threads, (ntw + 2 * 3 * 4 * fft_ls(n)) * sizeof(Cx<float>),
                       st>>>(gout, spec, plan, tw, 4);
  k_interp<float, false><<<(nb + 7) / 8, 256, 0, st>>>(nb, pos4, gout, y, n, P, (float)h, (float)alpha,
                                               (float)(cn * h * h * h), TauArg());
  k_na_stage_out<<<(nb + 127) / 128, 128, 0, st>>>(nb, y, out);
  if (cudaGetLastError() != cudaSuccess) return FSD_ECUDA;
  return FSD_OK;
}
