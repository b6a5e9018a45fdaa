// Krylov primitives for the GMRES of Algorithm 1 step 4: fused multi-vector
// dot products (classical Gram-Schmidt, applied twice), fused multi-vector
// updates, scaling.  The basis is stored as k vectors of length n with
// leading dimension ld, in FP64 or (inner solve of the mixed path) FP32.
// Reductions are two-stage and deterministic (fixed block partials, fixed
// reduction order).
#include "fsd_internal.cuh"

#include <algorithm>

namespace fsd {

constexpr int kDotBlocks = kDotPartials;
constexpr int kDotChunk = 16;        // basis vectors per pass

// partial[j * nb + blk] = sum over this block's grid-stride slice of V_j . w
__global__ void __launch_bounds__(256) k_dot_partial(const double *__restrict__ V, int64_t ld,
                                                     int k0, int kc, const double *__restrict__ w,
                                                     int64_t n, double *partial) {
  double acc[kDotChunk];
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) acc[j] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < kDotChunk; ++j)
      if (j < kc) acc[j] += V[(int64_t)(k0 + j) * ld + i] * wi;
  }
  __shared__ double red[kDotChunk][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[j][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kc) {
    double s = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[threadIdx.x][wv];
    partial[(int64_t)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

// k_dev (when non-null) gives the count on the device: k = *k_dev + k_add.
__global__ void k_dot_final(const double *__restrict__ partial, int nb, int k, const int *k_dev,
                            int k_add, double *out) {
  if (k_dev) k = *k_dev + k_add;
  const int j = blockIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)j * nb + b];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

void dot_multi(Ctx &c, const double *V, int64_t ld, int k, const double *w, double *out_dev) {
  ProfScope ps(c, PG_KRYLOV);
  const int64_t n = c.nunk;
  for (int k0 = 0; k0 < k; k0 += kDotChunk) {
    int kc = std::min(kDotChunk, k - k0);
    k_dot_partial<<<kDotBlocks, 256, 0, c.stream>>>(V, ld, k0, kc, w, n, c.partial.p);
    FSD_LAUNCHED(c);
  }
  k_dot_final<<<k, 256, 0, c.stream>>>(c.partial.p, kDotBlocks, k, nullptr, 0, out_dev);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// Fused classical Gram-Schmidt passes over the basis V (k vectors):
//   MODE 0:  partial dots  V_j . w
//   MODE 1:  w -= sum_j coef_j V_j, then partial dots V_j . w
//   MODE 2:  w -= sum_j coef_j V_j, then partial ||w||^2
// Each thread owns up to kE elements spaced by the grid's thread count
// (coalesced); basis vectors are taken four at a time so that 4 kE loads are
// in flight per thread; block partials go to partial[j * blocks + block] and
// the last block to finish reduces them into out (fixed reduction order
// throughout).  The grid is a whole number of waves over the SMs (two blocks
// per SM on the benchmark's 417 792 unknowns), so that every SM carries the
// same share of the FP64 multiply-adds that bound these passes; six elements
// per thread keep the warp reductions of the dot products (1.5 FP64 adds per
// basis vector and warp) small beside the 6 multiply-adds they sum.
//
// The basis element type B is double (the FP64 solve and the Lanczos square
// roots: every product and sum in FP64) or float (the inner GMRES of the
// mixed solve, whose operator is FP32 anyway).  With a float basis the
// products and the sums within a warp are FP32 (exact products of two FP32
// numbers would need FP64, whose rate is 1/74 of FP32 on this part), the
// update sum_j coef_j V_j is formed in FP32 and subtracted from the FP64 w,
// and the cross-warp sums stay FP64.
constexpr int kE = 6;

// Warp sums of four values with six shuffles: after the exchange across
// lane bit 4 each lane keeps two of the four partial sums, after bit 3 one;
// bits 2..0 finish it.  Lane 8 q holds the full sum of value q.
template <typename R>
__device__ __forceinline__ R warp_sum4(const R a[4], int lane) {
  const bool h4 = lane & 16;
  const R s0 = h4 ? a[0] : a[2], s1 = h4 ? a[1] : a[3];
  R b0 = (h4 ? a[2] : a[0]) + __shfl_xor_sync(0xffffffffu, s0, 16);
  R b1 = (h4 ? a[3] : a[1]) + __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool h3 = lane & 8;
  R c = (h3 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h3 ? b0 : b1, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

template <int MODE, typename B>
__global__ void __launch_bounds__(256) k_cgs(const B *__restrict__ V, int64_t ld, int k,
                                             const int *k_dev, int k_add, double *w,
                                             const double *__restrict__ coef, int64_t n,
                                             double *partial, double *out, unsigned *ticket) {
  constexpr bool f64 = sizeof(B) == 8;
  if (k_dev) k = *k_dev + k_add;
  __shared__ B cs[kMaxBasis];
  __shared__ double wred[kMaxBasis][8];  // per basis vector, per warp
  __shared__ int last;
  // FP64: the update is a chain of fused multiply-adds with -coef (no
  // separate products and sums on the FP64 pipe, which bounds these passes)
  if (MODE > 0)
    for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = f64 ? (B)(-coef[j]) : (B)coef[j];
  __syncthreads();
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // a thread whose kE elements are all in range loads without predicates
  const bool full = t0 + (kE - 1) * T < n;
  double wv[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const int64_t i = t0 + e * T;
    wv[e] = i < n ? w[i] : 0.0;
  }
  auto ld_col = [&](const B *vj, B *out_) {
    if (full) {
#pragma unroll
      for (int e = 0; e < kE; ++e) out_[e] = vj[e * T];
    } else {
#pragma unroll
      for (int e = 0; e < kE; ++e) out_[e] = t0 + e * T < n ? vj[e * T] : (B)0;
    }
  };
  if (MODE > 0) {
    const B *vj = V + t0;
    B us[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) us[e] = (B)0;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      B v[4][kE];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_col(vj + q * ld, v[q]);
      vj += 4 * ld;
#pragma unroll
      for (int e = 0; e < kE; ++e) {
        if constexpr (f64) {
          wv[e] = fma(cs[j], v[0][e], wv[e]);
          wv[e] = fma(cs[j + 1], v[1][e], wv[e]);
          wv[e] = fma(cs[j + 2], v[2][e], wv[e]);
          wv[e] = fma(cs[j + 3], v[3][e], wv[e]);
        } else {
          us[e] += cs[j] * v[0][e] + cs[j + 1] * v[1][e] + cs[j + 2] * v[2][e] + cs[j + 3] * v[3][e];
        }
      }
    }
    for (; j < k; ++j, vj += ld) {
      B v[kE];
      ld_col(vj, v);
#pragma unroll
      for (int e = 0; e < kE; ++e) {
        if constexpr (f64)
          wv[e] = fma(cs[j], v[e], wv[e]);
        else
          us[e] += cs[j] * v[e];
      }
    }
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      if constexpr (!f64) wv[e] -= (double)us[e];
      if (t0 + e * T < n) w[t0 + e * T] = wv[e];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (MODE == 2) {
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < kE; ++e) acc = fma(wv[e], wv[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wred[0][warp] = acc;
  } else {
    B wb[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) wb[e] = (B)wv[e];
    const B *vj = V + t0;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      B v[4][kE], acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_col(vj + q * ld, v[q]);
      vj += 4 * ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = (B)0;
#pragma unroll
        for (int e = 0; e < kE; ++e) acc[q] = fma(v[q][e], wb[e], acc[q]);
      }
      const B r = warp_sum4<B>(acc, lane);
      if ((lane & 7) == 0) wred[j + (lane >> 3)][warp] = (double)r;
    }
    for (; j < k; ++j, vj += ld) {
      B v[kE];
      ld_col(vj, v);
      B acc = (B)0;
#pragma unroll
      for (int e = 0; e < kE; ++e) acc += v[e] * wb[e];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) wred[j][warp] = (double)acc;
    }
  }
  // block partials (warps summed in a fixed order), then the last block to
  // finish sums the block partials in a fixed order: no second launch, and
  // the result does not depend on which block finishes last
  const int kr = MODE == 2 ? 1 : k;
  __syncthreads();
  if (threadIdx.x < kr) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += wred[threadIdx.x][q];
    partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  const int nb = (int)gridDim.x;
  for (int jj = warp; jj < kr; jj += 8) {
    // two independent sums per lane (a dependent FP64 add is long on this
    // part), in an order fixed by the grid size
    const double *pj = partial + (int64_t)jj * nb;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < nb; b += 64) {
      s0 += __ldcg(pj + b);
      s1 += __ldcg(pj + b + 32);
    }
    if (b < nb) s0 += __ldcg(pj + b);
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[jj] = s;
  }
  if (threadIdx.x == 0) atomicExch(ticket, 0u);
}

// enough blocks for kE elements per thread, rounded up to whole waves of
// the SMs once there are more blocks than SMs
static int cgs_blocks(int64_t n, int nsm) {
  const int64_t b = std::max<int64_t>(1, ceil_div(n, 256LL * kE));
  if (nsm < 1 || b <= nsm) return (int)b;
  return (int)(ceil_div(b, (int64_t)nsm) * nsm);
}

// out[j] = V_j . w (j < k); mode 1 / 2 first apply w -= V coef (mode 2:
// out[0] = ||w||^2).  With k_dev non-null the basis size is read on the
// device (k = *k_dev + k_add <= kmax), so the pass can sit in a captured loop
// whose trip count the host never sees.  One launch per pass.
template <typename B>
static void cgs_launch(Ctx &c, int mode, const B *V, int64_t ld, int k, const int *k_dev,
                       int k_add, int kmax, double *w, const double *coef_dev, double *out_dev) {
  ProfScope ps(c, PG_KRYLOV);
  if (std::max(k, kmax) > kMaxBasis) throw Invalid{"Krylov basis longer than 64 vectors"};
  const int64_t n = c.nunk;
  const int blocks = cgs_blocks(n, c.num_sms);
  unsigned *tk = c.cgs_ticket.p;
  double *pp = c.partial.p;
  if (mode == 0)
    k_cgs<0, B><<<blocks, 256, 0, c.stream>>>(V, ld, k, k_dev, k_add, w, coef_dev, n, pp, out_dev, tk);
  else if (mode == 1)
    k_cgs<1, B><<<blocks, 256, 0, c.stream>>>(V, ld, k, k_dev, k_add, w, coef_dev, n, pp, out_dev, tk);
  else
    k_cgs<2, B><<<blocks, 256, 0, c.stream>>>(V, ld, k, k_dev, k_add, w, coef_dev, n, pp, out_dev, tk);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void cgs_pass(Ctx &c, int mode, const double *V, int64_t ld, int k, double *w,
              const double *coef_dev, double *out_dev) {
  cgs_launch(c, mode, V, ld, k, nullptr, 0, k, w, coef_dev, out_dev);
}

void cgs_pass(Ctx &c, int mode, const float *V, int64_t ld, int k, double *w,
              const double *coef_dev, double *out_dev) {
  cgs_launch(c, mode, V, ld, k, nullptr, 0, k, w, coef_dev, out_dev);
}

void cgs_pass_dev(Ctx &c, int mode, const double *V, int64_t ld, const int *k_dev, int k_add,
                  int kmax, double *w, const double *coef_dev, double *out_dev) {
  cgs_launch(c, mode, V, ld, 0, k_dev, k_add, kmax, w, coef_dev, out_dev);
}

void cgs_pass_dev(Ctx &c, int mode, const float *V, int64_t ld, const int *k_dev, int k_add,
                  int kmax, double *w, const double *coef_dev, double *out_dev) {
  cgs_launch(c, mode, V, ld, 0, k_dev, k_add, kmax, w, coef_dev, out_dev);
}

int64_t cgs_partial_size(int64_t nunk, int kmax, int nsm) {
  return (int64_t)cgs_blocks(nunk, nsm) * (kmax + 1);
}

// w[i] += sign * sum_j coef[j] V_j[i]; with a float basis the sum over j is
// FP32 and is added to the FP64 w.
template <typename B>
__global__ void k_axpy_multi(double *w, const B *__restrict__ V, int64_t ld, int k,
                             const int *k_dev, const double *__restrict__ coef, double sign,
                             int64_t n) {
  if (k_dev) k = *k_dev;
  __shared__ B cs[128];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = (B)(sign * coef[j]);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if constexpr (sizeof(B) == 8) {
      double s = w[i];
      for (int j = 0; j < k; ++j) s += cs[j] * V[(int64_t)j * ld + i];
      w[i] = s;
    } else {
      B s = (B)0;
      for (int j = 0; j < k; ++j) s += cs[j] * V[(int64_t)j * ld + i];
      w[i] += (double)s;
    }
  }
}

template <typename B>
static void axpy_multi_launch(Ctx &c, double *w, const B *V, int64_t ld, int k, const int *k_dev,
                              const double *coef_dev, double sign) {
  ProfScope ps(c, PG_KRYLOV);
  const int64_t n = c.nunk;
  int blocks = std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)c.num_sms);
  k_axpy_multi<B><<<blocks, 256, 0, c.stream>>>(w, V, ld, k, k_dev, coef_dev, sign, n);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void axpy_multi(Ctx &c, double *w, const double *V, int64_t ld, int k, const double *coef_dev,
                double sign) {
  if (k > 0) axpy_multi_launch(c, w, V, ld, k, nullptr, coef_dev, sign);
}

void axpy_multi(Ctx &c, double *w, const float *V, int64_t ld, int k, const double *coef_dev,
                double sign) {
  if (k > 0) axpy_multi_launch(c, w, V, ld, k, nullptr, coef_dev, sign);
}

// w += sign * sum_{j < *k_dev} coef[j] V_j (count read on the device)
void axpy_multi_dev(Ctx &c, double *w, const double *V, int64_t ld, const int *k_dev,
                    const double *coef_dev, double sign) {
  axpy_multi_launch(c, w, V, ld, 0, k_dev, coef_dev, sign);
}

void axpy_multi_dev(Ctx &c, double *w, const float *V, int64_t ld, const int *k_dev,
                    const double *coef_dev, double sign) {
  axpy_multi_launch(c, w, V, ld, 0, k_dev, coef_dev, sign);
}

__global__ void k_scale(double *y, const double *__restrict__ x, double s, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = x[i] * s;
}

__global__ void k_axpby(double *y, double a, const double *__restrict__ x, double b, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = a * x[i] + b * y[i];
}

void vec_scale_host(Ctx &c, double *y, const double *x, double s) {
  ProfScope ps(c, PG_KRYLOV);
  int blocks = std::min<int64_t>(ceil_div(c.nunk, 256), 8 * (int64_t)c.num_sms);
  k_scale<<<blocks, 256, 0, c.stream>>>(y, x, s, c.nunk);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// y = (float)(s x)
__global__ void k_scale_f32(float *y, const double *__restrict__ x, double s, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = (float)(x[i] * s);
}

void vec_scale_host(Ctx &c, float *y, const double *x, double s) {
  ProfScope ps(c, PG_KRYLOV);
  int blocks = std::min<int64_t>(ceil_div(c.nunk, 256), 8 * (int64_t)c.num_sms);
  k_scale_f32<<<blocks, 256, 0, c.stream>>>(y, x, s, c.nunk);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

// y = (double) x
__global__ void k_widen(double *y, const float *__restrict__ x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = (double)x[i];
}

// z32 = (float) z and z = (double) z32: the FP32 copy and the operator input
// hold the same values
__global__ void k_round_f32(float *z32, double *z, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = (float)z[i];
    z32[i] = v;
    z[i] = (double)v;
  }
}

void vec_widen(Ctx &c, double *y, const float *x) {
  ProfScope ps(c, PG_KRYLOV);
  int blocks = std::min<int64_t>(ceil_div(c.nunk, 256), 8 * (int64_t)c.num_sms);
  k_widen<<<blocks, 256, 0, c.stream>>>(y, x, c.nunk);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void vec_round_f32(Ctx &c, float *z32, double *z) {
  ProfScope ps(c, PG_KRYLOV);
  int blocks = std::min<int64_t>(ceil_div(c.nunk, 256), 8 * (int64_t)c.num_sms);
  k_round_f32<<<blocks, 256, 0, c.stream>>>(z32, z, c.nunk);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void vec_axpby(Ctx &c, double *y, double a, const double *x, double b, int64_t n) {
  ProfScope ps(c, PG_KRYLOV);
  int blocks = std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)c.num_sms);
  k_axpby<<<blocks, 256, 0, c.stream>>>(y, a, x, b, n);
  FSD_LAUNCHED(c);
  FSD_CUDA(cudaGetLastError());
}

void norm2_dev(Ctx &c, const double *x, double *out_dev) {
  dot_multi(c, x, 0, 1, x, out_dev);
}

}  // namespace fsd
