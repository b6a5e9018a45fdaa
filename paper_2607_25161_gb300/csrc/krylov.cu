// FP64 Krylov primitives for the GMRES of Algorithm 1 step 4: fused
// multi-vector dot products (classical Gram-Schmidt, applied twice), fused
// multi-vector updates, scaling.  The basis is stored as k vectors of
// length n with leading dimension ld.  Reductions are two-stage and
// deterministic (fixed block partials, fixed reduction order).
#include "fsd_internal.cuh"

#include <algorithm>

namespace fsd {

constexpr int kDotBlocks = 4 * 152;  // partial sums per dot (multiple of the SM count)
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

__global__ void k_dot_final(const double *__restrict__ partial, int nb, int k, double *out) {
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
  const int64_t n = c.nunk;
  for (int k0 = 0; k0 < k; k0 += kDotChunk) {
    int kc = std::min(kDotChunk, k - k0);
    k_dot_partial<<<kDotBlocks, 256, 0, c.stream>>>(V, ld, k0, kc, w, n, c.partial.p);
  }
  k_dot_final<<<k, 256, 0, c.stream>>>(c.partial.p, kDotBlocks, k, out_dev);
  FSD_CUDA(cudaGetLastError());
}

// w[i] += sign * sum_j coef[j] V_j[i]
__global__ void k_axpy_multi(double *w, const double *__restrict__ V, int64_t ld, int k,
                             const double *__restrict__ coef, double sign, int64_t n) {
  __shared__ double cs[128];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = sign * coef[j];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double s = w[i];
    for (int j = 0; j < k; ++j) s += cs[j] * V[(int64_t)j * ld + i];
    w[i] = s;
  }
}

void axpy_multi(Ctx &c, double *w, const double *V, int64_t ld, int k, const double *coef_dev,
                double sign) {
  if (k <= 0) return;
  const int64_t n = c.nunk;
  int blocks = std::min<int64_t>(ceil_div(n, 256), 8 * 152);
  k_axpy_multi<<<blocks, 256, 0, c.stream>>>(w, V, ld, k, coef_dev, sign, n);
  FSD_CUDA(cudaGetLastError());
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
  int blocks = std::min<int64_t>(ceil_div(c.nunk, 256), 8 * 152);
  k_scale<<<blocks, 256, 0, c.stream>>>(y, x, s, c.nunk);
  FSD_CUDA(cudaGetLastError());
}

void vec_axpby(Ctx &c, double *y, double a, const double *x, double b, int64_t n) {
  int blocks = std::min<int64_t>(ceil_div(n, 256), 8 * 152);
  k_axpby<<<blocks, 256, 0, c.stream>>>(y, a, x, b, n);
  FSD_CUDA(cudaGetLastError());
}

void norm2_dev(Ctx &c, const double *x, double *out_dev) {
  dot_multi(c, x, 0, 1, x, out_dev);
}

}  // namespace fsd
