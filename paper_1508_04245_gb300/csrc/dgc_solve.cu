// Linear combinations of vectors (the extrapolated convection velocity of
// Sec. 3.2.2 as a combination of earlier exactly divergence-free velocities),
// and the kernels of the pseudo-time (Richardson) solve of the implicit convection
// problem v + tau (M^V)^{-1} C^V v = g of the modified fractional-step-theta
// scheme (Sec. 3.3.2):
//
//   rho_i = g - v_i - tau r_i,   r_i = (M^V)^{-1} C^V v_i,   v_{i+1} = v_i + ds rho_i,
//
// stopped at the first i with ||rho_i|| <= reduction ||rho_0|| or i = max_iter,
// ||x||^2 = sum_T |det J_T| sum_{c,j} x^2 (the L2 norm of the DG function in the
// orthonormal basis).  The loop runs on the device: a graph WHILE node repeats
// [update, operator, residual + norm partials, control] while the control
// kernel sets its condition; the host never waits on a norm.
//
// The norm is reduced deterministically: each residual block writes one
// partial sum (fixed grid, fixed in-block order) and the control kernel adds
// the partials in a fixed order, so every run takes the same decisions.
#include <cuda_runtime.h>

#include <cmath>

#include "dgc_kernels.h"

namespace dgc {
namespace {

constexpr int kBlock = 256;

// sum over the block of one double per thread, fixed order (warp tree, then warps)
__device__ double block_sum(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;   // valid in thread 0
}

// rho = g - v - tau r over all n = E * DN values, and per block sum |det J| rho^2
__global__ void __launch_bounds__(kBlock) rich_resid_kernel(const double* __restrict__ g,
                                                             const double* __restrict__ v,
                                                             const double* __restrict__ r, double tau,
                                                             double* __restrict__ rho,
                                                             const double* __restrict__ detJ, int DN, long n,
                                                             double* __restrict__ partials) {
  __shared__ double sh[kBlock / 32];
  double acc = 0.0;
  for (long j = (long)blockIdx.x * kBlock + threadIdx.x; j < n; j += (long)gridDim.x * kBlock) {
    const double x = g[j] - v[j] - tau * r[j];
    rho[j] = x;
    acc += fabs(detJ[j / DN]) * x * x;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// v += ds rho
__global__ void __launch_bounds__(kBlock) rich_update_kernel(double* __restrict__ v,
                                                              const double* __restrict__ rho, double ds, long n) {
  for (long j = (long)blockIdx.x * kBlock + threadIdx.x; j < n; j += (long)gridDim.x * kBlock) v[j] += ds * rho[j];
}

// state[0] = ||rho_0||, state[1] = i (as a double); first != 0 starts the count
__global__ void __launch_bounds__(kBlock) rich_control_kernel(const double* __restrict__ partials, int np,
                                                               double* state, int* iters, double* res,
                                                               double reduction, int max_iter, int first,
                                                               cudaGraphConditionalHandle h, int* status) {
  __shared__ double sh[kBlock / 32];
  double acc = 0.0;
  for (int j = threadIdx.x; j < np; j += kBlock) acc += partials[j];
  const double s = block_sum(acc, sh);
  if (threadIdx.x != 0) return;
  const double norm = sqrt(s);
  if (first) {
    state[0] = norm;
    state[1] = 0.0;
  }
  const int i = (int)state[1];
  if (res) res[i] = norm;
  const bool finite = isfinite(norm);
  if (!finite) atomicOr(status, 4);
  const bool stop = !finite || norm <= reduction * state[0] || i >= max_iter;
  if (!stop) state[1] = (double)(i + 1);   // the body's update makes v = v_{i+1}
  *iters = stop ? i : i + 1;
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// out = sum_t c_t x_t (up to kMaxTerms vectors; out may be one of the x_t)
__global__ void __launch_bounds__(kBlock) combine_kernel(double* out, CombineArgs a, long n) {
  for (long j = (long)blockIdx.x * kBlock + threadIdx.x; j < n; j += (long)gridDim.x * kBlock) {
    double s = 0.0;
    for (int t = 0; t < a.nterms; ++t) s += a.c[t] * a.x[t][j];
    out[j] = s;
  }
}

__global__ void __launch_bounds__(kBlock) to_float_kernel(const double* __restrict__ x, float* __restrict__ y, long n) {
  for (long j = (long)blockIdx.x * kBlock + threadIdx.x; j < n; j += (long)gridDim.x * kBlock) y[j] = (float)x[j];
}

}  // namespace

cudaError_t launch_to_float(const double* x, float* y, long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long b = (n + kBlock - 1) / kBlock;
  to_float_kernel<<<(unsigned)(b > 4096 ? 4096 : b), kBlock, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_combine(double* out, const CombineArgs& a, long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long b = (n + kBlock - 1) / kBlock;
  combine_kernel<<<(unsigned)(b > 4096 ? 4096 : b), kBlock, 0, s>>>(out, a, n);
  return cudaGetLastError();
}

int rich_blocks(long n) {
  long b = (n + kBlock * 4 - 1) / (kBlock * 4);
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_rich_resid(const double* g, const double* v, const double* r, double tau, double* rho,
                              const double* detJ, int DN, long n, double* partials, int nblocks, cudaStream_t s) {
  rich_resid_kernel<<<nblocks, kBlock, 0, s>>>(g, v, r, tau, rho, detJ, DN, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_rich_update(double* v, const double* rho, double ds, long n, cudaStream_t s) {
  long b = (n + kBlock - 1) / kBlock;
  rich_update_kernel<<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), kBlock, 0, s>>>(v, rho, ds, n);
  return cudaGetLastError();
}

cudaError_t launch_rich_control(const double* partials, int np, double* state, int* iters, double* res,
                                double reduction, int max_iter, bool first, cudaGraphConditionalHandle h,
                                int* status, cudaStream_t s) {
  rich_control_kernel<<<1, kBlock, 0, s>>>(partials, np, state, iters, res, reduction, max_iter, first ? 1 : 0, h,
                                           status);
  return cudaGetLastError();
}

}  // namespace dgc
