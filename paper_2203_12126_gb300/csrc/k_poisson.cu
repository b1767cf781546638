// Kernels of the Poisson limit (Sec. 5.4, App. C, App. D), float64.
//
// Completed IBDL (App. C) works on z = (Q, u_bar) of length M + 1:
//   rows 0..M-1: Q/2 - S* Delta_0^{-1} (S~ + eta S) Q + u_bar
//   row M:       eta sum_i w_i Q_i
// The field part is the ordinary spread / solve / interpolation with the
// plain spread added (coefficient eta); the kernels here add the bordered
// column (u_bar) and row (eta w^T Q).  The weight sum is taken before the
// interpolation writes y, so q and y may alias.
//
// Reductions are two-level with a fixed launch shape (kRedBlocks blocks,
// fixed per-block order), so results are deterministic.
#include "ibdl_internal.cuh"

namespace ibdl {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_total(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // thread 0
}

// part[b] = sum over block b's stride of a[i] * (b ? b[i] : 1);
// part[kRedBlocks] = *keep when keep is given (block 0).
__global__ void __launch_bounds__(kT) k_partial_dot(int64_t n, const double* __restrict__ a,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ part,
                                                    const double* keep) {
  __shared__ double sh[kT / 32];
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    s += b ? a[i] * b[i] : a[i];
  s = block_total(s, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    if (keep && blockIdx.x == 0) part[kRedBlocks] = *keep;
  }
}

// y[i] += part[kRedBlocks] (i < m); block 0: y[m] = scale * sum part[0..kRedBlocks).
__global__ void __launch_bounds__(kT) k_completed_tail(int m, double* __restrict__ y,
                                                       const double* __restrict__ part,
                                                       double scale) {
  __shared__ double sh[kT / 32];
  const double ubar = part[kRedBlocks];
  for (int i = blockIdx.x * kT + threadIdx.x; i < m; i += gridDim.x * kT) y[i] += ubar;
  if (blockIdx.x == 0) {
    double s = 0;
    for (int t = threadIdx.x; t < kRedBlocks; t += kT) s += part[t];
    s = block_total(s, sh);
    if (threadIdx.x == 0) y[m] = scale * s;
  }
}

// out[0] = scale * sum part[0..kRedBlocks)
__global__ void __launch_bounds__(kT) k_finish_sum(const double* __restrict__ part, double scale,
                                                   double* out) {
  __shared__ double sh[kT / 32];
  double s = 0;
  for (int t = threadIdx.x; t < kRedBlocks; t += kT) s += part[t];
  s = block_total(s, sh);
  if (threadIdx.x == 0) out[0] = scale * s;
}

__global__ void __launch_bounds__(kT) k_add_scalar(int64_t n, double* __restrict__ u,
                                                   const double* s) {
  const double v = *s;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    u[i] += v;
}

__global__ void __launch_bounds__(kT) k_fill(int64_t n, double* __restrict__ x, double v) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    x[i] = v;
}

// App. D: chi_h = u - u(corner node 0); chi = chi_h > 1/2.
__global__ void __launch_bounds__(kT) k_indicator(int64_t n, const double* __restrict__ u,
                                                  double* __restrict__ chi_h,
                                                  unsigned char* __restrict__ chi) {
  const double c = u[0];
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kT) {
    const double v = u[i] - c;
    if (chi_h) chi_h[i] = v;
    if (chi) chi[i] = v > 0.5 ? 1 : 0;
  }
}

int grid_blocks(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}

}  // namespace

cudaError_t launch_completed_head(int m, const double* w, const double* q, double* part,
                                  cudaStream_t st) {
  prof_begin(st);
  k_partial_dot<<<kRedBlocks, kT, 0, st>>>(m, w, q, part, q + m);
  count_launch("completed_head", st);
  return check_launch();
}

cudaError_t launch_completed_tail(int m, double* y, const double* part, double scale,
                                  cudaStream_t st) {
  prof_begin(st);
  k_completed_tail<<<grid_blocks(m), kT, 0, st>>>(m, y, part, scale);
  count_launch("completed_tail", st);
  return check_launch();
}

cudaError_t launch_scaled_sum(int64_t n, const double* a, double scale, double* part,
                              double* out, cudaStream_t st) {
  prof_begin(st);
  k_partial_dot<<<kRedBlocks, kT, 0, st>>>(n, a, nullptr, part, nullptr);
  count_launch("grid_sum", st);
  cudaError_t e = check_launch();
  if (e) return e;
  prof_begin(st);
  k_finish_sum<<<1, kT, 0, st>>>(part, scale, out);
  count_launch("grid_sum_finish", st);
  return check_launch();
}

cudaError_t launch_add_scalar(int64_t n, double* u, const double* s, cudaStream_t st) {
  prof_begin(st);
  k_add_scalar<<<grid_blocks(n), kT, 0, st>>>(n, u, s);
  count_launch("add_scalar", st);
  return check_launch();
}

cudaError_t launch_fill(int64_t n, double* x, double v, cudaStream_t st) {
  prof_begin(st);
  k_fill<<<grid_blocks(n), kT, 0, st>>>(n, x, v);
  count_launch("fill", st);
  return check_launch();
}

cudaError_t launch_indicator(int64_t n, const double* u, double* chi_h, unsigned char* chi,
                             cudaStream_t st) {
  prof_begin(st);
  k_indicator<<<grid_blocks(n), kT, 0, st>>>(n, u, chi_h, chi);
  count_launch("indicator", st);
  return check_launch();
}

}  // namespace ibdl
