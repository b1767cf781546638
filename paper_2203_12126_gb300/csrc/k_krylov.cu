// GMRES kernels (Sec. 5.3: unpreconditioned GMRES on the non-symmetric
// boundary operator, relative residual test).  Always float64.
//
// One Arnoldi step j (basis V_0..V_j, new vector w = V_{j+1} = A V_j):
//   classical Gram-Schmidt applied twice (CGS2):
//     h  = V^T w ;  w -= V h          (twice, h accumulated into H[:, j])
//     H[j+1, j] = ||w|| ;  V_{j+1} = w / ||w||
//   then the Givens rotations of the least-squares problem are applied to
//   column j on one thread, and |g_{j+1}| (the residual norm of the current
//   least-squares iterate) is written for the host's convergence test.
// Reductions are two-level: per-block partial sums in `partial`, re-reduced
// redundantly by every block of the next kernel, so no atomics are used and
// results are deterministic.
#include <math.h>

#include "ibdl_internal.cuh"

namespace ibdl {

constexpr int kBs = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid on thread 0
}

__device__ __forceinline__ void chunk(int m, int& lo, int& hi) {
  const int c = (m + gridDim.x - 1) / gridDim.x;
  lo = min(m, blockIdx.x * c);
  hi = min(m, lo + c);
}

// partial[blk * stride + c] = sum_{i in blk} V_c[i] w[i], c < ncols
__global__ void __launch_bounds__(kBs) k_dots(const double* __restrict__ V, int ld, int ncols,
                                              const double* __restrict__ w, int m,
                                              double* __restrict__ partial, int stride) {
  __shared__ double sh[32];
  int lo, hi;
  chunk(m, lo, hi);
  for (int c = 0; c < ncols; ++c) {
    const double* v = V + (size_t)c * ld;
    double s = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) s += v[i] * w[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * stride + c] = s;
  }
}

// h_c = sum_b partial[b][c];  w -= sum_c h_c V_c;  Hcol[c] (+)= h_c;
// norm partial of the updated w into partial[b * stride + ncols].
__global__ void __launch_bounds__(kBs) k_orth_update(const double* __restrict__ V, int ld,
                                                     int ncols, double* __restrict__ w, int m,
                                                     double* __restrict__ partial, int stride,
                                                     double* __restrict__ Hcol, int accumulate) {
  __shared__ double h[64];
  __shared__ double sh[32];
  const int nb = gridDim.x;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += partial[b * stride + c];
    h[c] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x)
      Hcol[c] = accumulate ? Hcol[c] + h[c] : h[c];
  }
  int lo, hi;
  chunk(m, lo, hi);
  double nrm = 0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double v = w[i];
    for (int c = 0; c < ncols; ++c) v -= h[c] * V[(size_t)c * ld + i];
    w[i] = v;
    nrm += v * v;
  }
  __syncthreads();  // all blocks have read `partial` before anyone rewrites it
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x * stride + ncols] = nrm;
}

// H[j+1, j] = ||w||, w /= ||w||; then Givens on column j (block 0, thread 0).
__global__ void __launch_bounds__(kBs) k_normalize(double* __restrict__ w, int m,
                                                   const double* __restrict__ partial,
                                                   int stride, int nparts, int slot,
                                                   double* Hcol) {
  __shared__ double hn;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int b = 0; b < nparts; ++b) s += partial[b * stride + slot];
    hn = sqrt(s);
    if (blockIdx.x == 0) Hcol[slot] = hn;
  }
  __syncthreads();
  const double inv = (hn > 0 && isfinite(hn)) ? 1.0 / hn : 0.0;
  if (inv == 0.0) return;
  int lo, hi;
  chunk(m, lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) w[i] *= inv;
}

// Apply rotations 0..j-1 to column j, build rotation j, update g.
// scal[0] = |g_{j+1}| / bnorm, scal[1] = H[j+1, j] before rotation.
__global__ void k_givens(double* H, int ldh, double* cs, double* sn, double* g, int j,
                         double bnorm, double* scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ldh;
  scal[1] = col[j + 1];
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double den = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (den > 0) {
    c = a / den;
    s = b / den;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  scal[0] = fabs(g[j + 1]) / bnorm;
}

// Back substitution R y = g (R = leading k x k of the rotated H), 1 thread.
__global__ void k_backsolve(const double* H, int ldh, const double* g, int k, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * ldh + i] * y[l];
    const double d = H[(size_t)i * ldh + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// x += sum_c y_c V_c
__global__ void __launch_bounds__(kBs) k_update_x(const double* __restrict__ V, int ld, int k,
                                                  const double* __restrict__ y,
                                                  double* __restrict__ x, int m) {
  __shared__ double ys[64];
  for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = y[c];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double v = x[i];
    for (int c = 0; c < k; ++c) v += ys[c] * V[(size_t)c * ld + i];
    x[i] = v;
  }
}

// V0 = r / ||r||, g = (||r||, 0, ...), scal[2] = ||r||
__global__ void __launch_bounds__(kBs) k_start(const double* __restrict__ r, double* V0, int m,
                                               const double* __restrict__ partial, int stride,
                                               double* g, int glen, double* scal) {
  __shared__ double beta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int b = 0; b < gridDim.x; ++b) s += partial[b * stride];
    beta = sqrt(s);
    if (blockIdx.x == 0) scal[2] = beta;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < glen; c += blockDim.x) g[c] = (c == 0) ? beta : 0.0;
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  int lo, hi;
  chunk(m, lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) V0[i] = r[i] * inv;
}

__global__ void k_axpby(int m, double a, const double* x, double b, const double* y,
                        double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

__global__ void k_nonfinite(int m, const double* x, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 1;
}

// ---- host launchers ---------------------------------------------------------

cudaError_t krylov_dot_norm(const KrylovWs& k, const double* x, double* out_sq,
                            cudaStream_t st) {
  const int stride = k.restart + 2;
  prof_begin(st);
  k_dots<<<k.nblk, kBs, 0, st>>>(x, 0, 1, x, k.m, k.partial, stride);
  count_launch("dots", st);
  cudaError_t e = check_launch();
  if (e) return e;
  // reduce the block partials on one block into out_sq[0]
  prof_begin(st);
  k_normalize<<<1, 32, 0, st>>>(nullptr, 0, k.partial, stride, k.nblk, 0, out_sq);
  count_launch("normalize", st);
  return check_launch();
}

cudaError_t krylov_start(const KrylovWs& k, const double* r, double* /*unused*/,
                         cudaStream_t st) {
  const int stride = k.restart + 2;
  prof_begin(st);
  k_dots<<<k.nblk, kBs, 0, st>>>(r, 0, 1, r, k.m, k.partial, stride);
  count_launch("dots", st);
  cudaError_t e = check_launch();
  if (e) return e;
  prof_begin(st);
  k_start<<<k.nblk, kBs, 0, st>>>(r, k.V, k.m, k.partial, stride, k.gvec, k.restart + 1,
                                  k.scal);
  count_launch("start", st);
  return check_launch();
}

cudaError_t krylov_arnoldi(const KrylovWs& k, int j, double bnorm, cudaStream_t st) {
  const int stride = k.restart + 2;
  const int ldh = k.restart + 1;
  double* w = k.V + (size_t)(j + 1) * k.ld;
  double* Hcol = k.H + (size_t)j * ldh;
  cudaError_t e;
  for (int pass = 0; pass < 2; ++pass) {
    prof_begin(st);
    k_dots<<<k.nblk, kBs, 0, st>>>(k.V, k.ld, j + 1, w, k.m, k.partial, stride);
    count_launch("dots", st);
    if ((e = check_launch())) return e;
    prof_begin(st);
    k_orth_update<<<k.nblk, kBs, 0, st>>>(k.V, k.ld, j + 1, w, k.m, k.partial, stride, Hcol,
                                          pass);
    count_launch("orth_update", st);
    if ((e = check_launch())) return e;
  }
  prof_begin(st);
  k_normalize<<<k.nblk, kBs, 0, st>>>(w, k.m, k.partial, stride, k.nblk, j + 1, Hcol);
  count_launch("normalize", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_givens<<<1, 32, 0, st>>>(k.H, ldh, k.cs, k.sn, k.gvec, j, bnorm, k.scal);
  count_launch("givens", st);
  return check_launch();
}

cudaError_t krylov_finish(const KrylovWs& k, int kdim, double* x, cudaStream_t st) {
  cudaError_t e;
  prof_begin(st);
  k_backsolve<<<1, 32, 0, st>>>(k.H, k.restart + 1, k.gvec, kdim, k.ysol);
  count_launch("backsolve", st);
  if ((e = check_launch())) return e;
  const int blocks = (k.m + kBs - 1) / kBs;
  prof_begin(st);
  k_update_x<<<blocks < 1 ? 1 : blocks, kBs, 0, st>>>(k.V, k.ld, kdim, k.ysol, x, k.m);
  count_launch("update_x", st);
  return check_launch();
}

cudaError_t launch_axpby(int m, double a, const double* x, double b, const double* y,
                         double* out, cudaStream_t st) {
  int blocks = (m + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  prof_begin(st);
  k_axpby<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(m, a, x, b, y, out);
  count_launch("axpby", st);
  return check_launch();
}

cudaError_t launch_nonfinite_check(int m, const double* x, int* flag, cudaStream_t st) {
  int blocks = (m + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  prof_begin(st);
  k_nonfinite<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(m, x, flag);
  count_launch("nonfinite", st);
  return check_launch();
}

}  // namespace ibdl
