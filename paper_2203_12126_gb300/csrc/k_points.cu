// Point-side kernels: delta weights, tile binning and interpolation S*.
//
// Sec. 5.2: delta_h(x) = h^{-d} prod_c phi(x_c / h) with Peskin's 4-point
// phi (eq. (delta eqn 2)) or the cosine 4-point kernel; interpolation
// (S* u)(X) = sum_j u_j delta_h(x_j - X) h^d, whose h^{-d} h^d cancel, so a
// point reads the 4^d nodes base_c + t (t = 0..3) with weights prod_c W[c][t].
#include <math.h>

#include "ibdl_device.cuh"

namespace ibdl {

__device__ __forceinline__ double phi_peskin4(double r) {
  const double a = fabs(r);
  if (a <= 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
  if (a < 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(fmax(0.0, -7.0 + 12.0 * a - 4.0 * a * a)));
  return 0.0;
}

__device__ __forceinline__ double phi_cos4(double r) {
  const double a = fabs(r);
  return a < 2.0 ? 0.25 * (1.0 + cospi(0.5 * a)) : 0.0;
}

// Per point and axis: base index and the four phi weights.
__global__ void k_point_prep(GridDesc g, int m, const double* __restrict__ X0,
                             const double* __restrict__ X1, const double* __restrict__ X2,
                             int* b0, int* b1, int* b2, double* W0, double* W1, double* W2,
                             float* V0, float* V1, float* V2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double* X[3] = {X0, X1, X2};
  int* B[3] = {b0, b1, b2};
  double* W[3] = {W0, W1, W2};
  float* V[3] = {V0, V1, V2};
  for (int c = 0; c < g.dim; ++c) {
    const double s = (X[c][i] - g.origin[c]) / g.h;
    const int base = (int)floor(s) - 1;
    B[c][i] = base;
    for (int t = 0; t < 4; ++t) {
      const double r = (double)(base + t) - s;
      const double v = g.delta == IBDL_DELTA_COS4 ? phi_cos4(r) : phi_peskin4(r);
      W[c][t * m + i] = v;
      V[c][t * m + i] = (float)v;
    }
  }
}

cudaError_t launch_point_prep(const GridDesc& g, int m, const double* const X[3],
                              int* const base[3], double* const W64[3],
                              float* const W32[3], cudaStream_t st) {
  const int bs = 256;
  prof_begin(st);
  k_point_prep<<<(m + bs - 1) / bs, bs, 0, st>>>(g, m, X[0], X[1], X[2], base[0], base[1],
                                                base[2], W64[0], W64[1], W64[2], W32[0],
                                                W32[1], W32[2]);
  count_launch("point_prep", st);
  return check_launch();
}

// ---- binning ---------------------------------------------------------------
// A point's spread-divergence touches rows y in [by-1, by+4] and (3D) planes
// z in [bz-1, bz+4] (periodic).  Tile id = z * (n/R) + y / R.  The 6 rows map
// to at most 3 consecutive row groups (R >= 4) or, for small n, groups that
// repeat only in runs, so de-duplicating against the previous group suffices
// when R <= n - 5.

template <bool FILL>
__global__ void k_bins(GridDesc g, PointData p, int rows, int* counts, int* pts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.m) return;
  const int mask = g.n - 1;
  const int ngroups = g.n / rows;
  const int by = p.base[1][i];
  const int nz = g.dim == 3 ? kBoxSide : 1;
  for (int cz = 0; cz < nz; ++cz) {
    const int z = g.dim == 3 ? ((p.base[2][i] - 1 + cz) & mask) : 0;
    int prev = -1;
    for (int b = 0; b < kBoxSide; ++b) {
      const int grp = ((by - 1 + b) & mask) / rows;
      if (grp == prev) continue;
      prev = grp;
      const int tile = z * ngroups + grp;
      const int pos = atomicAdd(&counts[tile], 1);
      if (FILL) pts[pos] = i;
    }
  }
}

// Single-block exclusive scan: start[t] = sum_{s < t} counts[s], start[T] = nnz.
__global__ void k_scan(const int* counts, int* start, int* cursor, int ntiles) {
  __shared__ int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int chunk = (ntiles + nt - 1) / nt;
  const int lo = min(ntiles, tid * chunk), hi = min(ntiles, lo + chunk);
  int s = 0;
  for (int t = lo; t < hi; ++t) s += counts[t];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nt; ++t) {
      const int v = part[t];
      part[t] = acc;
      acc += v;
    }
    start[ntiles] = acc;
  }
  __syncthreads();
  int acc = part[tid];
  for (int t = lo; t < hi; ++t) {
    start[t] = acc;
    cursor[t] = acc;
    acc += counts[t];
  }
}

// Tile lists: count, scan, fill.  The order of points inside a tile is the
// order of the fill's atomics; it does not matter, since the spread adds a
// tile's contributions with shared-memory atomics anyway (the sum is the
// same up to rounding in any order).  pts has room for the largest possible
// count (bins_capacity), so no host round trip sizes it.
cudaError_t launch_bins(const GridDesc& g, const PointData& p, int rows, int ntiles,
                        int* start, int* cursor, int* counts, int* pts, cudaStream_t st) {
  cudaError_t e;
  const int bs = 256;
  const int gb = (p.m + bs - 1) / bs;
  if ((e = cudaMemsetAsync(cursor, 0, sizeof(int) * (ntiles + 1), st))) return e;
  prof_begin(st);
  k_bins<false><<<gb, bs, 0, st>>>(g, p, rows, cursor, nullptr);
  count_launch("bins", st);
  if ((e = check_launch())) return e;
  if ((e = cudaMemcpyAsync(counts, cursor, sizeof(int) * (ntiles + 1),
                           cudaMemcpyDeviceToDevice, st)))
    return e;
  prof_begin(st);
  k_scan<<<1, 1024, 0, st>>>(counts, start, cursor, ntiles);
  count_launch("scan", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_bins<true><<<gb, bs, 0, st>>>(g, p, rows, cursor, pts);
  count_launch("bins", st);
  return check_launch();
}

int64_t bins_capacity(int dim, int rows, int64_t m) {
  // the 6 support rows meet at most 1 + ceil(5 / R) row groups, on 6 planes in 3D
  const int64_t groups = 1 + (5 + rows - 1) / rows;
  return m * groups * (dim == 3 ? 6 : 1);
}

// zempty[z] = 1 when no tile of plane z lists a point (3D).
__global__ void k_plane_flags(const int* start, int ngroups, int n, unsigned char* zempty) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) zempty[z] = start[(z + 1) * ngroups] == start[z * ngroups] ? 1 : 0;
}

cudaError_t launch_plane_flags(const int* start, int ngroups, int n, unsigned char* zempty,
                               cudaStream_t st) {
  prof_begin(st);
  k_plane_flags<<<(n + 127) / 128, 128, 0, st>>>(start, ngroups, n, zempty);
  count_launch("plane_flags", st);
  return check_launch();
}

// ---- interpolation ------------------------------------------------------------

// y_i = S* grid at X_i (+ jump * jvec_i).
template <typename T, int D>
__global__ void __launch_bounds__(128) k_interp(GridDesc g, PointData p, const T* grid,
                                                const double* jvec, double jump, double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.m) return;
  // the grid comes from an earlier launch: cached loads are coherent here
  double out = (double)interp_point<T, D, true>(g, p, grid, i);
  if (jvec) out += jump * jvec[i];
  y[i] = out;
}

template <typename T>
cudaError_t launch_interp(const GridDesc& g, const PointData& p, const T* grid,
                          const double* jvec, double jump, double* y, cudaStream_t st) {
  const int bs = 128;
  const int gb = (p.m + bs - 1) / bs;
  prof_begin(st);
  if (g.dim == 2)
    k_interp<T, 2><<<gb, bs, 0, st>>>(g, p, grid, jvec, jump, y);
  else
    k_interp<T, 3><<<gb, bs, 0, st>>>(g, p, grid, jvec, jump, y);
  count_launch(sizeof(T) == 8 ? "interp_f64" : "interp_f32", st);
  return check_launch();
}

template cudaError_t launch_interp<double>(const GridDesc&, const PointData&, const double*,
                                           const double*, double, double*, cudaStream_t);
template cudaError_t launch_interp<float>(const GridDesc&, const PointData&, const float*,
                                          const double*, double, double*, cudaStream_t);

__global__ void k_to_float(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

cudaError_t launch_grid_to_float(const double* src, float* dst, int64_t count,
                                 cudaStream_t st) {
  prof_begin(st);
  k_to_float<<<608, 256, 0, st>>>(src, dst, count);
  count_launch("to_float", st);
  return check_launch();
}

}  // namespace ibdl
