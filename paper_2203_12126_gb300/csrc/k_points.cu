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

// Writes each tile's list, ordered by the point's first support column
// xs = (base_x - 1) mod n and then by point index, to spts: a counting sort
// over the n columns (histogram, scan, scatter), then each column's bucket
// sorted by index in place by one thread.  The gather spread finds a node's
// sources in the sorted list (a contiguous run of columns), and the fixed
// order makes that spread bitwise reproducible.  Dynamic shared memory:
// 2 (n + 1) ints.
__global__ void __launch_bounds__(256) k_sort_bins(GridDesc g, const int* __restrict__ base0,
                                                   const int* __restrict__ start,
                                                   const int* __restrict__ pts, int* spts,
                                                   int ntiles) {
  extern __shared__ int sh[];
  const int n = g.n, mask = n - 1, tid = threadIdx.x, nt = blockDim.x;
  int* cnt = sh;          // n + 1: counts, then running ends
  int* beg = sh + n + 1;  // n + 1: bucket starts
  __shared__ int part[32];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int lo = start[t], hi = start[t + 1];
    if (hi - lo < 2) {
      if (hi > lo && tid == 0) spts[lo] = pts[lo];
      continue;
    }
    for (int x = tid; x <= n; x += nt) cnt[x] = 0;
    __syncthreads();
    for (int e = lo + tid; e < hi; e += nt) atomicAdd(&cnt[(base0[pts[e]] - 1) & mask], 1);
    __syncthreads();
    // exclusive scan of cnt[0..n) into beg: per-thread runs, then the warp
    // sums of the run totals
    const int per = (n + nt - 1) / nt, x0 = min(n, tid * per), x1 = min(n, x0 + per);
    int run = 0;
    for (int x = x0; x < x1; ++x) run += cnt[x];
    int incl = run;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = lane < (nt >> 5) ? part[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += v;
      }
      if (lane < (nt >> 5)) part[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    int acc = incl - run + (wid > 0 ? part[wid - 1] : 0);
    for (int x = x0; x < x1; ++x) {
      const int c = cnt[x];
      beg[x] = acc;
      cnt[x] = acc;  // running end of bucket x
      acc += c;
    }
    __syncthreads();
    for (int e = lo + tid; e < hi; e += nt) {
      const int i = pts[e];
      const int pos = atomicAdd(&cnt[(base0[i] - 1) & mask], 1);
      spts[lo + pos] = i;
    }
    __syncthreads();
    // each bucket by point index (buckets hold the few points of a column)
    for (int x = tid; x < n; x += nt) {
      const int b0 = lo + beg[x], b1 = lo + cnt[x];
      for (int a = b0 + 1; a < b1; ++a) {
        const int v = spts[a];
        int b = a;
        while (b > b0 && spts[b - 1] > v) {
          spts[b] = spts[b - 1];
          --b;
        }
        spts[b] = v;
      }
    }
    __syncthreads();
  }
}

// Tile lists: count, scan, fill (pts: fill order), then each tile's list
// ordered by first support column and point index into spts (k_sort_bins).
// pts and spts have room for the largest possible count (bins_capacity), so
// no host round trip sizes them.
cudaError_t launch_bins(const GridDesc& g, const PointData& p, int rows, int ntiles,
                        int* start, int* cursor, int* counts, int* pts, int* spts,
                        cudaStream_t st) {
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
  if ((e = check_launch())) return e;
  prof_begin(st);
  const int sb = ntiles < 2048 ? ntiles : 2048;
  k_sort_bins<<<sb, 256, 2 * (g.n + 1) * sizeof(int), st>>>(g, p.base[0], start, pts, spts,
                                                              ntiles);
  count_launch("sort_bins", st);
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

// The four x taps grid[x0 .. x0 + 3] (mod n) of one grid row: away from the
// row's end, from the aligned 16-byte vectors that cover them (one or two
// loads instead of four), else one load per tap with the periodic wrap.  The
// row starts a multiple of n >= 16 elements into the grid, so with VEC (a
// 16-byte aligned grid) the vectors are aligned.
template <bool VEC>
__device__ __forceinline__ void row_taps(const float* row, int x0, int n, float t[4]) {
  x0 &= n - 1;
  const int a0 = x0 & ~3, sh = x0 & 3;
  if (VEC && a0 + 8 <= n) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(row + a0));
    if (sh == 0) {
      t[0] = u.x;
      t[1] = u.y;
      t[2] = u.z;
      t[3] = u.w;
      return;
    }
    const float4 w = __ldg(reinterpret_cast<const float4*>(row + a0 + 4));
    const float v[8] = {u.x, u.y, u.z, u.w, w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = sh == 1 ? v[k + 1] : (sh == 2 ? v[k + 2] : v[k + 3]);
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = __ldg(row + ((x0 + k) & (n - 1)));
}
template <bool VEC>
__device__ __forceinline__ void row_taps(const double* row, int x0, int n, double t[4]) {
  x0 &= n - 1;
  const int a0 = x0 & ~1, sh = x0 & 1;
  if (VEC && a0 + 6 <= n) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(row + a0));
    const double2 w = __ldg(reinterpret_cast<const double2*>(row + a0 + 2));
    if (sh == 0) {
      t[0] = u.x;
      t[1] = u.y;
      t[2] = w.x;
      t[3] = w.y;
      return;
    }
    const double2 z = __ldg(reinterpret_cast<const double2*>(row + a0 + 4));
    t[0] = u.y;
    t[1] = w.x;
    t[2] = w.y;
    t[3] = z.x;
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = __ldg(row + ((x0 + k) & (n - 1)));
}

// y_i = S* grid at X_i (+ jump * jvec_i).  Four threads share a point, one
// per tap plane (3D: z = bz + t) or tap row (2D: y = by + t), so a warp keeps
// four times as many independent grid loads in flight; the four partial sums
// are combined by a fixed butterfly of shuffles (a deterministic order).
// In 3D lane t of a point loads the point's tap weights W_c[t] and base
// index c = t and hands them to the other three by shuffles, and the x taps
// of a row come in vector loads (row_taps): that kernel is bound by its load
// instructions, not by their bytes (C3 float32: 14.4 -> 11.4 us).
template <typename T, int D, bool VEC>
__global__ void __launch_bounds__(128) k_interp(GridDesc g, PointData p, const T* grid,
                                                const double* jvec, double jump, double* y) {
  pdl_wait();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt >> 2, sub = gt & 3;
  const bool live = i < p.m;
  const int ii = live ? i : 0;
  const int n = g.n, mask = n - 1, m = p.m;
  // the grid comes from an earlier launch: cached loads are coherent here
  T acc = 0;
  if constexpr (D == 2) {
    // 2D: each lane loads its own weights and indices (a shuffle hand-off
    // lengthens this latency-bound kernel's chain: measured 6.1 -> 7.2 us)
    T wx[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) wx[t] = interp_w<T>(p, 0, t, ii, m);
    const int bx = p.base[0][ii], by = p.base[1][ii];
    const T* row = grid + (size_t)((by + sub) & mask) * n;
    T r = 0;
#pragma unroll
    for (int tx = 0; tx < 4; ++tx) r += __ldg(row + ((bx + tx) & mask)) * wx[tx];
    acc = r * interp_w<T>(p, 1, sub, ii, m);
  } else {
    // 3D: 16 rows of 4 taps per point, bound by load instructions: lane t of
    // a point loads W_c[t] and base index c = t for the other three lanes
    const int lead = threadIdx.x & 28;  // lane of the point's sub = 0 thread
    const T wxs = interp_w<T>(p, 0, sub, ii, m);
    const T wys = interp_w<T>(p, 1, sub, ii, m);
    const T wzs = interp_w<T>(p, 2, sub, ii, m);
    const int* bp = sub == 0 ? p.base[0] : (sub == 1 ? p.base[1] : p.base[2]);
    const int bsub = sub < 3 ? __ldg(bp + ii) : 0;
    T wx[4], wy[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      wx[t] = __shfl_sync(0xffffffffu, wxs, lead + t);
      wy[t] = __shfl_sync(0xffffffffu, wys, lead + t);
    }
    const int bx = __shfl_sync(0xffffffffu, bsub, lead);
    const int by = __shfl_sync(0xffffffffu, bsub, lead + 1);
    const int bz = __shfl_sync(0xffffffffu, bsub, lead + 2);
    const T* plane = grid + (size_t)((bz + sub) & mask) * n * n;
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
      const T* row = plane + (size_t)((by + ty) & mask) * n;
      T tp[4];
      row_taps<VEC>(row, bx, n, tp);
      T r = 0;
#pragma unroll
      for (int tx = 0; tx < 4; ++tx) r += tp[tx] * wx[tx];
      acc += r * wy[ty];
    }
    acc *= wzs;
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (live && sub == 0) {
    double out = (double)acc;
    if (jvec) out += jump * jvec[i];
    y[i] = out;
  }
  pdl_release();
}

template <typename T>
cudaError_t launch_interp(const GridDesc& g, const PointData& p, const T* grid,
                          const double* jvec, double jump, double* y, cudaStream_t st) {
  const int bs = 128;
  const int gb = (int)((4 * (int64_t)p.m + bs - 1) / bs);
  // vector tap loads need a 16-byte aligned grid (the library's own grids
  // are; one passed in by a caller may not be)
  const bool vec = (reinterpret_cast<uintptr_t>(grid) & 15) == 0;
  prof_begin(st);
  if (g.dim == 2) {
    if (vec)
      launch_dependent(k_interp<T, 2, true>, gb, bs, 0, st, g, p, grid, jvec, jump, y);
    else
      launch_dependent(k_interp<T, 2, false>, gb, bs, 0, st, g, p, grid, jvec, jump, y);
  } else {
    if (vec)
      launch_dependent(k_interp<T, 3, true>, gb, bs, 0, st, g, p, grid, jvec, jump, y);
    else
      launch_dependent(k_interp<T, 3, false>, gb, bs, 0, st, g, p, grid, jvec, jump, y);
  }
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
