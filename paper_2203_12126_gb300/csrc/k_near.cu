// Near-boundary values (Sec. 5.5, App. A), 2D, float64.
//
// Grid nodes of Omega (inside = 1) whose nearest boundary point is closer
// than m1 h get a value interpolated along the line from the chord point
// x_A (on the segment of the two nearest boundary points, carrying the
// boundary values) to x_B, m2 h further into Omega (bilinear in the grid
// field):
//   1. mark: each boundary point flags the nodes of the (2 m1 + 2)^2 box
//      around it (a superset of the nodes within m1 h);
//   2. compact: flagged nodes with inside = 1 are appended to a list;
//   3. cells: the points are counting-sorted into square cells of side
//      s = max(m1 + 2, 8) h;
//   4. fix: one thread per listed node finds the three nearest points (ordered
//      by squared distance, then index) among the 3 x 3 cells around it.
//      Every point outside those cells is at least s away (0.999 s, a margin
//      for the rounding of the cell assignment), and s > m1 h: a node whose
//      nearest found point is not within m1 h is not near, and the three
//      found are the three nearest overall whenever the third is within
//      0.999 s; otherwise the warp scans all points.  Then the steps of
//      App. A, and u_out.
// u_out starts as a copy of u_in, and the fix reads only u_in, so the result
// does not depend on the order in which nodes are corrected.
//
// This file is compiled with -fmad=false: distances, the chord parameter and
// the cell of x_B are rounded operation by operation, so the integer
// decisions (near or not, which points, which branch) are those of a plain
// IEEE evaluation of the same expressions.
#include <math.h>

#include "ibdl_internal.cuh"

namespace ibdl {

namespace {

constexpr int kT = 256;

__global__ void __launch_bounds__(kT) k_near_mark(int m, const double* __restrict__ X,
                                                  const double* __restrict__ Y, double ox,
                                                  double oy, double h, int n, int m1,
                                                  unsigned char* __restrict__ flag) {
  __shared__ int cell[2];
  const int w = 2 * m1 + 2;
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    if (threadIdx.x == 0) {  // one thread does the (slow) float64 divisions
      double rx = (X[i] - ox) / h, ry = (Y[i] - oy) / h;
      rx = fmin(fmax(rx, -1073741824.0), 1073741824.0);
      ry = fmin(fmax(ry, -1073741824.0), 1073741824.0);
      cell[0] = (int)floor(rx);
      cell[1] = (int)floor(ry);
    }
    __syncthreads();
    const int cx = cell[0], cy = cell[1];
    for (int e = threadIdx.x; e < w * w; e += kT) {
      const int ix = cx - m1 + e % w, iy = cy - m1 + e / w;
      if (ix >= 0 && ix < n && iy >= 0 && iy < n) flag[(size_t)iy * n + ix] = 1;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kT) k_near_compact(int64_t nn,
                                                     const unsigned char* __restrict__ flag,
                                                     const unsigned char* __restrict__ inside,
                                                     int* __restrict__ list, int* count,
                                                     int cap) {
  for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < nn;
       j += (int64_t)gridDim.x * kT) {
    if (flag[j] && inside[j]) {
      const int k = atomicAdd(count, 1);
      if (k < cap) list[k] = (int)j;
    }
  }
}

__device__ __forceinline__ double chord_t(double px, double py, double x1, double y1, double x2,
                                          double y2) {
  const double e0 = x1 - x2, e1 = y1 - y2;
  return ((px - x2) * e0 + (py - y2) * e1) / (e0 * e0 + e1 * e1);
}

__device__ __forceinline__ double dist(double ax, double ay, double bx, double by) {
  const double dx = ax - bx, dy = ay - by;
  return sqrt(dx * dx + dy * dy);
}

// (d, index) order; index -1 (no point) sorts last
__device__ __forceinline__ bool before(double d, int i, double e, int k) {
  return d < e || (d == e && (unsigned)i < (unsigned)k);
}

struct Top3 {
  double d0 = INFINITY, d1 = INFINITY, d2 = INFINITY;
  int i0 = -1, i1 = -1, i2 = -1;
  __device__ __forceinline__ void add(double d, int i) {
    if (!before(d, i, d2, i2)) return;
    if (before(d, i, d1, i1)) {
      d2 = d1, i2 = i1;
      if (before(d, i, d0, i0)) {
        d1 = d0, i1 = i0;
        d0 = d, i0 = i;
      } else {
        d1 = d, i1 = i;
      }
    } else {
      d2 = d, i2 = i;
    }
  }
};

__global__ void __launch_bounds__(kT) k_cell_count(int m, const double* __restrict__ X,
                                                   const double* __restrict__ Y, double ox,
                                                   double oy, double s, int nc,
                                                   int* __restrict__ cell_of,
                                                   int* __restrict__ counts) {
  for (int i = blockIdx.x * kT + threadIdx.x; i < m; i += gridDim.x * kT) {
    const double rx = fmin(fmax(floor((X[i] - ox) / s), 0.0), (double)(nc - 1));
    const double ry = fmin(fmax(floor((Y[i] - oy) / s), 0.0), (double)(nc - 1));
    const int c = (int)ry * nc + (int)rx;
    cell_of[i] = c;
    atomicAdd(counts + c, 1);
  }
}

// exclusive scan of counts into start (ncell + 1) and cursor, one block
// walking coalesced tiles of 1024 cells
__global__ void __launch_bounds__(1024) k_cell_scan(const int* __restrict__ counts,
                                                    int* __restrict__ start,
                                                    int* __restrict__ cursor, int ncell) {
  __shared__ int wsum[32];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) base = 0;
  __syncthreads();
  for (int t0 = 0; t0 < ncell; t0 += 1024) {
    const int t = t0 + tid;
    const int v = t < ncell ? counts[t] : 0;
    int x = v;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int excl = base + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    if (t < ncell) {
      start[t] = excl;
      cursor[t] = excl;
    }
    __syncthreads();
    if (tid == 1023) base += wsum[31];
    __syncthreads();
  }
  if (tid == 0) start[ncell] = base;
}

__global__ void __launch_bounds__(kT) k_cell_fill(int m, const int* __restrict__ cell_of,
                                                  int* __restrict__ cursor,
                                                  int* __restrict__ sorted) {
  for (int i = blockIdx.x * kT + threadIdx.x; i < m; i += gridDim.x * kT)
    sorted[atomicAdd(cursor + cell_of[i], 1)] = i;
}

// One thread per listed node (the work per node is a few dozen points and
// a few dozen float64 operations; GB300's float64 pipe is narrow, so no
// lane repeats another's arithmetic).
constexpr int kFixT = 64;  // small blocks spread the few thousand nodes over all SMs

__global__ void __launch_bounds__(kFixT) k_near_fix(const int* __restrict__ list, const int* count,
                                                 int cap, int n, double ox, double oy, double h,
                                                 int m, const double* __restrict__ X,
                                                 const double* __restrict__ Y,
                                                 const double* __restrict__ ub,
                                                 const double* __restrict__ uin, double thresh,
                                                 double m2h, int cw, int nc,
                                                 const int* __restrict__ cstart,
                                                 const int* __restrict__ sorted,
                                                 double guard2, double* __restrict__ uout) {
  const int cnt = min(*count, cap);
  for (int k = blockIdx.x * kFixT + threadIdx.x; k < cnt; k += gridDim.x * kFixT) {
    const int j = list[k];
    const int ix = j % n, iy = j / n;
    const double px = ox + (double)ix * h, py = oy + (double)iy * h;
    Top3 t3;
    const int cx = min(ix / cw, nc - 1), cy = min(iy / cw, nc - 1);
    for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by)
      for (int bx = max(cx - 1, 0); bx <= min(cx + 1, nc - 1); ++bx) {
        const int c = by * nc + bx;
        for (int t = cstart[c]; t < cstart[c + 1]; ++t) {
          const int i = sorted[t];
          const double dx = px - __ldg(X + i), dy = py - __ldg(Y + i);
          t3.add(dx * dx + dy * dy, i);
        }
      }
    // every point closer than the guard (> m1 h) was searched: a node whose
    // nearest found point is not within m1 h has none
    if (!(t3.d0 < thresh)) continue;
    if (!(t3.d2 < guard2)) {
      // the third nearest may lie outside the searched cells: scan all points
      t3 = Top3();
      for (int i = 0; i < m; ++i) {
        const double dx = px - __ldg(X + i), dy = py - __ldg(Y + i);
        t3.add(dx * dx + dy * dy, i);
      }
    }
    const double dd[3] = {t3.d0, t3.d1, t3.d2};
    const int ii[3] = {t3.i0, t3.i1, t3.i2};
    const double d0 = dd[0];
    const int i0 = ii[0], i1 = ii[1], i2 = ii[2];
    // i1, i2 stay -1 only if squared distances overflow (points near 1e154)
    if (!(d0 < thresh) || i1 < 0 || i2 < 0) continue;
    int a = i0, b = i1;
    double t = chord_t(px, py, X[a], Y[a], X[b], Y[b]);
    if (!(t >= 0.0 && t <= 1.0)) {
      // the two of the three nearest that lie farthest apart
      const int pa[3] = {i0, i0, i1}, pb[3] = {i1, i2, i2};
      double best = -1.0;
      for (int q = 0; q < 3; ++q) {
        const double e0 = X[pa[q]] - X[pb[q]], e1 = Y[pa[q]] - Y[pb[q]];
        const double s = e0 * e0 + e1 * e1;
        if (s > best) best = s, a = pa[q], b = pb[q];
      }
      t = fmin(fmax(chord_t(px, py, X[a], Y[a], X[b], Y[b]), 0.0), 1.0);
    }
    const double x1 = X[a], y1 = Y[a], x2 = X[b], y2 = Y[b];
    const double xa = x2 + t * (x1 - x2), ya = y2 + t * (y1 - y2);
    const double L12 = dist(x2, y2, x1, y1);
    const double uA = ub[a] * dist(xa, ya, x2, y2) / L12 + ub[b] * dist(xa, ya, x1, y1) / L12;
    const double dA = dist(px, py, xa, ya);
    if (dA == 0.0) {
      uout[j] = uA;
      continue;
    }
    const double xb = xa + (px - xa) / dA * m2h, yb = ya + (py - ya) / dA * m2h;
    const double rx = (xb - ox) / h, ry = (yb - oy) / h;
    const double fjx = floor(rx), fjy = floor(ry);
    const double fx = rx - fjx, fy = ry - fjy;
    constexpr double kBig = 4503599627370496.0;  // 2^52: keeps the casts defined
    const long long jx = (long long)fmin(fmax(fjx, -kBig), kBig);
    const long long jy = (long long)fmin(fmax(fjy, -kBig), kBig);
    const int x0 = (int)(((jx % n) + n) % n), y0 = (int)(((jy % n) + n) % n);
    const int x1i = (x0 + 1) % n, y1i = (y0 + 1) % n;
    const double u00 = uin[(size_t)y0 * n + x0], u10 = uin[(size_t)y0 * n + x1i];
    const double u01 = uin[(size_t)y1i * n + x0], u11 = uin[(size_t)y1i * n + x1i];
    double uB = fx * fy * u11;
    uB = uB + fy * (1.0 - fx) * u01;
    uB = uB + fx * (1.0 - fy) * u10;
    uB = uB + (1.0 - fx - fy + fx * fy) * u00;
    const double LAB = dist(xb, yb, xa, ya);
    uout[j] = uA * dist(xb, yb, px, py) / LAB + uB * dA / LAB;
  }
}

int blocks_for(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b));
}

}  // namespace

int64_t near_list_capacity(int n, int m, int m1) {
  const int64_t w = 2 * (int64_t)m1 + 2;
  const int64_t a = (int64_t)n * n, b = (int64_t)m * w * w;
  return a < b ? a : b;
}

// cell side in grid spacings: at least m1 + 2 (the guaranteed search radius
// must exceed m1 h), at least 8 (bounds the cell count for small m1)
static int near_cell_width(int m1) { return m1 + 2 > 8 ? m1 + 2 : 8; }
static int near_cells(int n, int m1) {
  const int cw = near_cell_width(m1);
  return (n + cw - 1) / cw;
}

size_t near_scratch_bytes(int n, int m, int m1) {
  const int64_t nc = near_cells(n, m1);
  const size_t flag = ((size_t)n * n + 15) / 16 * 16;
  return flag + sizeof(int) * (4 + (size_t)near_list_capacity(n, m, m1) + 3 * (nc * nc + 1) +
                               2 * (size_t)m);
}

cudaError_t launch_near_boundary(const GridDesc& g, const PointData& p, const double* ub,
                                 const double* uin, const unsigned char* inside, int m1,
                                 double m2, double* uout, void* scratch, cudaStream_t st) {
  const int n = g.n;
  const int64_t nn = (int64_t)n * n;
  const int cap = (int)near_list_capacity(n, p.m, m1);
  const int nc = near_cells(n, m1);
  const int ncell = nc * nc;
  unsigned char* flag = static_cast<unsigned char*>(scratch);
  int* count = reinterpret_cast<int*>(flag + ((size_t)nn + 15) / 16 * 16);
  int* list = count + 4;
  int* counts = list + cap;
  int* cstart = counts + ncell + 1;
  int* cursor = cstart + ncell + 1;
  int* cell_of = cursor + ncell + 1;
  int* sorted = cell_of + p.m;
  cudaError_t e;
  if ((e = cudaMemsetAsync(flag, 0, (size_t)nn, st))) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(int), st))) return e;
  if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * ((size_t)ncell + 1), st))) return e;
  if ((e = cudaMemcpyAsync(uout, uin, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st)))
    return e;
  const int cw = near_cell_width(m1);
  const double s = (double)cw * g.h;
  prof_begin(st);
  k_cell_count<<<blocks_for(p.m), kT, 0, st>>>(p.m, p.X[0], p.X[1], g.origin[0], g.origin[1], s,
                                               nc, cell_of, counts);
  count_launch("near_cells", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_cell_scan<<<1, 1024, 0, st>>>(counts, cstart, cursor, ncell);
  count_launch("near_cell_scan", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_cell_fill<<<blocks_for(p.m), kT, 0, st>>>(p.m, cell_of, cursor, sorted);
  count_launch("near_cell_fill", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_near_mark<<<p.m < 8 * 152 ? p.m : 8 * 152, kT, 0, st>>>(p.m, p.X[0], p.X[1], g.origin[0],
                                                           g.origin[1], g.h, n, m1, flag);
  count_launch("near_mark", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_near_compact<<<blocks_for(nn), kT, 0, st>>>(nn, flag, inside, list, count, cap);
  count_launch("near_compact", st);
  if ((e = check_launch())) return e;
  const double mh = (double)m1 * g.h;
  const double guard = 0.999 * s;
  prof_begin(st);
  const int64_t fb = (cap + kFixT - 1) / kFixT;
  k_near_fix<<<(int)(fb < 32 * 152 ? fb : 32 * 152), kFixT, 0, st>>>(
      list, count, cap, n, g.origin[0], g.origin[1], g.h, p.m, p.X[0], p.X[1], ub, uin, mh * mh,
      m2 * g.h, cw, nc, cstart, sorted, guard * guard, uout);
  count_launch("near_fix", st);
  return check_launch();
}

}  // namespace ibdl
