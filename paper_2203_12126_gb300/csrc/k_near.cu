// Near-boundary values (Sec. 5.5, App. A in 2D; its 3D generalisation of
// Sec. 6.7), float64.
//
// Grid nodes of Omega (inside = 1) whose nearest boundary point is closer
// than m1 h get a value interpolated along the line from a point x_A on the
// discretised boundary (carrying the boundary values) to x_B, m2 h further
// into Omega (bilinear / trilinear in the grid field).  2D: x_A on the chord
// of the two nearest boundary points.  3D: x_A the foot of x_p on the plane
// of the three nearest, barycentric coordinates clamped to the triangle.
//   1. mark: each boundary point flags the nodes of the (2 m1 + 2)^d box
//      around it (a superset of the nodes within m1 h);
//   2. compact: flagged nodes with inside = 1 are appended to a list;
//   3. cells: the points are counting-sorted into cubic cells of side
//      s = max(m1 + 2, 8) h;
//   4. fix: one thread per listed node finds the three nearest points (ordered
//      by squared distance, then index) among the 3^d cells around it.
//      Every point outside those cells is at least s away (0.999 s, a margin
//      for the rounding of the cell assignment), and s > m1 h: a node whose
//      nearest found point is not within m1 h is not near, and the three
//      found are the three nearest overall whenever the third is within
//      0.999 s; otherwise the thread scans all points.  Then the steps of
//      App. A, and u_out.
// u_out starts as a copy of u_in, and the fix reads only u_in, so the result
// does not depend on the order in which nodes are corrected.
//
// This file is compiled with -fmad=false: distances, the chord parameter and
// the cell of x_B are rounded operation by operation, so the integer
// decisions (near or not, which points, which branch) are those of a plain
// IEEE evaluation of the same expressions.
#include <math.h>
#include <stdint.h>

#include "ibdl_internal.cuh"

namespace ibdl {

namespace {

constexpr int kT = 256;

struct Pts {
  const double* X[3];
  double o[3];
};

template <int D>
__global__ void __launch_bounds__(kT) k_near_mark(int m, Pts P, double h, int n, int m1,
                                                  unsigned char* __restrict__ flag) {
  __shared__ int cell[3];
  const int w = 2 * m1 + 2;
  const int wd = D == 3 ? w * w * w : w * w;
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    if (threadIdx.x == 0) {  // one thread does the (slow) float64 divisions
      for (int c = 0; c < D; ++c) {
        double r = (P.X[c][i] - P.o[c]) / h;
        r = fmin(fmax(r, -1073741824.0), 1073741824.0);
        cell[c] = (int)floor(r);
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < wd; e += kT) {
      const int ix = cell[0] - m1 + e % w, iy = cell[1] - m1 + (e / w) % w;
      const int iz = D == 3 ? cell[2] - m1 + e / (w * w) : 0;
      if (ix >= 0 && ix < n && iy >= 0 && iy < n && iz >= 0 && iz < n)
        flag[((size_t)iz * n + iy) * n + ix] = 1;
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

template <int D>
__global__ void __launch_bounds__(kT) k_cell_count(int m, Pts P, double s, int nc,
                                                   int* __restrict__ cell_of,
                                                   int* __restrict__ counts) {
  for (int i = blockIdx.x * kT + threadIdx.x; i < m; i += gridDim.x * kT) {
    int c = 0;
    for (int a = D - 1; a >= 0; --a) {
      const double r = fmin(fmax(floor((P.X[a][i] - P.o[a]) / s), 0.0), (double)(nc - 1));
      c = c * nc + (int)r;
    }
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

// Points in cell order: the index, and float copies of the coordinates for
// the distance filter of the fix.
template <int D>
__global__ void __launch_bounds__(kT) k_cell_fill(int m, Pts P, const int* __restrict__ cell_of,
                                                  int* __restrict__ cursor,
                                                  int* __restrict__ sorted,
                                                  float4* __restrict__ pts4) {
  for (int i = blockIdx.x * kT + threadIdx.x; i < m; i += gridDim.x * kT) {
    const int t = atomicAdd(cursor + cell_of[i], 1);
    sorted[t] = i;
    pts4[t] = make_float4((float)P.X[0][i], (float)P.X[1][i], D == 3 ? (float)P.X[2][i] : 0.0f,
                          0.0f);
  }
}

constexpr int kFixT = 64;  // small blocks spread the few thousand nodes over all SMs

template <int D>
__device__ __forceinline__ double sqdist(const double* p, const Pts& P, int i) {
  const double dx = p[0] - __ldg(P.X[0] + i), dy = p[1] - __ldg(P.X[1] + i);
  if (D == 2) return dx * dx + dy * dy;
  const double dz = p[2] - __ldg(P.X[2] + i);
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ double norm3(double a, double b, double c) {
  return sqrt(a * a + b * b + c * c);
}

template <int D>
__global__ void __launch_bounds__(kFixT) k_near_fix(const int* __restrict__ list, const int* count,
                                                    int cap, int n, Pts P, double h, int m,
                                                    const double* __restrict__ ub,
                                                    const double* __restrict__ uin,
                                                    double thresh, double m2h, int cw, int nc,
                                                    const int* __restrict__ cstart,
                                                    const int* __restrict__ sorted,
                                                    const float4* __restrict__ pts4,
                                                    float ferr, double guard2,
                                                    double* __restrict__ uout) {
  const int cnt = min(*count, cap);
  const double* X = P.X[0];
  const double* Y = P.X[1];
  const double* Z = P.X[2];
  const double ox = P.o[0], oy = P.o[1], oz = P.o[2];
  for (int k = blockIdx.x * kFixT + threadIdx.x; k < cnt; k += gridDim.x * kFixT) {
    const int j = list[k];
    const int ix = j % n, iy = (j / n) % n, iz = D == 3 ? j / (n * n) : 0;
    double p[3];
    p[0] = ox + (double)ix * h;
    p[1] = oy + (double)iy * h;
    p[2] = D == 3 ? oz + (double)iz * h : 0.0;
    Top3 t3;
    const int cx = min(ix / cw, nc - 1), cy = min(iy / cw, nc - 1);
    const int cz = D == 3 ? min(iz / cw, nc - 1) : 0;
    // float32 filter: |d2f - d2| <= ferr for every point of these cells, so
    // a point with d2f > (third best, rounded up) + ferr cannot enter the
    // three nearest; the others are ranked by their float64 distance
    const float pxf = (float)p[0], pyf = (float)p[1], pzf = (float)p[2];
    float third = INFINITY;
    for (int bz = (D == 3 ? max(cz - 1, 0) : 0); bz <= (D == 3 ? min(cz + 1, nc - 1) : 0); ++bz)
      for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by)
        for (int bx = max(cx - 1, 0); bx <= min(cx + 1, nc - 1); ++bx) {
          const int c = (bz * nc + by) * nc + bx;
          for (int t = cstart[c]; t < cstart[c + 1]; ++t) {
            const float4 q = __ldg(pts4 + t);
            const float fx = pxf - q.x, fy = pyf - q.y, fz = pzf - q.z;
            const float d2f = D == 3 ? fx * fx + fy * fy + fz * fz : fx * fx + fy * fy;
            if (d2f > third + ferr) continue;
            const int i = sorted[t];
            t3.add(sqdist<D>(p, P, i), i);
            third = __double2float_ru(t3.d2);
          }
        }
    // every point closer than the guard (> m1 h) was searched: a node whose
    // nearest found point is not within m1 h has none
    if (!(t3.d0 < thresh)) continue;
    if (!(t3.d2 < guard2)) {
      // the third nearest may lie outside the searched cells: scan all points
      t3 = Top3();
      for (int i = 0; i < m; ++i) t3.add(sqdist<D>(p, P, i), i);
    }
    const int i0 = t3.i0, i1 = t3.i1, i2 = t3.i2;
    // i1, i2 stay -1 only if squared distances overflow (points near 1e154)
    if (!(t3.d0 < thresh) || i1 < 0 || i2 < 0) continue;
    const double px = p[0], py = p[1], pz = p[2];
    if (D == 3) {
      // x_A: the foot on the plane of the three nearest points, barycentric
      // coordinates clamped to the triangle and renormalised
      double xa = X[i0], ya = Y[i0], za = Z[i0], uA = ub[i0];
      const double e1x = X[i1] - X[i0], e1y = Y[i1] - Y[i0], e1z = Z[i1] - Z[i0];
      const double e2x = X[i2] - X[i0], e2y = Y[i2] - Y[i0], e2z = Z[i2] - Z[i0];
      const double wx = px - X[i0], wy = py - Y[i0], wz = pz - Z[i0];
      const double d11 = e1x * e1x + e1y * e1y + e1z * e1z;
      const double d12 = e1x * e2x + e1y * e2y + e1z * e2z;
      const double d22 = e2x * e2x + e2y * e2y + e2z * e2z;
      const double w1 = wx * e1x + wy * e1y + wz * e1z;
      const double w2 = wx * e2x + wy * e2y + wz * e2z;
      const double det = d11 * d22 - d12 * d12;
      if (det > 0.0) {
        const double l2 = (d22 * w1 - d12 * w2) / det;
        const double l3 = (d11 * w2 - d12 * w1) / det;
        double a0 = fmax(1.0 - l2 - l3, 0.0), a1 = fmax(l2, 0.0), a2 = fmax(l3, 0.0);
        const double sm = a0 + a1 + a2;
        a0 = a0 / sm;
        a1 = a1 / sm;
        a2 = a2 / sm;
        xa = a0 * X[i0] + a1 * X[i1] + a2 * X[i2];
        ya = a0 * Y[i0] + a1 * Y[i1] + a2 * Y[i2];
        za = a0 * Z[i0] + a1 * Z[i1] + a2 * Z[i2];
        uA = a0 * ub[i0] + a1 * ub[i1] + a2 * ub[i2];
      }
      const double dA = norm3(px - xa, py - ya, pz - za);
      if (dA == 0.0) {
        uout[j] = uA;
        continue;
      }
      const double xb = xa + (px - xa) / dA * m2h, yb = ya + (py - ya) / dA * m2h;
      const double zb = za + (pz - za) / dA * m2h;
      const double rr[3] = {(xb - ox) / h, (yb - oy) / h, (zb - oz) / h};
      int q0[3];
      double ff[3];
      for (int c = 0; c < 3; ++c) {
        const double fj = floor(rr[c]);
        ff[c] = rr[c] - fj;
        constexpr double kBig = 4503599627370496.0;  // 2^52: keeps the casts defined
        const long long jj = (long long)fmin(fmax(fj, -kBig), kBig);
        q0[c] = (int)(((jj % n) + n) % n);
      }
      double uB = 0.0;
      for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            const double wgt = ((dx ? ff[0] : 1.0 - ff[0]) * (dy ? ff[1] : 1.0 - ff[1])) *
                               (dz ? ff[2] : 1.0 - ff[2]);
            const size_t at = ((size_t)((q0[2] + dz) % n) * n + (q0[1] + dy) % n) * n +
                              (q0[0] + dx) % n;
            uB = uB + wgt * uin[at];
          }
      const double LAB = norm3(xb - xa, yb - ya, zb - za);
      uout[j] = uA * norm3(xb - px, yb - py, zb - pz) / LAB + uB * dA / LAB;
      continue;
    }
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

int64_t near_list_capacity(int dim, int n, int m, int m1) {
  const int64_t w = 2 * (int64_t)m1 + 2;
  const int64_t a = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const int64_t b = (int64_t)m * w * w * (dim == 3 ? w : 1);
  return a < b ? a : b;
}

// cell side in grid spacings: at least m1 + 2 (the guaranteed search radius
// must exceed m1 h), at least 8 (bounds the cell count for small m1)
static int near_cell_width(int m1) { return m1 + 2 > 8 ? m1 + 2 : 8; }
static int near_cells(int n, int m1) {
  const int cw = near_cell_width(m1);
  return (n + cw - 1) / cw;
}
static int64_t near_cell_count(int dim, int n, int m1) {
  const int64_t nc = near_cells(n, m1);
  return dim == 3 ? nc * nc * nc : nc * nc;
}

size_t near_scratch_bytes(int dim, int n, int m, int m1) {
  const int64_t nn = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const size_t flag = ((size_t)nn + 15) / 16 * 16;
  return flag + sizeof(int) * (4 + (size_t)near_list_capacity(dim, n, m, m1) +
                               3 * ((size_t)near_cell_count(dim, n, m1) + 1) + 2 * (size_t)m) +
         16 + sizeof(float4) * (size_t)m;
}

cudaError_t launch_near_boundary(const GridDesc& g, const PointData& p, const double* ub,
                                 const double* uin, const unsigned char* inside, int m1,
                                 double m2, double cmax, double* uout, void* scratch,
                                 cudaStream_t st) {
  const int n = g.n, D = g.dim;
  const int64_t nn = D == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const int cap = (int)near_list_capacity(D, n, p.m, m1);
  const int nc = near_cells(n, m1);
  const int ncell = (int)near_cell_count(D, n, m1);
  unsigned char* flag = static_cast<unsigned char*>(scratch);
  int* count = reinterpret_cast<int*>(flag + ((size_t)nn + 15) / 16 * 16);
  int* list = count + 4;
  int* counts = list + cap;
  int* cstart = counts + ncell + 1;
  int* cursor = cstart + ncell + 1;
  int* cell_of = cursor + ncell + 1;
  int* sorted = cell_of + p.m;
  float4* pts4 = reinterpret_cast<float4*>(
      (reinterpret_cast<uintptr_t>(sorted + p.m) + 15) / 16 * 16);
  Pts P;
  for (int c = 0; c < 3; ++c) {
    P.X[c] = p.X[c];
    P.o[c] = g.origin[c];
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(flag, 0, (size_t)nn, st))) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(int), st))) return e;
  if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * ((size_t)ncell + 1), st))) return e;
  if ((e = cudaMemcpyAsync(uout, uin, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st)))
    return e;
  const int cw = near_cell_width(m1);
  const double s = (double)cw * g.h;
  prof_begin(st);
  if (D == 3)
    k_cell_count<3><<<blocks_for(p.m), kT, 0, st>>>(p.m, P, s, nc, cell_of, counts);
  else
    k_cell_count<2><<<blocks_for(p.m), kT, 0, st>>>(p.m, P, s, nc, cell_of, counts);
  count_launch("near_cells", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_cell_scan<<<1, 1024, 0, st>>>(counts, cstart, cursor, ncell);
  count_launch("near_cell_scan", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  if (D == 3)
    k_cell_fill<3><<<blocks_for(p.m), kT, 0, st>>>(p.m, P, cell_of, cursor, sorted, pts4);
  else
    k_cell_fill<2><<<blocks_for(p.m), kT, 0, st>>>(p.m, P, cell_of, cursor, sorted, pts4);
  count_launch("near_cell_fill", st);
  if ((e = check_launch())) return e;
  const int mb = p.m < 8 * 152 ? p.m : 8 * 152;
  prof_begin(st);
  if (D == 3)
    k_near_mark<3><<<mb, kT, 0, st>>>(p.m, P, g.h, n, m1, flag);
  else
    k_near_mark<2><<<mb, kT, 0, st>>>(p.m, P, g.h, n, m1, flag);
  count_launch("near_mark", st);
  if ((e = check_launch())) return e;
  prof_begin(st);
  k_near_compact<<<blocks_for(nn), kT, 0, st>>>(nn, flag, inside, list, count, cap);
  count_launch("near_compact", st);
  if ((e = check_launch())) return e;
  const double mh = (double)m1 * g.h;
  const double guard = 0.999 * s;
  // Error of d2 in float32 for a point of the 3^d cells (|dx_c| <= 2s):
  // rounding the coordinates (|.| <= cmax) and the difference gives
  // |dxf - dx| <= 4 u cmax =: e, so the squares sum to within e (2 sum|dx| + d e)
  // of d2, and rounding the squares and sums adds 4 u d2; twice that.
  const double u = 5.9604644775390625e-8;  // 2^-24
  const double ec = 4.0 * u * cmax, rmax = 2.0 * s;
  const double ferr_d = 2.0 * (ec * (2.0 * D * rmax + D * ec) + 4.0 * u * D * rmax * rmax);
  float ferr = (float)ferr_d;  // rounded up
  if ((double)ferr < ferr_d) ferr = nextafterf(ferr, INFINITY);
  const int64_t fb = (cap + kFixT - 1) / kFixT;
  const int nfb = (int)(fb < 32 * 152 ? fb : 32 * 152);
  prof_begin(st);
  if (D == 3)
    k_near_fix<3><<<nfb, kFixT, 0, st>>>(list, count, cap, n, P, g.h, p.m, ub, uin, mh * mh,
                                         m2 * g.h, cw, nc, cstart, sorted, pts4, ferr,
                                         guard * guard, uout);
  else
    k_near_fix<2><<<nfb, kFixT, 0, st>>>(list, count, cap, n, P, g.h, p.m, ub, uin, mh * mh,
                                         m2 * g.h, cw, nc, cstart, sorted, pts4, ferr,
                                         guard * guard, uout);
  count_launch("near_fix", st);
  return check_launch();
}

}  // namespace ibdl
