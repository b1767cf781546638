// Device-side building blocks of the IBDL matvec, shared by the one-kernel-
// per-pass launchers (k_fft.cu, k_points.cu) and the persistent solver
// (k_solver.cu).  Each "phase" function processes one work item (a row tile,
// a group of pencils, a point) with all threads of the calling block.
//
// Data produced by another block of the same launch (spectrum, grids, Krylov
// vectors) is read with ld.global.cg (__ldcg), which bypasses L1: inside a
// persistent kernel an SM's L1 may hold a line from an earlier phase.
#pragma once

#include "ibdl_internal.cuh"

namespace ibdl {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
  C r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
  C r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
template <typename C> __device__ __forceinline__ C cmuli(C a) {  // i * a
  C r;
  r.x = -a.y;
  r.y = a.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}

// Stockham FFT of `npen` pencils of length n held in src (pencil-major),
// radix 4 with one radix-2 stage when log2 n is odd.  All threads of the
// block take part; the caller synchronises before the call.  Returns the
// buffer (src or dst) holding the result; the block is synchronised.
template <typename T, bool INV>
__device__ cx_t<T>* fft_pencils(cx_t<T>* src, cx_t<T>* dst, int n, int npen,
                                const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  while (Ns < n) {
    if (((n / Ns) & 3) == 0) {
      const int nb = n >> 2;
      const int twstep = n / (Ns * 4);
      for (int e = tid; e < npen * nb; e += nt) {
        const int pen = e / nb;
        const int j = e - pen * nb;
        const int k = j & (Ns - 1);
        const C* x = src + (size_t)pen * n;
        C* y = dst + (size_t)pen * n;
        C a0 = x[j], a1 = x[j + nb], a2 = x[j + 2 * nb], a3 = x[j + 3 * nb];
        if (Ns > 1) {
          const int m1 = k * twstep;
          C w1 = tw[m1], w2 = tw[2 * m1], w3 = tw[3 * m1];
          if (INV) {
            w1 = cconj(w1);
            w2 = cconj(w2);
            w3 = cconj(w3);
          }
          a1 = cmul(a1, w1);
          a2 = cmul(a2, w2);
          a3 = cmul(a3, w3);
        }
        const C t0 = cadd(a0, a2), t1 = csub(a0, a2);
        const C t2 = cadd(a1, a3), it3 = cmuli(csub(a1, a3));
        const int o = (j - k) * 4 + k;
        y[o] = cadd(t0, t2);
        y[o + 2 * Ns] = csub(t0, t2);
        if (INV) {
          y[o + Ns] = cadd(t1, it3);
          y[o + 3 * Ns] = csub(t1, it3);
        } else {
          y[o + Ns] = csub(t1, it3);
          y[o + 3 * Ns] = cadd(t1, it3);
        }
      }
      Ns *= 4;
    } else {
      const int nb = n >> 1;
      const int twstep = n / (Ns * 2);
      for (int e = tid; e < npen * nb; e += nt) {
        const int pen = e / nb;
        const int j = e - pen * nb;
        const int k = j & (Ns - 1);
        const C* x = src + (size_t)pen * n;
        C* y = dst + (size_t)pen * n;
        C a0 = x[j], a1 = x[j + nb];
        if (Ns > 1) {
          C w1 = tw[k * twstep];
          if (INV) w1 = cconj(w1);
          a1 = cmul(a1, w1);
        }
        const int o = (j - k) * 2 + k;
        y[o] = cadd(a0, a1);
        y[o + Ns] = csub(a0, a1);
      }
      Ns *= 2;
    }
    __syncthreads();
    C* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

template <typename T> __device__ __forceinline__ T wload(const PointData& p, int c, int t, int i);
template <> __device__ __forceinline__ double wload<double>(const PointData& p, int c, int t,
                                                            int i) {
  return (t >= 0 && t < 4) ? p.W64[c][t * p.m + i] : 0.0;
}
template <> __device__ __forceinline__ float wload<float>(const PointData& p, int c, int t,
                                                          int i) {
  return (t >= 0 && t < 4) ? p.W32[c][t * p.m + i] : 0.0f;
}

template <typename T>
__host__ __device__ __forceinline__ size_t rows_smem_bytes(int n, int rows) {
  return 2 * (size_t)(rows / 2) * n * sizeof(cx_t<T>);
}

// ---- fused spread + forward x pass ------------------------------------------
//
// Tile = R rows y0..y0+R-1 at plane z.  The rows are zeroed (or seeded with
// coef_grid * f) in shared memory, then every (point, box node) pair of the
// tile's bin adds its share with a shared-memory atomic:
//
//   S~q at node (bx-1+a, by-1+b, bz-1+c) (Sec. 5.2, the centred difference of
//   the spread of q n, fused):  q w/h^d [ nx dW_x[a] W_y[b-1] W_z[c-1]
//        + ny W_x[a-1] dW_y[b] W_z[c-1] + nz W_x[a-1] W_y[b-1] dW_z[c] ],
//   dW[a] = (W[a] - W[a-2]) / (2h),  W[t] = 0 outside t = 0..3;
//   S v at the same node:  v w/h^d W_x[a-1] W_y[b-1] W_z[c-1].
//
// Then two real rows are packed as one complex row, FFT'd along x, separated
// (A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i)) and written
// to the transposed half spectrum spec[k][z][y], k = 0..n/2.
template <typename T, int D>
__device__ void phase_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                               const SpreadSrc& src, cx_t<T>* spec,
                               const cx_t<T>* __restrict__ tw, double* write_grid, int tile,
                               unsigned char* smem) {
  using C = cx_t<T>;
  const int n = g.n, mask = n - 1, R = b.rows, npen = R >> 1;
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)npen * n;
  T* rows = reinterpret_cast<T*>(bufA);  // row r, column x at [((r>>1)*n + x)*2 + (r&1)]
  const int ngroups = n / R;
  const int z = (D == 3) ? tile / ngroups : 0;
  const int y0 = (tile % ngroups) * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t row0 = ((size_t)z * n + y0) * n;

  for (int e = tid; e < R * n; e += nt) {
    const int r = e / n, x = e - r * n;
    T v = 0;
    if (src.f_grid) v = (T)(src.coef_grid * src.f_grid[row0 + (size_t)r * n + x]);
    rows[((size_t)(r >> 1) * n + x) * 2 + (r & 1)] = v;
  }
  __syncthreads();

  // One thread per (point, support row bb): the point's weights are loaded
  // once and its (up to) 6 x nodes on that row are added from registers.
  // With c = the plane offset (3D) and W[t] = 0 outside t = 0..3:
  //   node a: W_x[a-1] * cA + (W_x[a] - W_x[a-2]) * cB,
  //   cA = q w/h^d (ny dW_y[bb] W_z[c-1] + nz W_y[bb-1] dW_z[c]) + v w/h^d W_y[bb-1] W_z[c-1]
  //   cB = q w/h^d nx W_y[bb-1] W_z[c-1] / (2h).
  const int lo = b.start[tile], hi = b.start[tile + 1];
  const int units = (hi - lo) * kBoxSide;
  const T inv2h = (T)(0.5 / g.h);
  for (int e = tid; e < units; e += nt) {
    const int pi = e / kBoxSide, bb = e - pi * kBoxSide;
    const int i = b.pts[lo + pi];
    const int ry = ((p.base[1][i] - 1 + bb) & mask) - y0;
    if ((unsigned)ry >= (unsigned)R) continue;
    int cz = 1;
    if (D == 3) {
      cz = (z - (p.base[2][i] - 1)) & mask;
      if (cz >= kBoxSide) continue;
    }
    const T wyb = wload<T>(p, 1, bb - 1, i);
    const T dyb = (wload<T>(p, 1, bb, i) - wload<T>(p, 1, bb - 2, i)) * inv2h;
    T wzc = (T)1, dzc = (T)0;
    if (D == 3) {
      wzc = wload<T>(p, 2, cz - 1, i);
      dzc = (wload<T>(p, 2, cz, i) - wload<T>(p, 2, cz - 2, i)) * inv2h;
    }
    T cA = 0, cB = 0;
    if (src.q_div) {
      const T amp = (T)(src.coef_div * __ldcg(src.q_div + i) * p.w[i]);
      T t = (T)p.nrm[1][i] * dyb * wzc;
      if (D == 3) t += (T)p.nrm[2][i] * wyb * dzc;
      cA = amp * t;
      cB = amp * (T)p.nrm[0][i] * wyb * wzc * inv2h;
    }
    if (src.v_plain)
      cA += (T)(src.coef_plain * __ldcg(src.v_plain + i) * p.w[i]) * wyb * wzc;
    if (cA == (T)0 && cB == (T)0) continue;
    T wx[6];
    wx[0] = 0;
    wx[5] = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) wx[t + 1] = wload<T>(p, 0, t, i);  // wx[k] = W_x[k-1]
    T* rowp = rows + (size_t)(ry >> 1) * n * 2 + (ry & 1);
    const int xb = p.base[0][i] - 1;
#pragma unroll
    for (int a = 0; a < kBoxSide; ++a) {
      // W_x[a] - W_x[a-2] = wx[a+1] - wx[a-1]
      const T wa1 = wx[a];
      const T wa = (a + 1 < 6) ? wx[a + 1] : (T)0;
      const T wam2 = (a >= 1) ? wx[a - 1] : (T)0;
      const T val = wa1 * cA + (wa - wam2) * cB;
      if (val != (T)0) atomicAdd(rowp + (size_t)((xb + a) & mask) * 2, val);
    }
  }
  __syncthreads();

  if (write_grid) {
    for (int e = tid; e < R * n; e += nt) {
      const int r = e / n, x = e - r * n;
      write_grid[row0 + (size_t)r * n + x] =
          (double)rows[((size_t)(r >> 1) * n + x) * 2 + (r & 1)];
    }
    __syncthreads();
    return;
  }

  C* res = fft_pencils<T, false>(bufA, bufB, n, npen, tw);

  const int half = n >> 1;
  const size_t slab = (D == 3) ? (size_t)n * n : (size_t)n;
  const size_t pos0 = (size_t)z * n + y0;
  for (int e = tid; e < (half + 1) * npen; e += nt) {
    const int k = e / npen, a = e - k * npen;
    const C zk = res[(size_t)a * n + k];
    const C zm = res[(size_t)a * n + ((n - k) & mask)];
    C A, B;
    A.x = (T)0.5 * (zk.x + zm.x);
    A.y = (T)0.5 * (zk.y - zm.y);
    B.x = (T)0.5 * (zk.y + zm.y);
    B.y = (T)-0.5 * (zk.x - zm.x);
    C* out = spec + (size_t)k * slab + pos0 + 2 * a;
    out[0] = A;
    out[1] = B;
  }
  __syncthreads();  // the block's shared buffers are reused by the next item
}

// ---- pencil passes on the transposed half spectrum -----------------------
struct PencilLayout {
  int64_t gstride, bstride, estride;
  int pg;        // pencils per group
  int npencils;  // total pencils
  int c;         // pencils per block
};

template <typename T>
__host__ __device__ inline PencilLayout pencil_layout(int n, int64_t gstride, int64_t bstride,
                                                      int64_t estride, int pg, int npencils) {
  PencilLayout L;
  L.gstride = gstride;
  L.bstride = bstride;
  L.estride = estride;
  L.pg = pg;
  L.npencils = npencils;
  int c = (int)(65536 / (2 * (size_t)n * sizeof(cx_t<T>)));
  if (c < 1) c = 1;
  if (c > 16) c = 16;
  if (estride != 1 && c > pg) c = pg;
  L.c = c;
  return L;
}

// The pencil passes of one Helmholtz solve: 2D has one (kx slabs, y pencils,
// forward + multiply + inverse); 3D has three: y forward on (kx, z),
// z forward + multiply + inverse on (kx, y), y inverse on (kx, z).
template <typename T>
__host__ __device__ inline PencilLayout solve_layout(int dim, int n, int which) {
  const int half = n / 2;
  if (dim == 2) return pencil_layout<T>(n, n, 0, 1, 1, half + 1);
  const int64_t n2 = (int64_t)n * n;
  if (which == 1) return pencil_layout<T>(n, n2, 1, n, n, (half + 1) * n);
  return pencil_layout<T>(n, n2, n, 1, n, (half + 1) * n);
}

template <typename T>
__host__ __device__ inline size_t pencil_smem_bytes(const PencilLayout& L, int n) {
  return 2 * (size_t)L.c * n * sizeof(cx_t<T>);
}

// MODE 0: forward, 1: inverse, 2: forward, multiply by
// scale0 / (1 + cfac * sum_c sin^2(pi k_c / n)), inverse.
template <typename T, int MODE>
__device__ void phase_pencils(const GridDesc& g, const PencilLayout& L, cx_t<T>* data,
                              const cx_t<T>* __restrict__ tw, const T* __restrict__ s2,
                              T cfac, T scale0, int blk, unsigned char* smem) {
  using C = cx_t<T>;
  const int n = g.n, c = L.c;
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)c * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p0 = blk * c;
  const bool tfast = (L.estride == 1);

  for (int e = tid; e < c * n; e += nt) {
    int pl, t;
    if (tfast) {
      pl = e / n;
      t = e - pl * n;
    } else {
      t = e / c;
      pl = e - t * c;
    }
    const int p = p0 + pl;
    C v;
    v.x = 0;
    v.y = 0;
    if (p < L.npencils) {
      const int gi = p / L.pg, q = p - gi * L.pg;
      v = __ldcg(data + gi * L.gstride + q * L.bstride + t * L.estride);
    }
    bufA[(size_t)pl * n + t] = v;
  }
  __syncthreads();

  C* res = fft_pencils<T, MODE == 1>(bufA, bufB, n, c, tw);
  if (MODE == 2) {
    for (int e = tid; e < c * n; e += nt) {
      const int pl = e / n, t = e - pl * n;
      const int p = p0 + pl;
      if (p >= L.npencils) continue;
      const int gi = p / L.pg, q = p - gi * L.pg;
      T ssum = s2[gi] + s2[t];
      if (g.dim == 3) ssum += s2[q];
      const T f = scale0 / ((T)1 + cfac * ssum);
      C v = res[(size_t)pl * n + t];
      v.x *= f;
      v.y *= f;
      res[(size_t)pl * n + t] = v;
    }
    __syncthreads();
    C* other = (res == bufA) ? bufB : bufA;
    res = fft_pencils<T, true>(res, other, n, c, tw);
  }

  for (int e = tid; e < c * n; e += nt) {
    int pl, t;
    if (tfast) {
      pl = e / n;
      t = e - pl * n;
    } else {
      t = e / c;
      pl = e - t * c;
    }
    const int p = p0 + pl;
    if (p < L.npencils) {
      const int gi = p / L.pg, q = p - gi * L.pg;
      data[gi * L.gstride + q * L.bstride + t * L.estride] = res[(size_t)pl * n + t];
    }
  }
  __syncthreads();
}

// ---- inverse x pass: complex-to-real ----------------------------------------
// Rebuild the full spectrum of the packed pair a + i b from the half spectra
// A, B (Hermitian): Z_k = A_k + i B_k, Z_{n-k} = conj A_k + i conj B_k.
template <typename T, int D, typename OutT>
__device__ void phase_rows_inv(const GridDesc& g, const Bins& b, const cx_t<T>* spec,
                               const cx_t<T>* __restrict__ tw, OutT* out, int tile,
                               unsigned char* smem) {
  using C = cx_t<T>;
  const int n = g.n, R = b.rows, npen = R >> 1;
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)npen * n;
  const int ngroups = n / R;
  const int z = (D == 3) ? tile / ngroups : 0;
  const int y0 = (tile % ngroups) * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = n >> 1;
  const size_t slab = (D == 3) ? (size_t)n * n : (size_t)n;
  const size_t pos0 = (size_t)z * n + y0;

  for (int e = tid; e < (half + 1) * npen; e += nt) {
    const int k = e / npen, a = e - k * npen;
    const C* in = spec + (size_t)k * slab + pos0 + 2 * a;
    C A = __ldcg(in), B = __ldcg(in + 1);
    if (k == 0 || k == half) {
      A.y = 0;
      B.y = 0;
    }
    C zk, zm;
    zk.x = A.x - B.y;
    zk.y = A.y + B.x;
    bufA[(size_t)a * n + k] = zk;
    if (k > 0 && k < half) {
      zm.x = A.x + B.y;
      zm.y = B.x - A.y;
      bufA[(size_t)a * n + (n - k)] = zm;
    }
  }
  __syncthreads();
  C* res = fft_pencils<T, true>(bufA, bufB, n, npen, tw);
  const size_t row0 = ((size_t)z * n + y0) * n;
  for (int e = tid; e < R * n; e += nt) {
    const int r = e / n, x = e - r * n;
    const C v = res[(size_t)(r >> 1) * n + x];
    out[row0 + (size_t)r * n + x] = (OutT)((r & 1) ? v.y : v.x);
  }
  __syncthreads();
}

// ---- interpolation of one point ---------------------------------------------

template <typename T> __device__ __forceinline__ const T* wtab(const PointData& p, int c);
template <> __device__ __forceinline__ const double* wtab<double>(const PointData& p, int c) {
  return p.W64[c];
}
template <> __device__ __forceinline__ const float* wtab<float>(const PointData& p, int c) {
  return p.W32[c];
}

// sum over the 4^d taps of grid * prod_c W[c][t]  (S* u at X_i, Sec. 5.2)
template <typename T, int D>
__device__ __forceinline__ T interp_point(const GridDesc& g, const PointData& p, const T* grid,
                                          int i) {
  const int n = g.n, mask = n - 1, m = p.m;
  T wx[4], wy[4];
  const T* Wx = wtab<T>(p, 0);
  const T* Wy = wtab<T>(p, 1);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    wx[t] = Wx[t * m + i];
    wy[t] = Wy[t * m + i];
  }
  int col[4];
  const int bx = p.base[0][i], by = p.base[1][i];
#pragma unroll
  for (int t = 0; t < 4; ++t) col[t] = (bx + t) & mask;
  T acc = 0;
  if (D == 2) {
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
      const T* row = grid + (size_t)((by + ty) & mask) * n;
      T r = 0;
#pragma unroll
      for (int tx = 0; tx < 4; ++tx) r += __ldcg(row + col[tx]) * wx[tx];
      acc += r * wy[ty];
    }
  } else {
    const T* Wz = wtab<T>(p, 2);
    const int bz = p.base[2][i];
    for (int tz = 0; tz < 4; ++tz) {
      const T wz = Wz[tz * m + i];
      const T* plane = grid + (size_t)((bz + tz) & mask) * n * n;
      T pz = 0;
#pragma unroll
      for (int ty = 0; ty < 4; ++ty) {
        const T* row = plane + (size_t)((by + ty) & mask) * n;
        T r = 0;
#pragma unroll
        for (int tx = 0; tx < 4; ++tx) r += __ldcg(row + col[tx]) * wx[tx];
        pz += r * wy[ty];
      }
      acc += pz * wz;
    }
  }
  return acc;
}

}  // namespace ibdl
