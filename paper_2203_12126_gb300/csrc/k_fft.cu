// Periodic Helmholtz solve v = kappa L'^{-1} f, L' = I - kappa Delta_h, by
// diagonalising the 5-point (2D) / 7-point (3D) stencil with the FFT
// (Sec. 5.1: a periodic box "to make use of efficient ... methods").  The
// eigenvalue of L' on exp(2 pi i k.j / n) is
//     sigma(k) = 1 + (4 kappa / h^2) sum_c sin^2(pi k_c / n),
// so v = IFFT( FFT(f) * kappa / sigma ) with the 1/n^d of the inverse folded
// into the same multiplier.
//
// Passes (2D): [rows_fwd] spread into row tiles + x FFT + real-to-complex
// unpack, written as the transposed half spectrum; [pencils] y FFT, multiply,
// inverse y FFT on contiguous kx slabs; [rows_inv] complex-to-real x inverse.
// 3D adds a y FFT pass before and an inverse y pass after the z pass, which
// carries the multiplier.
//
// FFTs are shared-memory Stockham transforms (radix 4, one radix-2 stage for
// odd log2 n), ping-ponging between two shared buffers; twiddles come from a
// table exp(-2 pi i j / n) in global memory.  Two real rows are packed into
// one complex row (real part / imaginary part) and separated after the FFT
// with Z_k and conj(Z_{n-k}).
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
// i * a
template <typename C> __device__ __forceinline__ C cmuli(C a) {
  C r;
  r.x = -a.y;
  r.y = a.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}

// Stockham FFT of `npen` pencils of length n held in src (pencil-major).
// All threads of the block take part; the caller synchronises before the
// call.  Returns the buffer (src or dst) that holds the result; the block is
// synchronised on return.
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

// ---- fused spread + forward x pass ------------------------------------------
//
// Tile = R rows y0..y0+R-1 at plane z.  The tile's rows are zeroed (or
// seeded with coef_grid * f) in shared memory, then every (point, box node)
// pair of the tile's bin adds its share with a shared-memory atomic:
//
//   S~q at node (bx-1+a, by-1+b, bz-1+c) (Sec. 5.2, the centred difference of
//   the spread of q n, fused):  q w/h^d [ nx dW_x[a] W_y[b-1] W_z[c-1]
//        + ny W_x[a-1] dW_y[b] W_z[c-1] + nz W_x[a-1] W_y[b-1] dW_z[c] ],
//   dW[a] = (W[a] - W[a-2]) / (2h),  W[t] = 0 outside t = 0..3;
//   S v at the same node:  v w/h^d W_x[a-1] W_y[b-1] W_z[c-1].
template <typename T, int D>
__global__ void __launch_bounds__(1024) k_rows_fwd(GridDesc g, PointData p, Bins b,
                                                   SpreadSrc src, cx_t<T>* __restrict__ spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   double* __restrict__ write_grid) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, mask = n - 1, R = b.rows, npen = R >> 1;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)npen * n;
  T* rows = reinterpret_cast<T*>(bufA);  // row r, column x at [((r>>1)*n + x)*2 + (r&1)]
  const int ngroups = n / R;
  const int tile = blockIdx.x;
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

  const int lo = b.start[tile], hi = b.start[tile + 1];
  const int total = (hi - lo) * (kBoxSide * kBoxSide);
  const T inv2h = (T)(0.5 / g.h);
  for (int e = tid; e < total; e += nt) {
    const int pi = e / (kBoxSide * kBoxSide);
    const int l = e - pi * (kBoxSide * kBoxSide);
    const int a = l % kBoxSide, bb = l / kBoxSide;
    const int i = b.pts[lo + pi];
    const int ry = ((p.base[1][i] - 1 + bb) & mask) - y0;
    if ((unsigned)ry >= (unsigned)R) continue;
    int cz = 1;
    if (D == 3) {
      cz = (z - (p.base[2][i] - 1)) & mask;
      if (cz >= kBoxSide) continue;
    }
    const T wxa = wload<T>(p, 0, a - 1, i);
    const T wyb = wload<T>(p, 1, bb - 1, i);
    const T wzc = (D == 3) ? wload<T>(p, 2, cz - 1, i) : (T)1;
    T val = 0;
    if (src.q_div) {
      const T amp = (T)(src.coef_div * src.q_div[i] * p.w[i]);
      const T dx = (wload<T>(p, 0, a, i) - wload<T>(p, 0, a - 2, i)) * inv2h;
      const T dy = (wload<T>(p, 1, bb, i) - wload<T>(p, 1, bb - 2, i)) * inv2h;
      T s = (T)p.nrm[0][i] * dx * wyb * wzc + (T)p.nrm[1][i] * wxa * dy * wzc;
      if (D == 3) {
        const T dz = (wload<T>(p, 2, cz, i) - wload<T>(p, 2, cz - 2, i)) * inv2h;
        s += (T)p.nrm[2][i] * wxa * wyb * dz;
      }
      val += amp * s;
    }
    if (src.v_plain) val += (T)(src.coef_plain * src.v_plain[i] * p.w[i]) * wxa * wyb * wzc;
    if (val != (T)0) {
      const int x = (p.base[0][i] - 1 + a) & mask;
      atomicAdd(&rows[((size_t)(ry >> 1) * n + x) * 2 + (ry & 1)], val);
    }
  }
  __syncthreads();

  if (write_grid) {
    for (int e = tid; e < R * n; e += nt) {
      const int r = e / n, x = e - r * n;
      write_grid[row0 + (size_t)r * n + x] = (double)rows[((size_t)(r >> 1) * n + x) * 2 + (r & 1)];
    }
    return;
  }

  C* res = fft_pencils<T, false>(bufA, bufB, n, npen, tw);

  // Z = FFT(a + i b): A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i)
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
}

// ---- pencil passes on the transposed half spectrum -----------------------
struct PencilLayout {
  int64_t gstride, bstride, estride;
  int pg;        // pencils per group
  int npencils;  // total pencils
  int c;         // pencils per block
};

// MODE 0: forward, 1: inverse, 2: forward, multiply, inverse.
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_pencils(GridDesc g, PencilLayout L,
                                                 cx_t<T>* __restrict__ data,
                                                 const cx_t<T>* __restrict__ tw,
                                                 const T* __restrict__ s2, T cfac, T scale0) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, c = L.c;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)c * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p0 = blockIdx.x * c;
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
      v = data[gi * L.gstride + q * L.bstride + t * L.estride];
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
}

// ---- inverse x pass: complex-to-real ----------------------------------------
// Rebuild the full spectrum of the packed pair a + i b from the half
// spectra A, B (Hermitian): Z_k = A_k + i B_k, Z_{n-k} = conj A_k + i conj B_k.
template <typename T, int D, typename OutT>
__global__ void __launch_bounds__(1024) k_rows_inv(GridDesc g, Bins b,
                                                   const cx_t<T>* __restrict__ spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   OutT* __restrict__ out) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, R = b.rows, npen = R >> 1;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)npen * n;
  const int ngroups = n / R;
  const int tile = blockIdx.x;
  const int z = (D == 3) ? tile / ngroups : 0;
  const int y0 = (tile % ngroups) * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = n >> 1;
  const size_t slab = (D == 3) ? (size_t)n * n : (size_t)n;
  const size_t pos0 = (size_t)z * n + y0;

  for (int e = tid; e < (half + 1) * npen; e += nt) {
    const int k = e / npen, a = e - k * npen;
    const C* in = spec + (size_t)k * slab + pos0 + 2 * a;
    C A = in[0], B = in[1];
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
}

// ---- launchers ----------------------------------------------------------------

static int rows_threads(int n, int npen) {
  int t = npen * n / 4;
  if (t < 64) t = 64;
  if (t > 1024) t = 1024;
  return t;
}

template <typename T>
static size_t rows_smem(int n, int rows) {
  return 2 * (size_t)(rows / 2) * n * sizeof(cx_t<T>);
}

template <typename T>
cudaError_t launch_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                            const SpreadSrc& src, SpectralWs<T>& ws, double* write_grid,
                            cudaStream_t st) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem<T>(g.n, b.rows);
  const int thr = rows_threads(g.n, npen);
  prof_begin(st);
  if (g.dim == 2)
    k_rows_fwd<T, 2><<<b.ntiles, thr, smem, st>>>(g, p, b, src, ws.spec, ws.tw, write_grid);
  else
    k_rows_fwd<T, 3><<<b.ntiles, thr, smem, st>>>(g, p, b, src, ws.spec, ws.tw, write_grid);
  count_launch(sizeof(T) == 8 ? "rows_fwd_f64" : "rows_fwd_f32", st);
  return check_launch();
}

template <typename T, typename OutT>
cudaError_t launch_rows_inv(const GridDesc& g, const Bins& b, SpectralWs<T>& ws, OutT* out,
                            cudaStream_t st) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem<T>(g.n, b.rows);
  const int thr = rows_threads(g.n, npen);
  prof_begin(st);
  if (g.dim == 2)
    k_rows_inv<T, 2, OutT><<<b.ntiles, thr, smem, st>>>(g, b, ws.spec, ws.tw, out);
  else
    k_rows_inv<T, 3, OutT><<<b.ntiles, thr, smem, st>>>(g, b, ws.spec, ws.tw, out);
  count_launch(sizeof(T) == 8 ? "rows_inv_f64" : "rows_inv_f32", st);
  return check_launch();
}

template <typename T>
static PencilLayout pencil_layout(int n, int64_t gstride, int64_t bstride, int64_t estride,
                                  int pg, int npencils) {
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

template <typename T, int MODE>
static cudaError_t run_pencils(const GridDesc& g, const PencilLayout& L, SpectralWs<T>& ws,
                               cudaStream_t st) {
  const int blocks = (L.npencils + L.c - 1) / L.c;
  int thr = L.c * g.n / 4;
  if (thr < 64) thr = 64;
  if (thr > 512) thr = 512;
  const size_t smem = 2 * (size_t)L.c * g.n * sizeof(cx_t<T>);
  const double nd = g.dim == 3 ? (double)g.n * g.n * g.n : (double)g.n * g.n;
  const T cfac = (T)(4.0 * g.kappa / (g.h * g.h));
  const T scale0 = (T)(g.kappa / nd);
  prof_begin(st);
  k_pencils<T, MODE><<<blocks, thr, smem, st>>>(g, L, ws.spec, ws.tw, ws.s2, cfac, scale0);
  static const char* names[2][3] = {{"pencils_fwd_f32", "pencils_inv_f32", "pencils_solve_f32"},
                                    {"pencils_fwd_f64", "pencils_inv_f64", "pencils_solve_f64"}};
  count_launch(names[sizeof(T) == 8 ? 1 : 0][MODE], st);
  return check_launch();
}

template <typename T>
cudaError_t launch_spectral_solve(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st) {
  const int n = g.n, half = n / 2;
  cudaError_t e;
  if (g.dim == 2) {
    // slab kx = contiguous y pencil
    PencilLayout L = pencil_layout<T>(n, n, 0, 1, 1, half + 1);
    return run_pencils<T, 2>(g, L, ws, st);
  }
  const int64_t n2 = (int64_t)n * n;
  PencilLayout Ly = pencil_layout<T>(n, n2, n, 1, n, (half + 1) * n);   // (kx, z) -> y
  PencilLayout Lz = pencil_layout<T>(n, n2, 1, n, n, (half + 1) * n);   // (kx, y) -> z
  if ((e = run_pencils<T, 0>(g, Ly, ws, st))) return e;
  if ((e = run_pencils<T, 2>(g, Lz, ws, st))) return e;
  return run_pencils<T, 1>(g, Ly, ws, st);
}

template <typename T>
int fft_kernels_per_solve(int dim) {
  return dim == 2 ? 3 : 5;
}

template <typename F>
static void raise_smem(F* f) {
  cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
}

cudaError_t configure_fft_kernels(int, int) {
  static bool done = false;
  if (done) return cudaSuccess;
  raise_smem(k_rows_fwd<double, 2>);
  raise_smem(k_rows_fwd<double, 3>);
  raise_smem(k_rows_fwd<float, 2>);
  raise_smem(k_rows_fwd<float, 3>);
  raise_smem(k_rows_inv<double, 2, double>);
  raise_smem(k_rows_inv<double, 3, double>);
  raise_smem(k_rows_inv<float, 2, float>);
  raise_smem(k_rows_inv<float, 3, float>);
  raise_smem(k_rows_inv<float, 2, double>);
  raise_smem(k_rows_inv<float, 3, double>);
  raise_smem(k_pencils<double, 0>);
  raise_smem(k_pencils<double, 1>);
  raise_smem(k_pencils<double, 2>);
  raise_smem(k_pencils<float, 0>);
  raise_smem(k_pencils<float, 1>);
  raise_smem(k_pencils<float, 2>);
  done = true;
  return cudaGetLastError();
}

template cudaError_t launch_rows_fwd<double>(const GridDesc&, const PointData&, const Bins&,
                                             const SpreadSrc&, SpectralWs<double>&, double*,
                                             cudaStream_t);
template cudaError_t launch_rows_fwd<float>(const GridDesc&, const PointData&, const Bins&,
                                            const SpreadSrc&, SpectralWs<float>&, double*,
                                            cudaStream_t);
template cudaError_t launch_rows_inv<double, double>(const GridDesc&, const Bins&,
                                                     SpectralWs<double>&, double*, cudaStream_t);
template cudaError_t launch_rows_inv<float, float>(const GridDesc&, const Bins&,
                                                   SpectralWs<float>&, float*, cudaStream_t);
template cudaError_t launch_rows_inv<float, double>(const GridDesc&, const Bins&,
                                                    SpectralWs<float>&, double*, cudaStream_t);
template cudaError_t launch_spectral_solve<double>(const GridDesc&, SpectralWs<double>&,
                                                   cudaStream_t);
template cudaError_t launch_spectral_solve<float>(const GridDesc&, SpectralWs<float>&,
                                                  cudaStream_t);
template int fft_kernels_per_solve<double>(int);
template int fft_kernels_per_solve<float>(int);

}  // namespace ibdl
