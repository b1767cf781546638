// Periodic Helmholtz solve v = kappa L'^{-1} f, L' = I - kappa Delta_h, by
// diagonalising the 5-point (2D) / 7-point (3D) stencil with the FFT on the
// periodic box of Sec. 5.1.  The eigenvalue of L' on exp(2 pi i k.j / n) is
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
// FFTs are shared-memory Stockham transforms (ibdl_device.cuh): a first pass
// of radix 16, then the remaining bits of log2 n split as evenly as possible
// into passes of radix <= 16 (1024 = 16 * 8 * 8, 256 = 16 * 16), ping-ponging
// between two shared buffers, with per-pass twiddle tables.  Two real rows
// are packed into one complex row (real part / imaginary part) and separated
// after the FFT with Z_k and conj(Z_{n-k}).
#include <mutex>

#include "ibdl_device.cuh"

namespace ibdl {

template <typename T, int D>
__global__ void __launch_bounds__(512) k_rows_fwd(GridDesc g, PointData p, Bins b,
                                                   SpreadSrc src, cx_t<T>* spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   double* write_grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  phase_rows_fwd<T, D>(g, p, b, src, spec, tw, write_grid, blockIdx.x, smem_raw);
  pdl_release();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_pencils(GridDesc g, PencilLayout L, cx_t<T>* data,
                                                 const cx_t<T>* __restrict__ tw,
                                                 const T* __restrict__ s2, T cfac, T scale0,
                                                 const int* zskip, int ngroups,
                                                 const unsigned char* zempty) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  phase_pencils<T, MODE>(g, L, data, tw, s2, cfac, scale0, blockIdx.x, smem_raw, zskip,
                         ngroups, zempty);
  pdl_release();
}

template <typename T, int D, typename OutT>
__global__ void __launch_bounds__(512) k_rows_inv(GridDesc g, Bins b, const cx_t<T>* spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   OutT* out, bool band_only) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  phase_rows_inv<T, D, OutT>(g, b, spec, tw, out, blockIdx.x, smem_raw, band_only);
  pdl_release();
}

// ---- launchers ----------------------------------------------------------------

// Threads per block.  Pencil items: one per butterfly of the FFT pass with
// the most butterflies (n over the smallest radix of the plan, per pencil)
// -- more would idle in the FFT passes and thin the per-thread work over
// which an item's fixed cost is spread.  Row tiles take n/8 per pencil:
// their spread stage wants the extra threads.
static int rows_threads(int n, int npen) { return clamp_threads(npen * n / 8); }

// launch-profile label by element type: float, double, double-float
template <typename T> static const char* tag3(const char* f32, const char* f64, const char* d2) {
  return std::is_same<T, dd>::value ? d2 : (sizeof(T) == 8 ? f64 : f32);
}

template <typename T>
cudaError_t launch_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                            const SpreadSrc& src, SpectralWs<T>& ws, double* write_grid,
                            cudaStream_t st) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem_bytes<T>(g.n, b.rows);
  const int thr = rows_threads(g.n, npen);
  prof_begin(st);
  if (g.dim == 2)
    launch_dependent(k_rows_fwd<T, 2>, b.ntiles, thr, smem, st, g, p, b, src, ws.spec,
                     (const cx_t<T>*)ws.tw, write_grid);
  else
    launch_dependent(k_rows_fwd<T, 3>, b.ntiles, thr, smem, st, g, p, b, src, ws.spec,
                     (const cx_t<T>*)ws.tw, write_grid);
  count_launch(tag3<T>("rows_fwd_f32", "rows_fwd_f64", "rows_fwd_dd"), st);
  return check_launch();
}

template <typename T, typename OutT>
cudaError_t launch_rows_inv(const GridDesc& g, const Bins& b, SpectralWs<T>& ws, OutT* out,
                            cudaStream_t st, bool band_only) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem_bytes<T>(g.n, b.rows);
  // float32 x inverse tiles (no spread stage): one thread per radix-16
  // butterfly, twice the resident tiles (C3 x inverse 20.3 -> 17.5 us; the C2
  // one unchanged); float64 and double-float keep n/8 per pencil
  const int thr = std::is_same<T, float>::value ? clamp_threads(npen * g.n / 16)
                                                : rows_threads(g.n, npen);
  prof_begin(st);
  if (g.dim == 2)
    launch_dependent(k_rows_inv<T, 2, OutT>, b.ntiles, thr, smem, st, g, b,
                     (const cx_t<T>*)ws.spec, (const cx_t<T>*)ws.tw, out, band_only);
  else
    launch_dependent(k_rows_inv<T, 3, OutT>, b.ntiles, thr, smem, st, g, b,
                     (const cx_t<T>*)ws.spec, (const cx_t<T>*)ws.tw, out, band_only);
  count_launch(tag3<T>("rows_inv_f32", "rows_inv_f64", "rows_inv_dd"), st);
  return check_launch();
}

template <typename T, int MODE>
static cudaError_t run_pencils(const GridDesc& g, const PencilLayout& L, SpectralWs<T>& ws,
                               cudaStream_t st, const int* zskip = nullptr, int ngroups = 0,
                               const unsigned char* zempty = nullptr) {
  const int blocks = (L.npencils + L.c - 1) / L.c;
  const int thr = pencil_threads(g.n, L.c);
  const size_t smem = pencil_smem_bytes<T>(L, g.n);
  const T cfac = (T)symbol_cfac(g);
  const T scale0 = (T)symbol_scale0(g);
  prof_begin(st);
  launch_dependent(k_pencils<T, MODE>, blocks, thr, smem, st, g, L, ws.spec,
                   (const cx_t<T>*)ws.tw, (const T*)ws.s2, cfac, scale0, zskip, ngroups, zempty);
  static const char* names[3][3] = {{"pencils_fwd_f32", "pencils_inv_f32", "pencils_solve_f32"},
                                    {"pencils_fwd_f64", "pencils_inv_f64", "pencils_solve_f64"},
                                    {"pencils_fwd_dd", "pencils_inv_dd", "pencils_solve_dd"}};
  count_launch(names[std::is_same<T, dd>::value ? 2 : (sizeof(T) == 8 ? 1 : 0)][MODE], st);
  return check_launch();
}

template <typename T>
cudaError_t launch_spectral_solve(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st,
                                  const Bins* skip, bool skip_fwd) {
  cudaError_t e;
  if (g.dim == 2) return run_pencils<T, 2>(g, solve_layout<T>(g, 1), ws, st);
  PencilLayout Ly = solve_layout<T>(g, 0);   // (kx, z) -> y
  PencilLayout Lz = solve_layout<T>(g, 1);   // (kx, y) -> z
  const int ngroups = g.n / (skip ? skip->rows : 1);
  if ((e = run_pencils<T, 0>(g, Ly, ws, st, (skip && skip_fwd) ? skip->start : nullptr,
                             ngroups)))
    return e;
  const unsigned char* zfw = (skip && skip_fwd) ? skip->zempty : nullptr;
  if constexpr (std::is_same<T, float>::value) {
    // float32: the z pass with its pencils staged by bulk tensor copies
    if (ws.zmap) {
      if ((e = launch_zsolve_tma<T>(g, ws, zfw, st))) return e;
      return run_pencils<T, 1>(g, Ly, ws, st, skip ? skip->start : nullptr, ngroups);
    }
  }
  if ((e = run_pencils<T, 2>(g, Lz, ws, st, nullptr, 0, zfw))) return e;
  return run_pencils<T, 1>(g, Ly, ws, st, skip ? skip->start : nullptr, ngroups);
}

template <typename T>
cudaError_t launch_pencils_forward(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st) {
  if (g.dim == 2) return run_pencils<T, 0>(g, solve_layout<T>(g, 1), ws, st);
  cudaError_t e = run_pencils<T, 0>(g, solve_layout<T>(g, 0), ws, st);
  if (e) return e;
  return run_pencils<T, 0>(g, solve_layout<T>(g, 1), ws, st);
}

template <typename T>
cudaError_t launch_pencils_inverse(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st) {
  if (g.dim == 2) return run_pencils<T, 1>(g, solve_layout<T>(g, 1), ws, st);
  cudaError_t e = run_pencils<T, 1>(g, solve_layout<T>(g, 1), ws, st);
  if (e) return e;
  return run_pencils<T, 1>(g, solve_layout<T>(g, 0), ws, st);
}

// Combination of spectral source terms on the transposed half spectrum
// ([kx][y] in 2D, [kx][z][y] in 3D; kx = 0..n/2).  Signed wavenumber of
// index k: k (k < n/2), k - n (k > n/2); the Nyquist index n/2 gets a zero
// first derivative and (pi/2)^2 in the Laplacian.
template <typename T>
__global__ void __launch_bounds__(256) k_spec_combine(int dim, int n, cx_t<T>* __restrict__ spec,
                                                      cx_t<T>* __restrict__ acc, int64_t count,
                                                      int deriv_c, int accumulate, int final,
                                                      T two_pi_over_L, T c0, T cfac, T scale0) {
  const int lg = 31 - __clz(n);
  const int half = n >> 1;
  const T pin = (T)3.14159265358979323846 / (T)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k[3];
    k[1] = (int)(e & (n - 1));  // y
    if (dim == 2) {
      k[0] = (int)(e >> lg);
      k[2] = 0;
    } else {
      k[2] = (int)((e >> lg) & (n - 1));  // z
      k[0] = (int)(e >> (2 * lg));
    }
    cx_t<T> t = spec[e];
    if (deriv_c >= 0) {
      const int kc = k[deriv_c];
      const T f = kc == half ? (T)0 : two_pi_over_L * (T)(kc < half ? kc : kc - n);
      const T re = -f * t.y, im = f * t.x;
      t.x = re;
      t.y = im;
    }
    if (accumulate) {
      const cx_t<T> a = acc[e];
      t.x += a.x;
      t.y += a.y;
    }
    if (final) {
      T ssum = 0;
      for (int c = 0; c < dim; ++c) {
        const T kt = (T)(k[c] <= half ? k[c] : k[c] - n) * pin;
        ssum += kt * kt;
      }
      const T den = c0 + cfac * ssum;
      const T f = den > (T)0 ? scale0 / den : (T)0;
      t.x *= f;
      t.y *= f;
      spec[e] = t;
    } else {
      acc[e] = t;
    }
  }
}

template <typename T>
cudaError_t launch_spec_combine(const GridDesc& g, SpectralWs<T>& ws, int deriv_c,
                                bool accumulate, bool final, cudaStream_t st) {
  const int64_t count = (int64_t)(g.n / 2 + 1) * g.n * (g.dim == 3 ? g.n : 1);
  int64_t blocks = (count + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  const double L = g.h * g.n;
  prof_begin(st);
  k_spec_combine<T><<<(int)blocks, 256, 0, st>>>(
      g.dim, g.n, ws.spec, ws.acc, count, deriv_c, accumulate ? 1 : 0, final ? 1 : 0,
      (T)(6.283185307179586476925 / L), (T)(g.poisson ? 0.0 : 1.0), (T)symbol_cfac(g),
      (T)symbol_scale0(g));
  count_launch(sizeof(T) == 4 ? "spec_combine_f32" : "spec_combine_f64", st);
  return check_launch();
}

template cudaError_t launch_pencils_forward<double>(const GridDesc&, SpectralWs<double>&,
                                                    cudaStream_t);
template cudaError_t launch_pencils_forward<float>(const GridDesc&, SpectralWs<float>&,
                                                   cudaStream_t);
template cudaError_t launch_pencils_inverse<double>(const GridDesc&, SpectralWs<double>&,
                                                    cudaStream_t);
template cudaError_t launch_pencils_inverse<float>(const GridDesc&, SpectralWs<float>&,
                                                   cudaStream_t);
template cudaError_t launch_spec_combine<double>(const GridDesc&, SpectralWs<double>&, int, bool,
                                                 bool, cudaStream_t);
template cudaError_t launch_spec_combine<float>(const GridDesc&, SpectralWs<float>&, int, bool,
                                                bool, cudaStream_t);

template <typename T>
int fft_kernels_per_solve(int dim) {
  return dim == 2 ? 3 : 5;
}

template <typename F>
static void raise_smem(F* f) {
  cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
}

// Raises the dynamic shared-memory limit of every FFT kernel, once per
// device (the attribute is per device), with that device current.
cudaError_t configure_fft_kernels(int, int) {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
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
  raise_smem(k_rows_fwd<dd, 2>);
  raise_smem(k_rows_fwd<dd, 3>);
  raise_smem(k_rows_inv<dd, 2, double>);
  raise_smem(k_rows_inv<dd, 3, double>);
  raise_smem(k_pencils<dd, 0>);
  raise_smem(k_pencils<dd, 1>);
  raise_smem(k_pencils<dd, 2>);
  e = cudaGetLastError();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

template cudaError_t launch_rows_fwd<double>(const GridDesc&, const PointData&, const Bins&,
                                             const SpreadSrc&, SpectralWs<double>&, double*,
                                             cudaStream_t);
template cudaError_t launch_rows_fwd<float>(const GridDesc&, const PointData&, const Bins&,
                                            const SpreadSrc&, SpectralWs<float>&, double*,
                                            cudaStream_t);
template cudaError_t launch_rows_inv<double, double>(const GridDesc&, const Bins&,
                                                     SpectralWs<double>&, double*, cudaStream_t,
                                                     bool);
template cudaError_t launch_rows_inv<float, float>(const GridDesc&, const Bins&,
                                                   SpectralWs<float>&, float*, cudaStream_t,
                                                   bool);
template cudaError_t launch_rows_inv<float, double>(const GridDesc&, const Bins&,
                                                    SpectralWs<float>&, double*, cudaStream_t,
                                                    bool);
template cudaError_t launch_spectral_solve<double>(const GridDesc&, SpectralWs<double>&,
                                                   cudaStream_t, const Bins*, bool);
template cudaError_t launch_rows_fwd<dd>(const GridDesc&, const PointData&, const Bins&,
                                         const SpreadSrc&, SpectralWs<dd>&, double*,
                                         cudaStream_t);
template cudaError_t launch_rows_inv<dd, double>(const GridDesc&, const Bins&, SpectralWs<dd>&,
                                                 double*, cudaStream_t, bool);
template cudaError_t launch_spectral_solve<dd>(const GridDesc&, SpectralWs<dd>&, cudaStream_t,
                                               const Bins*, bool);
template cudaError_t launch_spectral_solve<float>(const GridDesc&, SpectralWs<float>&,
                                                  cudaStream_t, const Bins*, bool);
template int fft_kernels_per_solve<double>(int);
template int fft_kernels_per_solve<float>(int);

}  // namespace ibdl
