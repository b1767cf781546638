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
#include "ibdl_device.cuh"

namespace ibdl {

template <typename T, int D>
__global__ void __launch_bounds__(512) k_rows_fwd(GridDesc g, PointData p, Bins b,
                                                   SpreadSrc src, cx_t<T>* spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   double* write_grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  phase_rows_fwd<T, D>(g, p, b, src, spec, tw, write_grid, blockIdx.x, smem_raw);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_pencils(GridDesc g, PencilLayout L, cx_t<T>* data,
                                                 const cx_t<T>* __restrict__ tw,
                                                 const T* __restrict__ s2, T cfac, T scale0,
                                                 const int* zskip, int ngroups,
                                                 const unsigned char* zempty) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  phase_pencils<T, MODE>(g, L, data, tw, s2, cfac, scale0, blockIdx.x, smem_raw, zskip,
                         ngroups, zempty);
}

template <typename T, int D, typename OutT>
__global__ void __launch_bounds__(512) k_rows_inv(GridDesc g, Bins b, const cx_t<T>* spec,
                                                   const cx_t<T>* __restrict__ tw,
                                                   OutT* out, bool band_only) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  phase_rows_inv<T, D, OutT>(g, b, spec, tw, out, blockIdx.x, smem_raw, band_only);
}

// ---- launchers ----------------------------------------------------------------

// Threads per block.  Pencil items: one per butterfly of the FFT pass with
// the most butterflies (n over the smallest radix of the plan, per pencil)
// -- more would idle in the FFT passes and thin the per-thread work over
// which an item's fixed cost is spread.  Row tiles take n/8 per pencil:
// their spread stage wants the extra threads.
static int clamp_threads(int t) { return t < 64 ? 64 : (t > 512 ? 512 : t); }

static int pencil_threads(int n, int c) {
  const int lg = ilog2(n);
  int min_lr = 4;
  for (int s = 0; s < plan_npass(lg); ++s)
    if (plan_lr(lg, s) < min_lr) min_lr = plan_lr(lg, s);
  return clamp_threads(c * (n >> min_lr));
}

static int rows_threads(int n, int npen) { return clamp_threads(npen * n / 8); }

template <typename T>
cudaError_t launch_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                            const SpreadSrc& src, SpectralWs<T>& ws, double* write_grid,
                            cudaStream_t st) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem_bytes<T>(g.n, b.rows);
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
                            cudaStream_t st, bool band_only) {
  const int npen = b.rows / 2;
  const size_t smem = rows_smem_bytes<T>(g.n, b.rows);
  const int thr = rows_threads(g.n, npen);
  prof_begin(st);
  if (g.dim == 2)
    k_rows_inv<T, 2, OutT><<<b.ntiles, thr, smem, st>>>(g, b, ws.spec, ws.tw, out, band_only);
  else
    k_rows_inv<T, 3, OutT><<<b.ntiles, thr, smem, st>>>(g, b, ws.spec, ws.tw, out, band_only);
  count_launch(sizeof(T) == 8 ? "rows_inv_f64" : "rows_inv_f32", st);
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
  k_pencils<T, MODE><<<blocks, thr, smem, st>>>(g, L, ws.spec, ws.tw, ws.s2, cfac, scale0,
                                                 zskip, ngroups, zempty);
  static const char* names[2][3] = {{"pencils_fwd_f32", "pencils_inv_f32", "pencils_solve_f32"},
                                    {"pencils_fwd_f64", "pencils_inv_f64", "pencils_solve_f64"}};
  count_launch(names[sizeof(T) == 8 ? 1 : 0][MODE], st);
  return check_launch();
}

template <typename T>
cudaError_t launch_spectral_solve(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st,
                                  const Bins* skip, bool skip_fwd) {
  cudaError_t e;
  if (g.dim == 2) return run_pencils<T, 2>(g, solve_layout<T>(2, g.n, 1), ws, st);
  PencilLayout Ly = solve_layout<T>(3, g.n, 0);   // (kx, z) -> y
  PencilLayout Lz = solve_layout<T>(3, g.n, 1);   // (kx, y) -> z
  const int ngroups = g.n / (skip ? skip->rows : 1);
  if ((e = run_pencils<T, 0>(g, Ly, ws, st, (skip && skip_fwd) ? skip->start : nullptr,
                             ngroups)))
    return e;
  if ((e = run_pencils<T, 2>(g, Lz, ws, st, nullptr, 0,
                             (skip && skip_fwd) ? skip->zempty : nullptr)))
    return e;
  return run_pencils<T, 1>(g, Ly, ws, st, skip ? skip->start : nullptr, ngroups);
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
template cudaError_t launch_spectral_solve<float>(const GridDesc&, SpectralWs<float>&,
                                                  cudaStream_t, const Bins*, bool);
template int fft_kernels_per_solve<double>(int);
template int fft_kernels_per_solve<float>(int);

}  // namespace ibdl
