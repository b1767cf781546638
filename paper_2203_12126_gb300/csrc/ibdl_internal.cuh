// Internal declarations shared by the translation units of libibdl.
//
// Data layout in device memory (one geometry handle):
//   points   : SoA float64 x/y/z, normals, weights (length m)
//   base[c]  : int32 floor((X_c - origin_c)/h) - 1, the first of the 4 nodes
//              per axis where phi((x_j - X_c)/h) can be non-zero (Sec. 5.2)
//   W[c][t]  : phi(base_c + t - s_c), t = 0..3, in float64 and float32
//   bins     : CSR lists of the points whose 6-node support box touches each
//              row tile (R consecutive y rows at one z), for the fused
//              spread + forward x-FFT kernel
//   grid     : real n^d field, x fastest
//   spectrum : after the x real-to-complex transform, stored TRANSPOSED as
//              (n/2 + 1) contiguous slabs, slab kx holding [z][y] (3D) or [y]
//              (2D); the y/z pencils are then contiguous or uniformly strided
//              and the Nyquist slab needs no special case.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ibdl.h"

namespace ibdl {

// Device ordinals with per-device state (kernel attributes, symbol addresses)
constexpr int kMaxDevices = 64;
// Largest grid per axis: 2D 2048 (a float64 pencil item of 4096 points would
// need more than the 227 KB of shared memory a block can have), 3D 512.
constexpr int kMaxN2 = 2048;
constexpr int kMaxN3 = 512;

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <typename T> using cx_t = typename Cx<T>::type;

// Double-float: the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 48 significant bits.  The float64-grade transforms of the refined
// solver's residual and right-hand side run in it: GB300 issues float32
// arithmetic at some sixty times its float64 rate.  Arithmetic (device,
// ibdl_device.cuh): Knuth's two-sum for sums, the fused-multiply-add form of
// Dekker's two-product for products, each renormalised by Dekker's fast
// two-sum.
struct __align__(8) dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ dd(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dd(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) cdd {
  dd x, y;
};
template <> struct Cx<dd> { using type = cdd; };

// Row tile height of the fused spread + x-FFT and x-iFFT kernels.
constexpr int kBoxSide = 6;   // nodes per axis touched by the centred
                              // difference of a 4-point delta

struct PointData {
  int m = 0;
  const double* X[3] = {nullptr, nullptr, nullptr};
  const double* nrm[3] = {nullptr, nullptr, nullptr};
  const double* w = nullptr;       // quadrature weight / h^d
  const float* nrm32[3] = {nullptr, nullptr, nullptr};  // float copies for the
  const float* w32 = nullptr;                            // float32 spread
  const int* base[3] = {nullptr, nullptr, nullptr};
  const double* W64[3] = {nullptr, nullptr, nullptr};  // [t*m + i]
  const float* W32[3] = {nullptr, nullptr, nullptr};
};

struct Bins {
  int rows = 4;              // R: y rows per tile (even)
  int ntiles = 0;            // n^(d-2) * (n / R)
  const int* start = nullptr;  // ntiles + 1
  const int* pts = nullptr;    // per tile: points in fill order (about index order)
  const int* spts = nullptr;   // the same lists sorted by first support column, then
                               // index (the gather spread's order)
  const unsigned char* zempty = nullptr;  // 3D: 1 for z planes no point touches
};

struct GridDesc {
  int dim = 2;
  int n = 0;
  int log2n = 0;
  double h = 0, kappa = 0;
  double inv2h = 0;  // 1 / (2h) of the centred difference, set with h (a
                     // float64 divide per thread is slow on GB300's FP64 pipe)
  double origin[3] = {0, 0, 0};
  int delta = 0;
  // 1: the Poisson limit kappa = inf (Sec. 5.4): the solve applies the
  // mean-zero -Delta_0^{-1} (symbol 1 / lambda(k), the k = 0 mode dropped)
  // in place of kappa L'^{-1}.
  int poisson = 0;
  // 1: the Fourier-spectral discretisation (Sec. 5.1, Sec. 6.2.1): spectral
  // Laplacian in the solve, spectral divergence in S~ (Sec. 5.2)
  int spectral = 0;
  // pencils per work item of the pencil passes, chosen by the autotuner:
  // [0] float32 layouts, [1] float64 and double-float layouts; [.][0] the 3D
  // y passes, [.][1] the solve pass (2D y, 3D z).  0: the fixed rule.
  int pcap[2][2] = {{0, 0}, {0, 0}};
  // pencils per work item of the persistent solver's solve pass (2D y, 3D
  // z), per element type [0] float64, [1] float32, [2] double-float; 0: the
  // fixed rule
  int scap[3] = {0, 0, 0};
  // FFT plan variant of the float32 transforms (plan_lr: 0 radices as even
  // as possible, 1 radix-16 passes first), chosen by the autotuner; the
  // float32 twiddle table is of the same variant
  int fplan = 0;
};

// Host constants of the symbol multiply: the solve scales mode k by
// scale0 / (c0 + cfac * sum_c sin^2(pi k_c / n)), and by 0 where that
// denominator is 0 (only k = 0 in the Poisson limit).
__host__ __device__ inline double symbol_cfac(const GridDesc& g) {
  return 4.0 * (g.poisson ? 1.0 : g.kappa) / (g.h * g.h);
}
__host__ __device__ inline double symbol_scale0(const GridDesc& g) {
  double nd = 1.0;
  for (int c = 0; c < g.dim; ++c) nd *= g.n;
  return (g.poisson ? 1.0 : g.kappa) / nd;
}

// Storage of a CUDA tensor map (the 128-byte CUtensorMap of the driver API),
// kept opaque outside the translation unit that encodes and uses it.
struct alignas(64) TmaDesc {
  unsigned char bytes[128];
};

template <typename T>
struct SpectralWs {
  typename Cx<T>::type* spec = nullptr;  // (n/2+1) * n^(d-1) complex
  T* grid = nullptr;                      // n^d real
  const typename Cx<T>::type* tw = nullptr;  // tw[j] = exp(-2 pi i j / n)
  const T* s2 = nullptr;                  // sin^2(pi k / n), k < n
  typename Cx<T>::type* acc = nullptr;    // spectral discretisation: source accumulator
  // 3D float32: tensor map of spec for the bulk-copy staged z pass (k_tma.cu),
  // or null; err: device word raised when a bounded wait there gives up
  const TmaDesc* zmap = nullptr;
  unsigned* err = nullptr;
};

// Sources of the fused spread kernel: out = coef_div * S~ q_div
//   + coef_plain * S v_plain + coef_grid * f_grid (null pointers skip a term).
struct SpreadSrc {
  const double* q_div = nullptr;
  double coef_div = 0;
  const double* v_plain = nullptr;
  double coef_plain = 0;
  int plain_nrm = -1;  // >= 0: the plain term spreads v_plain * n_c, c = plain_nrm
  const double* f_grid = nullptr;
  double coef_grid = 0;
  // 3D, no grid source, grid feeding only the interpolation: tiles of
  // planes without points are not written (the z pass reads them as zero)
  bool skip_empty_planes = false;
};

// ---- dependent launches ----------------------------------------------------
// The kernels of a matvec chain (x forward, pencil passes, x inverse,
// interpolation) are launched with programmatic stream serialisation: the
// next kernel of the stream may be launched before this one has finished,
// its blocks taking the SMs this one's blocks leave.  Every such kernel
// starts with pdl_wait() -- it returns once the grids it depends on have
// completed and their memory operations are visible -- before touching any
// memory, and lets its own successor launch when a block has done its work
// (pdl_release at the end: released at the start, the successor's waiting
// blocks sat beside the running ones and slowed the double-float chain).
// Without a programmatic predecessor both are no-ops.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kernel<<<grid, block, smem, st>>>(args...) as a programmatic
// dependent of the stream's previous kernel (the kernel must begin with
// pdl_wait()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                    size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// ---- launch bookkeeping -------------------------------------------------
// prof_begin records a start event when profiling is on; count_launch counts
// the launch and records its end event (name must be a string literal).
void prof_begin(cudaStream_t st);
void count_launch(const char* name, cudaStream_t st);
cudaError_t check_launch();
// Device buffer of per-phase times of the persistent solver while profiling
// is on (nullptr otherwise); kPhaseSlots (id) pairs of (ns, count).
constexpr int kPhaseSlots = 16;
// The same buffer holds the solver's item trace after the phase times: word
// kTraceFlag switches it on (nonzero) for the launches that follow, word
// kTraceFlag + 1 is spare, then kTraceCap records of three words (start ns,
// end ns, and block << 40 | instance << 24 | phase << 20 | prec << 18 |
// item), each block of a launch writing its own kTraceCap / blocks of them
// (start 0: unused).  Phase 15 marks a hand-off: the finishing block
// choosing and publishing the next phase (item = that phase, or 15 when the
// instance stops).
constexpr int kTraceFlag = 2 * kPhaseSlots;
constexpr int kTraceCap = 1 << 16;
constexpr size_t kProfWords = 2 * kPhaseSlots + 2 + 3 * (size_t)kTraceCap;
unsigned long long* prof_phase_buffer();
// Sets the per-thread message of ibdl_last_error_message and returns s.
ibdl_status set_last_error(ibdl_status s, const char* msg);

// ---- point kernels (k_points.cu) -----------------------------------------
cudaError_t launch_point_prep(const GridDesc& g, int m, const double* const X[3],
                              int* const base[3], double* const W64[3],
                              float* const W32[3], cudaStream_t st);
// Bin building: counts, scan, fill into pts, then each tile's list sorted by
// first support column and point index into spts (asynchronous).  counts:
// ntiles + 1 ints of scratch; pts, spts: bins_capacity(dim, rows, m) ints.
cudaError_t launch_bins(const GridDesc& g, const PointData& p, int rows, int ntiles,
                        int* start, int* cursor, int* counts, int* pts, int* spts,
                        cudaStream_t st);
int64_t bins_capacity(int dim, int rows, int64_t m);
// 3D: zempty[z] = 1 for planes whose tiles list no point.
cudaError_t launch_plane_flags(const int* start, int ngroups, int n, unsigned char* zempty,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_interp(const GridDesc& g, const PointData& p, const T* grid,
                          const double* jvec, double jump, double* y, cudaStream_t st);
cudaError_t launch_grid_to_float(const double* src, float* dst, int64_t count,
                                 cudaStream_t st);

// ---- FFT / Helmholtz kernels (k_fft.cu) ------------------------------------
// Forward pass: spread sources into row tiles, x-FFT, write the transposed
// half spectrum.  If write_grid != nullptr the tile rows are written to that
// real grid instead (no FFT).
template <typename T>
cudaError_t launch_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                            const SpreadSrc& src, SpectralWs<T>& ws, double* write_grid,
                            cudaStream_t st);
// y/z passes on the spectrum; solve multiplies by kappa / (sigma(k) n^d).
// skip (3D, may be null): the bins, to skip y-pass items of planes without
// points -- in the inverse pass always, in the forward pass when skip_fwd
// (the forward input of such planes is zero: no grid source).
template <typename T>
cudaError_t launch_spectral_solve(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st,
                                  const Bins* skip = nullptr, bool skip_fwd = false);
// Inverse x pass: transposed half spectrum -> real grid (T or double).
// band_only: produce only the tiles that hold points (the grid then feeds
// the interpolation alone).
template <typename T, typename OutT>
cudaError_t launch_rows_inv(const GridDesc& g, const Bins& b, SpectralWs<T>& ws,
                            OutT* out, cudaStream_t st, bool band_only = false);
template <typename T>
int fft_kernels_per_solve(int dim);
cudaError_t configure_fft_kernels(int n, int rows);

// ---- bulk-copy staged z pass (k_tma.cu, 3D float32) --------------------------
// Shared memory of one block of the staged z pass with c pencils per item.
template <typename T>
size_t zsolve_smem(int n, int c);
// Encodes the tensor map of a (n/2+1) x n x n transposed half spectrum.
template <typename T>
cudaError_t make_zsolve_map(const GridDesc& g, const typename Cx<T>::type* spec, TmaDesc* out);
// Forward z FFT, symbol, inverse z FFT of the 3D solve, in place on ws.spec
// (ws.zmap set); zempty: planes without points (read as zero, not stored).
template <typename T>
cudaError_t launch_zsolve_tma(const GridDesc& g, SpectralWs<T>& ws, const unsigned char* zempty,
                              cudaStream_t st);

// ---- Krylov kernels (k_krylov.cu) -----------------------------------------
struct KrylovWs {
  int m = 0;            // vector length
  int ld = 0;           // leading dimension of V (>= m, multiple of 32)
  int restart = 0;
  double* V = nullptr;  // (restart + 1) x ld
  double* H = nullptr;  // column j at H[j * (restart + 1)]
  double* cs = nullptr;
  double* sn = nullptr;
  double* gvec = nullptr;   // restart + 1
  double* ysol = nullptr;   // restart
  double* partial = nullptr;  // nblk * (restart + 2)
  double* scal = nullptr;     // device scalars: [0] residual estimate, ...
  int nblk = 0;
};
cudaError_t krylov_dot_norm(const KrylovWs& k, const double* x, double* out_sq,
                            cudaStream_t st);   // out_sq[0] = ||x||^2 (device)
cudaError_t krylov_start(const KrylovWs& k, const double* r, double* out_scal,
                         cudaStream_t st);      // V0 = r/||r||, g = (||r||,0..)
cudaError_t krylov_arnoldi(const KrylovWs& k, int j, double bnorm, cudaStream_t st);
cudaError_t krylov_finish(const KrylovWs& k, int kdim, double* x, cudaStream_t st);
cudaError_t launch_axpby(int m, double a, const double* x, double b, const double* y,
                         double* out, cudaStream_t st);  // out = a x + b y
cudaError_t launch_nonfinite_check(int m, const double* x, int* flag, cudaStream_t st);

// Fourier-spectral discretisation (k_fft.cu).  The forward passes after the
// x pass (y; 3D y then z) and the inverse passes before the x inverse, in
// place on ws.spec.  combine: term = spec, times i 2 pi k_c / L when
// deriv_c >= 0 (0 at the Nyquist mode); accumulate adds ws.acc; final
// writes (term) * scale0 / (c0 + cfac sum_c (pi k_c / n)^2) into ws.spec
// (0 where the denominator is 0), else stores term into ws.acc.
template <typename T>
cudaError_t launch_pencils_forward(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st);
template <typename T>
cudaError_t launch_pencils_inverse(const GridDesc& g, SpectralWs<T>& ws, cudaStream_t st);
template <typename T>
cudaError_t launch_spec_combine(const GridDesc& g, SpectralWs<T>& ws, int deriv_c,
                                bool accumulate, bool final, cudaStream_t st);

// Poisson limit (k_poisson.cu).  Reduction buffers hold kRedBlocks + 1 doubles.
constexpr int kRedBlocks = 152;
// part = block partials of w^T q and part[kRedBlocks] = q[m] (u_bar)
cudaError_t launch_completed_head(int m, const double* w, const double* q, double* part,
                                  cudaStream_t st);
// y[i] += u_bar (i < m), y[m] = scale * w^T q
cudaError_t launch_completed_tail(int m, double* y, const double* part, double scale,
                                  cudaStream_t st);
// out[0] = scale * sum a
cudaError_t launch_scaled_sum(int64_t n, const double* a, double scale, double* part,
                              double* out, cudaStream_t st);
cudaError_t launch_add_scalar(int64_t n, double* u, const double* s, cudaStream_t st);
cudaError_t launch_fill(int64_t n, double* x, double v, cudaStream_t st);
// chi_h = u - u[0], chi = chi_h > 1/2 (either output may be null)
cudaError_t launch_indicator(int64_t n, const double* u, double* chi_h, unsigned char* chi,
                             cudaStream_t st);

// Near-boundary values, 2D and 3D (k_near.cu); scratch: near_scratch_bytes,
// 16-byte aligned.
int64_t near_list_capacity(int dim, int n, int m, int m1);
size_t near_scratch_bytes(int dim, int n, int m, int m1);
// cmax: a bound on |coordinate| of every point and grid node (the float32
// distance filter's error bound scales with it)
cudaError_t launch_near_boundary(const GridDesc& g, const PointData& p, const double* ub,
                                 const double* uin, const unsigned char* inside, int m1,
                                 double m2, double cmax, double* uout, void* scratch,
                                 cudaStream_t st);

}  // namespace ibdl
