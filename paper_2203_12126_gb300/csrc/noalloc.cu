// ibdl_helmholtz_2d_noalloc: the periodic 2D Helmholtz solve of
// ibdl_helmholtz (v = kappa L'^{-1} f) for callers that cannot allocate
// device memory -- code running where cudaMalloc is unavailable or
// forbidden, such as inside a host callback, a plugin whose host framework
// owns every allocation, or a process that must not grow its device
// footprint after start-up.  All scratch (half spectrum, twiddles, symbol
// table, empty tile lists) lives in one file-scope __device__ array that
// every GPU loading this library holds until the process exits.
#include <math.h>

#include <mutex>

#include "ibdl_device.cuh"

namespace ibdl {

constexpr int kNoAllocMaxN = 512;  // largest grid: 512 x 512
constexpr size_t kSpecBytes = (size_t)(kNoAllocMaxN / 2 + 1) * kNoAllocMaxN * sizeof(double2);
constexpr size_t kTwBytes = 2 * (size_t)kNoAllocMaxN * sizeof(double2);  // >= fft_tw_count(n)
constexpr size_t kS2Bytes = (size_t)kNoAllocMaxN * sizeof(double);
constexpr size_t kStartBytes = 256 * 4;  // >= (n/4 + 1) ints for n <= 512
constexpr size_t kScratchBytes = kSpecBytes + kTwBytes + kS2Bytes + kStartBytes;

// The scratch: ~2.1 MB per GPU.  Host code must not use this name as a
// device address; it takes the address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// FFT pass twiddles (fft_tw_count(n) entries) and sin^2(pi j / n), j < n,
// rewritten by every call.
__global__ void k_noalloc_tables(int n, int ntw, double2* tw, double* s2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ntw) {
    int num, den;
    fft_tw_angle(n, j, &num, &den);
    double s, c;
    sincospi(2.0 * (double)(num % den) / den, &s, &c);
    tw[j] = make_double2(c, -s);
  }
  if (j < n) {
    const double h = sinpi((double)j / n);
    s2[j] = h * h;
  }
}

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};
}  // namespace

}  // namespace ibdl

using namespace ibdl;

extern "C" ibdl_status ibdl_helmholtz_2d_noalloc(int32_t n, double box_len, double kappa,
                                                 const double* f, double* v_out,
                                                 void* stream) {
  if (n < 16 || n > kNoAllocMaxN || (n & (n - 1)) != 0)
    return set_last_error(IBDL_ERR_INVALID_ARG,
                          "ibdl_helmholtz_2d_noalloc: n must be a power of two in [16, 512] "
                          "(the static scratch holds a 512 x 512 spectrum)");
  if (!(box_len > 0) || !isfinite(box_len) || !(kappa > 0) || !isfinite(kappa))
    return set_last_error(IBDL_ERR_INVALID_ARG,
                          "ibdl_helmholtz_2d_noalloc: box_len and kappa must be positive "
                          "and finite");
  if (!f || !v_out)
    return set_last_error(IBDL_ERR_INVALID_ARG, "ibdl_helmholtz_2d_noalloc: NULL f or v_out");
  for (const void* p : {(const void*)f, (const void*)v_out}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return set_last_error(IBDL_ERR_INVALID_ARG,
                            "ibdl_helmholtz_2d_noalloc: f and v_out must be device memory "
                            "(this entry point stages nothing)");
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return set_last_error(IBDL_ERR_CUDA, "ibdl_helmholtz_2d_noalloc: cudaGetDevice failed");
  unsigned char* base = nullptr;
  {
    // once per device, with that device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return set_last_error(IBDL_ERR_CUDA,
                              "ibdl_helmholtz_2d_noalloc: cudaGetSymbolAddress failed");
      g_noalloc_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  }
  if ((e = configure_fft_kernels(n, 4)) != cudaSuccess)
    return set_last_error(IBDL_ERR_CUDA, "ibdl_helmholtz_2d_noalloc: kernel configuration");

  double2* spec = reinterpret_cast<double2*>(base);
  double2* tw = reinterpret_cast<double2*>(base + kSpecBytes);
  double* s2 = reinterpret_cast<double*>(base + kSpecBytes + kTwBytes);
  int* start = reinterpret_cast<int*>(base + kSpecBytes + kTwBytes + kS2Bytes);

  // the tile lists must be empty: no boundary points take part
  if ((e = cudaMemsetAsync(start, 0, kStartBytes, st)) != cudaSuccess)
    return set_last_error(IBDL_ERR_CUDA, "ibdl_helmholtz_2d_noalloc: clearing scratch");
  prof_begin(st);
  const int ntw = fft_tw_count(n);
  k_noalloc_tables<<<(2 * n + 127) / 128, 128, 0, st>>>(n, ntw, tw, s2);
  count_launch("noalloc_tables", st);
  if ((e = check_launch()) != cudaSuccess)
    return set_last_error(IBDL_ERR_CUDA, "ibdl_helmholtz_2d_noalloc: table kernel");

  GridDesc g;
  g.dim = 2;
  g.n = n;
  while ((1 << g.log2n) < n) g.log2n++;
  g.h = box_len / n;
  g.inv2h = 0.5 / g.h;
  g.kappa = kappa;
  PointData p;  // m = 0
  Bins b;
  b.rows = 4;
  b.ntiles = n / 4;
  b.start = start;
  b.pts = nullptr;
  SpectralWs<double> ws;
  ws.spec = spec;
  ws.grid = nullptr;
  ws.tw = tw;
  ws.s2 = s2;
  SpreadSrc src;
  src.f_grid = f;
  src.coef_grid = 1.0;
  if ((e = launch_rows_fwd<double>(g, p, b, src, ws, nullptr, st)) != cudaSuccess ||
      (e = launch_spectral_solve<double>(g, ws, st)) != cudaSuccess ||
      (e = launch_rows_inv<double, double>(g, b, ws, v_out, st)) != cudaSuccess)
    return set_last_error(IBDL_ERR_CUDA, cudaGetErrorString(e));
  return IBDL_OK;
}
