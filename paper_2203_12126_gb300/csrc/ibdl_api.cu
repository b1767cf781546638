// C ABI of libibdl and the host-side orchestration of the IBDL hot path.
//
// Operators (Leathers & Guy, arXiv:2203.12126, with L' = I - kappa Delta_h):
//   Dirichlet matvec  A_D q = q/2 + kappa S* L'^{-1} S~ q      (Sec. 5.3)
//   Neumann matvec    A_N u = kappa S* L'^{-1} S~ u - u/2      (Sec. 4.4)
//   Dirichlet rhs     b = U_b + kappa S* L'^{-1} g~
//   Neumann rhs       b = kappa S* L'^{-1} (g~ - S V_b)
//   field             u = kappa L'^{-1} (S~ q [+ S V_b] - g~)  (Sec. 4.1 step 2)
// One matvec = rows_fwd (spread-divergence fused with the x FFT), the y (and
// z) pencil passes with the symbol, rows_inv (x inverse FFT) and interp
// (gather + jump term): 4 kernels in 2D, 6 in 3D.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ibdl_device.cuh"
#include "ibdl_solver.cuh"

namespace ibdl {

static std::atomic<long long> g_launches{0};

// Opt-in kernel timing: a CUDA event pair on the launching stream around
// every launch, resolved when the statistics are read.
struct ProfPending {
  const char* name;
  cudaEvent_t a, b;
};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
static std::vector<ProfPending> g_pending;
static std::vector<cudaEvent_t> g_ev_pool;
static std::map<std::string, std::pair<long long, double>> g_prof_stats;
static thread_local cudaEvent_t t_begin = nullptr;
static unsigned long long* g_phase_buf = nullptr;  // persistent-solver phase times

static cudaEvent_t prof_event() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

unsigned long long* prof_phase_buffer() {
  return g_prof.load(std::memory_order_relaxed) ? g_phase_buf : nullptr;
}

void prof_begin(cudaStream_t st) {
  if (!g_prof.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  t_begin = prof_event();
  if (t_begin) cudaEventRecord(t_begin, st);
}

void count_launch(const char* name, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof.load(std::memory_order_relaxed) || !t_begin) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = prof_event();
  if (!e) return;
  cudaEventRecord(e, st);
  g_pending.push_back({name, t_begin, e});
  t_begin = nullptr;
}

cudaError_t check_launch() { return cudaGetLastError(); }

static thread_local std::string g_err;

static ibdl_status fail(ibdl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

ibdl_status set_last_error(ibdl_status s, const char* msg) { return fail(s, msg); }

static ibdl_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? IBDL_ERR_OOM : IBDL_ERR_CUDA;
}

#define IBDL_CU(expr)                                  \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

#define IBDL_TRY(expr)                  \
  do {                                  \
    ibdl_status s_ = (expr);            \
    if (s_ != IBDL_OK) return s_;       \
  } while (0)

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace ibdl

using namespace ibdl;

namespace {

// Device workspaces of geometry handles come from one stream-ordered memory
// pool per device that keeps freed blocks for reuse (release threshold at
// its maximum): creating and destroying many handles -- the serving engine
// does one per request -- then costs no cudaMalloc/cudaFree round trips.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaError_t workspace_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    if ((e = cudaMemPoolCreate(&pool, &props))) return e;
    uint64_t keep = ~0ull;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep))) return e;
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

constexpr int kHistCapHost = 256;  // residual history entries (kHistCap)
// the solver's work items per phase are counted in 16 bits: at most 65535
// vector chunks of kSolverThreads points
constexpr int64_t kMaxPoints = 65535LL * kSolverThreads;

struct ibdl_geometry_s {
  GridDesc grid;
  int bc = 0, precision = 0, m = 0;
  // completed IBDL (eta > 0, Poisson limit): the system unknown is
  // (Q, u_bar), nsys = m + 1; otherwise nsys = m
  int nsys = 0;
  double eta = 0;
  double* cpart = nullptr;  // kRedBlocks + 1 reduction partials
  double xmax = 0;          // max |coordinate| over the points
  Bins bins;
  PointData pd;
  SpectralWs<double> ws64;
  SpectralWs<float> ws32;
  SpectralWs<dd> wsdd;  // double-float view of the float64 buffers (own tables)
  bool have32 = false;
  TmaDesc zmap32;            // 3D: tensor map of ws32.spec for the staged z pass
  unsigned* d_err = nullptr;  // raised by a bounded wait inside a transform
  KrylovWs kry;
  double *vb = nullptr, *vx = nullptr, *vr = nullptr, *vt = nullptr, *vd = nullptr;
  double *stage_a = nullptr, *stage_b = nullptr;
  double* grid_stage = nullptr;   // n^d doubles, allocated on first host grid
  double* host_scal = nullptr;    // pinned
  int* d_flag = nullptr;
  // persistent solver context
  SolveInst* d_inst = nullptr;
  SolveState* d_state = nullptr;
  unsigned* d_bar = nullptr;
  double* ppart = nullptr;
  double* d_hist = nullptr;
  int nchunk = 0;
  int nsec = 0;
  int solver_smem = 0;
  SolveInst* h_inst = nullptr;    // pinned
  SolveState* h_state = nullptr;  // pinned
  double* h_hist = nullptr;       // pinned
  int64_t bytes = 0;
  int64_t ncells = 0;
  std::vector<void*> dev_allocs;

  cudaStream_t alloc_st = nullptr;  // stream of the creating call

  // Pool allocation, ordered on the creating stream (which the creation
  // synchronises before returning, so other streams may use the memory).
  template <typename P>
  ibdl_status alloc(P** out, size_t count) {
    void* p = nullptr;
    const size_t nbytes = count * sizeof(P);
    cudaMemPool_t pool;
    cudaError_t e = workspace_pool(&pool);
    if (!e) e = cudaMallocFromPoolAsync(&p, nbytes > 0 ? nbytes : 16, pool, alloc_st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? fail(IBDL_ERR_OOM, "device workspace")
                                            : cuda_fail(e, "cudaMallocFromPoolAsync");
    }
    dev_allocs.push_back(p);
    bytes += (int64_t)nbytes;
    *out = static_cast<P*>(p);
    return IBDL_OK;
  }
  // Pinned host scratch of ibdl_solve, made on its first call.
  ibdl_status ensure_host() {
    if (host_scal) return IBDL_OK;
    cudaError_t e = cudaMallocHost((void**)&h_inst, sizeof(SolveInst));
    if (!e) e = cudaMallocHost((void**)&h_state, sizeof(SolveState));
    if (!e) e = cudaMallocHost((void**)&h_hist, kHistCapHost * sizeof(double));
    if (!e) e = cudaMallocHost((void**)&host_scal, 16 * sizeof(double));
    if (e) return cuda_fail(e, "cudaMallocHost");
    return IBDL_OK;
  }
  // The handle's users have finished (ibdl_destroy_geometry synchronises
  // the device first): the blocks go back to the pool.
  ~ibdl_geometry_s() {
    for (void* p : dev_allocs) cudaFreeAsync(p, 0);
    if (host_scal) cudaFreeHost(host_scal);
    if (h_inst) cudaFreeHost(h_inst);
    if (h_state) cudaFreeHost(h_state);
    if (h_hist) cudaFreeHost(h_hist);
  }
};

namespace {

// cos and sin of 2 pi num / den (0 <= num < den): exact quadrant and octant
// reduction, then the double library functions on |angle| <= pi/4.
void cis_2pi(int64_t num, int64_t den, double* c, double* s) {
  num %= den;
  const double x = (double)num / (double)den;  // exact: den is a power of two
  const int k = (int)(4.0 * x);                 // quadrant
  double y = x - 0.25 * k;                      // [0, 1/4), exact
  const bool swap = y > 0.125;
  if (swap) y = 0.25 - y;
  const double t = 6.283185307179586476925286766559 * y;
  double cc = cos(t), ss = sin(t);
  if (swap) {
    const double u = cc;
    cc = ss;
    ss = u;
  }
  switch (k & 3) {
    case 0: *c = cc; *s = ss; break;
    case 1: *c = -ss; *s = cc; break;
    case 2: *c = -cc; *s = -ss; break;
    default: *c = ss; *s = -cc; break;
  }
}

// FFT pass twiddles and sin^2(pi j / n) tables, read-only and the same for
// every handle with the same n: made once per (device, n, precision) and
// kept for the life of the process.
std::mutex g_tab_mu;
std::map<std::tuple<int, int, int>, std::pair<const void*, const void*>> g_tabs;

// v: the plan variant of the twiddle table (float32 only; see plan_lr).
template <typename T>
ibdl_status fft_tables(int n, const typename Cx<T>::type** tw_out, const T** s2_out, int v = 0) {
  int dev = 0;
  IBDL_CU(cudaGetDevice(&dev));
  if (v != 0 && !std::is_same<T, float>::value)
    return fail(IBDL_ERR_INVALID_ARG, "FFT tables: only float32 tables have plan variants");
  std::lock_guard<std::mutex> lk(g_tab_mu);
  const int tag = (std::is_same<T, dd>::value ? 2 : (sizeof(T) == 8 ? 1 : 0)) + 3 * v;
  const auto key = std::make_tuple(dev, n, tag);
  auto it = g_tabs.find(key);
  if (it == g_tabs.end()) {
    const int ntw = fft_tw_count(n, v);
    if (ntw < 0) return fail(IBDL_ERR_INVALID_ARG, "FFT tables: unsupported n or plan");
    std::vector<typename Cx<T>::type> htw(ntw);
    std::vector<T> hs2(n);
    for (int j = 0; j < ntw; ++j) {
      int num, den;
      fft_tw_angle(n, j, &num, &den, v);
      double c, s;
      cis_2pi(num, den, &c, &s);
      htw[j].x = (T)c;
      htw[j].y = (T)-s;
    }
    for (int j = 0; j < n; ++j) {
      double c, s;
      cis_2pi(j, 2 * (int64_t)n, &c, &s);  // sin(pi j / n)
      hs2[j] = (T)(s * s);
    }
    void *dtw = nullptr, *ds2 = nullptr;
    IBDL_CU(cudaMalloc(&dtw, sizeof(htw[0]) * ntw));
    IBDL_CU(cudaMalloc(&ds2, sizeof(T) * n));
    IBDL_CU(cudaMemcpy(dtw, htw.data(), sizeof(htw[0]) * ntw, cudaMemcpyHostToDevice));
    IBDL_CU(cudaMemcpy(ds2, hs2.data(), sizeof(T) * n, cudaMemcpyHostToDevice));
    it = g_tabs.emplace(key, std::make_pair((const void*)dtw, (const void*)ds2)).first;
  }
  *tw_out = static_cast<const typename Cx<T>::type*>(it->second.first);
  *s2_out = static_cast<const T*>(it->second.second);
  return IBDL_OK;
}

template <typename T>
ibdl_status alloc_spectral(ibdl_geometry_s* g, SpectralWs<T>& ws, cudaStream_t) {
  const int n = g->grid.n;
  const int64_t spec_count = (int64_t)(n / 2 + 1) * (g->ncells / n);
  typename Cx<T>::type* spec;
  T* grid;
  const typename Cx<T>::type* tw;
  const T* s2;
  IBDL_TRY(g->alloc(&spec, (size_t)spec_count));
  IBDL_TRY(g->alloc(&grid, (size_t)g->ncells));
  IBDL_TRY(fft_tables<T>(n, &tw, &s2, plan_variant_of<T>(g->grid)));
  if (g->grid.spectral) IBDL_TRY(g->alloc(&ws.acc, (size_t)spec_count));
  ws.spec = spec;
  ws.grid = grid;
  ws.tw = tw;
  ws.s2 = s2;
  return IBDL_OK;
}

// Switches the geometry's float32 transforms to plan variant v: its float32
// twiddle table is replaced by that variant's (the buffers and budgets are
// sized for either, fft_tw_capacity).  No-op before the float32 workspace
// exists; ensure32 then takes the table of g->grid.fplan.
ibdl_status set_float_plan(ibdl_geometry_s* g, int v) {
  if (v < 0 || v >= kPlanVariants || !plan_offered(g->grid.log2n, v))
    return fail(IBDL_ERR_INVALID_ARG, "plan variant not offered for this size");
  if (g->have32) {
    const cx_t<float>* tw;
    const float* s2;
    IBDL_TRY(fft_tables<float>(g->grid.n, &tw, &s2, v));
    g->ws32.tw = tw;
  }
  g->grid.fplan = v;
  return IBDL_OK;
}

ibdl_status ensure32(ibdl_geometry_s* g, cudaStream_t st) {
  if (g->have32) return IBDL_OK;
  IBDL_TRY(alloc_spectral<float>(g, g->ws32, st));
  g->ws32.err = g->d_err;
  // 3D: the z pass stages its pencils with bulk tensor copies when the
  // driver can encode the tensor map (otherwise the plain pass runs)
  if (g->grid.dim == 3 && !g->grid.spectral &&
      make_zsolve_map<float>(g->grid, g->ws32.spec, &g->zmap32) == cudaSuccess)
    g->ws32.zmap = &g->zmap32;
  cudaGetLastError();
  g->have32 = true;
  return IBDL_OK;
}

// Device view of a caller array of `count` doubles: the pointer itself when
// it is device memory, else a copy in `stage`.
ibdl_status dev_in(const double* p, size_t count, double* stage, const double** out,
                   cudaStream_t st) {
  if (is_device_ptr(p)) {
    *out = p;
    return IBDL_OK;
  }
  IBDL_CU(cudaMemcpyAsync(stage, p, count * sizeof(double), cudaMemcpyHostToDevice, st));
  *out = stage;
  return IBDL_OK;
}

ibdl_status grid_in(ibdl_geometry_s* g, const double* p, const double** out, cudaStream_t st) {
  if (!p) {
    *out = nullptr;
    return IBDL_OK;
  }
  if (is_device_ptr(p)) {
    *out = p;
    return IBDL_OK;
  }
  if (!g->grid_stage) IBDL_TRY(g->alloc(&g->grid_stage, (size_t)g->ncells));
  IBDL_CU(cudaMemcpyAsync(g->grid_stage, p, g->ncells * sizeof(double),
                          cudaMemcpyHostToDevice, st));
  *out = g->grid_stage;
  return IBDL_OK;
}

template <typename T>
SpectralWs<T>& wsof(ibdl_geometry_s* g);
template <>
SpectralWs<double>& wsof<double>(ibdl_geometry_s* g) {
  return g->ws64;
}
template <>
SpectralWs<float>& wsof<float>(ibdl_geometry_s* g) {
  return g->ws32;
}
template <>
SpectralWs<dd>& wsof<dd>(ibdl_geometry_s* g) {
  return g->wsdd;
}

// Precision of the float64-grade matvecs of a solve (residuals, right-hand
// side): a float32-refined geometry takes double-float transforms (float64
// spread and interpolation); IBDL_FP64 geometries, the spectral
// discretisation and the completed system stay in native float64.
int resid_prec(const ibdl_geometry_s* g) {
  return g->precision == IBDL_FP32_REFINED && !g->grid.spectral && g->eta <= 0
             ? IBDL_FP64_DF
             : IBDL_FP64;
}

// Fourier-spectral discretisation (Sec. 5.1, Sec. 6.2.1): the divergence in
// S~ is spectral too (Sec. 5.2), so each component S(q n_c) is transformed
// on its own and combined as i 2 pi k_c / L times its transform; the
// scalar sources (plain spread, grid) are added as they are; the last
// combination applies kappa / sigma(k) and the inverse passes follow.
template <typename T, typename OutT>
ibdl_status spectral_field_solve(ibdl_geometry_s* g, const SpreadSrc& src, OutT* out,
                                 cudaStream_t st) {
  SpectralWs<T>& ws = wsof<T>(g);
  const GridDesc& gd = g->grid;
  struct Term {
    SpreadSrc s;
    int deriv;
  };
  Term terms[4];
  int nt = 0;
  if (src.q_div)
    for (int c = 0; c < gd.dim; ++c) {
      SpreadSrc t;
      t.v_plain = src.q_div;
      t.coef_plain = src.coef_div;
      t.plain_nrm = c;
      terms[nt++] = {t, c};
    }
  if (src.v_plain || src.f_grid) {
    SpreadSrc t;
    t.v_plain = src.v_plain;
    t.coef_plain = src.coef_plain;
    t.plain_nrm = src.plain_nrm;
    t.f_grid = src.f_grid;
    t.coef_grid = src.coef_grid;
    terms[nt++] = {t, -1};
  }
  if (nt == 0) return fail(IBDL_ERR_INVALID_ARG, "no source");
  for (int k = 0; k < nt; ++k) {
    IBDL_CU(launch_rows_fwd<T>(gd, g->pd, g->bins, terms[k].s, ws, nullptr, st));
    IBDL_CU(launch_pencils_forward<T>(gd, ws, st));
    IBDL_CU(launch_spec_combine<T>(gd, ws, terms[k].deriv, k > 0, k == nt - 1, st));
  }
  IBDL_CU(launch_pencils_inverse<T>(gd, ws, st));
  IBDL_CU((launch_rows_inv<T, OutT>(gd, g->bins, ws, out, st, false)));
  return IBDL_OK;
}

// grid = kappa L'^{-1} (sources), T-precision spectral passes, output OutT grid.
// band_only: the grid feeds only the interpolation (matvec, right-hand
// side), so tiles and planes without points are not produced.
template <typename T, typename OutT>
ibdl_status field_solve(ibdl_geometry_s* g, const SpreadSrc& src, OutT* out, cudaStream_t st,
                        bool band_only = false) {
  if constexpr (!std::is_same<T, dd>::value) {
    if (g->grid.spectral) return spectral_field_solve<T, OutT>(g, src, out, st);
  }
  SpectralWs<T>& ws = wsof<T>(g);
  SpreadSrc s = src;
  s.skip_empty_planes = band_only && !src.f_grid;
  IBDL_CU(launch_rows_fwd<T>(g->grid, g->pd, g->bins, s, ws, nullptr, st));
  IBDL_CU(launch_spectral_solve<T>(g->grid, ws, st, band_only ? &g->bins : nullptr,
                                   band_only && !src.f_grid));
  IBDL_CU((launch_rows_inv<T, OutT>(g->grid, g->bins, ws, out, st, band_only)));
  return IBDL_OK;
}

// y = A q with the T-precision spectral path.  q, y device, may alias.
template <typename T>
ibdl_status matvec(ibdl_geometry_s* g, const double* q, double* y, cudaStream_t st) {
  SpreadSrc src;
  src.q_div = q;
  src.coef_div = 1.0;
  SpectralWs<T>& ws = wsof<T>(g);
  IBDL_TRY((field_solve<T, T>(g, src, ws.grid, st, true)));
  const double jump = g->bc == IBDL_DIRICHLET ? 0.5 : -0.5;
  IBDL_CU(launch_interp<T>(g->grid, g->pd, ws.grid, q, jump, y, st));
  return IBDL_OK;
}

// y = A q with float64 spread / interpolation and double-float transforms.
ibdl_status matvec_dd(ibdl_geometry_s* g, const double* q, double* y, cudaStream_t st) {
  SpreadSrc src;
  src.q_div = q;
  src.coef_div = 1.0;
  IBDL_TRY((field_solve<dd, double>(g, src, g->ws64.grid, st, true)));
  const double jump = g->bc == IBDL_DIRICHLET ? 0.5 : -0.5;
  IBDL_CU(launch_interp<double>(g->grid, g->pd, g->ws64.grid, q, jump, y, st));
  return IBDL_OK;
}

ibdl_status matvec_prec(ibdl_geometry_s* g, int prec, const double* q, double* y,
                        cudaStream_t st) {
  if (prec == IBDL_FP64_DF) return matvec_dd(g, q, y, st);
  if (prec == IBDL_FP32_REFINED) {
    IBDL_TRY(ensure32(g, st));
    return matvec<float>(g, q, y, st);
  }
  return matvec<double>(g, q, y, st);
}

double cell_volume(const GridDesc& g) {
  return g.dim == 3 ? g.h * g.h * g.h : g.h * g.h;
}

// Completed IBDL (Sec. 5.4, App. C), z = (Q, u_bar):
//   y[0:m] = Q/2 + S* (-Delta_0^{-1}) (S~ + eta S) Q + u_bar,  y[m] = eta sum w_i Q_i.
// The weight sum and u_bar are read before the interpolation writes y.
template <typename T>
ibdl_status completed_matvec(ibdl_geometry_s* g, const double* q, double* y, cudaStream_t st) {
  IBDL_CU(launch_completed_head(g->m, g->pd.w, q, g->cpart, st));
  SpreadSrc src;
  src.q_div = q;
  src.coef_div = 1.0;
  src.v_plain = q;
  src.coef_plain = g->eta;
  SpectralWs<T>& ws = wsof<T>(g);
  IBDL_TRY((field_solve<T, T>(g, src, ws.grid, st, true)));
  IBDL_CU(launch_interp<T>(g->grid, g->pd, ws.grid, q, 0.5, y, st));
  // pd.w holds w_i / h^d
  IBDL_CU(launch_completed_tail(g->m, y, g->cpart, g->eta * cell_volume(g->grid), st));
  return IBDL_OK;
}

// The operator of the geometry's boundary system (length nsys).
ibdl_status sys_matvec(ibdl_geometry_s* g, int prec, const double* q, double* y,
                       cudaStream_t st) {
  if (prec == IBDL_FP64_DF && (g->eta > 0 || g->grid.spectral))
    return fail(IBDL_ERR_UNSUPPORTED, "double-float transforms: finite-difference, plain "
                                      "system only");
  if (g->eta <= 0) return matvec_prec(g, prec, q, y, st);
  if (prec == IBDL_FP32_REFINED) {
    IBDL_TRY(ensure32(g, st));
    return completed_matvec<float>(g, q, y, st);
  }
  return completed_matvec<double>(g, q, y, st);
}

// b = right-hand side of the boundary system (float64).
ibdl_status build_rhs(ibdl_geometry_s* g, const double* bdata, const double* ggrid, double* b,
                      cudaStream_t st) {
  if (g->bc == IBDL_DIRICHLET) {
    if (g->eta > 0) {
      // completed system: last row h^d sum g~ (App. C solvability condition)
      if (ggrid)
        IBDL_CU(launch_scaled_sum(g->ncells, ggrid, cell_volume(g->grid), g->cpart, b + g->m,
                                  st));
      else
        IBDL_CU(cudaMemsetAsync(b + g->m, 0, sizeof(double), st));
    }
    if (!ggrid) {
      IBDL_CU(cudaMemcpyAsync(b, bdata, sizeof(double) * g->m, cudaMemcpyDeviceToDevice, st));
      return IBDL_OK;
    }
    SpreadSrc src;
    src.f_grid = ggrid;
    src.coef_grid = 1.0;
    if (resid_prec(g) == IBDL_FP64_DF)
      IBDL_TRY((field_solve<dd, double>(g, src, g->ws64.grid, st, true)));
    else
      IBDL_TRY((field_solve<double, double>(g, src, g->ws64.grid, st, true)));
    IBDL_CU(launch_interp<double>(g->grid, g->pd, g->ws64.grid, bdata, 1.0, b, st));
    return IBDL_OK;
  }
  SpreadSrc src;
  src.v_plain = bdata;
  src.coef_plain = -1.0;
  if (ggrid) {
    src.f_grid = ggrid;
    src.coef_grid = 1.0;
  }
  if (resid_prec(g) == IBDL_FP64_DF)
    IBDL_TRY((field_solve<dd, double>(g, src, g->ws64.grid, st, true)));
  else
    IBDL_TRY((field_solve<double, double>(g, src, g->ws64.grid, st, true)));
  IBDL_CU(launch_interp<double>(g->grid, g->pd, g->ws64.grid, nullptr, 0.0, b, st));
  return IBDL_OK;
}

double read_scalar(ibdl_geometry_s* g, const double* dptr, int slot, cudaStream_t st,
                   cudaError_t* err) {
  *err = cudaMemcpyAsync(g->host_scal + slot, dptr, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (*err == cudaSuccess) *err = cudaStreamSynchronize(st);
  return g->host_scal[slot];
}

struct GmresRun {
  int iters = 0;
  int matvecs = 0;
  double rel = 0;   // final relative residual (true, if checked)
  std::vector<double> hist;
};

// Restarted GMRES on A_prec x = b (x in/out, device).  If true_check, a
// converged estimate is confirmed with the true residual ||b - A x|| (the
// same precision), as MATLAB's gmres does; otherwise the estimate is final.
ibdl_status gmres(ibdl_geometry_s* g, int prec, const double* b, double* x, bool x_is_zero,
                  double bnorm, double tol, int restart, int maxit, bool true_check,
                  GmresRun* run, cudaStream_t st) {
  KrylovWs& k = g->kry;
  cudaError_t ce;
  bool zero = x_is_zero;
  bool est_converged = false;
  for (;;) {
    if (zero) {
      IBDL_CU(cudaMemcpyAsync(g->vr, b, sizeof(double) * g->nsys, cudaMemcpyDeviceToDevice, st));
    } else {
      IBDL_TRY(sys_matvec(g, prec, x, g->vt, st));
      run->matvecs++;
      IBDL_CU(launch_axpby(g->nsys, 1.0, b, -1.0, g->vt, g->vr, st));
    }
    if (est_converged && !true_check) break;
    IBDL_CU(krylov_start(k, g->vr, nullptr, st));
    const double beta = read_scalar(g, k.scal + 2, 0, st, &ce);
    if (ce) return cuda_fail(ce, "read residual");
    run->rel = beta / bnorm;
    if (!isfinite(beta)) return fail(IBDL_ERR_NONFINITE, "non-finite residual");
    if (run->rel <= tol) return IBDL_OK;
    if (run->iters >= maxit) return fail(IBDL_ERR_NOT_CONVERGED, "GMRES reached max_iters");
    int kdim = 0;
    bool breakdown = false;
    est_converged = false;
    for (int j = 0; j < restart; ++j) {
      IBDL_TRY(sys_matvec(g, prec, k.V + (size_t)j * k.ld, k.V + (size_t)(j + 1) * k.ld, st));
      run->matvecs++;
      IBDL_CU(krylov_arnoldi(k, j, bnorm, st));
      IBDL_CU(cudaMemcpyAsync(g->host_scal, k.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              st));
      IBDL_CU(cudaStreamSynchronize(st));
      const double est = g->host_scal[0], hnext = g->host_scal[1];
      run->iters++;
      run->hist.push_back(est);
      kdim = j + 1;
      if (!isfinite(est) || !isfinite(hnext))
        return fail(IBDL_ERR_NONFINITE, "non-finite value in the Arnoldi process");
      if (est <= tol) {
        est_converged = true;
        break;
      }
      if (hnext == 0.0) {
        breakdown = true;
        break;
      }
      if (run->iters >= maxit) break;
    }
    IBDL_CU(krylov_finish(k, kdim, x, st));
    zero = false;
    if (breakdown) est_converged = true;
    if (est_converged && !true_check) {
      run->rel = g->host_scal[0];
      return IBDL_OK;
    }
  }
  return IBDL_OK;
}

constexpr int kHistCap = 256;
// IBDL_SOLVER_MULTIBLOCK=1 forces the multi-block vector phases for every
// instance (used by the tests to cover both code paths on small problems).
const bool g_force_multi = [] {
  const char* e = getenv("IBDL_SOLVER_MULTIBLOCK");
  return e && e[0] == '1';
}();

// batch_size: instances in the launch.  One block per instance for the
// vector work pays off only when many instances share the rounds; a lone
// instance is faster with its vector work spread over many blocks.
SolveInst make_inst(ibdl_geometry_s* g, const ibdl_solve_opts& o, int batch_size) {
  SolveInst I;
  memset(&I, 0, sizeof(I));
  I.g = g->grid;
  I.p = g->pd;
  I.b = g->bins;
  I.w64 = g->ws64;
  I.w32 = g->ws32;
  I.wdd = g->wsdd;
  I.dd64 = resid_prec(g) == IBDL_FP64_DF && batch_size <= kDdMaxBatch;
  I.V = g->kry.V;
  I.ld = g->kry.ld;
  I.restart = o.restart;
  I.H = g->kry.H;
  I.cs = g->kry.cs;
  I.sn = g->kry.sn;
  I.gv = g->kry.gvec;
  I.ysol = g->kry.ysol;
  I.part = g->ppart;
  I.nchunk = g->nchunk;
  I.nsec = g->nsec;
  I.pstride = g->kry.restart + 2;
  I.bvec = g->vb;
  I.x = g->vx;
  I.r = g->vr;
  I.dvec = g->vt;  // free in the persistent engine (the host loop's scratch)
  I.upd_resid = g->precision == IBDL_FP32_REFINED;
  I.cgs1 = g->precision == IBDL_FP32_REFINED;
  I.bc = g->bc;
  I.refined = g->precision == IBDL_FP32_REFINED;
  I.maxit = o.max_iters;
  I.max_refine = o.max_refine;
  I.tol = o.tol;
  I.inner_tol = o.inner_tol;
  I.hist = g->d_hist;
  I.hist_cap = kHistCap;
  I.single = g->m <= kSingleMax && batch_size >= kSingleMinBatch && !g_force_multi;
  // 2D solves alone in their launch: the Arnoldi steps interpolate in their
  // x-inverse tiles, one phase fewer per step on the instance's chain (C2
  // solve 0.993 -> 0.957 ms, C1 0.726 -> 0.711 ms).  Instances that share a
  // launch keep phase D: the fused x-inverse items do more work in all (a
  // point's share in up to two tiles' bins, a dot-product row per tile), and
  // sharing the blocks that costs more than the phase saves (the C2 pair
  // 1.261 -> 1.281 ms).  Float64 steps only for small instances: their
  // float64 interpolation lengthens the x-inverse items (the C2 float64 pair
  // 2.99 -> 3.30 ms when fused).
  if (batch_size == 1 && g->grid.dim == 2 && !I.single && g->nsec >= g->bins.ntiles)
    I.fuse_interp = g->m <= 1024 ? 2 : 1;
  // A few 2D instances in one launch share the blocks: float32 solve items
  // of 4 pencils (about 129 per instance) let them run side by side (the C2
  // pair: 1.268 -> 1.251 ms against the rule's 2 pencils), where the item
  // fits the geometry's reservation and no choice was set on the geometry.
  if (I.g.dim == 2 && batch_size >= 2 && batch_size <= kDdMaxBatch && I.g.scap[1] == 0) {
    const PencilLayout base = solve_layout<float>(2, I.g.n, 1);
    GridDesc gd = I.g;
    gd.scap[1] = 4;
    size_t need[3];
    solver_item_smem(gd, I.b.rows, 1, need);
    if (pencils_admissible<float>(I.g.n, base.estride, base.pg, 4) &&
        need[1] <= (size_t)g->solver_smem)
      I.g.scap[1] = 4;
  }
  solver_fill_items(I);
  return I;
}

// rhs_in_kernel: the Neumann right-hand side is built by the solver's first
// action (ACT_RHS) from V_b in inst.vdata.  A float32-refined instance then
// builds it in float32 (it only starts the first inner solve) and adds
// S V_b to every float64-grade residual's spread instead (I.rhs_resid):
// r = b - A x = -kappa S* L'^{-1} (S~ x + S V_b) + x / 2 in one Helmholtz
// solve, so a solve needs one float64-grade field solve fewer.
SolveState initial_state(SolveInst& I, bool x_zero, bool rhs_in_kernel = false) {
  SolveState s;
  memset(&s, 0, sizeof(s));
  s.action = x_zero ? ACT_RESID_ZERO : ACT_MV_RESIDUAL;
  I.rhs_resid = rhs_in_kernel && I.refined ? 1 : 0;
  I.rhs_r0 = rhs_in_kernel && x_zero ? 1 : 0;
  if (rhs_in_kernel) {
    s.action = ACT_RHS;
    s.prec = I.rhs_resid;
  }
  s.xinit = x_zero ? 0 : 1;
  s.status = IBDL_ERR_NOT_CONVERGED;
  s.bnorm = -1.0;
  return s;
}

void info_from_state(const SolveState& st, const double* hist, ibdl_solve_info* info) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  info->iters = st.iters;
  info->refine_steps = st.outer;
  info->matvecs = st.matvecs;
  info->residual_updates = st.nupd;
  info->rel_residual = st.rel;
  const int nh = st.nhist < 256 ? st.nhist : 256;
  info->n_history = nh;
  for (int i = 0; i < nh; ++i) info->residual_history[i] = hist[i];
}

ibdl_status vec_norm(ibdl_geometry_s* g, const double* v, double* out, cudaStream_t st) {
  IBDL_CU(krylov_dot_norm(g->kry, v, g->kry.scal + 4, st));
  cudaError_t ce;
  *out = read_scalar(g, g->kry.scal + 4, 4, st, &ce);
  if (ce) return cuda_fail(ce, "read norm");
  return IBDL_OK;
}

// Tile lists of `rows` rows per tile into `out` (3D: with the empty-plane
// flags in dz), from caller-provided buffers; asynchronous on st.
cudaError_t build_tiles(ibdl_geometry_s* g, int rows, int* start, int* cursor, int* counts,
                        int* pts, int* spts, unsigned char* dz, Bins* out, cudaStream_t st) {
  const GridDesc& gd = g->grid;
  const int n = gd.n;
  // the x passes index a tile's pencils with shifts
  if (rows < 2 || (rows & (rows - 1))) return cudaErrorInvalidValue;
  const int ntiles = (n / rows) * (gd.dim == 3 ? n : 1);
  cudaError_t e = launch_bins(gd, g->pd, rows, ntiles, start, cursor, counts, pts, spts, st);
  if (e) return e;
  out->rows = rows;
  out->ntiles = ntiles;
  out->start = start;
  out->pts = pts;
  out->spts = spts;
  out->zempty = nullptr;
  if (gd.dim == 3) {
    // planes no point touches: their spectrum stays zero through the x and
    // y passes of a matvec
    if ((e = launch_plane_flags(start, n / rows, n, dz, st))) return e;
    out->zempty = dz;
  }
  return cudaSuccess;
}

// ---- autotuner ---------------------------------------------------------------
// Rows per tile of the x passes (the spread bin size, and how many pencils a
// row tile transforms together) for each (device, dim, n, precision): the
// first geometry of a kind times a matvec (band-only field solve and
// interpolation, in its inner precision) for every admissible tiling -- an
// even R with n/R >= 4 tiles per plane, R <= n - 5 (the tile-list rule) and
// float64 row buffers within the persistent solver's 100 KB -- and the
// fastest is kept for the process.  Off (ibdl_tuning_enable(0)), the fixed
// rule rows_per_tile applies.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;

// the tilings the tuner times (and ibdl_tuning_set accepts)
bool tiling_admissible(int n, int R) {
  return R >= 2 && R <= 32 && (R & (R - 1)) == 0 && n / R >= 4 && R <= n - 5 &&
         rows_smem_bytes<double>(n, R) <= 100 * 1024;
}
std::atomic<int> g_tuning_on{1};
// set while the server builds a request's geometry: it takes a cached
// tiling or the rule, never times candidates beside a running slice
thread_local bool tl_no_tune = false;

// Per-matvec time of a candidate: one warm-up matvec, three timed ones,
// and, when those took under a millisecond (small grids, where a few
// launches are all noise), as many more as fill about a millisecond (at
// most 64), which are the ones timed.
ibdl_status time_matvecs(ibdl_geometry_s* g, const double* q, double* y, cudaEvent_t e0,
                         cudaEvent_t e1, cudaStream_t st, float* per_ms) {
  ibdl_status status = matvec_prec(g, g->precision, q, y, st);
  int reps = 3;
  for (int round = 0; round < 2 && status == IBDL_OK; ++round) {
    cudaError_t e = cudaEventRecord(e0, st);
    for (int rep = 0; rep < reps && !e && status == IBDL_OK; ++rep)
      status = matvec_prec(g, g->precision, q, y, st);
    float ms = 0;
    if (!e && status == IBDL_OK) e = cudaEventRecord(e1, st);
    if (!e && status == IBDL_OK) e = cudaEventSynchronize(e1);
    if (!e && status == IBDL_OK) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e) return cuda_fail(e, "autotuner timing");
    if (status != IBDL_OK) break;
    *per_ms = ms / reps;
    if (ms >= 1.0f) break;
    const float t = ms / reps > 1e-4f ? ms / reps : 1e-4f;
    reps = (int)(1.0f / t) + 1;
    if (reps > 64) reps = 64;
  }
  return status;
}

ibdl_status tuned_rows(ibdl_geometry_s* g, int* rows_out, cudaStream_t st) {
  const GridDesc& gd = g->grid;
  const int n = gd.n, dim = gd.dim;
  if (!g_tuning_on.load()) return IBDL_OK;
  int dev = 0;
  IBDL_CU(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, dim, n, g->precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      *rows_out = it->second;
      return IBDL_OK;
    }
  }
  if (tl_no_tune || g->grid.spectral) return IBDL_OK;
  std::vector<int> cand;
  for (int R = 2; R <= 32; R *= 2)
    if (tiling_admissible(n, R)) cand.push_back(R);
  if (cand.size() < 2) return IBDL_OK;
  cudaMemPool_t pool;
  IBDL_CU(workspace_pool(&pool));
  const int m = g->m;
  double *q = nullptr, *y = nullptr;
  IBDL_CU(cudaMallocFromPoolAsync((void**)&q, sizeof(double) * m, pool, st));
  IBDL_CU(cudaMallocFromPoolAsync((void**)&y, sizeof(double) * m, pool, st));
  {
    std::vector<double> hq(m);
    uint64_t r = 0x9e3779b97f4a7c15ull;
    for (int i = 0; i < m; ++i) {
      r ^= r << 13;
      r ^= r >> 7;
      r ^= r << 17;
      hq[i] = (double)(r >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    IBDL_CU(cudaMemcpyAsync(q, hq.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
  }
  cudaEvent_t e0, e1;
  IBDL_CU(cudaEventCreate(&e0));
  IBDL_CU(cudaEventCreate(&e1));
  const Bins saved = g->bins;
  std::vector<float> times;
  ibdl_status status = IBDL_OK;
  for (int R : cand) {
    const int ntiles = (n / R) * (dim == 3 ? n : 1);
    void* buf = nullptr;
    const size_t ni = 3 * ((size_t)ntiles + 1) + 2 * (size_t)bins_capacity(dim, R, m);
    cudaError_t e = cudaMallocFromPoolAsync(&buf, ni * sizeof(int) + n, pool, st);
    if (e) {
      status = cuda_fail(e, "autotuner buffers");
      break;
    }
    int* start = static_cast<int*>(buf);
    int* cursor = start + ntiles + 1;
    int* counts = cursor + ntiles + 1;
    int* pts = counts + ntiles + 1;
    int* spts = pts + bins_capacity(dim, R, m);
    unsigned char* dz = reinterpret_cast<unsigned char*>(spts + bins_capacity(dim, R, m));
    e = build_tiles(g, R, start, cursor, counts, pts, spts, dz, &g->bins, st);
    float ms = 0;
    if (e) status = cuda_fail(e, "autotuner tiles");
    if (status == IBDL_OK) status = time_matvecs(g, q, y, e0, e1, st, &ms);
    cudaFreeAsync(buf, st);
    if (status != IBDL_OK) break;
    times.push_back(ms);
  }
  // the largest tiling within 15% of the fastest: fewer, larger tiles cost
  // a lone matvec little on a small grid, but they shorten the persistent
  // solver's phases when many instances share its blocks (256 C4 stars:
  // 39.2 ms per launch with the 2-row tiles a 3-matvec timing picked at
  // 128^2 and 256^2, 26-30 ms with 32 and 16 rows; with a 5% margin the
  // picks still moved between runs)
  int best = cand[0];
  if (status == IBDL_OK && !times.empty()) {
    float tmin = times[0];
    for (float t : times) tmin = t < tmin ? t : tmin;
    for (size_t k = 0; k < times.size(); ++k)
      if (times[k] <= 1.15f * tmin) best = cand[k];
  }
  g->bins = saved;
  cudaFreeAsync(q, st);
  cudaFreeAsync(y, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != IBDL_OK) return status;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  }
  *rows_out = best;
  return IBDL_OK;
}

// Pencils per work item of the pencil passes, per (device, dim, n,
// precision): after the tiling, the first geometry of a kind times a matvec
// of its inner precision (float32 for a refined geometry, float64 else) for
// every admissible c of each pencil layout in turn (3D: the solve pass, then
// the y passes; c a power of two <= 16 whose item fits 100 KB of shared
// memory, strided items at least 2), keeping the fastest.  The other
// precision class keeps the fixed rule.
std::map<std::tuple<int, int, int, int>, std::array<int, 2>> g_tuned_pc;

// The tensor map of the staged z pass encodes its box (c pencils): encode
// again whenever the float32 solve layout changes.
ibdl_status refresh_maps(ibdl_geometry_s* g) {
  if (!g->ws32.zmap) return IBDL_OK;
  IBDL_CU(make_zsolve_map<float>(g->grid, g->ws32.spec, &g->zmap32));
  return IBDL_OK;
}

ibdl_status tuned_pencils(ibdl_geometry_s* g, cudaStream_t st) {
  GridDesc& gd = g->grid;
  const int n = gd.n, dim = gd.dim, cls = g->precision == IBDL_FP32_REFINED ? 0 : 1;
  if (!g_tuning_on.load() || gd.spectral || g->eta > 0) return IBDL_OK;
  int dev = 0;
  IBDL_CU(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, dim, n, g->precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_pc.find(key);
    if (it != g_tuned_pc.end()) {
      gd.pcap[cls][0] = it->second[0];
      gd.pcap[cls][1] = it->second[1];
      return refresh_maps(g);
    }
  }
  if (tl_no_tune) return IBDL_OK;
  cudaMemPool_t pool;
  IBDL_CU(workspace_pool(&pool));
  const int m = g->m;
  double *q = nullptr, *y = nullptr;
  IBDL_CU(cudaMallocFromPoolAsync((void**)&q, sizeof(double) * m, pool, st));
  IBDL_CU(cudaMallocFromPoolAsync((void**)&y, sizeof(double) * m, pool, st));
  IBDL_CU(cudaMemsetAsync(q, 0, sizeof(double) * m, st));
  IBDL_CU(launch_fill(m, q, 1.0, st));
  cudaEvent_t e0, e1;
  IBDL_CU(cudaEventCreate(&e0));
  IBDL_CU(cudaEventCreate(&e1));
  ibdl_status status = IBDL_OK;
  const int passes[2] = {1, 0};
  for (int w = 0; w < (dim == 3 ? 2 : 1) && status == IBDL_OK; ++w) {
    const int which = passes[w];
    const PencilLayout base = cls == 0 ? solve_layout<float>(dim, n, which)
                                       : solve_layout<double>(dim, n, which);
    std::vector<int> cand;
    for (int c = 1; c <= 16; c *= 2) {
      const bool ok = cls == 0 ? pencils_admissible<float>(n, base.estride, base.pg, c)
                               : pencils_admissible<double>(n, base.estride, base.pg, c);
      if (ok) cand.push_back(c);
    }
    if (cand.size() < 2) continue;
    int best = 0;
    float best_ms = 1e30f;
    for (int c : cand) {
      gd.pcap[cls][which] = c;
      if ((status = refresh_maps(g)) != IBDL_OK) break;
      float ms = 0;
      if ((status = time_matvecs(g, q, y, e0, e1, st, &ms)) != IBDL_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    gd.pcap[cls][which] = best;
  }
  cudaFreeAsync(q, st);
  cudaFreeAsync(y, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status == IBDL_OK) status = refresh_maps(g);
  if (status != IBDL_OK) return status;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_pc[key] = {gd.pcap[cls][0], gd.pcap[cls][1]};
  return IBDL_OK;
}

// FFT plan variant of the float32 transforms, per (device, dim, n,
// precision): a float32-refined 2D geometry of a size with two plans
// (n = 512, 1024: radices as even as possible, or radix-16 passes first,
// plan_lr) times its float32 matvec in each, after the tiling and the
// pencils per item, and keeps the radix-16-first plan only when it is at
// least 2% faster.  3D geometries and float64 precision keep the balanced
// plan (the double-float and float64 transforms have one plan each).
std::map<std::tuple<int, int, int, int>, int> g_tuned_plan;

ibdl_status tuned_plan(ibdl_geometry_s* g, cudaStream_t st) {
  GridDesc& gd = g->grid;
  const int n = gd.n, dim = gd.dim;
  if (!g_tuning_on.load() || gd.spectral || g->eta > 0) return IBDL_OK;
  if (g->precision != IBDL_FP32_REFINED || !plan_offered(gd.log2n, 1)) return IBDL_OK;
  int dev = 0;
  IBDL_CU(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, dim, n, g->precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_plan.find(key);
    if (it != g_tuned_plan.end()) return dim == 2 ? set_float_plan(g, it->second) : IBDL_OK;
  }
  if (tl_no_tune || dim != 2) return IBDL_OK;
  cudaMemPool_t pool;
  IBDL_CU(workspace_pool(&pool));
  const int m = g->m;
  double *q = nullptr, *y = nullptr;
  IBDL_CU(cudaMallocFromPoolAsync((void**)&q, sizeof(double) * m, pool, st));
  IBDL_CU(cudaMallocFromPoolAsync((void**)&y, sizeof(double) * m, pool, st));
  IBDL_CU(cudaMemsetAsync(q, 0, sizeof(double) * m, st));
  IBDL_CU(launch_fill(m, q, 1.0, st));
  cudaEvent_t e0, e1;
  IBDL_CU(cudaEventCreate(&e0));
  IBDL_CU(cudaEventCreate(&e1));
  float ms[kPlanVariants] = {0, 0};
  ibdl_status status = IBDL_OK;
  for (int v = 0; v < kPlanVariants && status == IBDL_OK; ++v) {
    if ((status = set_float_plan(g, v)) != IBDL_OK) break;
    status = time_matvecs(g, q, y, e0, e1, st, &ms[v]);
  }
  const int best = (status == IBDL_OK && ms[1] < 0.98f * ms[0]) ? 1 : 0;
  cudaFreeAsync(q, st);
  cudaFreeAsync(y, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const ibdl_status s2 = set_float_plan(g, best);
  if (status != IBDL_OK) return status;
  if (s2 != IBDL_OK) return s2;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_plan[key] = best;
  return IBDL_OK;
}

ibdl_status check_handle(ibdl_geometry g) {
  if (!g) return fail(IBDL_ERR_INVALID_ARG, "NULL geometry handle");
  return IBDL_OK;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================

extern "C" {

void ibdl_solve_opts_default(ibdl_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->restart = 30;
  o->max_iters = 500;
  o->max_refine = 8;
  o->engine = 0;
  o->inner_tol = 1e-5;
  o->x0 = nullptr;
}

ibdl_status ibdl_create_geometry(const ibdl_geometry_desc* d, void* stream, ibdl_geometry* out) {
  g_err.clear();
  if (!d || !out) return fail(IBDL_ERR_INVALID_ARG, "NULL desc or out");
  cudaStream_t st = (cudaStream_t)stream;
  const int dim = d->dim, n = d->n;
  if (dim != 2 && dim != 3) return fail(IBDL_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (n < 16 || (n & (n - 1)) != 0 || n > (dim == 2 ? kMaxN2 : kMaxN3))
    return fail(IBDL_ERR_INVALID_ARG, "n must be a power of two in [16, 2048] (2D) / [16, 512] (3D)");
  if (d->m < 1 || d->m > kMaxPoints)
    return fail(IBDL_ERR_INVALID_ARG, "m out of range (1 .. 16776960)");
  if (!(d->box_len > 0) || !isfinite(d->box_len))
    return fail(IBDL_ERR_INVALID_ARG, "box_len must be positive and finite");
  if (!(d->kappa > 0))
    return fail(IBDL_ERR_INVALID_ARG, "kappa must be positive (or +inf for Poisson)");
  if (isinf(d->kappa) && d->bc != IBDL_DIRICHLET)
    return fail(IBDL_ERR_UNSUPPORTED, "the Poisson limit (kappa = inf) is Dirichlet only");
  if (!(d->eta >= 0) || !isfinite(d->eta))
    return fail(IBDL_ERR_INVALID_ARG, "eta must be finite and >= 0");
  if (d->eta > 0 && !isinf(d->kappa))
    return fail(IBDL_ERR_INVALID_ARG, "eta > 0 (completed IBDL) needs kappa = inf");
  if (d->disc != IBDL_DISC_FD && d->disc != IBDL_DISC_SPECTRAL)
    return fail(IBDL_ERR_INVALID_ARG, "unknown discretisation");
  if (d->disc == IBDL_DISC_SPECTRAL && d->eta > 0)
    return fail(IBDL_ERR_UNSUPPORTED, "the completed system uses the finite-difference "
                                      "discretisation");
  if (d->delta != IBDL_DELTA_PESKIN4 && d->delta != IBDL_DELTA_COS4)
    return fail(IBDL_ERR_INVALID_ARG, "unknown delta");
  if (d->bc != IBDL_DIRICHLET && d->bc != IBDL_NEUMANN)
    return fail(IBDL_ERR_INVALID_ARG, "unknown bc");
  if (d->precision != IBDL_FP64 && d->precision != IBDL_FP32_REFINED)
    return fail(IBDL_ERR_INVALID_ARG, "unknown precision");
  for (int c = 0; c < 3; ++c)
    if (!isfinite(d->origin[c])) return fail(IBDL_ERR_INVALID_ARG, "origin not finite");
  if (!d->x || !d->y || !d->nx || !d->ny || !d->w || (dim == 3 && (!d->z || !d->nz)))
    return fail(IBDL_ERR_INVALID_ARG, "NULL point, normal or weight array");

  ibdl_geometry_s* g = new ibdl_geometry_s();
  g->alloc_st = st;
  auto cleanup = [&](ibdl_status s) {
    cudaStreamSynchronize(st);  // nothing in flight may use the freed blocks
    delete g;
    return s;
  };
  const int m = (int)d->m;
  g->m = m;
  g->eta = d->eta;
  g->nsys = d->eta > 0 ? m + 1 : m;
  g->bc = d->bc;
  g->precision = d->precision;
  GridDesc& gd = g->grid;
  gd.dim = dim;
  gd.n = n;
  gd.log2n = 0;
  while ((1 << gd.log2n) < n) gd.log2n++;
  gd.h = d->box_len / n;
  gd.inv2h = 0.5 / gd.h;
  gd.kappa = d->kappa;
  gd.poisson = isinf(d->kappa) ? 1 : 0;
  gd.spectral = d->disc == IBDL_DISC_SPECTRAL ? 1 : 0;
  gd.delta = d->delta;
  for (int c = 0; c < 3; ++c) gd.origin[c] = c < dim ? d->origin[c] : 0.0;
  g->ncells = (int64_t)n * n * (dim == 3 ? n : 1);

  ibdl_status s;
  double* pts;
  if ((s = g->alloc(&pts, (size_t)7 * m))) return cleanup(s);
  const double* src_arr[7] = {d->x, d->y, dim == 3 ? d->z : nullptr, d->nx, d->ny,
                              dim == 3 ? d->nz : nullptr, d->w};
  for (int a = 0; a < 7; ++a) {
    if (!src_arr[a]) {
      cudaMemsetAsync(pts + (size_t)a * m, 0, sizeof(double) * m, st);
      continue;
    }
    cudaError_t e = cudaMemcpyAsync(pts + (size_t)a * m, src_arr[a], sizeof(double) * m,
                                    cudaMemcpyDefault, st);
    if (e) return cleanup(cuda_fail(e, "copy geometry"));
  }
  // weights scaled by h^-d on the host side of the device copy
  {
    std::vector<double> hw(m);
    cudaError_t e = cudaMemcpyAsync(hw.data(), pts + (size_t)6 * m, sizeof(double) * m,
                                    cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cleanup(cuda_fail(e, "read weights"));
    std::vector<double> hx(m);
    const double hd = dim == 3 ? gd.h * gd.h * gd.h : gd.h * gd.h;
    for (int i = 0; i < m; ++i) {
      if (!isfinite(hw[i])) return cleanup(fail(IBDL_ERR_INVALID_ARG, "non-finite weight"));
      hw[i] /= hd;
    }
    for (int c = 0; c < dim; ++c) {
      e = cudaMemcpyAsync(hx.data(), pts + (size_t)c * m, sizeof(double) * m,
                          cudaMemcpyDeviceToHost, st);
      if (!e) e = cudaStreamSynchronize(st);
      if (e) return cleanup(cuda_fail(e, "read points"));
      for (int i = 0; i < m; ++i) {
        if (!isfinite(hx[i])) return cleanup(fail(IBDL_ERR_INVALID_ARG, "non-finite point"));
        g->xmax = fmax(g->xmax, fabs(hx[i]));
      }
    }
    e = cudaMemcpyAsync(pts + (size_t)6 * m, hw.data(), sizeof(double) * m,
                        cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cleanup(cuda_fail(e, "write weights"));
  }
  int* base;
  double* W64;
  float* W32;
  if ((s = g->alloc(&base, (size_t)3 * m))) return cleanup(s);
  if ((s = g->alloc(&W64, (size_t)12 * m))) return cleanup(s);
  if ((s = g->alloc(&W32, (size_t)12 * m))) return cleanup(s);
  PointData& pd = g->pd;
  pd.m = m;
  const double* X[3];
  int* B[3];
  double* WW[3];
  float* VV[3];
  for (int c = 0; c < 3; ++c) {
    X[c] = pts + (size_t)c * m;
    pd.X[c] = X[c];
    pd.nrm[c] = pts + (size_t)(3 + c) * m;
    B[c] = base + (size_t)c * m;
    WW[c] = W64 + (size_t)4 * c * m;
    VV[c] = W32 + (size_t)4 * c * m;
    pd.base[c] = B[c];
    pd.W64[c] = WW[c];
    pd.W32[c] = VV[c];
  }
  pd.w = pts + (size_t)6 * m;
  {
    // float copies of the normals and scaled weights for the float32 spread
    float* p32;
    if ((s = g->alloc(&p32, (size_t)4 * m))) return cleanup(s);
    cudaError_t e = launch_grid_to_float(pts + (size_t)3 * m, p32, (int64_t)3 * m, st);
    if (!e) e = launch_grid_to_float(pts + (size_t)6 * m, p32 + (size_t)3 * m, m, st);
    if (e) return cleanup(cuda_fail(e, "float copies"));
    for (int c = 0; c < 3; ++c) pd.nrm32[c] = p32 + (size_t)c * m;
    pd.w32 = p32 + (size_t)3 * m;
  }
  {
    cudaError_t e = launch_point_prep(gd, m, X, B, WW, VV, st);
    if (e) return cleanup(cuda_fail(e, "point prep"));
  }
  {
    cudaError_t e = configure_fft_kernels(n, 0);
    if (e) return cleanup(cuda_fail(e, "configure kernels"));
  }
  if ((s = g->alloc(&g->d_err, (size_t)1))) return cleanup(s);
  {
    cudaError_t e = cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), st);
    if (e) return cleanup(cuda_fail(e, "clear error word"));
  }
  if ((s = alloc_spectral<double>(g, g->ws64, st))) return cleanup(s);
  g->ws64.err = g->d_err;
  {
    // the double-float view shares the float64 spectrum (same 16-byte
    // complex) and grid; it has its own twiddle and sin^2 tables
    SpectralWs<dd>& w = g->wsdd;
    w.spec = reinterpret_cast<cdd*>(g->ws64.spec);
    w.grid = reinterpret_cast<dd*>(g->ws64.grid);
    w.acc = reinterpret_cast<cdd*>(g->ws64.acc);
    if ((s = fft_tables<dd>(n, &w.tw, &w.s2))) return cleanup(s);
  }
  if (d->precision == IBDL_FP32_REFINED) {
    if ((s = ensure32(g, st))) return cleanup(s);
  }

  // tile lists, with the rows per tile chosen by the autotuner
  int rows = rows_per_tile(dim, n);
  if ((s = tuned_rows(g, &rows, st))) return cleanup(s);
  {
    const int ntiles = (n / rows) * (dim == 3 ? n : 1);
    int *start, *cursor, *counts, *bpts, *spts;
    unsigned char* dz = nullptr;
    if ((s = g->alloc(&start, (size_t)ntiles + 1))) return cleanup(s);
    if ((s = g->alloc(&cursor, (size_t)ntiles + 1))) return cleanup(s);
    if ((s = g->alloc(&counts, (size_t)ntiles + 1))) return cleanup(s);
    if ((s = g->alloc(&bpts, (size_t)bins_capacity(dim, rows, m)))) return cleanup(s);
    if ((s = g->alloc(&spts, (size_t)bins_capacity(dim, rows, m)))) return cleanup(s);
    if (dim == 3 && (s = g->alloc(&dz, (size_t)n))) return cleanup(s);
    cudaError_t e = build_tiles(g, rows, start, cursor, counts, bpts, spts, dz, &g->bins, st);
    if (e) return cleanup(cuda_fail(e, "binning"));
  }
  // pencils per item of the pencil passes, then the float32 FFT plan, with
  // the autotuner
  if ((s = tuned_pencils(g, st))) return cleanup(s);
  if ((s = tuned_plan(g, st))) return cleanup(s);

  // Krylov workspace (float64, restart up to 64)
  KrylovWs& k = g->kry;
  k.m = g->nsys;
  k.ld = (g->nsys + 31) / 32 * 32;
  k.restart = 64;
  k.nblk = (m + 2047) / 2048;
  if (k.nblk > 148) k.nblk = 148;
  if ((s = g->alloc(&k.V, (size_t)(k.restart + 1) * k.ld))) return cleanup(s);
  if ((s = g->alloc(&k.H, (size_t)(k.restart + 1) * k.restart))) return cleanup(s);
  if ((s = g->alloc(&k.cs, (size_t)k.restart))) return cleanup(s);
  if ((s = g->alloc(&k.sn, (size_t)k.restart))) return cleanup(s);
  if ((s = g->alloc(&k.gvec, (size_t)k.restart + 1))) return cleanup(s);
  if ((s = g->alloc(&k.ysol, (size_t)k.restart))) return cleanup(s);
  if ((s = g->alloc(&k.partial, (size_t)k.nblk * (k.restart + 2)))) return cleanup(s);
  if ((s = g->alloc(&k.scal, (size_t)8))) return cleanup(s);
  double* vecs;
  if ((s = g->alloc(&vecs, (size_t)7 * k.ld))) return cleanup(s);
  g->vb = vecs;
  g->vx = vecs + k.ld;
  g->vr = vecs + 2 * (size_t)k.ld;
  g->vt = vecs + 3 * (size_t)k.ld;
  g->vd = vecs + 4 * (size_t)k.ld;
  g->stage_a = vecs + 5 * (size_t)k.ld;
  g->stage_b = vecs + 6 * (size_t)k.ld;
  if ((s = g->alloc(&g->d_flag, (size_t)4))) return cleanup(s);
  if ((s = g->alloc(&g->cpart, (size_t)kRedBlocks + 1))) return cleanup(s);
  g->nchunk = (m + kSolverThreads - 1) / kSolverThreads;
  // a section holds one row per vector chunk, or per x tile in 2D (the
  // Arnoldi steps' first dot products come from the x-inverse tiles)
  g->nsec = g->nchunk > (dim == 2 ? g->bins.ntiles : 0) ? g->nchunk : g->bins.ntiles;
  if ((s = g->alloc(&g->ppart, (size_t)3 * g->nsec * (k.restart + 2)))) return cleanup(s);
  if ((s = g->alloc(&g->d_hist, (size_t)kHistCap))) return cleanup(s);
  if ((s = g->alloc(&g->d_inst, (size_t)1))) return cleanup(s);
  if ((s = g->alloc(&g->d_state, (size_t)1))) return cleanup(s);
  if ((s = g->alloc(&g->d_bar, (size_t)(4 + kSchedWords)))) return cleanup(s);

  g->solver_smem = solver_smem_bytes(gd, g->bins.rows, 1);
  if (g->solver_smem < 0) return cleanup(fail(IBDL_ERR_INVALID_ARG, "solver shared memory"));
  {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e) return cleanup(cuda_fail(e, "create sync"));
  }
  *out = g;
  return IBDL_OK;
}

void ibdl_destroy_geometry(ibdl_geometry g) {
  if (!g) return;
  cudaDeviceSynchronize();
  delete g;
}

ibdl_status ibdl_apply_precision(ibdl_geometry g, const double* q, double* y, int32_t precision,
                                 void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!q || !y) return fail(IBDL_ERR_INVALID_ARG, "NULL q or y");
  if (precision != IBDL_FP64 && precision != IBDL_FP32_REFINED && precision != IBDL_FP64_DF)
    return fail(IBDL_ERR_INVALID_ARG, "unknown precision");
  cudaStream_t st = (cudaStream_t)stream;
  const double* qd;
  IBDL_TRY(dev_in(q, g->nsys, g->stage_a, &qd, st));
  const bool ydev = is_device_ptr(y);
  double* yd = ydev ? y : g->stage_b;
  IBDL_TRY(sys_matvec(g, precision, qd, yd, st));
  if (!ydev) {
    IBDL_CU(cudaMemcpyAsync(y, yd, sizeof(double) * g->nsys, cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaStreamSynchronize(st));
  }
  return IBDL_OK;
}

ibdl_status ibdl_apply(ibdl_geometry g, const double* q, double* y, void* stream) {
  IBDL_TRY(check_handle(g));
  return ibdl_apply_precision(g, q, y, g->precision, stream);
}

ibdl_status ibdl_solve(ibdl_geometry g, const double* bdata, const double* g_grid, double* q_out,
                       const ibdl_solve_opts* opts_in, ibdl_solve_info* info, void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!bdata || !q_out) return fail(IBDL_ERR_INVALID_ARG, "NULL bdata or q_out");
  ibdl_solve_opts o;
  ibdl_solve_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (!(o.tol > 0) || !isfinite(o.tol)) return fail(IBDL_ERR_INVALID_ARG, "tol must be > 0");
  if (o.restart < 1 || o.restart > 64) return fail(IBDL_ERR_INVALID_ARG, "restart in 1..64");
  if (o.max_iters < 1) return fail(IBDL_ERR_INVALID_ARG, "max_iters >= 1");
  if (o.max_refine < 1) o.max_refine = 1;
  if (!(o.inner_tol > 0) || o.inner_tol >= 1) o.inner_tol = 1e-5;
  if (o.engine != 0 && o.engine != 1) return fail(IBDL_ERR_INVALID_ARG, "engine is 0 or 1");
  // the completed system (length m + 1) and the spectral discretisation run
  // on the launch-based engine
  if (g->eta > 0 || g->grid.spectral) o.engine = 1;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = g->m;
  const int ns = g->nsys;
  IBDL_TRY(g->ensure_host());
  // inputs
  IBDL_CU(cudaMemcpyAsync(g->stage_a, bdata, sizeof(double) * m, cudaMemcpyDefault, st));
  const double* gg = nullptr;
  IBDL_TRY(grid_in(g, g_grid, &gg, st));
  IBDL_CU(cudaMemsetAsync(g->d_flag, 0, sizeof(int), st));
  IBDL_CU(launch_nonfinite_check(m, g->stage_a, g->d_flag, st));
  // the persistent engine builds an unforced Neumann right-hand side itself
  const bool rhs_in_kernel = o.engine == 0 && g->bc == IBDL_NEUMANN && !gg;
  if (!rhs_in_kernel) IBDL_TRY(build_rhs(g, g->stage_a, gg, g->vb, st));
  bool x_zero = true;
  if (o.x0) {
    IBDL_CU(cudaMemcpyAsync(g->vx, o.x0, sizeof(double) * ns, cudaMemcpyDefault, st));
    IBDL_CU(launch_nonfinite_check(ns, g->vx, g->d_flag, st));
    x_zero = false;
  } else {
    IBDL_CU(cudaMemsetAsync(g->vx, 0, sizeof(double) * ns, st));
  }
  if (o.engine == 0) {
    // one persistent launch runs the whole solve; the host waits once
    *g->h_inst = make_inst(g, o, 1);
    g->h_inst->vdata = g->stage_a;
    *g->h_state = initial_state(*g->h_inst, x_zero, rhs_in_kernel);
    IBDL_CU(cudaMemcpyAsync(g->d_inst, g->h_inst, sizeof(SolveInst), cudaMemcpyHostToDevice, st));
    IBDL_CU(cudaMemcpyAsync(g->d_state, g->h_state, sizeof(SolveState), cudaMemcpyHostToDevice,
                            st));
    {
      char why[256];
      if (!solver_smem_fits(g->h_inst, 1, g->solver_smem, why, sizeof(why)))
        return fail(IBDL_ERR_INVALID_ARG, why);
    }
    IBDL_CU(launch_persistent_solve(g->d_inst, g->d_state, 1, g->d_bar, g->solver_smem, st));
    IBDL_CU(cudaMemcpyAsync(g->h_state, g->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost,
                            st));
    IBDL_CU(cudaMemcpyAsync(g->h_hist, g->d_hist, kHistCap * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    unsigned* hb = reinterpret_cast<unsigned*>(g->host_scal + 8);
    IBDL_CU(cudaMemcpyAsync(hb, g->d_bar, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    int* hflag = reinterpret_cast<int*>(g->host_scal + 10);
    IBDL_CU(cudaMemcpyAsync(hflag, g->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaMemcpyAsync(q_out, g->vx, sizeof(double) * m, cudaMemcpyDefault, st));
    IBDL_CU(cudaStreamSynchronize(st));
    info_from_state(*g->h_state, g->h_hist, info);
    if (*hflag) return fail(IBDL_ERR_NONFINITE, "non-finite boundary data or initial guess");
    if (hb[2]) return fail(IBDL_ERR_TIMEOUT, "persistent solver: a bounded device wait timed out");
    const int stt = g->h_state->status;
    if (stt == IBDL_ERR_NOT_CONVERGED) return fail(IBDL_ERR_NOT_CONVERGED, "GMRES reached max_iters");
    if (stt == IBDL_ERR_NONFINITE) return fail(IBDL_ERR_NONFINITE, "non-finite residual");
    return (ibdl_status)stt;
  }
  int flag = 0;
  IBDL_CU(cudaMemcpyAsync(&flag, g->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  IBDL_CU(cudaStreamSynchronize(st));
  if (flag) return fail(IBDL_ERR_NONFINITE, "non-finite boundary data or initial guess");
  double bnorm = 0;
  IBDL_TRY(vec_norm(g, g->vb, &bnorm, st));
  if (!isfinite(bnorm)) return fail(IBDL_ERR_NONFINITE, "non-finite right-hand side");

  GmresRun run;
  int refine = 0;
  ibdl_status status = IBDL_OK;
  if (bnorm == 0.0) {
    IBDL_CU(cudaMemsetAsync(g->vx, 0, sizeof(double) * ns, st));
    run.rel = 0;
  } else if (g->precision == IBDL_FP64) {
    status = gmres(g, IBDL_FP64, g->vb, g->vx, x_zero, bnorm, o.tol, o.restart, o.max_iters,
                   true, &run, st);
  } else {
    // FP32 operator inside GMRES (float64 Arnoldi/Givens), float64 residuals
    // outside: r = b - A64 x;  solve A32 d = r to inner_tol;  x += d.
    if (x_zero) {
      IBDL_CU(cudaMemcpyAsync(g->vr, g->vb, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
    } else {
      IBDL_TRY(sys_matvec(g, resid_prec(g), g->vx, g->vt, st));
      run.matvecs++;
      IBDL_CU(launch_axpby(ns, 1.0, g->vb, -1.0, g->vt, g->vr, st));
    }
    double rnorm = 0;
    IBDL_TRY(vec_norm(g, g->vr, &rnorm, st));
    run.rel = rnorm / bnorm;
    status = IBDL_ERR_NOT_CONVERGED;
    for (refine = 0; refine <= o.max_refine; ++refine) {
      if (!isfinite(run.rel)) {
        status = fail(IBDL_ERR_NONFINITE, "non-finite residual");
        break;
      }
      if (run.rel <= o.tol) {
        status = IBDL_OK;
        break;
      }
      if (refine == o.max_refine || run.iters >= o.max_iters) {
        status = fail(IBDL_ERR_NOT_CONVERGED, "refinement did not reach tol");
        break;
      }
      // inner solve: the residual vector is moved to vd's right-hand side slot
      IBDL_CU(cudaMemcpyAsync(g->vt, g->vr, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
      IBDL_CU(cudaMemsetAsync(g->vd, 0, sizeof(double) * ns, st));
      GmresRun inner;
      inner.iters = run.iters;
      const double itol = fmax(o.inner_tol, 0.5 * o.tol * bnorm / rnorm);
      double* rhs = g->stage_b;  // keep r intact while gmres reuses vr/vt
      IBDL_CU(cudaMemcpyAsync(rhs, g->vr, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
      ibdl_status si = gmres(g, IBDL_FP32_REFINED, rhs, g->vd, true, rnorm, itol, o.restart,
                             o.max_iters, false, &inner, st);
      run.iters = inner.iters;
      run.matvecs += inner.matvecs;
      if (si != IBDL_OK && si != IBDL_ERR_NOT_CONVERGED) {
        status = si;
        break;
      }
      IBDL_CU(launch_axpby(ns, 1.0, g->vx, 1.0, g->vd, g->vx, st));
      IBDL_TRY(sys_matvec(g, resid_prec(g), g->vx, g->vt, st));
      run.matvecs++;
      IBDL_CU(launch_axpby(ns, 1.0, g->vb, -1.0, g->vt, g->vr, st));
      IBDL_TRY(vec_norm(g, g->vr, &rnorm, st));
      run.rel = rnorm / bnorm;
      run.hist.push_back(run.rel);
    }
  }
  IBDL_CU(cudaMemcpyAsync(q_out, g->vx, sizeof(double) * ns, cudaMemcpyDefault, st));
  unsigned* herr = reinterpret_cast<unsigned*>(g->host_scal + 12);
  IBDL_CU(cudaMemcpyAsync(herr, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  IBDL_CU(cudaStreamSynchronize(st));
  if (*herr) {
    // a bounded wait inside a transform gave up: the result is not valid
    cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), st);
    status = fail(IBDL_ERR_TIMEOUT, "a bounded wait for a staged copy timed out");
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = run.iters;
    info->refine_steps = refine;
    info->matvecs = run.matvecs;
    info->rel_residual = run.rel;
    const int nh = (int)run.hist.size() < 256 ? (int)run.hist.size() : 256;
    info->n_history = nh;
    for (int i = 0; i < nh; ++i) info->residual_history[i] = run.hist[i];
  }
  return status;
}

ibdl_status ibdl_evaluate(ibdl_geometry g, const double* q, const double* vb, const double* g_grid,
                          double* u_out, void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!q || !u_out) return fail(IBDL_ERR_INVALID_ARG, "NULL q or u_out");
  if (g->bc == IBDL_DIRICHLET && vb) return fail(IBDL_ERR_INVALID_ARG, "vb is Neumann-only");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = g->m;
  IBDL_CU(cudaMemcpyAsync(g->stage_a, q, sizeof(double) * g->nsys, cudaMemcpyDefault, st));
  if (vb) IBDL_CU(cudaMemcpyAsync(g->stage_b, vb, sizeof(double) * m, cudaMemcpyDefault, st));
  const double* gg = nullptr;
  IBDL_TRY(grid_in(g, g_grid, &gg, st));
  SpreadSrc src;
  src.q_div = g->stage_a;
  src.coef_div = 1.0;
  if (vb) {
    src.v_plain = g->stage_b;
    src.coef_plain = 1.0;
  }
  if (g->eta > 0) {
    // completed: u = -Delta_0^{-1} ((S~ + eta S) Q - g~) + u_bar
    src.v_plain = g->stage_a;
    src.coef_plain = g->eta;
  }
  if (gg) {
    src.f_grid = gg;
    src.coef_grid = -1.0;
  }
  const bool udev = is_device_ptr(u_out);
  double* ud = udev ? u_out : g->ws64.grid;
  IBDL_TRY((field_solve<double, double>(g, src, ud, st)));
  if (g->eta > 0) IBDL_CU(launch_add_scalar(g->ncells, ud, g->stage_a + m, st));
  if (!udev) {
    IBDL_CU(cudaMemcpyAsync(u_out, ud, sizeof(double) * g->ncells, cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaStreamSynchronize(st));
  }
  return IBDL_OK;
}

static ibdl_status grid_out_begin(ibdl_geometry g, double* out, double** dev) {
  if (is_device_ptr(out)) {
    *dev = out;
    return IBDL_OK;
  }
  if (!g->grid_stage) IBDL_TRY(g->alloc(&g->grid_stage, (size_t)g->ncells));
  *dev = g->grid_stage;
  return IBDL_OK;
}

static ibdl_status grid_out_end(ibdl_geometry g, double* out, double* dev, cudaStream_t st) {
  if (dev == out) return IBDL_OK;
  IBDL_CU(cudaMemcpyAsync(out, dev, sizeof(double) * g->ncells, cudaMemcpyDeviceToHost, st));
  IBDL_CU(cudaStreamSynchronize(st));
  return IBDL_OK;
}

static ibdl_status spread_common(ibdl_geometry g, const double* v, double* f_out, int precision,
                                 bool div, void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (div && g->grid.spectral)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_spread_div is the finite-difference S~");
  if (!v || !f_out) return fail(IBDL_ERR_INVALID_ARG, "NULL input or output");
  if (precision != 0 && precision != 1) return fail(IBDL_ERR_INVALID_ARG, "precision");
  cudaStream_t st = (cudaStream_t)stream;
  IBDL_CU(cudaMemcpyAsync(g->stage_a, v, sizeof(double) * g->m, cudaMemcpyDefault, st));
  SpreadSrc src;
  if (div) {
    src.q_div = g->stage_a;
    src.coef_div = 1.0;
  } else {
    src.v_plain = g->stage_a;
    src.coef_plain = 1.0;
  }
  double* fd;
  IBDL_TRY(grid_out_begin(g, f_out, &fd));
  if (precision == 1) {
    IBDL_TRY(ensure32(g, st));
    IBDL_CU(launch_rows_fwd<float>(g->grid, g->pd, g->bins, src, g->ws32, fd, st));
  } else {
    IBDL_CU(launch_rows_fwd<double>(g->grid, g->pd, g->bins, src, g->ws64, fd, st));
  }
  return grid_out_end(g, f_out, fd, st);
}

ibdl_status ibdl_spread_div(ibdl_geometry g, const double* q, double* f_out, int32_t precision,
                            void* stream) {
  return spread_common(g, q, f_out, precision, true, stream);
}

ibdl_status ibdl_spread(ibdl_geometry g, const double* v, double* f_out, int32_t precision,
                        void* stream) {
  return spread_common(g, v, f_out, precision, false, stream);
}

ibdl_status ibdl_helmholtz(ibdl_geometry g, const double* f, double* v_out, int32_t precision,
                           void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (g->grid.spectral)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_helmholtz is the finite-difference solve");
  if (!f || !v_out) return fail(IBDL_ERR_INVALID_ARG, "NULL input or output");
  if (precision != 0 && precision != 1) return fail(IBDL_ERR_INVALID_ARG, "precision");
  cudaStream_t st = (cudaStream_t)stream;
  const double* fd;
  IBDL_TRY(grid_in(g, f, &fd, st));
  double* vd;
  if (is_device_ptr(v_out)) {
    vd = v_out;
  } else {
    // the staging grid may hold f; the float64 workspace grid is free here
    vd = g->ws64.grid;
  }
  SpreadSrc src;
  src.f_grid = fd;
  src.coef_grid = 1.0;
  if (precision == 1) {
    IBDL_TRY(ensure32(g, st));
    IBDL_TRY((field_solve<float, double>(g, src, vd, st)));
  } else {
    IBDL_TRY((field_solve<double, double>(g, src, vd, st)));
  }
  if (vd != v_out) {
    IBDL_CU(cudaMemcpyAsync(v_out, vd, sizeof(double) * g->ncells, cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaStreamSynchronize(st));
  }
  return IBDL_OK;
}

ibdl_status ibdl_interp(ibdl_geometry g, const double* u, double* y_out, int32_t precision,
                        void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!u || !y_out) return fail(IBDL_ERR_INVALID_ARG, "NULL input or output");
  if (precision != 0 && precision != 1) return fail(IBDL_ERR_INVALID_ARG, "precision");
  cudaStream_t st = (cudaStream_t)stream;
  const double* ud;
  IBDL_TRY(grid_in(g, u, &ud, st));
  const bool ydev = is_device_ptr(y_out);
  double* yd = ydev ? y_out : g->stage_b;
  if (precision == 1) {
    IBDL_TRY(ensure32(g, st));
    IBDL_CU(launch_grid_to_float(ud, g->ws32.grid, g->ncells, st));
    IBDL_CU(launch_interp<float>(g->grid, g->pd, g->ws32.grid, nullptr, 0.0, yd, st));
  } else {
    IBDL_CU(launch_interp<double>(g->grid, g->pd, ud, nullptr, 0.0, yd, st));
  }
  if (!ydev) {
    IBDL_CU(cudaMemcpyAsync(y_out, yd, sizeof(double) * g->m, cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaStreamSynchronize(st));
  }
  return IBDL_OK;
}

ibdl_status ibdl_indicator(ibdl_geometry g, double* chi_h_out, uint8_t* chi_out, void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!chi_h_out && !chi_out) return fail(IBDL_ERR_INVALID_ARG, "no output requested");
  cudaStream_t st = (cudaStream_t)stream;
  // Delta u = -S~ 1: spread-divergence of Q = 1, then the mean-zero Poisson
  // solve whatever the geometry's kappa
  IBDL_CU(launch_fill(g->m, g->stage_a, 1.0, st));
  SpreadSrc src;
  src.q_div = g->stage_a;
  src.coef_div = 1.0;
  const GridDesc saved = g->grid;
  g->grid.poisson = 1;
  const ibdl_status fs = field_solve<double, double>(g, src, g->ws64.grid, st);
  g->grid = saved;
  IBDL_TRY(fs);
  double* hd = nullptr;
  if (chi_h_out) IBDL_TRY(grid_out_begin(g, chi_h_out, &hd));
  unsigned char* cd = nullptr;
  const bool cdev = chi_out && is_device_ptr(chi_out);
  cudaMemPool_t pool;
  if (chi_out && !cdev) {
    IBDL_CU(workspace_pool(&pool));
    IBDL_CU(cudaMallocFromPoolAsync((void**)&cd, (size_t)g->ncells, pool, st));
  } else {
    cd = reinterpret_cast<unsigned char*>(chi_out);
  }
  cudaError_t e = launch_indicator(g->ncells, g->ws64.grid, hd, cd, st);
  if (!e && chi_out && !cdev) {
    e = cudaMemcpyAsync(chi_out, cd, (size_t)g->ncells, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(cd, st);
    if (!e) e = cudaStreamSynchronize(st);
  }
  if (e) return cuda_fail(e, "indicator");
  if (chi_h_out) IBDL_TRY(grid_out_end(g, chi_h_out, hd, st));
  return IBDL_OK;
}

ibdl_status ibdl_near_boundary(ibdl_geometry g, const double* u_in, const double* ub,
                               const uint8_t* inside, int32_t m1, double m2, double* u_out,
                               void* stream) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  if (!u_in || !ub || !inside || !u_out) return fail(IBDL_ERR_INVALID_ARG, "NULL argument");
  if (g->m < 3) return fail(IBDL_ERR_INVALID_ARG, "at least three boundary points are needed");
  if (m1 < 1 || m1 > g->grid.n / 2) return fail(IBDL_ERR_INVALID_ARG, "m1 in 1 .. n/2");
  if (!(m2 > 0) || !isfinite(m2)) return fail(IBDL_ERR_INVALID_ARG, "m2 must be > 0");
  const int64_t nn = g->ncells;
  if (u_out < u_in + nn && u_in < u_out + nn)
    return fail(IBDL_ERR_INVALID_ARG, "u_in and u_out overlap");
  cudaStream_t st = (cudaStream_t)stream;
  const double* ubd;
  IBDL_TRY(dev_in(ub, g->m, g->stage_a, &ubd, st));
  const double* uind;
  IBDL_TRY(grid_in(g, u_in, &uind, st));
  const bool udev = is_device_ptr(u_out);
  double* uoutd = udev ? u_out : g->ws64.grid;
  const bool idev = is_device_ptr(inside);
  // scratch: the kernels' buffers, then a copy of a host mask
  const size_t kb = (near_scratch_bytes(g->grid.dim, g->grid.n, g->m, m1) + 15) / 16 * 16;
  const size_t bytes = kb + (idev ? 0 : (size_t)nn);
  cudaMemPool_t pool;
  IBDL_CU(workspace_pool(&pool));
  unsigned char* scratch = nullptr;
  IBDL_CU(cudaMallocFromPoolAsync((void**)&scratch, bytes, pool, st));
  const unsigned char* insd = inside;
  cudaError_t e = cudaSuccess;
  if (!idev) {
    e = cudaMemcpyAsync(scratch + kb, inside, (size_t)nn, cudaMemcpyHostToDevice, st);
    insd = scratch + kb;
  }
  double cmax = g->xmax;  // bounds every point and node coordinate
  for (int c = 0; c < g->grid.dim; ++c)
    cmax = fmax(cmax, fabs(g->grid.origin[c]) + g->grid.h * g->grid.n);
  if (!e)
    e = launch_near_boundary(g->grid, g->pd, ubd, uind, insd, m1, m2, cmax, uoutd, scratch, st);
  if (!e && !udev)
    e = cudaMemcpyAsync(u_out, uoutd, sizeof(double) * nn, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(scratch, st);
  if (!e && (!udev || !idev)) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(e, "near-boundary values");
  return IBDL_OK;
}

ibdl_status ibdl_selftest_bounded_wait(uint32_t spin_limit, void* stream) {
  g_err.clear();
  if (spin_limit < 1 || spin_limit > (1u << 24))
    return fail(IBDL_ERR_INVALID_ARG, "spin_limit in 1 .. 2^24");
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemPool_t pool;
  IBDL_CU(workspace_pool(&pool));
  unsigned* bar = nullptr;
  IBDL_CU(cudaMallocFromPoolAsync((void**)&bar, 4 * sizeof(unsigned), pool, st));
  unsigned flag = 0;
  cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st);
  if (!e) e = launch_barrier_selftest(bar, spin_limit, st);
  if (!e) e = cudaMemcpyAsync(&flag, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(bar, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(e, "bounded-wait self-test");
  if (flag) return fail(IBDL_ERR_TIMEOUT, "the self-test wait gave up, as designed");
  return IBDL_OK;
}

ibdl_status ibdl_get_geometry_info(ibdl_geometry g, ibdl_geometry_info* info) {
  IBDL_TRY(check_handle(g));
  if (!info) return fail(IBDL_ERR_INVALID_ARG, "NULL info");
  memset(info, 0, sizeof(*info));
  info->dim = g->grid.dim;
  info->n = g->grid.n;
  info->m = g->m;
  info->h = g->grid.h;
  info->kappa = g->grid.kappa;
  info->bc = g->bc;
  info->delta = g->grid.delta;
  info->precision = g->precision;
  info->device_bytes = g->bytes;
  info->fft_passes = fft_kernels_per_solve<double>(g->grid.dim);
  info->rows_per_tile = g->bins.rows;
  info->fft_plan = g->grid.fplan;
  // the pencils per item the passes of the geometry's inner precision use
  if (g->precision == IBDL_FP32_REFINED) {
    info->pencils_per_item[0] = solve_layout<float>(g->grid, 1).c;
    info->pencils_per_item[1] = g->grid.dim == 3 ? solve_layout<float>(g->grid, 0).c : 0;
  } else {
    info->pencils_per_item[0] = solve_layout<double>(g->grid, 1).c;
    info->pencils_per_item[1] = g->grid.dim == 3 ? solve_layout<double>(g->grid, 0).c : 0;
  }
  return IBDL_OK;
}


struct ibdl_batch_s {
  int cap = 0;
  SolveInst* d_inst = nullptr;
  SolveState* d_state = nullptr;
  unsigned* d_bar = nullptr;
  SolveInst* h_inst = nullptr;
  SolveState* h_state = nullptr;
  ~ibdl_batch_s() {
    if (d_inst) cudaFree(d_inst);
    if (d_state) cudaFree(d_state);
    if (d_bar) cudaFree(d_bar);
    if (h_inst) cudaFreeHost(h_inst);
    if (h_state) cudaFreeHost(h_state);
  }
};

ibdl_status ibdl_batch_create(int32_t capacity, ibdl_batch* out) {
  g_err.clear();
  if (!out) return fail(IBDL_ERR_INVALID_ARG, "NULL out");
  if (capacity < 1 || capacity > kMaxBatch)
    return fail(IBDL_ERR_INVALID_ARG, "capacity must be in [1, 512]");
  ibdl_batch_s* b = new ibdl_batch_s();
  b->cap = capacity;
  cudaError_t e = cudaMalloc((void**)&b->d_inst, sizeof(SolveInst) * capacity);
  if (!e) e = cudaMalloc((void**)&b->d_state, sizeof(SolveState) * capacity);
  if (!e) e = cudaMalloc((void**)&b->d_bar, (4 + kSchedWords * (size_t)capacity) * sizeof(unsigned));
  if (!e) e = cudaMallocHost((void**)&b->h_inst, sizeof(SolveInst) * capacity);
  if (!e) e = cudaMallocHost((void**)&b->h_state, sizeof(SolveState) * capacity);
  if (e) {
    delete b;
    return cuda_fail(e, "ibdl_batch_create");
  }
  *out = b;
  return IBDL_OK;
}

void ibdl_batch_destroy(ibdl_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  delete b;
}

ibdl_status ibdl_solve_batched(ibdl_batch b, int32_t count, const ibdl_geometry* geoms,
                               const double* const* bdata, double* const* q_out,
                               const ibdl_solve_opts* opts_in, ibdl_solve_info* infos,
                               ibdl_status* statuses, void* stream) {
  g_err.clear();
  if (!b || !geoms || !bdata || !q_out) return fail(IBDL_ERR_INVALID_ARG, "NULL argument");
  if (count < 1 || count > b->cap) return fail(IBDL_ERR_INVALID_ARG, "count out of range");
  ibdl_solve_opts o;
  ibdl_solve_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (!(o.tol > 0) || !isfinite(o.tol)) return fail(IBDL_ERR_INVALID_ARG, "tol must be > 0");
  if (o.restart < 1 || o.restart > 64) return fail(IBDL_ERR_INVALID_ARG, "restart in 1..64");
  if (o.max_iters < 1) return fail(IBDL_ERR_INVALID_ARG, "max_iters >= 1");
  if (o.max_refine < 1) o.max_refine = 1;
  if (!(o.inner_tol > 0) || o.inner_tol >= 1) o.inner_tol = 1e-5;
  for (int k = 0; k < count; ++k) {
    if (!geoms[k] || !bdata[k] || !q_out[k])
      return fail(IBDL_ERR_INVALID_ARG, "NULL geometry, bdata or q_out entry");
    if (geoms[k]->eta > 0 || geoms[k]->grid.spectral)
      return fail(IBDL_ERR_UNSUPPORTED,
                  "completed or spectral geometries solve with ibdl_solve");
    IBDL_TRY(geoms[k]->ensure_host());
    for (int l = 0; l < k; ++l)
      if (geoms[l] == geoms[k])
        return fail(IBDL_ERR_INVALID_ARG, "a geometry handle appears twice in one batch");
  }
  cudaStream_t st = (cudaStream_t)stream;
  int smem = 0;
  for (int k = 0; k < count; ++k) {
    ibdl_geometry g = geoms[k];
    IBDL_CU(cudaMemcpyAsync(g->stage_a, bdata[k], sizeof(double) * g->m, cudaMemcpyDefault, st));
    const bool rhs_in_kernel = g->bc == IBDL_NEUMANN;
    if (!rhs_in_kernel) IBDL_TRY(build_rhs(g, g->stage_a, nullptr, g->vb, st));
    IBDL_CU(cudaMemsetAsync(g->vx, 0, sizeof(double) * g->m, st));
    b->h_inst[k] = make_inst(g, o, count);
    b->h_inst[k].vdata = g->stage_a;
    b->h_state[k] = initial_state(b->h_inst[k], true, rhs_in_kernel);
    if (g->solver_smem > smem) smem = g->solver_smem;
  }
  IBDL_CU(cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(SolveInst) * count,
                          cudaMemcpyHostToDevice, st));
  IBDL_CU(cudaMemcpyAsync(b->d_state, b->h_state, sizeof(SolveState) * count,
                          cudaMemcpyHostToDevice, st));
  {
    char why[256];
    if (!solver_smem_fits(b->h_inst, count, smem, why, sizeof(why)))
      return fail(IBDL_ERR_INVALID_ARG, why);
  }
  IBDL_CU(launch_persistent_solve(b->d_inst, b->d_state, count, b->d_bar, smem, st));
  IBDL_CU(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(SolveState) * count,
                          cudaMemcpyDeviceToHost, st));
  for (int k = 0; k < count; ++k) {
    ibdl_geometry g = geoms[k];
    if (infos)
      IBDL_CU(cudaMemcpyAsync(g->h_hist, g->d_hist, kHistCap * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
    IBDL_CU(cudaMemcpyAsync(q_out[k], g->vx, sizeof(double) * g->m, cudaMemcpyDefault, st));
  }
  unsigned hb[4] = {0, 0, 0, 0};
  IBDL_CU(cudaMemcpyAsync(hb, b->d_bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
  IBDL_CU(cudaStreamSynchronize(st));
  if (hb[2]) return fail(IBDL_ERR_TIMEOUT, "persistent solver: a bounded device wait timed out");
  ibdl_status worst = IBDL_OK;
  for (int k = 0; k < count; ++k) {
    const ibdl_status sk = (ibdl_status)b->h_state[k].status;
    if (statuses) statuses[k] = sk;
    if (infos) info_from_state(b->h_state[k], geoms[k]->h_hist, &infos[k]);
    if (sk != IBDL_OK && worst == IBDL_OK) worst = sk;
  }
  if (worst != IBDL_OK) return fail(worst, "at least one instance did not converge");
  return IBDL_OK;
}

int64_t ibdl_kernel_launch_count(void) { return (int64_t)g_launches.load(); }

ibdl_status ibdl_solver_smem_query(int32_t dim, int32_t n, int32_t rows, int32_t elem,
                                   int64_t* need_out, int64_t* budget_out, int32_t* twiddles_out) {
  g_err.clear();
  if ((dim != 2 && dim != 3) || n < 16 || (n & (n - 1)) != 0 || n > (dim == 2 ? kMaxN2 : kMaxN3))
    return fail(IBDL_ERR_INVALID_ARG, "n must be a power of two in [16, 2048] (2D) / [16, 512] (3D)");
  if (rows < 2 || rows > n || (rows & (rows - 1)) != 0)
    return fail(IBDL_ERR_INVALID_ARG, "rows: a power of two in [2, n]");
  if (elem < 0 || elem > 2) return fail(IBDL_ERR_INVALID_ARG, "elem: 0, 1 or 2");
  GridDesc g;
  g.dim = dim;
  g.n = n;
  g.log2n = ilog2(n);
  size_t need[3];
  solver_item_smem(g, rows, elem, need);
  if (need_out)
    for (int k = 0; k < 3; ++k) need_out[k] = (int64_t)need[k];
  if (budget_out) *budget_out = solver_smem_bytes(g, rows, 1);
  if (twiddles_out) *twiddles_out = fft_tw_count(n);
  return IBDL_OK;
}

void ibdl_tuning_enable(int32_t on) { g_tuning_on.store(on != 0); }

ibdl_status ibdl_tuning_set_pencils(int32_t dim, int32_t n, int32_t precision, int32_t c_solve,
                                    int32_t c_y) {
  g_err.clear();
  if ((dim != 2 && dim != 3) || n < 16 || n > (dim == 2 ? kMaxN2 : kMaxN3) || (n & (n - 1)) ||
      precision < IBDL_FP64 || precision > IBDL_FP32_REFINED)
    return fail(IBDL_ERR_INVALID_ARG, "dim, n or precision");
  if (dim == 2 && c_y != 0) return fail(IBDL_ERR_INVALID_ARG, "2D has no y passes: c_y = 0");
  const int cs[2] = {c_y, c_solve};
  for (int which = 0; which < 2; ++which) {
    const int c = cs[which];
    if (c == 0 || (dim == 2 && which == 0)) continue;
    const PencilLayout base = precision == IBDL_FP32_REFINED
                                  ? solve_layout<float>(dim, n, which)
                                  : solve_layout<double>(dim, n, which);
    const bool ok = precision == IBDL_FP32_REFINED
                        ? pencils_admissible<float>(n, base.estride, base.pg, c)
                        : pencils_admissible<double>(n, base.estride, base.pg, c);
    if (!ok) return fail(IBDL_ERR_INVALID_ARG, "pencils per item: not admissible");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(IBDL_ERR_CUDA, "cudaGetDevice");
  const auto key = std::make_tuple(dev, (int)dim, (int)n, (int)precision);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (c_solve == 0 && c_y == 0)
    g_tuned_pc.erase(key);
  else
    g_tuned_pc[key] = {c_y, c_solve};
  return IBDL_OK;
}

ibdl_status ibdl_tuning_set_plan(int32_t dim, int32_t n, int32_t precision, int32_t plan) {
  g_err.clear();
  if (dim != 2 || n < 16 || n > kMaxN2 || (n & (n - 1)) || precision != IBDL_FP32_REFINED)
    return fail(IBDL_ERR_INVALID_ARG,
                "dim, n or precision (plan variants: 2D, float32-refined only)");
  if (plan < -1 || plan >= kPlanVariants || (plan >= 0 && !plan_offered(ilog2(n), plan)))
    return fail(IBDL_ERR_INVALID_ARG, "plan variant not offered for this size");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(IBDL_ERR_CUDA, "cudaGetDevice");
  const auto key = std::make_tuple(dev, (int)dim, (int)n, (int)precision);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (plan < 0)
    g_tuned_plan.erase(key);
  else
    g_tuned_plan[key] = plan;
  return IBDL_OK;
}

ibdl_status ibdl_geometry_set_solver_pencils(ibdl_geometry g, int32_t c_f64, int32_t c_f32,
                                             int32_t c_dd) {
  g_err.clear();
  IBDL_TRY(check_handle(g));
  GridDesc gd = g->grid;
  const int cs[3] = {c_f64, c_f32, c_dd};
  for (int e = 0; e < 3; ++e) {
    const int c = cs[e];
    if (c == 0) continue;
    const PencilLayout base = solve_layout<double>(gd.dim, gd.n, 1);
    const bool ok = e == 1 ? pencils_admissible<float>(gd.n, base.estride, base.pg, c)
                  : e == 2 ? pencils_admissible<dd>(gd.n, base.estride, base.pg, c)
                           : pencils_admissible<double>(gd.n, base.estride, base.pg, c);
    if (!ok) return fail(IBDL_ERR_INVALID_ARG, "solver pencils per item: not admissible");
    gd.scap[e] = c;
  }
  for (int e = 0; e < 3; ++e)
    if (cs[e] == 0) gd.scap[e] = 0;
  const int smem = solver_smem_bytes(gd, g->bins.rows, 1);
  if (smem < 0 || smem > 227 * 1024)
    return fail(IBDL_ERR_INVALID_ARG, "solver pencils per item: items exceed shared memory");
  g->grid = gd;
  g->solver_smem = smem;
  return IBDL_OK;
}

ibdl_status ibdl_tuning_set(int32_t dim, int32_t n, int32_t precision, int32_t rows) {
  if ((dim != 2 && dim != 3) || n < 16 || n > (dim == 2 ? kMaxN2 : kMaxN3) || (n & (n - 1)) ||
      precision < IBDL_FP64 || precision > IBDL_FP32_REFINED || rows < 0)
    return IBDL_ERR_INVALID_ARG;
  if (rows && !tiling_admissible(n, rows)) return IBDL_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IBDL_ERR_CUDA;
  const auto key = std::make_tuple(dev, (int)dim, (int)n, (int)precision);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (rows)
    g_tuned[key] = rows;
  else
    g_tuned.erase(key);
  return IBDL_OK;
}

void ibdl_profile_enable(int32_t on) {
  if (on && !g_phase_buf) {
    // allocated when profiling is switched on, never on the solve path
    if (cudaMalloc((void**)&g_phase_buf, kProfWords * sizeof(unsigned long long)) ==
        cudaSuccess)
      cudaMemset(g_phase_buf, 0, kProfWords * sizeof(unsigned long long));
    else
      g_phase_buf = nullptr;
  }
  g_prof.store(on != 0);
}

ibdl_status ibdl_profile_trace(int32_t on) {
  g_err.clear();
  if (!g_phase_buf) return fail(IBDL_ERR_INVALID_ARG, "profiling is off (ibdl_profile_enable)");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  const unsigned long long h[2] = {on ? 1ull : 0ull, 0ull};
  IBDL_CU(cudaDeviceSynchronize());
  IBDL_CU(cudaMemset(g_phase_buf + kTraceFlag + 2, 0,
                     3 * (size_t)kTraceCap * sizeof(unsigned long long)));
  IBDL_CU(cudaMemcpy(g_phase_buf + kTraceFlag, h, sizeof(h), cudaMemcpyHostToDevice));
  return IBDL_OK;
}

int64_t ibdl_profile_trace_read(uint64_t* out, int64_t max_records) {
  if (!g_phase_buf) return 0;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  std::vector<uint64_t> h(3 * (size_t)kTraceCap);
  if (cudaMemcpy(h.data(), g_phase_buf + kTraceFlag + 2, h.size() * sizeof(uint64_t),
                 cudaMemcpyDeviceToHost) ||
      cudaMemset(g_phase_buf + kTraceFlag + 2, 0, h.size() * sizeof(uint64_t)))
    return -1;
  int64_t k = 0;
  for (size_t r = 0; r < (size_t)kTraceCap; ++r) {
    if (h[3 * r] == 0) continue;
    if (out && k < max_records)
      for (int w = 0; w < 3; ++w) out[3 * k + w] = h[3 * r + w];
    ++k;
  }
  return k;
}

int32_t ibdl_profile_read(ibdl_kernel_stat* out, int32_t max_out, int32_t reset) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_phase_buf) {
    static const char* names[15] = {
        "phase:rows_fwd_f64", "phase:y_fwd_f64", "phase:solve_f64", "phase:y_inv_f64",
        "phase:rows_inv_f64", "phase:rows_fwd_f32", "phase:y_fwd_f32", "phase:solve_f32",
        "phase:y_inv_f32", "phase:rows_inv_f32", "phase:vector_phases", "phase:unused11",
        "phase:unused12", "phase:unused13", "phase:idle_blocks"};
    unsigned long long h[2 * kPhaseSlots];
    if (cudaMemcpy(h, g_phase_buf, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
      for (int id = 0; id < 15; ++id) {
        if (!h[2 * id + 1]) continue;
        auto& st = g_prof_stats[names[id]];
        st.first += (long long)h[2 * id + 1];
        st.second += (double)h[2 * id] * 1e-6;
      }
      cudaMemset(g_phase_buf, 0, sizeof(h));
    } else {
      cudaGetLastError();
    }
  }
  for (const ProfPending& p : g_pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& st = g_prof_stats[p.name];
      st.first += 1;
      st.second += ms;
    } else {
      cudaGetLastError();
    }
    g_ev_pool.push_back(p.a);
    g_ev_pool.push_back(p.b);
  }
  g_pending.clear();
  int32_t k = 0;
  for (const auto& kv : g_prof_stats) {
    if (out && k < max_out) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
      out[k].launches = kv.second.first;
      out[k].total_ms = kv.second.second;
    }
    ++k;
  }
  if (reset) g_prof_stats.clear();
  return k;
}

const char* ibdl_status_string(ibdl_status s) {
  switch (s) {
    case IBDL_OK: return "ok";
    case IBDL_ERR_INVALID_ARG: return "invalid argument";
    case IBDL_ERR_OOM: return "out of device memory";
    case IBDL_ERR_CUDA: return "CUDA error";
    case IBDL_ERR_NOT_CONVERGED: return "not converged";
    case IBDL_ERR_BREAKDOWN: return "GMRES breakdown";
    case IBDL_ERR_NONFINITE: return "non-finite value";
    case IBDL_ERR_TIMEOUT: return "device wait timed out";
    case IBDL_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* ibdl_last_error_message(void) { return g_err.c_str(); }

int32_t ibdl_version(void) { return 100 * IBDL_VERSION_MAJOR + IBDL_VERSION_MINOR; }

}  // extern "C"

// =============================================================================
// Serving engine (continuous batching over the persistent solver)
// =============================================================================

namespace {

double server_now() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Device bytes a request will hold, from the sizes ibdl_create_geometry
// allocates (tile lists at their largest: 3 tiles per point in 2D, 18 in 3D).
int64_t estimate_request_bytes(const ibdl_geometry_desc& d) {
  const int64_t n = d.n, m = d.m;
  const int64_t ncells = d.dim == 3 ? n * n * n : n * n;
  const int64_t spec = (n / 2 + 1) * (ncells / n);
  const int64_t ntw = fft_tw_count((int)n);
  const int64_t rows = rows_per_tile(d.dim, (int)n);
  const int64_t ntiles = (n / rows) * (d.dim == 3 ? n : 1);
  const int64_t ld = (m + 31) / 32 * 32;
  int64_t b = 7 * m * 8 + 3 * m * 4 + 12 * m * 8 + 12 * m * 4;      // points, delta weights
  b += 3 * (ntiles + 1) * 4 + 2 * (d.dim == 3 ? 18 : 3) * m * 4;    // tile lists (two orders)
  b += 4;                                                            // error word
  b += spec * 16 + ncells * 8 + ntw * 16 + n * 8;                   // float64 spectral
  if (d.precision == IBDL_FP32_REFINED) b += spec * 8 + ncells * 4 + ntw * 8 + n * 4;
  b += (65 * ld + 65 * 64 + 3 * 64 + 65 + 8 + 7 * ld) * 8;          // Krylov, vectors
  b += 3 * ((m + kSolverThreads - 1) / kSolverThreads) * 66 * 8 + kHistCap * 8;
  return b + (1 << 16);
}

}  // namespace

struct SrvReq {
  int64_t id = 0;
  ibdl_geometry_desc desc;
  std::vector<double> arr[7];  // x, y, z, nx, ny, nz, w
  std::vector<double> bdata;
  double t_arrival = 0, t_admit = 0, t_done = 0;
  int64_t est = 0, held = 0;
  ibdl_geometry g = nullptr;
  int slot = -1;
  ibdl_status status = IBDL_ERR_NOT_CONVERGED;
  ibdl_solve_info info;
  std::vector<double> q;
};

struct ibdl_server_s {
  ibdl_server_config cfg;
  int cap = 0;
  cudaStream_t solve_st = nullptr, setup_st = nullptr;
  SolveInst* d_inst = nullptr;
  SolveState* d_state = nullptr;
  unsigned* d_bar = nullptr;
  SolveInst* h_inst = nullptr;         // pinned: descriptors of fresh slots
  SolveState* h_state_in = nullptr;    // pinned: initial states of fresh slots
  SolveState* h_state_out = nullptr;   // pinned: states after a slice
  unsigned* h_bar = nullptr;           // pinned
  std::vector<SrvReq*> slot;
  std::vector<char> fresh;             // admitted since the last launch
  std::deque<SrvReq*> queue;
  std::map<int64_t, SrvReq*> done;
  std::vector<int64_t> just_done;      // finished during the current step
  int64_t next_id = 1, bytes = 0, peak = 0, steps = 0, launches = 0;
  double admit_seconds = 0, wait_seconds = 0;
  std::mutex mu;
  ~ibdl_server_s() {
    if (solve_st) cudaStreamSynchronize(solve_st);
    if (setup_st) cudaStreamSynchronize(setup_st);
    for (SrvReq* r : slot)
      if (r) {
        ibdl_destroy_geometry(r->g);
        delete r;
      }
    for (SrvReq* r : queue) delete r;
    for (auto& kv : done) delete kv.second;
    if (d_inst) cudaFree(d_inst);
    if (d_state) cudaFree(d_state);
    if (d_bar) cudaFree(d_bar);
    if (h_inst) cudaFreeHost(h_inst);
    if (h_state_in) cudaFreeHost(h_state_in);
    if (h_state_out) cudaFreeHost(h_state_out);
    if (h_bar) cudaFreeHost(h_bar);
    if (solve_st) cudaStreamDestroy(solve_st);
    if (setup_st) cudaStreamDestroy(setup_st);
  }
};

namespace {

ibdl_status sanitize_opts(ibdl_solve_opts* o) {
  if (!(o->tol > 0) || !isfinite(o->tol)) return fail(IBDL_ERR_INVALID_ARG, "tol must be > 0");
  if (o->restart < 1 || o->restart > 64) return fail(IBDL_ERR_INVALID_ARG, "restart in 1..64");
  if (o->max_iters < 1) return fail(IBDL_ERR_INVALID_ARG, "max_iters >= 1");
  if (o->max_refine < 1) o->max_refine = 1;
  if (!(o->inner_tol > 0) || o->inner_tol >= 1) o->inner_tol = 1e-5;
  o->x0 = nullptr;
  o->engine = 0;
  return IBDL_OK;
}

void finish_request(ibdl_server_s* s, SrvReq* r, ibdl_status st) {
  r->status = st;
  r->t_done = server_now();
  s->done[r->id] = r;
  s->just_done.push_back(r->id);
}

// Builds the request's geometry on the set-up stream and stages its data;
// the slot's descriptor and initial state wait in the pinned tables until
// the next launch.
ibdl_status admit_one(ibdl_server_s* s, SrvReq* r, int k) {
  ibdl_geometry g = nullptr;
  tl_no_tune = true;
  const ibdl_status cs = ibdl_create_geometry(&r->desc, s->setup_st, &g);
  tl_no_tune = false;
  IBDL_TRY(cs);
  const size_t mb = sizeof(double) * (size_t)g->m;
  // Dirichlet: b = U_b; Neumann: V_b, from which the solver's first action
  // builds b
  double* target = g->bc == IBDL_NEUMANN ? g->stage_a : g->vb;
  cudaError_t e = cudaMemcpyAsync(target, r->bdata.data(), mb, cudaMemcpyHostToDevice,
                                  s->setup_st);
  if (!e) e = cudaMemsetAsync(g->vx, 0, mb, s->setup_st);
  if (!e) e = cudaStreamSynchronize(s->setup_st);
  if (e) {
    ibdl_destroy_geometry(g);
    return cuda_fail(e, "server: staging request data");
  }
  r->g = g;
  r->slot = k;
  r->held = g->bytes;
  r->t_admit = server_now();
  s->h_inst[k] = make_inst(g, s->cfg.opts, s->cap);
  s->h_inst[k].vdata = g->stage_a;
  s->h_state_in[k] = initial_state(s->h_inst[k], true, g->bc == IBDL_NEUMANN);
  s->slot[k] = r;
  s->fresh[k] = 1;
  s->bytes += r->held;
  if (s->bytes > s->peak) s->peak = s->bytes;
  return IBDL_OK;
}

// Admits queued requests in arrival order while a slot is free and the
// budget allows; a request larger than the whole budget fails with OOM.
// While a slice runs, admission stops as soon as it has finished, so the
// GPU is not left idle behind host-side set-up; with no slice running at
// most kIdleAdmit requests are set up before the next launch.
constexpr int kIdleAdmit = 8;
void admit_queued(ibdl_server_s* s, bool slice_running) {
  int admitted = 0;
  const double t0 = server_now();
  while (!s->queue.empty()) {
    if (slice_running ? (admitted > 0 && cudaStreamQuery(s->solve_st) != cudaErrorNotReady)
                      : admitted >= kIdleAdmit)
      break;
    SrvReq* r = s->queue.front();
    if (r->est > s->cfg.memory_budget) {
      s->queue.pop_front();
      finish_request(s, r, IBDL_ERR_OOM);
      continue;
    }
    int k = -1;
    for (int j = 0; j < s->cap; ++j)
      if (!s->slot[j]) {
        k = j;
        break;
      }
    if (k < 0) return;
    if (s->bytes + r->est > s->cfg.memory_budget) return;
    s->queue.pop_front();
    const ibdl_status st = admit_one(s, r, k);
    if (st != IBDL_OK) finish_request(s, r, st);
    ++admitted;
  }
  s->admit_seconds += server_now() - t0;
}

// Retires slot k: result to the host, geometry released.
void retire(ibdl_server_s* s, int k, ibdl_status st, const SolveState* state) {
  SrvReq* r = s->slot[k];
  ibdl_geometry g = r->g;
  r->q.resize(g->m);
  cudaMemcpy(r->q.data(), g->vx, sizeof(double) * g->m, cudaMemcpyDeviceToHost);
  std::vector<double> hist(kHistCap);
  cudaMemcpy(hist.data(), g->d_hist, sizeof(double) * kHistCap, cudaMemcpyDeviceToHost);
  memset(&r->info, 0, sizeof(r->info));
  if (state) info_from_state(*state, hist.data(), &r->info);
  ibdl_destroy_geometry(g);
  r->g = nullptr;
  s->bytes -= r->held;
  s->slot[k] = nullptr;
  s->fresh[k] = 0;
  finish_request(s, r, st);
}

}  // namespace

void ibdl_server_config_default(ibdl_server_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->memory_budget = 0;
  cfg->max_active = 64;
  cfg->rounds_per_step = 8;
  cfg->reserve_sms = 8;
  ibdl_solve_opts_default(&cfg->opts);
}

double ibdl_server_clock(void) { return server_now(); }

ibdl_status ibdl_server_create(const ibdl_server_config* cfg_in, ibdl_server* out) {
  g_err.clear();
  if (!out) return fail(IBDL_ERR_INVALID_ARG, "NULL out");
  ibdl_server_config cfg;
  ibdl_server_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_active < 1 || cfg.max_active > kMaxBatch)
    return fail(IBDL_ERR_INVALID_ARG, "max_active must be in [1, 512]");
  if (cfg.rounds_per_step < 1) return fail(IBDL_ERR_INVALID_ARG, "rounds_per_step >= 1");
  if (cfg.memory_budget < 0) return fail(IBDL_ERR_INVALID_ARG, "memory_budget >= 0");
  IBDL_TRY(sanitize_opts(&cfg.opts));
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return cuda_fail(e, "server: device query");
  if (cfg.reserve_sms < 0 || cfg.reserve_sms >= sms)
    return fail(IBDL_ERR_INVALID_ARG, "reserve_sms must leave at least one SM to the solver");
  if (cfg.memory_budget == 0) {
    size_t fr = 0, tot = 0;
    if ((e = cudaMemGetInfo(&fr, &tot))) return cuda_fail(e, "server: cudaMemGetInfo");
    cfg.memory_budget = (int64_t)(0.8 * (double)fr);
  }
  ibdl_server_s* s = new ibdl_server_s();
  s->cfg = cfg;
  s->cap = cfg.max_active;
  const size_t nb = 4 + kSchedWords * (size_t)s->cap;
  e = cudaStreamCreateWithFlags(&s->solve_st, cudaStreamNonBlocking);
  if (!e) e = cudaStreamCreateWithFlags(&s->setup_st, cudaStreamNonBlocking);
  if (!e) e = cudaMalloc((void**)&s->d_inst, sizeof(SolveInst) * s->cap);
  if (!e) e = cudaMalloc((void**)&s->d_state, sizeof(SolveState) * s->cap);
  if (!e) e = cudaMalloc((void**)&s->d_bar, sizeof(unsigned) * nb);
  if (!e) e = cudaMallocHost((void**)&s->h_inst, sizeof(SolveInst) * s->cap);
  if (!e) e = cudaMallocHost((void**)&s->h_state_in, sizeof(SolveState) * s->cap);
  if (!e) e = cudaMallocHost((void**)&s->h_state_out, sizeof(SolveState) * s->cap);
  if (!e) e = cudaMallocHost((void**)&s->h_bar, sizeof(unsigned) * 4);
  if (e) {
    delete s;
    return cuda_fail(e, "ibdl_server_create");
  }
  // every slot starts empty: zero descriptors, DONE states
  memset(s->h_inst, 0, sizeof(SolveInst) * s->cap);
  for (int k = 0; k < s->cap; ++k) {
    memset(&s->h_state_out[k], 0, sizeof(SolveState));
    s->h_state_out[k].action = ACT_DONE;
  }
  e = cudaMemcpy(s->d_inst, s->h_inst, sizeof(SolveInst) * s->cap, cudaMemcpyHostToDevice);
  if (!e)
    e = cudaMemcpy(s->d_state, s->h_state_out, sizeof(SolveState) * s->cap,
                   cudaMemcpyHostToDevice);
  if (e) {
    delete s;
    return cuda_fail(e, "ibdl_server_create");
  }
  s->slot.assign(s->cap, nullptr);
  s->fresh.assign(s->cap, 0);
  *out = s;
  return IBDL_OK;
}

void ibdl_server_destroy(ibdl_server s) { delete s; }

ibdl_status ibdl_server_submit(ibdl_server s, const ibdl_geometry_desc* d, const double* bdata,
                               double t_arrival, int64_t* id_out) {
  g_err.clear();
  if (!s || !d || !bdata) return fail(IBDL_ERR_INVALID_ARG, "NULL server, desc or bdata");
  if (d->dim != 2 && d->dim != 3) return fail(IBDL_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (d->n < 16 || (d->n & (d->n - 1)) != 0 || d->n > (d->dim == 2 ? kMaxN2 : kMaxN3))
    return fail(IBDL_ERR_INVALID_ARG,
                "n must be a power of two in [16, 2048] (2D) / [16, 512] (3D)");
  if (d->m < 1 || d->m > kMaxPoints)
    return fail(IBDL_ERR_INVALID_ARG, "m out of range (1 .. 16776960)");
  if (!d->x || !d->y || !d->nx || !d->ny || !d->w || (d->dim == 3 && (!d->z || !d->nz)))
    return fail(IBDL_ERR_INVALID_ARG, "NULL point, normal or weight array");
  if (d->eta != 0 || d->disc != IBDL_DISC_FD)
    return fail(IBDL_ERR_UNSUPPORTED,
                "completed or spectral requests solve with ibdl_solve");
  SrvReq* r = new SrvReq();
  const size_t m = (size_t)d->m;
  const double* src[7] = {d->x, d->y, d->dim == 3 ? d->z : nullptr, d->nx, d->ny,
                          d->dim == 3 ? d->nz : nullptr, d->w};
  for (int a = 0; a < 7; ++a) {
    if (!src[a]) continue;
    r->arr[a].resize(m);
    if (cudaMemcpy(r->arr[a].data(), src[a], sizeof(double) * m, cudaMemcpyDefault)) {
      cudaGetLastError();
      delete r;
      return fail(IBDL_ERR_INVALID_ARG, "server: unreadable point array");
    }
  }
  r->bdata.resize(m);
  if (cudaMemcpy(r->bdata.data(), bdata, sizeof(double) * m, cudaMemcpyDefault)) {
    cudaGetLastError();
    delete r;
    return fail(IBDL_ERR_INVALID_ARG, "server: unreadable bdata");
  }
  for (double v : r->bdata)
    if (!isfinite(v)) {
      delete r;
      return fail(IBDL_ERR_NONFINITE, "non-finite boundary data");
    }
  r->desc = *d;
  double* dst[7];
  for (int a = 0; a < 7; ++a) dst[a] = r->arr[a].empty() ? nullptr : r->arr[a].data();
  r->desc.x = dst[0];
  r->desc.y = dst[1];
  r->desc.z = dst[2];
  r->desc.nx = dst[3];
  r->desc.ny = dst[4];
  r->desc.nz = dst[5];
  r->desc.w = dst[6];
  r->est = estimate_request_bytes(*d);
  r->t_arrival = t_arrival >= 0 ? t_arrival : server_now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  s->queue.push_back(r);
  if (id_out) *id_out = r->id;
  return IBDL_OK;
}

ibdl_status ibdl_server_step(ibdl_server s, int64_t* done_ids, int32_t max_ids,
                             int32_t* n_done) {
  g_err.clear();
  if (!s) return fail(IBDL_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->steps++;
  s->just_done.clear();
  // 1. one slice over the active slots, fresh slots uploaded first
  int hi = -1, smem = 0;
  for (int k = 0; k < s->cap; ++k)
    if (s->slot[k]) {
      hi = k;
      if (s->slot[k]->g->solver_smem > smem) smem = s->slot[k]->g->solver_smem;
    }
  ibdl_status slice_err = IBDL_OK;
  bool launched = false;
  if (hi >= 0) {
    // every item of every active slot must fit the slice's shared memory
    char why[256];
    for (int k = 0; k <= hi && slice_err == IBDL_OK; ++k)
      if (s->slot[k] && !solver_smem_fits(s->h_inst + k, 1, smem, why, sizeof(why)))
        slice_err = fail(IBDL_ERR_INVALID_ARG, why);
    if (slice_err != IBDL_OK)
      for (int k = 0; k <= hi; ++k) s->fresh[k] = 0;  // retire them all below
  }
  if (hi >= 0 && slice_err == IBDL_OK) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k <= hi && !e; ++k) {
      if (!s->fresh[k]) continue;
      e = cudaMemcpyAsync(s->d_inst + k, s->h_inst + k, sizeof(SolveInst),
                          cudaMemcpyHostToDevice, s->solve_st);
      if (!e)
        e = cudaMemcpyAsync(s->d_state + k, s->h_state_in + k, sizeof(SolveState),
                            cudaMemcpyHostToDevice, s->solve_st);
      s->fresh[k] = 0;
    }
    if (!e)
      e = launch_persistent_solve(s->d_inst, s->d_state, hi + 1, s->d_bar, smem, s->solve_st,
                                  s->cfg.rounds_per_step, s->cfg.reserve_sms);
    if (!e)
      e = cudaMemcpyAsync(s->h_state_out, s->d_state, sizeof(SolveState) * (hi + 1),
                          cudaMemcpyDeviceToHost, s->solve_st);
    if (!e)
      e = cudaMemcpyAsync(s->h_bar, s->d_bar, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost,
                          s->solve_st);
    if (e) {
      slice_err = cuda_fail(e, "server: slice launch");
    } else {
      launched = true;
      s->launches++;
    }
  }
  // 2. admit while the slice runs (set-up kernels use the reserved SMs)
  admit_queued(s, launched);
  // 3. wait, then retire finished solves
  if (launched) {
    const double tw = server_now();
    const cudaError_t e = cudaStreamSynchronize(s->solve_st);
    s->wait_seconds += server_now() - tw;
    if (e)
      slice_err = cuda_fail(e, "server: slice");
    else if (s->h_bar[2])
      slice_err = fail(IBDL_ERR_TIMEOUT, "server: a solver barrier timed out");
  }
  for (int k = 0; k <= hi; ++k) {
    SrvReq* r = s->slot[k];
    if (!r || s->fresh[k]) continue;  // empty, or admitted during this slice
    if (slice_err != IBDL_OK) {
      retire(s, k, slice_err, nullptr);
      continue;
    }
    const SolveState& st = s->h_state_out[k];
    if (st.action != ACT_DONE) continue;
    retire(s, k, (ibdl_status)st.status, &st);
  }
  const int32_t cnt = (int32_t)s->just_done.size();
  for (int32_t i = 0; done_ids && i < cnt && i < max_ids; ++i) done_ids[i] = s->just_done[i];
  if (n_done) *n_done = cnt;
  return slice_err;
}

ibdl_status ibdl_server_take(ibdl_server s, int64_t id, double* q_out,
                             ibdl_request_result* res) {
  g_err.clear();
  if (!s) return fail(IBDL_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(id);
  if (it == s->done.end()) return fail(IBDL_ERR_INVALID_ARG, "unknown or unfinished request");
  SrvReq* r = it->second;
  if (q_out && !r->q.empty()) {
    const cudaError_t e = cudaMemcpy(q_out, r->q.data(), sizeof(double) * r->q.size(),
                                     cudaMemcpyDefault);
    if (e) return cuda_fail(e, "server: copying the result");
  }
  if (res) {
    memset(res, 0, sizeof(*res));
    res->id = r->id;
    res->status = r->status;
    res->slot = r->slot;
    res->t_arrival = r->t_arrival;
    res->t_admit = r->t_admit;
    res->t_done = r->t_done;
    res->device_bytes = r->held;
    res->info = r->info;
  }
  s->done.erase(it);
  delete r;
  return IBDL_OK;
}

ibdl_status ibdl_server_get_stats(ibdl_server s, ibdl_server_stats* out) {
  if (!s || !out) return fail(IBDL_ERR_INVALID_ARG, "NULL server or out");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->queued = (int32_t)s->queue.size();
  for (SrvReq* r : s->slot)
    if (r) out->active++;
  out->finished = (int32_t)s->done.size();
  out->bytes_in_use = s->bytes;
  out->peak_bytes = s->peak;
  out->memory_budget = s->cfg.memory_budget;
  out->steps = s->steps;
  out->launches = s->launches;
  out->submitted = s->next_id - 1;
  out->admit_seconds = s->admit_seconds;
  out->wait_seconds = s->wait_seconds;
  return IBDL_OK;
}
