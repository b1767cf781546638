// The strided z pass of the 3D float32 solve (forward z FFT, the Helmholtz
// symbol of the 7-point stencil, Sec. 5.1, inverse z FFT) with its input
// pencils staged in shared memory by the Tensor Memory Accelerator.
//
// The transposed half spectrum holds slab kx as [z][y] (y fastest), so the
// c z-pencils of one work item (c consecutive y at one kx) form a 2D box of
// c contiguous complex values by n rows, n complex apart.  One bulk tensor
// copy (cp.async.bulk.tensor, a 3D tensor map over [kx][z][y] of 8-byte
// elements) moves the box into shared memory and completes on an mbarrier.
// A block runs items k, k + gridDim, ... (persistent): its first radix pass
// reads the box into a pencil buffer, the box then serves as the other
// ping-pong buffer of the transforms, and before the last inverse pass --
// when nothing reads the box any more -- the block's thread 0 starts the
// copy of its next item there; the copy overlaps that pass and its stores.
// One staging box doubles as a pencil buffer, so three blocks share an SM.
// Every wait on the mbarrier is bounded: on timeout the block
// raises an error word, waits (bounded) for its copy in flight and leaves.
//
// Only the GPU's own memory is addressed (no multicast, no clusters).
#include <cuda.h>
#include <string.h>

#include <mutex>

#include "ibdl_device.cuh"

namespace ibdl {

static_assert(sizeof(CUtensorMap) == sizeof(TmaDesc), "tensor map storage");
static_assert(alignof(TmaDesc) >= 64, "tensor map alignment");

namespace {

constexpr unsigned kTmaSpin = 1u << 26;  // polls of ~32 ns or more: seconds

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Polls the phase `parity` of bar at most `limit` times; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(512) k_zsolve_tma(GridDesc g, int c, int lgc, int nitems,
                                                    cx_t<T>* spec,
                                                    const __grid_constant__ CUtensorMap map,
                                                    const cx_t<T>* __restrict__ tw,
                                                    const T* __restrict__ s2, T cfac, T scale0,
                                                    const unsigned char* zempty, unsigned* err) {
  using C = cx_t<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ TmaItem ti;
  __shared__ int bad;
  const int n = g.n, lg = g.log2n, PS = pen_stride(n);
  const int ntw = fft_tw_count(n, plan_variant_of<T>(g));
  const int tid = threadIdx.x;
  C* box = reinterpret_cast<C*>(smem);  // dense [n][c] when staged; padded pencils later
  C* bufB = box + (size_t)c * PS;
  C* tws = bufB + (size_t)c * PS;
  T* s2s = reinterpret_cast<T*>(tws + ntw);

  // the tables once per block: it runs many items
  {
    TableStage<T, kTabBatch> ts;
    ts.load(tw, ntw, s2, n, 0);
    ts.store(tws, ntw, s2s, n, 0);
    ts.rest(tw, tws, ntw, s2, s2s, n);
  }
  if (tid == 0) {
    ti.map = &map;
    ti.bar = &bar;
    ti.box = box;
    ti.c = c;
    ti.n = n;
    ti.lgn = lg;
    ti.zb = n < 256 ? n : 256;
    ti.words = (int)(sizeof(C) / 8);
    ti.row_bytes = c * (int)sizeof(C);
    ti.bytes = (unsigned)((size_t)n * c * sizeof(C));
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  // the tables and the barrier do not depend on the previous kernel: they
  // are staged before its spectrum is waited for (a dependent launch)
  pdl_wait();
  if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  int k = blockIdx.x;
  if (tid == 0 && k < nitems) tma_issue_item(ti, k);
  unsigned parity = 0;
  for (; k < nitems; k += gridDim.x) {
    if (tid == 0 && !mbar_wait(&bar, parity, kTmaSpin)) bad = 1;
    __syncthreads();
    if (bad) break;
    parity ^= 1u;
    const int p0 = k * c, kx = p0 >> lg, q0 = p0 & (n - 1);
    SymbolEpi<T> epi;
    epi.s2s = s2s;
    epi.pre = s2s[kx];
    epi.c0 = g.poisson ? (T)0 : (T)1;
    epi.cfac = cfac;
    epi.scale0 = scale0;
    epi.pbase = q0;
    epi.npl = c;
    GlobalPencils<T> gio{};
    gio.p = spec + (size_t)kx * n * n + q0;
    gio.npl = c;
    gio.lgc = lgc;
    gio.zempty = zempty;
    gio.sin = box;
    gio.ld = c;
    // before the last inverse pass, thread 0 starts the copy of the block's
    // next item into the box
    gio.tma = &ti;
    gio.tma_next = k + (int)gridDim.x < nitems ? k + (int)gridDim.x : -1;
    fft_global<T, 2, true, true>(box, bufB, plan_code_of<T>(g), c, tws, epi, gio);  // ends with a barrier
  }
  if (bad) {
    // the copy engine did not deliver within the bound: report it, then wait
    // (bounded) for this block's copy still in flight before leaving
    if (tid == 0) {
      atomicExch(err, 1u);
      mbar_wait(&bar, parity, kTmaSpin);
    }
  }
  pdl_release();
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

}  // namespace

template <typename T>
size_t zsolve_smem(int n, int c) {
  const int ntw = fft_tw_capacity<T>(n);
  if (ntw < 0) return ~(size_t)0;
  // the staging box (dense n x c) lives in the first of the two padded
  // pencil buffers (c x pen_stride(n) >= n x c)
  return 2 * (size_t)c * pen_stride(n) * sizeof(cx_t<T>) + (size_t)ntw * sizeof(cx_t<T>) +
         (size_t)n * sizeof(T);
}

namespace {

// Items of c pencils: the autotuner's choice for the solve pass when it
// fits (g.pcap), else the largest power of two c <= 16 (and <= n) whose
// block (two pencil buffers, one the staging box, and the tables) fits
// 75 KB, so that three blocks share an SM.  c >= 2 keeps every copy's first
// coordinate a multiple of 16 bytes.
template <typename T>
int zsolve_pencils(const GridDesc& g) {
  const int n = g.n, want = g.pcap[sizeof(T) == 4 ? 0 : 1][1];
  if (want >= 2 && want <= 16 && want <= n && (want & (want - 1)) == 0 &&
      zsolve_smem<T>(n, want) <= 110 * 1024)
    return want;
  int c = n < 16 ? n : 16;
  while (c > 2 && zsolve_smem<T>(n, c) > 75 * 1024) c >>= 1;
  return c;
}

}  // namespace

template <typename T>
cudaError_t make_zsolve_map(const GridDesc& g, const cx_t<T>* spec, TmaDesc* out) {
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const int n = g.n;
  const int c = zsolve_pencils<T>(g);
  const int words = (int)(sizeof(cx_t<T>) / 8);
  // [kx][z][y] of 8-byte words: y (words per complex value) fastest
  const cuuint64_t dims[3] = {(cuuint64_t)n * words, (cuuint64_t)n, (cuuint64_t)(n / 2 + 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)n * sizeof(cx_t<T>),
                                 (cuuint64_t)n * n * sizeof(cx_t<T>)};
  const cuuint32_t box[3] = {(cuuint32_t)(c * words), (cuuint32_t)(n < 256 ? n : 256), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 3,
                         const_cast<cx_t<T>*>(spec), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_zsolve_tma(const GridDesc& g, SpectralWs<T>& ws, const unsigned char* zempty,
                              cudaStream_t st) {
  const int n = g.n;
  const int c = zsolve_pencils<T>(g);
  int lgc = 0;
  while ((1 << lgc) < c) ++lgc;
  const int nitems = (n / 2 + 1) * n / c;
  const size_t smem = zsolve_smem<T>(n, c);
  const int thr = pencil_threads(n, c);
  static std::mutex mu;
  static int blocks_per_sm[kMaxDevices][2] = {};
  static int sms[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const int ti = sizeof(T) == 4 ? 0 : 1;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!sms[dev] &&
        (e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)))
      return e;
    if ((e = cudaFuncSetAttribute((const void*)k_zsolve_tma<T>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zsolve_tma<T>, thr, smem)))
      return e;
    blocks_per_sm[dev][ti] = per < 1 ? 1 : per;
  }
  int blocks = sms[dev] * blocks_per_sm[dev][ti];
  if (blocks > nitems) blocks = nitems;
  CUtensorMap map;
  memcpy(&map, ws.zmap, sizeof(map));
  const T cfac = (T)symbol_cfac(g);
  const T scale0 = (T)symbol_scale0(g);
  prof_begin(st);
  launch_dependent(k_zsolve_tma<T>, blocks, thr, smem, st, g, c, lgc, nitems, ws.spec, map,
                   (const cx_t<T>*)ws.tw, (const T*)ws.s2, cfac, scale0, zempty, ws.err);
  count_launch(sizeof(T) == 4 ? "zsolve_tma_f32" : "zsolve_tma_f64", st);
  return check_launch();
}

template size_t zsolve_smem<float>(int, int);
template cudaError_t make_zsolve_map<float>(const GridDesc&, const float2*, TmaDesc*);
template cudaError_t launch_zsolve_tma<float>(const GridDesc&, SpectralWs<float>&,
                                              const unsigned char*, cudaStream_t);

}  // namespace ibdl
