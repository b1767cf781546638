// Device-side building blocks of the IBDL matvec, shared by the one-kernel-
// per-pass launchers (k_fft.cu, k_points.cu) and the persistent solver
// (k_solver.cu).  Each "phase" function processes one work item (a row tile,
// a group of pencils, a point) with all threads of the calling block.  The FFT
// cores are not inlined (their own register allocation; the persistent
// solver also calls each phase through a non-inlined wrapper).
//
// Data produced by another block of the same launch (spectrum, grids, Krylov
// vectors) is read with ld.global.cg (__ldcg), which bypasses L1: inside a
// persistent kernel an SM's L1 may hold a line from an earlier phase.
#pragma once

#include <type_traits>

#include "ibdl_internal.cuh"

namespace ibdl {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// ---- double-float arithmetic (the type dd, ibdl_internal.cuh) --------------
// These rely on every float operation being rounded on its own: no term
// below is a product added to something, so nothing is contracted into a
// fused multiply-add except where fmaf is written out.
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = a.hi + b.hi;  // two-sum of the high parts
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;        // fast two-sum: renormalise
  return dd(h, e - (h - s));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // exact error of the high product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float h = p + e;
  return dd(h, e - (h - p));
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }
__device__ __forceinline__ bool operator>(dd a, dd b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ cdd cmul(cdd a, cdd b) {
  cdd r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
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

// ---- shared-memory FFT ---------------------------------------------------------
//
// Pencils of length n = 2^lg are transformed in shared memory by a Stockham
// FFT whose passes have radix 16, 8, 4 or 2 (ceil(lg / 4) passes, radices as
// even as possible, larger first).  A thread loads the R inputs of one
// butterfly, multiplies them by the pass twiddles, does the R-point DFT in
// registers and stores the R outputs; passes ping-pong between two buffers
// with one block barrier each.
//
// Shared layout of a pencil: element t at padi(t) = t + t/16, pencils
// pen_stride(n) = n + n/16 + 1 apart.  The spare slot after every 16
// elements spreads the stride-R stores of the first pass and the stride-16
// loads of later passes over distinct banks, for 8- and 16-byte complex.
//
// Twiddles: pass s (radix R, Ns = product of the earlier radices) multiplies
// input q of butterfly j by w^(q k), w = exp(-2 pi i / (Ns R)), k = j mod Ns.
// Its table holds w^(q k) at [q * Ns + k], so a warp reads consecutive
// entries; the tables of all passes are concatenated (fft_tw_count entries).

__host__ __device__ constexpr int padi(int t) { return t + (t >> 4); }
__host__ __device__ constexpr int pen_stride(int n) { return n + (n >> 4) + 1; }

// Pass plan of an n = 2^lg point FFT, named by a plan code pl = lg + 16 v:
// a first pass of radix 16 (or n when n < 16), then the remaining bits in
// passes of radix <= 16, larger radices first -- split as evenly as
// possible (variant v = 0: 1024 = 16 * 8 * 8, 512 = 16 * 8 * 4), or radix-16
// passes first and the remainder last (v = 1: 1024 = 16 * 16 * 4,
// 512 = 16 * 16 * 2).  The two differ only for lg = 9 and 10, the only
// sizes where v = 1 is offered (the float32 transforms of 2D geometries,
// chosen by the autotuner).  After the first pass Ns >= 16, so the padded
// shared offsets of every later pass are compile-time constants.
constexpr int kPlanVariants = 2;
__host__ __device__ constexpr int plan_lg(int pl) { return pl & 15; }
__host__ __device__ constexpr int plan_variant(int pl) { return pl >> 4; }
__host__ __device__ constexpr int plan_npass(int pl) {
  return plan_lg(pl) <= 4 ? 1 : 1 + (plan_lg(pl) - 1) / 4;
}
__host__ __device__ constexpr int plan_lr(int pl, int s) {
  return s == 0 ? (plan_lg(pl) < 4 ? plan_lg(pl) : 4)
         : plan_variant(pl) == 1
             ? (s < plan_npass(pl) - 1 ? 4 : plan_lg(pl) - 4 - 4 * (plan_npass(pl) - 2))
             : (plan_lg(pl) - 4) / (plan_npass(pl) - 1) +
                   (s - 1 < (plan_lg(pl) - 4) % (plan_npass(pl) - 1) ? 1 : 0);
}
__host__ __device__ constexpr int plan_lgns(int pl, int s) {
  return s == 0 ? 0 : plan_lgns(pl, s - 1) + plan_lr(pl, s - 1);
}
__host__ __device__ constexpr int plan_off(int pl, int s) {
  return s == 0 ? 0 : plan_off(pl, s - 1) + (1 << (plan_lgns(pl, s - 1) + plan_lr(pl, s - 1)));
}
__host__ __device__ constexpr int plan_tw_total(int pl) { return plan_off(pl, plan_npass(pl)); }
// the variants that exist for an lg (v = 1 only where it differs from v = 0)
__host__ __device__ constexpr bool plan_offered(int lg, int v) {
  return v == 0 || (v == 1 && (lg == 9 || lg == 10));
}

__host__ __device__ inline int ilog2(int n) {
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  return lg;
}

// Twiddle-table entries of an n-point FFT (the passes' tables concatenated)
// in plan variant v, n = 2^lg with 4 <= lg <= 12 (16 ... 4096 points, the
// sizes the library accepts); -1 for any other n or a variant not offered
// for it, so a caller sizing a buffer from it fails instead of silently
// taking another size's table.
__host__ __device__ inline int fft_tw_count(int n, int v = 0) {
  const int lg = ilog2(n);
  if ((1 << lg) != n || v < 0 || v >= kPlanVariants || !plan_offered(lg, v)) return -1;
  switch (lg + 16 * v) {
    case 4: return plan_tw_total(4);
    case 5: return plan_tw_total(5);
    case 6: return plan_tw_total(6);
    case 7: return plan_tw_total(7);
    case 8: return plan_tw_total(8);
    case 9: return plan_tw_total(9);
    case 10: return plan_tw_total(10);
    case 11: return plan_tw_total(11);
    case 12: return plan_tw_total(12);
    case 16 + 9: return plan_tw_total(16 + 9);
    case 16 + 10: return plan_tw_total(16 + 10);
    default: return -1;
  }
}

// Entries a twiddle buffer of element type T holds: the float32 tables may
// be of either variant (the autotuner's choice, per geometry), so their
// buffers and shared-memory budgets take the larger; the others use v = 0.
template <typename T>
__host__ __device__ inline int fft_tw_capacity(int n) {
  const int t0 = fft_tw_count(n, 0);
  if (!std::is_same<T, float>::value || t0 < 0) return t0;
  const int t1 = fft_tw_count(n, 1);
  return t1 > t0 ? t1 : t0;
}

// Plan variant and plan code of a geometry's transforms of element type T
// (only the float32 transforms have a tuned variant).
template <typename T>
__host__ __device__ inline int plan_variant_of(const GridDesc& g) {
  return std::is_same<T, float>::value ? g.fplan : 0;
}
template <typename T>
__host__ __device__ inline int plan_code_of(const GridDesc& g) {
  return g.log2n + 16 * plan_variant_of<T>(g);
}

// Table entry idx of an n-point FFT in plan variant v is exp(-2 pi i num /
// den) (the passes' tables walked without recursion, for run-time n).
__host__ __device__ inline void fft_tw_angle(int n, int idx, int* num, int* den, int v = 0) {
  const int pl = ilog2(n) + 16 * v, np = plan_npass(pl);
  int off = 0, lgns = 0;
  for (int s = 0; s < np; ++s) {
    const int lr = plan_lr(pl, s);
    const int size = 1 << (lgns + lr);
    if (idx < off + size || s == np - 1) {
      const int local = idx - off;
      *num = (local >> lgns) * (local & ((1 << lgns) - 1));
      *den = size;
      return;
    }
    off += size;
    lgns += lr;
  }
}

// -i * a (forward) or +i * a (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
  C r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

template <typename C> __device__ __forceinline__ C cmulc(C a, double wr, double wi) {
  using T = decltype(a.x);
  const T cr = (T)wr, ci = (T)wi;
  C r;
  r.x = a.x * cr - a.y * ci;
  r.y = a.x * ci + a.y * cr;
  return r;
}

// In-register DFTs, natural order in and out; sign -1 (forward) or +1.
template <bool INV, typename C> __device__ __forceinline__ void dft2(C* a) {
  const C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const C t2 = cadd(a1, a3), t3 = rot90<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}
template <bool INV, typename C> __device__ __forceinline__ void dft4(C* a) {
  dft4<INV>(a[0], a[1], a[2], a[3]);
}

constexpr double kR2 = 0.70710678118654752440;   // cos(pi/4)
constexpr double kC8 = 0.92387953251128675613;   // cos(pi/8)
constexpr double kS8 = 0.38268343236508977173;   // sin(pi/8)

// X[p] = E[p] + w8^p O[p], X[p+4] = E[p] - w8^p O[p] (radix-2 split of 8)
template <bool INV, typename C> __device__ __forceinline__ void dft8(C* a) {
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const double sg = INV ? 1.0 : -1.0;
  o1 = cmulc(o1, kR2, sg * kR2);
  o2 = rot90<INV>(o2);
  o3 = cmulc(o3, -kR2, sg * kR2);
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1);
  a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3);
  a[7] = csub(e3, o3);
}

// 16 = 4 x 4: DFT-4 over q1 of a[q2 + 4 q1], twiddle w16^(p1 q2), DFT-4 over
// q2; output index p1 + 4 p2.
template <bool INV, typename C> __device__ __forceinline__ void dft16(C* a) {
#pragma unroll
  for (int q2 = 0; q2 < 4; ++q2) dft4<INV>(a[q2], a[q2 + 4], a[q2 + 8], a[q2 + 12]);
  // a[q2 + 4 p1] now holds B[q2][p1]
  const double sg = INV ? 1.0 : -1.0;
  a[5] = cmulc(a[5], kC8, sg * kS8);      // w^1
  a[9] = cmulc(a[9], kR2, sg * kR2);      // w^2
  a[13] = cmulc(a[13], kS8, sg * kC8);    // w^3
  a[6] = cmulc(a[6], kR2, sg * kR2);      // w^2
  a[10] = rot90<INV>(a[10]);              // w^4
  a[14] = cmulc(a[14], -kR2, sg * kR2);   // w^6
  a[7] = cmulc(a[7], kS8, sg * kC8);      // w^3
  a[11] = cmulc(a[11], -kR2, sg * kR2);   // w^6
  a[15] = cmulc(a[15], -kC8, -sg * kS8);  // w^9
#pragma unroll
  for (int p1 = 0; p1 < 4; ++p1) dft4<INV>(a[4 * p1], a[4 * p1 + 1], a[4 * p1 + 2], a[4 * p1 + 3]);
  // a[4 p1 + p2] holds X[p1 + 4 p2]: transpose the 4 x 4 index
  C t;
  t = a[1]; a[1] = a[4]; a[4] = t;
  t = a[2]; a[2] = a[8]; a[8] = t;
  t = a[3]; a[3] = a[12]; a[12] = t;
  t = a[6]; a[6] = a[9]; a[9] = t;
  t = a[7]; a[7] = a[13]; a[13] = t;
  t = a[11]; a[11] = a[14]; a[14] = t;
}

// cos and sin of 2 pi e / 16 (no recursion: used only in constant
// expressions, below as template arguments' constants)
__host__ __device__ constexpr double cos16(int e) {
  return ((e & 15) < 8 ? 1.0 : -1.0) *
         ((e & 7) == 0 ? 1.0 : (e & 7) == 1 ? kC8 : (e & 7) == 2 ? kR2 : (e & 7) == 3 ? kS8
          : (e & 7) == 4 ? 0.0 : (e & 7) == 5 ? -kS8 : (e & 7) == 6 ? -kR2 : -kC8);
}
__host__ __device__ constexpr double sin16(int e) { return cos16(e + 12); }

// a * w16^E0 (h false) or a * w16^E1 (h true), w16 = exp(-+2 pi i / 16) for
// the forward (inverse) direction: both constants fold at compile time and
// each thread selects one
template <bool INV, int E0, int E1, typename C>
__device__ __forceinline__ C cmul_w16_sel(C a, bool h) {
  using T = decltype(a.x);
  constexpr double sg = INV ? 1.0 : -1.0;
  constexpr double c0 = cos16(E0), s0 = sg * sin16(E0);
  constexpr double c1 = cos16(E1), s1 = sg * sin16(E1);
  const T r0 = (T)c0, i0 = (T)s0, r1 = (T)c1, i1 = (T)s1;
  const T wr = h ? r1 : r0, wi = h ? i1 : i0;
  C r;
  r.x = a.x * wr - a.y * wi;
  r.y = a.x * wi + a.y * wr;
  return r;
}

template <typename C> __device__ __forceinline__ C cneg_if(C a, bool neg) {
  C r;
  r.x = neg ? -a.x : a.x;
  r.y = neg ? -a.y : a.y;
  return r;
}

// value of lane ^ 16 (all 32 lanes of the warp take part)
template <typename C> __device__ __forceinline__ C shfl_xor16(C v) {
  static_assert(sizeof(C) % 4 == 0, "whole words");
  constexpr int W = sizeof(C) / 4;
  unsigned u[W];
  memcpy(u, &v, sizeof(C));
#pragma unroll
  for (int i = 0; i < W; ++i) u[i] = __shfl_xor_sync(0xffffffffu, u[i], 16);
  memcpy(&v, u, sizeof(C));
  return v;
}

template <int LR, bool INV, typename C> __device__ __forceinline__ void dft_reg(C* a) {
  if (LR == 1) dft2<INV>(a);
  if (LR == 2) dft4<INV>(a);
  if (LR == 3) dft8<INV>(a);
  if (LR == 4) dft16<INV>(a);
}

// 1/x for the symbol (x > 0).  float: the hardware approximate reciprocal.
// double: Newton-Raphson for 1/x, r <- r + r (1 - x r), from a
// float first guess; each step doubles the number of correct bits (24 ->
// 48 -> beyond 53), at four FMAs instead of a full double division.
template <typename T> __device__ __forceinline__ T recip_symbol(T x);
template <> __device__ __forceinline__ float recip_symbol<float>(float x) {
  // the hardware approximate reciprocal (one MUFU instruction, within about
  // an ulp): ample for the float32 operator, and once per spectral element
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <> __device__ __forceinline__ dd recip_symbol<dd>(dd x) {
  // Newton from the float reciprocal of the high part, two steps in
  // double-float (24 -> 48 bits)
  dd r(__frcp_rn(x.hi), 0.0f);
  r = r + r * (dd(1) - x * r);
  return r + r * (dd(1) - x * r);
}
template <> __device__ __forceinline__ double recip_symbol<double>(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// The Helmholtz symbol multiply (Sec. 6.2) applied as the last forward pass
// stores its outputs: element t of pencil pen is scaled by
// scale0 / (c0 + cfac (pre + s2s[pbase + pen] + s2s[t])), or zeroed where
// that denominator is 0 (the Poisson limit's k = 0 mode).  Pencils at or
// beyond npl hold no data of the item and are left as they are.
template <typename T> struct SymbolEpi {
  const T* s2s;
  T pre, c0, cfac, scale0;
  int pbase, npl;
};

// Pencils of an item in global memory: pencil pen, element t at
// p + pen n + t (contiguous) or p + t n + pen (strided: the 3D z pencils,
// whose planes flagged in zempty hold no point and read as zeros).
template <typename T> struct GlobalPencils {
  cx_t<T>* p;
  int npl;                     // pencils of the item (the rest are idle)
  int lgc;                     // log2 of the item's pencil count (strided)
  const unsigned char* zempty; // strided only; may be null
  // shared input (SIN): the item's strided pencils as a dense box in shared
  // memory, element t of pencil pen at sin[t * ld + pen] (a bulk tensor copy)
  const cx_t<T>* sin;
  int ld;
  // SIN: once the first pass has read the box, thread 0 starts the copy of
  // item tma_next (>= 0) into it
  const struct TmaItem* tma;
  int tma_next;
};

// The bulk tensor copy of one staged z-pass item (k_tma.cu): the tensor map,
// the mbarrier the copy completes on, the box in shared memory and the
// item geometry (c pencils per item, n points, zb z rows per copy).
struct TmaItem {
  const void* map;
  uint64_t* bar;
  void* box;
  int c, n, lgn, zb, words, row_bytes;
  unsigned bytes;
};

// Starts the copy of item k's box (thread 0 only): c pencils of slab kx from
// y0, all n z rows, in copies of at most zb rows.  The box was last read with
// ordinary loads, so the async proxy is fenced first.
__device__ __forceinline__ void tma_issue_item(const TmaItem& t, int k) {
  const int p0 = k * t.c, kx = p0 >> t.lgn, y0 = p0 & (t.n - 1);
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(t.bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(t.bytes)
               : "memory");
  for (int z0 = 0; z0 < t.n; z0 += t.zb) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(
        reinterpret_cast<unsigned char*>(t.box) + (size_t)z0 * t.row_bytes);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(t.map)), "r"(y0 * t.words), "r"(z0), "r"(kx), "r"(bar)
        : "memory");
  }
}

// Float and double transforms of the solver's pencil passes read their
// first inputs from and write their last outputs to global memory, and
// fold the symbol multiply into the last forward pass.  Double-float keeps
// the staged copies and a multiply sweep of its own: the reciprocal and the
// global accesses unrolled into every butterfly would grow its code, whose
// size already limits it.
template <typename T> struct DirectPencils { static constexpr bool value = true; };
template <> struct DirectPencils<dd> { static constexpr bool value = false; };

// The radix-16 first pass (Ns = 1: no pass twiddles) with each butterfly
// split over two threads, for passes with at most half as many butterflies
// as the block has threads: the unsplit pass would leave half the threads
// idle while each of the others runs the whole 16-point DFT.
//
// 16 = 4 x 4 as in dft16 (input q = q2 + 4 q1, output p = p1 + 4 p2).  Half
// h of a butterfly takes the inputs with q2 in {2h, 2h + 1}; its DFT-4s over
// q1 are taken with the odd-q1 inputs negated when h = 1, which rotates
// their outputs by two (register r holds p1 = (r + 2h) mod 4), so that
// registers r = 2, 3 always hold the values the other half needs.  After
// the w16^(p1 q2) twiddles the halves swap those four values (lanes l and
// l ^ 16 hold the two halves of one butterfly) and each does the DFT-4s
// over q2 for its p1 = 2h + r.  For h = 1 the swapped-in values are the
// inputs q2 = 0, 1 and its own q2 = 2, 3, a cyclic shift by two, so outputs
// with odd p2 come out negated and are negated back.  Inputs as in
// fft_pass (global, staged box or shared); the outputs go to shared memory.
template <typename T, int LG, bool INV, bool GIN, bool STR, bool SIN>
__device__ __forceinline__ void fft_pass16_split(const cx_t<T>* __restrict__ src,
                                                 cx_t<T>* __restrict__ dst, int npen,
                                                 const GlobalPencils<T>& gio) {
  using C = cx_t<T>;
  static_assert(plan_variant(LG) == 0, "double-float transforms use the balanced plan");
  constexpr int N = 1 << LG, LGNB = LG - 4, NB = 1 << LGNB, PS = pen_stride(N);
  const int e = threadIdx.x;
  // the caller checked 2 total <= blockDim and total % 16 == 0, so the
  // threads below 2 total are whole warps
  if (e < (npen << LGNB) * 2) {
    const bool h = (e >> 4) & 1;
    const int b = ((e >> 5) << 4) | (e & 15);
    int pen, j;
    if constexpr (STR) {
      pen = b & ((1 << gio.lgc) - 1);
      j = b >> gio.lgc;
    } else {
      pen = b >> LGNB;
      j = b & (NB - 1);
    }
    const bool live = !GIN || pen < gio.npl;
    auto in = [&](int q) -> C {
      C v;
      v.x = v.y = 0;
      if (!live) return v;
      const int t = j + q * NB;
      if constexpr (GIN && SIN) {
        if (!(gio.zempty && gio.zempty[t])) v = gio.sin[t * gio.ld + pen];
      } else if constexpr (GIN && STR) {
        if (!(gio.zempty && gio.zempty[t])) v = __ldcg(gio.p + (size_t)t * N + pen);
      } else if constexpr (GIN) {
        v = __ldcg(gio.p + (size_t)pen * N + t);
      } else {
        v = src[pen * PS + padi(t)];
      }
      return v;
    };
    C x[2][4];
#pragma unroll
    for (int q2l = 0; q2l < 2; ++q2l)
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1) x[q2l][q1] = in(2 * h + q2l + 4 * q1);
#pragma unroll
    for (int q2l = 0; q2l < 2; ++q2l) {
      x[q2l][1] = cneg_if(x[q2l][1], h);
      x[q2l][3] = cneg_if(x[q2l][3], h);
      dft4<INV>(x[q2l][0], x[q2l][1], x[q2l][2], x[q2l][3]);
    }
    // register (q2l, r): exponent p1 q2 = r q2l (h = 0), ((r + 2) mod 4)(2 + q2l) (h = 1)
    x[0][0] = cmul_w16_sel<INV, 0, 4>(x[0][0], h);
    x[0][1] = cmul_w16_sel<INV, 0, 6>(x[0][1], h);
    x[0][3] = cmul_w16_sel<INV, 0, 2>(x[0][3], h);
    x[1][0] = cmul_w16_sel<INV, 0, 6>(x[1][0], h);
    x[1][1] = cmul_w16_sel<INV, 1, 9>(x[1][1], h);
    x[1][2] = cmul_w16_sel<INV, 2, 0>(x[1][2], h);
    x[1][3] = cmul_w16_sel<INV, 3, 3>(x[1][3], h);
    C y[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      y[r][0] = x[0][r];
      y[r][1] = x[1][r];
      y[r][2] = shfl_xor16(x[0][r + 2]);
      y[r][3] = shfl_xor16(x[1][r + 2]);
      dft4<INV>(y[r][0], y[r][1], y[r][2], y[r][3]);
      y[r][1] = cneg_if(y[r][1], h);
      y[r][3] = cneg_if(y[r][3], h);
    }
    if (live) {
      // outputs p = p1 + 4 p2 of butterfly j at padi(16 j + p) = padi(16 j) + p
      C* yb = dst + pen * PS + padi(j << 4) + 2 * h;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int p2 = 0; p2 < 4; ++p2) yb[r + 4 * p2] = y[r][p2];
    }
  }
  __syncthreads();
}

// One radix pass (see above).  SYM: scale the outputs by the symbol (a last
// forward pass).  GIN: read the inputs from global memory (a first pass)
// instead of src; GOUT: write the outputs to global memory (a last pass)
// instead of dst; only pencils below gio.npl are touched then.  A first
// pass reads elements j + q NB and a last pass writes j + p NS (NS = NB
// there); the thread of butterfly e takes j fastest for contiguous pencils
// and the pencil fastest for strided ones (STR), so a warp's accesses are
// coalesced either way.  With a row type RO, GOUT instead writes pencil pen
// as two real rows, its real parts to rows[2 pen n + t] and its imaginary
// parts to rows[(2 pen + 1) n + t] (the x inverse pass).
template <typename T, int LG, int S, bool INV, bool SYM = false, bool GIN = false,
          bool GOUT = false, bool STR = false, typename RO = void, bool SIN = false>
__device__ __forceinline__ void fft_pass(const cx_t<T>* __restrict__ src,
                                         cx_t<T>* __restrict__ dst, int npen,
                                         const cx_t<T>* __restrict__ tws,
                                         const SymbolEpi<T>& epi = SymbolEpi<T>{},
                                         const GlobalPencils<T>& gio = GlobalPencils<T>{},
                                         RO* rows = nullptr) {
  using C = cx_t<T>;
  constexpr bool kSym = SYM && !INV && DirectPencils<T>::value;
  constexpr bool kGlobal = GIN || GOUT;
  // LG is a plan code (plan_lg(LG) = log2 n, plan_variant(LG) the variant)
  constexpr int N = 1 << plan_lg(LG);
  constexpr int LR = plan_lr(LG, S), LGNS = plan_lgns(LG, S), OFF = plan_off(LG, S);
  constexpr int R = 1 << LR, LGNB = plan_lg(LG) - LR, NB = 1 << LGNB, NS = 1 << LGNS;
  constexpr int PS = pen_stride(N);
  static_assert(!GIN || S == 0, "global inputs feed the first pass");
  static_assert(!STR || kGlobal, "the strided order is for global accesses");
  const int total = npen << LGNB;
  if constexpr (std::is_same<T, dd>::value && S == 0 && LR == 4 && plan_lg(LG) > 4 && !SYM &&
                !GOUT) {
    // a first pass that is not also the last (fft_passes also instantiates
    // unreached passes with S = 0, which keep the plain loop).  Only the
    // double-float butterflies are split: the split costs six more twiddle
    // multiplies per butterfly and the exchange, which pays where the
    // arithmetic of a butterfly is long, not for float or float64 items
    // (measured: float32 solve items 9.4 -> 10.6 us split)
    if (2 * total <= (int)blockDim.x && (total & 15) == 0) {
      fft_pass16_split<T, LG, INV, GIN, STR, SIN>(src, dst, npen, gio);
      return;
    }
  }
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int pen, j;
    if constexpr (STR) {
      pen = e & ((1 << gio.lgc) - 1);
      j = e >> gio.lgc;
    } else {
      pen = e >> LGNB;
      j = e & (NB - 1);
    }
    if (kGlobal && pen >= gio.npl) continue;
    const int k = j & (NS - 1);
    C a[R];
    if constexpr (GIN && SIN) {
      // the strided pencils staged as a dense box in shared memory
      const C* xs = gio.sin + j * gio.ld + pen;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if (gio.zempty && gio.zempty[j + q * NB]) {
          a[q].x = a[q].y = 0;
        } else {
          a[q] = xs[q * NB * gio.ld];
        }
      }
    } else if constexpr (GIN) {
      if constexpr (STR) {
        const C* xg = gio.p + (size_t)j * N + pen;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          if (gio.zempty && gio.zempty[j + q * NB]) {
            a[q].x = a[q].y = 0;
          } else {
            a[q] = __ldcg(xg + (size_t)q * NB * N);
          }
        }
      } else {
        const C* xg = gio.p + (size_t)pen * N + j;
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = __ldcg(xg + q * NB);
      }
    } else {
      const C* x = src + pen * PS;
      if (NB % 16 == 0) {
        // padi(j + q NB) = padi(j) + q (NB + NB/16)
        const C* xb = x + padi(j);
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = xb[q * (NB + NB / 16)];
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = x[padi(j + q * NB)];
      }
    }
    if (NS > 1) {
      const C* tw = tws + OFF + k;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        C w = tw[q * NS];
        if (INV) w.y = -w.y;
        a[q] = cmul(a[q], w);
      }
    }
    dft_reg<LR, INV>(a);
    const int o = ((j - k) << LR) + k;
    if (kSym && pen < epi.npl) {
      // the last pass writes frequency o + p NS of pencil pen
      const T pt = epi.pre + epi.s2s[epi.pbase + pen];
#pragma unroll
      for (int p = 0; p < R; ++p) {
        const T den = epi.c0 + epi.cfac * (pt + epi.s2s[o + p * NS]);
        const T f = den > (T)0 ? epi.scale0 * recip_symbol<T>(den) : (T)0;
        a[p].x *= f;
        a[p].y *= f;
      }
    }
    if constexpr (GOUT && !std::is_void<RO>::value) {
      RO* yr = rows + (size_t)(2 * pen) * N + o;
#pragma unroll
      for (int p = 0; p < R; ++p) {
        yr[p * NS] = (RO)a[p].x;
        yr[N + p * NS] = (RO)a[p].y;
      }
    } else if constexpr (GOUT) {
      if constexpr (STR) {
        // planes without points are never read by the y inverse pass
        C* yg = gio.p + (size_t)o * N + pen;
#pragma unroll
        for (int p = 0; p < R; ++p)
          if (!(gio.zempty && gio.zempty[o + p * NS])) yg[(size_t)p * NS * N] = a[p];
      } else {
        C* yg = gio.p + (size_t)pen * N + o;
#pragma unroll
        for (int p = 0; p < R; ++p) yg[p * NS] = a[p];
      }
    } else {
      C* yb = dst + pen * PS + padi(o);
      if (NS % 16 == 0) {
        // padi(o + p NS) = padi(o) + p (NS + NS/16)
#pragma unroll
        for (int p = 0; p < R; ++p) yb[p * (NS + NS / 16)] = a[p];
      } else {
        // NS == 1: o = R j, and o mod 16 + p < 16, so padi(o + p) = padi(o) + p
#pragma unroll
        for (int p = 0; p < R; ++p) yb[p] = a[p];
      }
    }
  }
  __syncthreads();
}

// All passes of one transform direction.  Pass s reads buffer s mod 2 and
// writes buffer (s + 1) mod 2 of (a, b); returns the buffer of the result
// (meaningless when GOUT).
// SIN: the first pass reads the staged box (gio.sin).  HOOK: before the last
// pass (after the barrier that ends the pass before it), thread 0 starts the
// bulk copy of the next item (gio.tma_next >= 0) into the staging box, which
// the passes before have finished with.
template <typename T, int LG, bool INV, bool SYM, bool GIN, bool GOUT, bool STR,
          typename RO = void, bool SIN = false, bool HOOK = false>
__device__ __forceinline__ cx_t<T>* fft_passes(cx_t<T>* a, cx_t<T>* b, int npen,
                                               const cx_t<T>* __restrict__ tws,
                                               const SymbolEpi<T>& epi,
                                               const GlobalPencils<T>& gio,
                                               RO* rows = nullptr) {
  constexpr int NP = plan_npass(LG);
  static_assert(NP <= 3, "n <= 4096");
  constexpr int S1 = NP > 1 ? 1 : 0, S2 = NP > 2 ? 2 : 0;
  // the strided order only where a pass touches global memory
  constexpr bool ST0 = STR && (GIN || (GOUT && NP == 1));
  constexpr bool ST1 = STR && GOUT && NP == 2, ST2 = STR && GOUT && NP == 3;
  if constexpr (HOOK && NP == 1) {
    if (threadIdx.x == 0 && gio.tma_next >= 0) tma_issue_item(*gio.tma, gio.tma_next);
  }
  fft_pass<T, LG, 0, INV, SYM && NP == 1, GIN, GOUT && NP == 1, ST0, RO, SIN && GIN>(
      a, b, npen, tws, epi, gio, rows);
  if (NP == 1) return b;
  if constexpr (HOOK && NP == 2) {
    if (threadIdx.x == 0 && gio.tma_next >= 0) tma_issue_item(*gio.tma, gio.tma_next);
  }
  fft_pass<T, LG, S1, INV, SYM && NP == 2, false, GOUT && NP == 2, ST1, RO>(b, a, npen, tws, epi,
                                                                             gio, rows);
  if (NP == 2) return a;
  if constexpr (HOOK && NP == 3) {
    if (threadIdx.x == 0 && gio.tma_next >= 0) tma_issue_item(*gio.tma, gio.tma_next);
  }
  fft_pass<T, LG, S2, INV, SYM, false, GOUT, ST2, RO>(a, b, npen, tws, epi, gio, rows);
  return b;
}

template <typename T, int LG, bool INV>
__device__ __noinline__ cx_t<T>* fft_run_lg(cx_t<T>* src, cx_t<T>* dst, int npen,
                                            const cx_t<T>* __restrict__ tws) {
  return fft_passes<T, LG, INV, false, false, false, false>(src, dst, npen, tws, SymbolEpi<T>{},
                                                            GlobalPencils<T>{});
}

// The pencil transforms of one item straight from and back to global
// memory (gio): MODE 0 forward, 1 inverse, 2 forward with the symbol
// multiply on its last pass, then inverse.  bufA/bufB are the shared pencil
// buffers of npen pencils.
template <typename T, int LG, int MODE, bool STR, bool SIN = false>
__device__ __noinline__ void fft_global_lg(cx_t<T>* bufA, cx_t<T>* bufB, int npen,
                                           const cx_t<T>* __restrict__ tws,
                                           const SymbolEpi<T> epi, const GlobalPencils<T> gio) {
  if constexpr (MODE == 2) {
    // SIN: bufA is the staging box (sized for a padded buffer), reused as a
    // ping-pong buffer once the first pass has read it
    cx_t<T>* r = fft_passes<T, LG, false, true, true, false, STR, void, SIN>(bufA, bufB, npen,
                                                                              tws, epi, gio);
    cx_t<T>* o = (r == bufA) ? bufB : bufA;
    fft_passes<T, LG, true, false, false, true, STR, void, false, SIN>(r, o, npen, tws, epi, gio);
  } else {
    fft_passes<T, LG, MODE == 1, false, true, true, STR>(bufA, bufB, npen, tws, epi, gio);
  }
}

template <typename T, int MODE, bool STR, bool SIN = false>
__device__ __forceinline__ void fft_global(cx_t<T>* bufA, cx_t<T>* bufB, int pl, int npen,
                                           const cx_t<T>* __restrict__ tws,
                                           const SymbolEpi<T>& epi, const GlobalPencils<T>& gio) {
  static_assert(DirectPencils<T>::value, "double-float stages its pencils");
  if constexpr (std::is_same<T, float>::value) {
    if (pl == 16 + 9) return fft_global_lg<T, 16 + 9, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    if (pl == 16 + 10)
      return fft_global_lg<T, 16 + 10, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
  }
  switch (plan_lg(pl)) {
    case 4: return fft_global_lg<T, 4, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 5: return fft_global_lg<T, 5, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 6: return fft_global_lg<T, 6, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 7: return fft_global_lg<T, 7, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 8: return fft_global_lg<T, 8, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 9: return fft_global_lg<T, 9, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 10: return fft_global_lg<T, 10, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    case 11: return fft_global_lg<T, 11, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
    default: return fft_global_lg<T, 12, MODE, STR, SIN>(bufA, bufB, npen, tws, epi, gio);
  }
}

// Inverse transform of the npen pencils in bufA (shared), the last pass
// writing each pencil as two real rows of `rows` (global, n apart).
template <typename T, int LG, typename OutT>
__device__ __noinline__ void fft_inverse_rows_lg(cx_t<T>* bufA, cx_t<T>* bufB, int npen,
                                                 const cx_t<T>* __restrict__ tws, OutT* rows) {
  GlobalPencils<T> gio{};
  gio.npl = npen;
  fft_passes<T, LG, true, false, false, true, false, OutT>(bufA, bufB, npen, tws,
                                                           SymbolEpi<T>{}, gio, rows);
}

template <typename T, typename OutT>
__device__ __forceinline__ void fft_inverse_rows(cx_t<T>* bufA, cx_t<T>* bufB, int pl, int npen,
                                                 const cx_t<T>* __restrict__ tws, OutT* rows) {
  static_assert(DirectPencils<T>::value, "double-float stages its rows");
  if constexpr (std::is_same<T, float>::value) {
    if (pl == 16 + 9) return fft_inverse_rows_lg<T, 16 + 9>(bufA, bufB, npen, tws, rows);
    if (pl == 16 + 10) return fft_inverse_rows_lg<T, 16 + 10>(bufA, bufB, npen, tws, rows);
  }
  switch (plan_lg(pl)) {
    case 4: return fft_inverse_rows_lg<T, 4>(bufA, bufB, npen, tws, rows);
    case 5: return fft_inverse_rows_lg<T, 5>(bufA, bufB, npen, tws, rows);
    case 6: return fft_inverse_rows_lg<T, 6>(bufA, bufB, npen, tws, rows);
    case 7: return fft_inverse_rows_lg<T, 7>(bufA, bufB, npen, tws, rows);
    case 8: return fft_inverse_rows_lg<T, 8>(bufA, bufB, npen, tws, rows);
    case 9: return fft_inverse_rows_lg<T, 9>(bufA, bufB, npen, tws, rows);
    case 10: return fft_inverse_rows_lg<T, 10>(bufA, bufB, npen, tws, rows);
    case 11: return fft_inverse_rows_lg<T, 11>(bufA, bufB, npen, tws, rows);
    default: return fft_inverse_rows_lg<T, 12>(bufA, bufB, npen, tws, rows);
  }
}

// Transforms npen pencils held in src (shared, padded layout); tws is the
// concatenated twiddle table in shared memory, of the plan pl (a plan code:
// log2 n + 16 * variant).  The caller synchronises before the call.
// Returns the buffer (src or dst) holding the result.
template <typename T, bool INV>
__device__ __forceinline__ cx_t<T>* fft_run(cx_t<T>* src, cx_t<T>* dst, int pl, int npen,
                                            const cx_t<T>* __restrict__ tws) {
  if constexpr (std::is_same<T, float>::value) {
    if (pl == 16 + 9) return fft_run_lg<T, 16 + 9, INV>(src, dst, npen, tws);
    if (pl == 16 + 10) return fft_run_lg<T, 16 + 10, INV>(src, dst, npen, tws);
  }
  switch (plan_lg(pl)) {
    case 4: return fft_run_lg<T, 4, INV>(src, dst, npen, tws);
    case 5: return fft_run_lg<T, 5, INV>(src, dst, npen, tws);
    case 6: return fft_run_lg<T, 6, INV>(src, dst, npen, tws);
    case 7: return fft_run_lg<T, 7, INV>(src, dst, npen, tws);
    case 8: return fft_run_lg<T, 8, INV>(src, dst, npen, tws);
    case 9: return fft_run_lg<T, 9, INV>(src, dst, npen, tws);
    case 10: return fft_run_lg<T, 10, INV>(src, dst, npen, tws);
    case 11: return fft_run_lg<T, 11, INV>(src, dst, npen, tws);
    default: return fft_run_lg<T, 12, INV>(src, dst, npen, tws);
  }
}

template <typename V>
__device__ __forceinline__ void copy_to_shared(V* dst, const V* __restrict__ src, int count);
// double-float tables move as their float vectors
__device__ __forceinline__ void copy_to_shared(cdd* dst, const cdd* __restrict__ src,
                                               int count) {
  copy_to_shared(reinterpret_cast<float4*>(dst), reinterpret_cast<const float4*>(src), count);
}
__device__ __forceinline__ void copy_to_shared(dd* dst, const dd* __restrict__ src, int count) {
  copy_to_shared(reinterpret_cast<float2*>(dst), reinterpret_cast<const float2*>(src), count);
}

// Copies `count` values from global (around L1) to shared memory.
template <typename V>
__device__ __forceinline__ void copy_to_shared(V* dst, const V* __restrict__ src, int count) {
  constexpr int U = 4;
  for (int e0 = threadIdx.x; e0 < count; e0 += U * blockDim.x) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < count) v[u] = __ldcg(src + e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < count) dst[e] = v[u];
    }
  }
}

// Shared-memory tables: the twiddles (ntw complex) and the sin^2 table (ns
// reals, ns = 0 for none), copied with all of a thread's loads of a batch in
// flight before its first store, so that tables of up to KB * blockDim
// entries cost one L2 round trip (a batch per KB * blockDim entries).  The
// loads are issued first, the stores come when `stage_tables_store` runs, so
// a caller can overlap other global loads with them.
template <typename V> struct TabVec { using type = V; };
template <> struct TabVec<cdd> { using type = float4; };
template <> struct TabVec<dd> { using type = float2; };

template <typename T, int KB> struct TableStage {
  using C = cx_t<T>;
  using VC = typename TabVec<C>::type;
  using VT = typename TabVec<T>::type;
  VC a[KB];
  VT b[KB];
  __device__ __forceinline__ void load(const C* __restrict__ tw, int ntw, const T* __restrict__ s2,
                                       int ns, int base) {
    const VC* tv = reinterpret_cast<const VC*>(tw);
    const VT* sv = reinterpret_cast<const VT*>(s2);
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int e = base + threadIdx.x + u * blockDim.x;
      if (e < ntw) a[u] = __ldcg(tv + e);
      if (e < ns) b[u] = __ldcg(sv + e);
    }
  }
  __device__ __forceinline__ void store(C* tws, int ntw, T* s2s, int ns, int base) const {
    VC* tv = reinterpret_cast<VC*>(tws);
    VT* sv = reinterpret_cast<VT*>(s2s);
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int e = base + threadIdx.x + u * blockDim.x;
      if (e < ntw) tv[e] = a[u];
      if (e < ns) sv[e] = b[u];
    }
  }
  // everything past the first batch (large n or few threads), copied at once
  __device__ __forceinline__ void rest(const C* __restrict__ tw, C* tws, int ntw,
                                       const T* __restrict__ s2, T* s2s, int ns) {
    for (int base = KB * blockDim.x; base < ntw || base < ns; base += KB * blockDim.x) {
      load(tw, ntw, s2, ns, base);
      store(tws, ntw, s2s, ns, base);
    }
  }
};

// Entries per thread of a table batch: twiddles of an n <= 1024 FFT
// (1168 entries) in one batch of 256 threads.
constexpr int kTabBatch = 5;

// Two consecutive complex values as one 16-byte access (float) or two
// (double).  Even element indices keep the float pair 16-byte aligned.
template <typename T> struct Pair;
template <> struct Pair<float> {
  float2 a, b;
  __device__ __forceinline__ void load(const float2* p) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
  __device__ __forceinline__ void store(float2* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  }
};
template <> struct Pair<double> {
  double2 a, b;
  __device__ __forceinline__ void load(const double2* p) {
    a = __ldcg(p);
    b = __ldcg(p + 1);
  }
  __device__ __forceinline__ void store(double2* p) const {
    p[0] = a;
    p[1] = b;
  }
};

template <> struct Pair<dd> {
  cdd a, b;
  __device__ __forceinline__ void load(const cdd* p) {
    const float4 u = __ldcg(reinterpret_cast<const float4*>(p));
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p + 1));
    a.x = dd(u.x, u.y);
    a.y = dd(u.z, u.w);
    b.x = dd(v.x, v.y);
    b.y = dd(v.z, v.w);
  }
  __device__ __forceinline__ void store(cdd* p) const {
    reinterpret_cast<float4*>(p)[0] = make_float4(a.x.hi, a.x.lo, a.y.hi, a.y.lo);
    reinterpret_cast<float4*>(p)[1] = make_float4(b.x.hi, b.x.lo, b.y.hi, b.y.lo);
  }
};

// The spread runs in the transforms' own arithmetic: float, float64, or
// double-float (the spread gathers without atomics, so any type works).
template <typename T> __device__ __forceinline__ T wload(const PointData& p, int c, int t, int i);
template <> __device__ __forceinline__ double wload<double>(const PointData& p, int c, int t,
                                                            int i) {
  return (t >= 0 && t < 4) ? p.W64[c][t * p.m + i] : 0.0;
}
template <> __device__ __forceinline__ float wload<float>(const PointData& p, int c, int t,
                                                          int i) {
  return (t >= 0 && t < 4) ? p.W32[c][t * p.m + i] : 0.0f;
}
template <> __device__ __forceinline__ dd wload<dd>(const PointData& p, int c, int t, int i) {
  return (t >= 0 && t < 4) ? dd(p.W64[c][t * p.m + i]) : dd(0);
}

// Point normal component c and weight / h^d in the spread's precision.
template <typename T> __device__ __forceinline__ T pt_nrm(const PointData& p, int c, int i);
template <> __device__ __forceinline__ double pt_nrm<double>(const PointData& p, int c, int i) {
  return p.nrm[c][i];
}
template <> __device__ __forceinline__ float pt_nrm<float>(const PointData& p, int c, int i) {
  return p.nrm32[c][i];
}
template <> __device__ __forceinline__ dd pt_nrm<dd>(const PointData& p, int c, int i) {
  return dd(p.nrm[c][i]);
}
template <typename T> __device__ __forceinline__ T pt_w(const PointData& p, int i);
template <> __device__ __forceinline__ double pt_w<double>(const PointData& p, int i) {
  return p.w[i];
}
template <> __device__ __forceinline__ float pt_w<float>(const PointData& p, int i) {
  return p.w32[i];
}
template <> __device__ __forceinline__ dd pt_w<dd>(const PointData& p, int i) {
  return dd(p.w[i]);
}

template <typename T> __device__ __forceinline__ bool is_zero(T v) { return v == (T)0; }
template <> __device__ __forceinline__ bool is_zero<dd>(dd v) { return v.hi == 0.0f; }

// First index in [p, np) whose sorted key sx[] is >= v (np if none), found by
// the 32 lanes of a warp together; every lane returns the same index.
__device__ __forceinline__ int warp_lower_bound(const int* sx, int p, int np, int v) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int idx = p + lane;
    const unsigned lt = __ballot_sync(0xffffffffu, idx < np && sx[idx] < v);
    if (lt != 0xffffffffu) return p + __popc(lt);  // keys are sorted: a prefix
    p += 32;
  }
}

// Rows per tile of the x passes: 2D keeps 4 (2 for n = 2048) so that even a
// 1024^2 grid has 256 tiles; 3D takes 8, so each kx of a tile is a 64-byte
// (float) or 128-byte (double) segment of the transposed spectrum.
__host__ __device__ inline int rows_per_tile(int dim, int n) {
  if (dim == 3) return 8;
  return n >= 2048 ? 2 : 4;
}

// Shared memory of a row tile: two pencil buffers and the twiddle table.
// (n outside the supported sizes: the largest size_t, which no budget meets)
template <typename T>
__host__ __device__ __forceinline__ size_t rows_smem_bytes(int n, int rows) {
  const int ntw = fft_tw_capacity<T>(n);
  if (ntw < 0) return ~(size_t)0;
  return (2 * (size_t)(rows / 2) * pen_stride(n) + (size_t)ntw) * sizeof(cx_t<T>);
}

// Gather spread of one tile (double-float).  rows holds the tile's R rows in
// the interleaved pencil layout; sbuf (bytes) is the staging space for the
// chunks' point records.  A tile's bin is sorted by the point's first
// support column xs (then by index), so the points that reach a run of
// columns are a contiguous run of the bin.  The 32 lanes of a warp own 32
// nodes -- R rows of 32/R neighbouring columns -- and walk that run
// together, each lane adding the shares that fall on its node in a register;
// a node has exactly one owner, so no atomics are needed and the sum's order
// is fixed (the spread is bitwise reproducible).  Warps take the column
// groups in turn.  The sorted lists are b.spts.
template <typename S, int D>
__device__ __forceinline__ void spread_gather(const GridDesc& g, const PointData& p, const Bins& b,
                                           const SpreadSrc& src, S* rows, unsigned char* sbuf,
                                           size_t sbytes, int z, int y0, int lo, int hi) {
  const int n = g.n, mask = n - 1, R = b.rows, lgR = __ffs(R) - 1;
  const int PS = pen_stride(n);
  const int tid = threadIdx.x, nt = blockDim.x;
  // The tile's points are taken in chunks of KP (contiguous runs of the
  // sorted bin).  Stage A (one thread per point) gathers each point's data
  // with independent loads and stages, in bufB (unused until the FFT), its
  // first column xs, first row yb and the node factors of its 6 x 6 box:
  //   node (xs + a, yb + bb):  U[a] cA[bb] + V[a] cB[bb],
  //   U[a] = W_x[a-1],  V[a] = W_x[a] - W_x[a-2],
  //   cA[bb] = P dW_y[bb] + Q W_y[bb-1],  cB[bb] = X W_y[bb-1],
  // P = q w/h^d ny W_z[c-1], Q = q w/h^d nz dW_z[c] + v w/h^d W_z[c-1],
  // X = q w/h^d nx W_z[c-1] / (2h), c the plane offset (3D), W[t] = 0
  // outside t = 0..3.  Stage B gathers (see above).
  const S inv2h = (S)g.inv2h;
  constexpr int kRec = 24;  // U[6], V[6], cA[6], cB[6]
  const int per_pt = kRec * (int)sizeof(S) + 2 * (int)sizeof(int);
  int KP = (int)(sbytes / per_pt);
  if (KP > 512) KP = 512;
  S* sv = reinterpret_cast<S*>(sbuf);  // [KP][kRec]
  int* sxs = reinterpret_cast<int*>(sv + (size_t)kRec * KP);
  int* syb = sxs + KP;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int cpg = 32 >> lgR;          // columns per lane group (R <= 32)
  const int lr = lane & (R - 1);      // this lane's row of the tile
  const int lc = lane >> lgR;         // this lane's column within the group
  const int ncg = n / cpg;            // column groups
  for (int c0 = lo; c0 < hi; c0 += KP) {
    const int np = min(KP, hi - c0);
    for (int t = tid; t < np; t += nt) {
      const int i = __ldg(b.spts + c0 + t);
      int ok = 1;
      S wz = (S)1, dz = (S)0;
      if (D == 3) {
        const int cz = (z - (__ldg(p.base[2] + i) - 1)) & mask;
        ok = cz < kBoxSide;
        wz = wload<S>(p, 2, cz - 1, i);
        dz = (wload<S>(p, 2, cz, i) - wload<S>(p, 2, cz - 2, i)) * inv2h;
      }
      S P = 0, Q = 0, X = 0;
      const S wi = pt_w<S>(p, i);
      if (src.q_div) {
        const S amp = (S)src.coef_div * (S)__ldcg(src.q_div + i) * wi;
        P = amp * pt_nrm<S>(p, 1, i) * wz;
        if (D == 3) Q = amp * pt_nrm<S>(p, 2, i) * dz;
        X = amp * pt_nrm<S>(p, 0, i) * wz * inv2h;
      }
      if (src.v_plain) {
        S v = (S)src.coef_plain * (S)__ldcg(src.v_plain + i) * wi * wz;
        if (src.plain_nrm >= 0) v *= pt_nrm<S>(p, src.plain_nrm, i);
        Q += v;
      }
      if (!ok) P = Q = X = 0;
      S wx[4], wy[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        wx[u] = wload<S>(p, 0, u, i);
        wy[u] = wload<S>(p, 1, u, i);
      }
      S* rec = sv + (size_t)t * kRec;
#pragma unroll
      for (int a = 0; a < kBoxSide; ++a) {
        const S w1 = (a >= 1 && a <= 4) ? wx[a - 1] : (S)0;
        const S w0 = a <= 3 ? wx[a] : (S)0;
        const S w2 = (a >= 2) ? wx[a - 2] : (S)0;
        rec[a] = w1;
        rec[6 + a] = w0 - w2;
        const S y1 = (a >= 1 && a <= 4) ? wy[a - 1] : (S)0;
        const S y0v = a <= 3 ? wy[a] : (S)0;
        const S y2 = (a >= 2) ? wy[a - 2] : (S)0;
        rec[12 + a] = P * (y0v - y2) * inv2h + Q * y1;
        rec[18 + a] = X * y1;
      }
      sxs[t] = (__ldg(p.base[0] + i) - 1) & mask;
      syb[t] = __ldg(p.base[1] + i) - 1;
    }
    __syncthreads();
    // Stage B: warp `warp` takes column groups warp, warp + nwarps, ...; the
    // candidates of group g (first column x0) have xs in [x0 - 5, x0 + cpg - 1]
    // (mod n).  plo / phi advance with g (the groups rise with x).
    int plo = 0, phi = 0;
    const bool all = cpg + kBoxSide - 1 >= n;  // the window covers every column
    for (int gi = warp; gi < ncg; gi += nwarps) {
      const int x0 = gi * cpg, x = x0 + lc;
      int e0, e1, w0 = np, w1 = np;  // [e0, e1): main run; [w0, w1): wrapped run
      if (all) {
        e0 = 0;
        e1 = np;
      } else {
        const int wl = x0 - (kBoxSide - 1);
        plo = warp_lower_bound(sxs, plo, np, wl < 0 ? 0 : wl);
        phi = warp_lower_bound(sxs, phi > plo ? phi : plo, np, x0 + cpg);
        e0 = plo;
        e1 = phi;
        if (wl < 0) w0 = warp_lower_bound(sxs, phi, np, n + wl);  // points near x = n
        if (e0 == e1 && w0 == w1) {
          // no candidate: skip to the next group of this warp that can have one
          if (plo >= np) break;
          const int first = sxs[plo];  // the next candidate's column
          const int gneed = (first - cpg + 1) / cpg;  // groups before it cannot reach it
          if (gneed > gi + nwarps) gi += ((gneed - gi) / nwarps) * nwarps - nwarps;
          continue;
        }
      }
      S acc = 0;
      const int yrow = y0 + lr;
      for (int pass = 0; pass < 2; ++pass) {
        const int ea = pass ? w0 : e0, eb = pass ? w1 : e1;
        for (int e = ea; e < eb; ++e) {
          const int a = (x - sxs[e]) & mask;
          const int bb = (yrow - syb[e]) & mask;
          if (a < kBoxSide && bb < kBoxSide) {
            const S* rec = sv + (size_t)e * kRec;
            acc += rec[a] * rec[12 + bb] + rec[6 + a] * rec[18 + bb];
          }
        }
      }
      if (!is_zero(acc)) rows[((lr >> 1) * PS + padi(x)) * 2 + (lr & 1)] += acc;
    }
    __syncthreads();
  }

}

// Scatter spread of one tile (float, float64): one thread per (point, support
// row) adds the 6 nodes of that row with shared-memory atomics (native for
// both types), so the sum's order varies with the atomics' order (rounding
// only).  The bin is in fill order (about the points' index order), so the
// threads of stage A load neighbouring points' data from neighbouring
// addresses.
template <typename S, int D>
__device__ __forceinline__ void spread_scatter(const GridDesc& g, const PointData& p, const Bins& b,
                                            const SpreadSrc& src, S* rows, unsigned char* sbuf,
                                            size_t sbytes, int z, int y0, int lo, int hi) {
  const int n = g.n, mask = n - 1, R = b.rows;
  const int PS = pen_stride(n);
  const int tid = threadIdx.x, nt = blockDim.x;
  // Stage A (one thread per point) gathers each point's data with
  // independent loads and folds it into per-point coefficients; stage B (one
  // thread per (point, support row bb)) adds the 6 x nodes of that row.
  // With c = the plane offset (3D) and W[t] = 0 outside t = 0..3:
  //   node a: W_x[a-1] * cA + (W_x[a] - W_x[a-2]) * cB,
  //   cA = q w/h^d (ny dW_y[bb] W_z[c-1] + nz W_y[bb-1] dW_z[c]) + v w/h^d W_y[bb-1] W_z[c-1]
  //   cB = q w/h^d nx W_y[bb-1] W_z[c-1] / (2h),
  // staged as  cA = P dW_y[bb] + Q W_y[bb-1],  cB = X W_y[bb-1].
  const S inv2h = (S)g.inv2h;
  constexpr int kWords = 11;  // wx[4], wy[4], P, Q, X
  const int per_pt = kWords * (int)sizeof(S) + 2 * (int)sizeof(int);
  int KP = (int)(sbytes / per_pt);
  if (KP > 256) KP = 256;
  S* sv = reinterpret_cast<S*>(sbuf);  // [kWords][KP]
  int* sxb = reinterpret_cast<int*>(sv + kWords * KP);
  int* syb = sxb + KP;
  for (int c0 = lo; c0 < hi; c0 += KP) {
    const int np = min(KP, hi - c0);
    for (int t = tid; t < np; t += nt) {
      const int i = __ldg(b.pts + c0 + t);
      int ok = 1;
      S wz = (S)1, dz = (S)0;
      if (D == 3) {
        const int cz = (z - (__ldg(p.base[2] + i) - 1)) & mask;
        ok = cz < kBoxSide;
        wz = wload<S>(p, 2, cz - 1, i);
        dz = (wload<S>(p, 2, cz, i) - wload<S>(p, 2, cz - 2, i)) * inv2h;
      }
      S P = 0, Q = 0, X = 0;
      // float32: one conversion (q) per staged point; the normals and
      // weights have float copies (float64 work is slow on GB300)
      const S wi = pt_w<S>(p, i);
      if (src.q_div) {
        const S amp = (S)src.coef_div * (S)__ldcg(src.q_div + i) * wi;
        P = amp * pt_nrm<S>(p, 1, i) * wz;
        if (D == 3) Q = amp * pt_nrm<S>(p, 2, i) * dz;
        X = amp * pt_nrm<S>(p, 0, i) * wz * inv2h;
      }
      if (src.v_plain) {
        S v = (S)src.coef_plain * (S)__ldcg(src.v_plain + i) * wi * wz;
        if (src.plain_nrm >= 0) v *= pt_nrm<S>(p, src.plain_nrm, i);
        Q += v;
      }
      if (!ok) P = Q = X = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sv[u * KP + t] = wload<S>(p, 0, u, i);
        sv[(4 + u) * KP + t] = wload<S>(p, 1, u, i);
      }
      sv[8 * KP + t] = P;
      sv[9 * KP + t] = Q;
      sv[10 * KP + t] = X;
      sxb[t] = __ldg(p.base[0] + i) - 1;
      syb[t] = __ldg(p.base[1] + i) - 1;
    }
    __syncthreads();
    for (int e = tid; e < np * kBoxSide; e += nt) {
      const int t = e / kBoxSide, bb = e - t * kBoxSide;
      const int ry = ((syb[t] + bb) & mask) - y0;
      if ((unsigned)ry >= (unsigned)R) continue;
      const S P = sv[8 * KP + t], Q = sv[9 * KP + t], X = sv[10 * KP + t];
      const S wyb = (bb >= 1 && bb <= 4) ? sv[(4 + bb - 1) * KP + t] : (S)0;
      const S wy0 = bb <= 3 ? sv[(4 + bb) * KP + t] : (S)0;
      const S wy2 = bb >= 2 ? sv[(4 + bb - 2) * KP + t] : (S)0;
      const S cA = P * (wy0 - wy2) * inv2h + Q * wyb;
      const S cB = X * wyb;
      if (cA == (S)0 && cB == (S)0) continue;
      S wx[6];
      wx[0] = 0;
      wx[5] = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) wx[u + 1] = sv[u * KP + t];  // wx[k] = W_x[k-1]
      S* rowp = rows + (size_t)(ry >> 1) * PS * 2 + (ry & 1);
      const int xb = sxb[t];
#pragma unroll
      for (int a = 0; a < kBoxSide; ++a) {
        // W_x[a] - W_x[a-2] = wx[a+1] - wx[a-1]
        const S wa1 = wx[a];
        const S wa = (a + 1 < 6) ? wx[a + 1] : (S)0;
        const S wam2 = (a >= 1) ? wx[a - 1] : (S)0;
        const S val = wa1 * cA + (wa - wam2) * cB;
        if (val != (S)0) atomicAdd(rowp + (size_t)padi((xb + a) & mask) * 2, val);
      }
    }
    __syncthreads();
  }
}

// The spread of a tile gathers (no atomics) in double-float, which has no
// atomic add and whose float64 alternative runs on GB300's slow float64
// pipe; float and float64 scatter with native shared-memory atomics, which
// measured faster for them (a gather walks every candidate point of a
// column group with all 32 lanes).
template <typename T> struct SpreadGathers { static constexpr bool value = false; };
template <> struct SpreadGathers<dd> { static constexpr bool value = true; };

// ---- fused spread + forward x pass ------------------------------------------
//
// Tile = R rows y0..y0+R-1 at plane z.  The rows are zeroed (or seeded with
// coef_grid * f) in shared memory, then every node of the tile gathers the
// shares of the points in the tile's bin:
//
//   S~q at node (bx-1+a, by-1+b, bz-1+c) (Sec. 5.2, the centred difference of
//   the spread of q n, fused):  q w/h^d [ nx dW_x[a] W_y[b-1] W_z[c-1]
//        + ny W_x[a-1] dW_y[b] W_z[c-1] + nz W_x[a-1] W_y[b-1] dW_z[c] ],
//   dW[a] = (W[a] - W[a-2]) / (2h),  W[t] = 0 outside t = 0..3;
//   S v at the same node:  v w/h^d W_x[a-1] W_y[b-1] W_z[c-1].
//
// Then two real rows are packed as one complex row, FFT'd along x, separated
// (A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i)) and written
// to the transposed half spectrum spec[k][z][y], k = 0..n/2.  The spread
// runs in the transforms' arithmetic T: scattered with atomics (float,
// float64) or gathered (double-float), see SpreadGathers.
template <typename T, int D>
__device__ __forceinline__ void phase_rows_fwd(const GridDesc& g, const PointData& p, const Bins& b,
                               const SpreadSrc& src, cx_t<T>* spec,
                               const cx_t<T>* __restrict__ tw, double* write_grid, int tile,
                               unsigned char* smem) {
  using C = cx_t<T>;
  using S = T;  // the spread's arithmetic
  const int n = g.n, lg = g.log2n, mask = n - 1, R = b.rows, npen = R >> 1;
  const int lgnp = __ffs(npen) - 1;  // R is a power of two (checked when the tiles are built)
  const int PS = pen_stride(n);
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)npen * PS;
  C* tws = bufB + (size_t)npen * PS;
  S* rows = reinterpret_cast<S*>(bufA);  // row r, column x at [((r>>1)*PS + padi(x))*2 + (r&1)]
  const int ngroups = n / R;
  const int z = (D == 3) ? tile / ngroups : 0;
  const int y0 = (tile % ngroups) * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t row0 = ((size_t)z * n + y0) * n;
  const int lo = b.start[tile], hi = b.start[tile + 1];
  const int half = n >> 1;
  const size_t slab = (D == 3) ? (size_t)n * n : (size_t)n;
  const size_t pos0 = (size_t)z * n + y0;

  if (D == 3 && src.skip_empty_planes && !src.f_grid && !write_grid && b.zempty &&
      b.zempty[z])
    return;  // a plane without points: zero, and read as zero by the z pass
  if (lo == hi && !src.f_grid) {
    // no source touches the tile: its rows, and so their spectrum, are zero
    if (write_grid) {
      for (int e = tid; e < R * n; e += nt) write_grid[row0 + e] = 0.0;
    } else {
      C zero;
      zero.x = 0;
      zero.y = 0;
      for (int e = tid; e < (half + 1) * R; e += nt) {
        const int k = e >> (lgnp + 1), a = e & (R - 1);
        spec[(size_t)k * slab + pos0 + a] = zero;
      }
    }
    return;
  }

  // the twiddles load now and land in shared memory after the spread, so
  // their L2 round trip overlaps the zero fill and the spread's own loads
  const int ntw = fft_tw_count(n, plan_variant_of<T>(g));
  TableStage<T, kTabBatch> ts;
  if (!write_grid) ts.load(tw, ntw, nullptr, 0, 0);
  for (int e = tid; e < R * n; e += nt) {
    const int r = e >> lg, x = e & mask;
    S v = 0;
    if (src.f_grid) v = (S)(src.coef_grid * src.f_grid[row0 + (size_t)r * n + x]);
    rows[((r >> 1) * PS + padi(x)) * 2 + (r & 1)] = v;
  }
  __syncthreads();

  const size_t sbytes = (size_t)npen * PS * sizeof(C);  // bufB, unused until the FFT
  if (lo < hi) {
    if constexpr (SpreadGathers<T>::value)
      spread_gather<S, D>(g, p, b, src, rows, reinterpret_cast<unsigned char*>(bufB), sbytes, z,
                          y0, lo, hi);
    else
      spread_scatter<S, D>(g, p, b, src, rows, reinterpret_cast<unsigned char*>(bufB), sbytes,
                           z, y0, lo, hi);
  }

  if (write_grid) {
    for (int e = tid; e < R * n; e += nt) {
      const int r = e >> lg, x = e & mask;
      write_grid[row0 + (size_t)r * n + x] = (double)rows[((r >> 1) * PS + padi(x)) * 2 + (r & 1)];
    }
    __syncthreads();
    return;
  }
  ts.store(tws, ntw, nullptr, 0, 0);
  ts.rest(tw, tws, ntw, nullptr, nullptr, 0);
  __syncthreads();

  C* res = fft_run<T, false>(bufA, bufB, plan_code_of<T>(g), npen, tws);

  for (int e = tid; e < (half + 1) * npen; e += nt) {
    const int k = e >> lgnp, a = e & (npen - 1);
    const C zk = res[a * PS + padi(k)];
    const C zm = res[a * PS + padi((n - k) & mask)];
    C A, B;
    A.x = (T)0.5 * (zk.x + zm.x);
    A.y = (T)0.5 * (zk.y - zm.y);
    B.x = (T)0.5 * (zk.y + zm.y);
    B.y = (T)-0.5 * (zk.x - zm.x);
    Pair<T> pr;
    pr.a = A;
    pr.b = B;
    pr.store(spec + (size_t)k * slab + pos0 + 2 * a);
  }
  __syncthreads();  // the block's shared buffers are reused by the next item
}

// ---- pencil passes on the transposed half spectrum -----------------------
struct PencilLayout {
  int64_t gstride, bstride, estride;
  int pg;        // pencils per group (a power of two)
  int npencils;  // total pencils
  int c;         // pencils per block (a power of two)
  int lgc, lgpg;
};

// c: pencils per work item (a power of two <= 16): at most pg when the
// pencils are strided, shared memory (pencil buffers + tables) within 100 KB
// so that two blocks of the persistent solver fit on an SM (with its ~7 KB
// of static shared memory), and -- by the fixed rule -- small enough that a
// pass over contiguous pencils has >= 256 items when it can.  want > 0 (the
// autotuner's choice) replaces the rule when it is admissible.
template <typename T>
__host__ __device__ inline size_t pencil_smem_for(int n, int c) {
  const int ntw = fft_tw_capacity<T>(n);
  if (ntw < 0) return ~(size_t)0;
  return (2 * (size_t)c * pen_stride(n) + (size_t)ntw) * sizeof(cx_t<T>) +
         (size_t)n * sizeof(T);
}

template <typename T>
__host__ __device__ inline bool pencils_admissible(int n, int64_t estride, int pg, int c) {
  if (c < 1 || c > 16 || (c & (c - 1))) return false;
  if (estride != 1 && (c < 2 || c > pg)) return false;
  return pencil_smem_for<T>(n, c) <= 100 * 1024;
}

template <typename T>
__host__ __device__ inline PencilLayout pencil_layout(int n, int64_t gstride, int64_t bstride,
                                                      int64_t estride, int pg, int npencils,
                                                      int want = 0) {
  PencilLayout L;
  L.gstride = gstride;
  L.bstride = bstride;
  L.estride = estride;
  L.pg = pg;
  L.npencils = npencils;
  int c = 16;
  if (estride != 1 && c > pg) c = pg;
  while (c > 1 && pencil_smem_for<T>(n, c) > 100 * 1024) c >>= 1;
  while (c > 1 && npencils / c < 256 && estride == 1) c >>= 1;
  if (estride != 1 && c < 2) c = 2;  // strided items move pencils in pairs
  if (want > 0 && pencils_admissible<T>(n, estride, pg, want)) c = want;
  L.c = c;
  L.lgc = 0;
  while ((1 << L.lgc) < c) ++L.lgc;
  L.lgpg = 0;
  while ((1 << L.lgpg) < pg) ++L.lgpg;
  return L;
}

// The pencil passes of one Helmholtz solve: 2D has one (kx slabs, y pencils,
// forward + multiply + inverse); 3D has three: y forward on (kx, z),
// z forward + multiply + inverse on (kx, y), y inverse on (kx, z).
template <typename T>
__host__ __device__ inline PencilLayout solve_layout(int dim, int n, int which, int want = 0) {
  const int half = n / 2;
  if (dim == 2) return pencil_layout<T>(n, n, 0, 1, 1, half + 1, want);
  const int64_t n2 = (int64_t)n * n;
  if (which == 1) return pencil_layout<T>(n, n2, 1, n, n, (half + 1) * n, want);
  return pencil_layout<T>(n, n2, n, 1, n, (half + 1) * n, want);
}

// The layout of a geometry's pencil pass `which` (1: the solve pass) in
// element type T, with the autotuner's pencils per item.
template <typename T>
__host__ __device__ inline PencilLayout solve_layout(const GridDesc& g, int which) {
  const int cls = sizeof(T) == 4 ? 0 : 1;
  return solve_layout<T>(g.dim, g.n, which, g.pcap[cls][g.dim == 2 ? 1 : which]);
}

// Element type code of the solver's per-type choices: 0 float64, 1 float32,
// 2 double-float.
template <typename T> struct ElemCode;
template <> struct ElemCode<double> { static constexpr int value = 0; };
template <> struct ElemCode<float> { static constexpr int value = 1; };
template <> struct ElemCode<dd> { static constexpr int value = 2; };

// The persistent solver's layout of pencil pass `which`: the solve pass
// takes the geometry's solver choice (g.scap), the 3D y passes the rule.
template <typename T>
__host__ __device__ inline PencilLayout solver_layout(const GridDesc& g, int which) {
  return solve_layout<T>(g.dim, g.n, which, which == 1 ? g.scap[ElemCode<T>::value] : 0);
}

// pencil buffers, twiddles, sin^2 table
template <typename T>
__host__ __device__ inline size_t pencil_smem_bytes(const PencilLayout& L, int n) {
  return pencil_smem_for<T>(n, L.c);
}

// Threads per block of the launch-based pencil passes: one per butterfly of
// the FFT pass with the most butterflies (n over the smallest radix of the
// plan, per pencil) -- more would idle in the FFT passes and thin the
// per-thread work over which an item's fixed cost is spread.  Row tiles take
// n/8 per pencil: their spread stage wants the extra threads.
inline int clamp_threads(int t) { return t < 64 ? 64 : (t > 512 ? 512 : t); }
inline int pencil_threads(int n, int c) {
  const int lg = ilog2(n);
  int min_lr = 4;
  for (int s = 0; s < plan_npass(lg); ++s)
    if (plan_lr(lg, s) < min_lr) min_lr = plan_lr(lg, s);
  return clamp_threads(c * (n >> min_lr));
}


// MODE 0: forward, 1: inverse, 2: forward, multiply by
// scale0 / (c0 + cfac * sum_c sin^2(pi k_c / n)) (c0 = 1; c0 = 0 and the
// k = 0 mode zeroed in the Poisson limit), inverse.
//
// An item's pencils are either contiguous (pencil p at data + p n: the 2D
// kx slabs and the 3D y pencils) or strided (3D z pencils: the item's c
// pencils are c consecutive y of one kx slab, element t at t n + pl), so one
// base pointer per item addresses everything.  Float and double items read
// and write the pencils in their first and last radix passes; double-float
// items (and the strided forward or inverse-only transforms) stage them
// through shared memory, elements moving in pairs.
template <typename T, int MODE>
__device__ __forceinline__ void phase_pencils(const GridDesc& g, const PencilLayout& L,
                                              cx_t<T>* data, const cx_t<T>* __restrict__ tw,
                                              const T* __restrict__ s2, T cfac, T scale0,
                                              int blk, unsigned char* smem,
                                              const int* zskip = nullptr, int ngroups = 0,
                                              const unsigned char* zempty = nullptr) {
  using C = cx_t<T>;
  const int n = g.n, lg = g.log2n, c = L.c, lgc = L.lgc, PS = pen_stride(n);
  const int ntw = fft_tw_count(n, plan_variant_of<T>(g));
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)c * PS;
  C* tws = bufB + (size_t)c * PS;
  T* s2s = reinterpret_cast<T*>(tws + ntw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p0 = blk * c;
  const int npl = min(c, L.npencils - p0);
  const bool tfast = (L.estride == 1);
  const int gi0 = p0 >> L.lgpg, q0 = p0 & (L.pg - 1);
  C* base = tfast ? data + (size_t)p0 * n : data + (size_t)gi0 * L.gstride + q0;
  const int npairs = (npl << lg) >> 1;
  // 3D y passes (pencils (kx, z), items of consecutive z): zskip = the tile
  // starts of the bins; an item whose planes hold no point is skipped -- a
  // forward pass would map zeros to zeros, and an inverse pass feeds only
  // the interpolation, which reads planes that hold points
  if (zskip && zskip[(q0 + npl) * ngroups] == zskip[q0 * ngroups]) return;

  if constexpr (DirectPencils<T>::value) {
    if (MODE == 2 || tfast) {
      // the transforms read and write global memory in their first and
      // last passes (the strided forward and inverse-only transforms of
      // the spectral discretisation stage their pencils below)
      {
        TableStage<T, kTabBatch> ts;
        const int ns = MODE == 2 ? n : 0;
        ts.load(tw, ntw, s2, ns, 0);
        ts.store(tws, ntw, s2s, ns, 0);
        ts.rest(tw, tws, ntw, s2, s2s, ns);
      }
      __syncthreads();
      // 2D: pencil kx = p0 + pl, position ky = t; 3D: kx = gi0, ky = q0 + pl, kz = t
      SymbolEpi<T> epi{};
      if (MODE == 2) {
        epi.s2s = s2s;
        epi.pre = g.dim == 3 ? s2s[gi0] : (T)0;
        epi.c0 = g.poisson ? (T)0 : (T)1;
        epi.cfac = cfac;
        epi.scale0 = scale0;
        epi.pbase = g.dim == 3 ? q0 : p0;
        epi.npl = npl;
      }
      GlobalPencils<T> gio{};
      gio.p = base;
      gio.npl = npl;
      gio.lgc = lgc;
      gio.zempty = zempty;
      if (tfast)
        fft_global<T, MODE, false>(bufA, bufB, plan_code_of<T>(g), c, tws, epi, gio);
      else if constexpr (MODE == 2)
        fft_global<T, MODE, true>(bufA, bufB, plan_code_of<T>(g), c, tws, epi, gio);
      return;  // the last pass ends with a block barrier
    }
  }

  // pair k: contiguous -> elements 2k, 2k+1 of the item (one pencil, t even);
  // strided -> pencils pl, pl+1 (pl even) at position t.  npl is even or 1
  // in the strided case (c | pg, pg a power of two), so pairs never straddle.
  // The first batch of pairs and the tables are loaded together (one L2
  // round trip), then stored.
  constexpr int U = 4;
  TableStage<T, kTabBatch> ts;
  const int ns = MODE == 2 ? n : 0;
  ts.load(tw, ntw, s2, ns, 0);
  for (int k0 = tid; k0 < npairs; k0 += U * nt) {
    Pair<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * nt;
      if (k < npairs) {
        if (tfast) {
          v[u].load(base + 2 * k);
        } else {
          // z pass: planes without points hold zeros (not written by the x pass)
          const int e = 2 * k, t = e >> lgc, pl = e & (c - 1);
          if (zempty && zempty[t]) {
            v[u].a.x = v[u].a.y = v[u].b.x = v[u].b.y = 0;
          } else {
            v[u].load(base + (size_t)t * n + pl);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * nt;
      if (k < npairs) {
        const int e = 2 * k;
        if (tfast) {
          const int pl = e >> lg, t = e & (n - 1);
          C* d = bufA + pl * PS + padi(t);  // padi(t + 1) = padi(t) + 1, t even
          d[0] = v[u].a;
          d[1] = v[u].b;
        } else {
          const int t = e >> lgc, pl = e & (c - 1);
          bufA[pl * PS + padi(t)] = v[u].a;
          bufA[(pl + 1) * PS + padi(t)] = v[u].b;
        }
      }
    }
  }
  ts.store(tws, ntw, s2s, ns, 0);
  ts.rest(tw, tws, ntw, s2, s2s, ns);
  __syncthreads();

  C* res = fft_run<T, MODE == 1>(bufA, bufB, plan_code_of<T>(g), c, tws);
  if (MODE == 2) {
    // double-float: the symbol multiply as a sweep of its own
    const T c0 = g.poisson ? (T)0 : (T)1;
    const T sfix = g.dim == 3 ? s2s[gi0] : (T)0;
    for (int e = tid; e < (npl << lg); e += nt) {
      const int pl = e >> lg, t = e & (n - 1);
      const T ssum = g.dim == 3 ? sfix + s2s[q0 + pl] + s2s[t] : s2s[p0 + pl] + s2s[t];
      const T den = c0 + cfac * ssum;
      const T f = den > (T)0 ? scale0 * recip_symbol<T>(den) : (T)0;
      C& v = res[pl * PS + padi(t)];
      v.x *= f;
      v.y *= f;
    }
    __syncthreads();
    C* other = (res == bufA) ? bufB : bufA;
    res = fft_run<T, true>(res, other, plan_code_of<T>(g), c, tws);
  }

  for (int k = tid; k < npairs; k += nt) {
    const int e = 2 * k;
    Pair<T> v;
    if (tfast) {
      const int pl = e >> lg, t = e & (n - 1);
      const C* sp = res + pl * PS + padi(t);
      v.a = sp[0];
      v.b = sp[1];
      v.store(base + 2 * k);
    } else {
      const int t = e >> lgc, pl = e & (c - 1);
      if (zempty && zempty[t]) continue;  // never read by the y inverse pass
      v.a = res[pl * PS + padi(t)];
      v.b = res[(pl + 1) * PS + padi(t)];
      v.store(base + (size_t)t * n + pl);
    }
  }
  __syncthreads();
}

// ---- inverse x pass: complex-to-real ----------------------------------------
// Rebuild the full spectrum of the packed pair a + i b from the half spectra
// A, B (Hermitian): Z_k = A_k + i B_k, Z_{n-k} = conj A_k + i conj B_k.
template <typename T, int D, typename OutT>
__device__ __forceinline__ void phase_rows_inv(const GridDesc& g, const Bins& b, const cx_t<T>* spec,
                               const cx_t<T>* __restrict__ tw, OutT* out, int tile,
                               unsigned char* smem, bool band_only = false) {
  // band_only: the grid feeds only the interpolation, whose stencil rows lie
  // in tiles that hold the point in their bin; other tiles are not produced
  if (band_only && b.start[tile] == b.start[tile + 1]) return;
  using C = cx_t<T>;
  const int n = g.n, lg = g.log2n, R = b.rows, npen = R >> 1;
  const int lgnp = __ffs(npen) - 1;  // R is a power of two (checked when the tiles are built)
  const int PS = pen_stride(n);
  C* bufA = reinterpret_cast<C*>(smem);
  C* bufB = bufA + (size_t)npen * PS;
  C* tws = bufB + (size_t)npen * PS;
  const int ngroups = n / R;
  const int z = (D == 3) ? tile / ngroups : 0;
  const int y0 = (tile % ngroups) * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = n >> 1;
  const size_t slab = (D == 3) ? (size_t)n * n : (size_t)n;
  const size_t pos0 = (size_t)z * n + y0;

  constexpr int U = sizeof(T) == 4 ? 4 : 2;
  const int total = (half + 1) * npen;
  // the twiddles load together with the first batch of the spectrum
  const int ntw = fft_tw_count(n, plan_variant_of<T>(g));
  TableStage<T, kTabBatch> ts;
  ts.load(tw, ntw, nullptr, 0, 0);
  for (int e0 = tid; e0 < total; e0 += U * nt) {
    C A[U], B[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      if (e < total) {
        const int k = e >> lgnp, a = e & (npen - 1);
        Pair<T> pr;
        pr.load(spec + (size_t)k * slab + pos0 + 2 * a);
        A[u] = pr.a;
        B[u] = pr.b;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      if (e < total) {
        const int k = e >> lgnp, a = e & (npen - 1);
        C Au = A[u], Bu = B[u];
        if (k == 0 || k == half) {
          Au.y = 0;
          Bu.y = 0;
        }
        C zk, zm;
        zk.x = Au.x - Bu.y;
        zk.y = Au.y + Bu.x;
        bufA[a * PS + padi(k)] = zk;
        if (k > 0 && k < half) {
          zm.x = Au.x + Bu.y;
          zm.y = Bu.x - Au.y;
          bufA[a * PS + padi(n - k)] = zm;
        }
      }
    }
  }
  ts.store(tws, ntw, nullptr, 0, 0);
  ts.rest(tw, tws, ntw, nullptr, nullptr, 0);
  __syncthreads();
  const size_t row0 = ((size_t)z * n + y0) * n;
  if constexpr (DirectPencils<T>::value) {
    // the last radix pass writes the rows (it ends with a block barrier)
    fft_inverse_rows<T, OutT>(bufA, bufB, plan_code_of<T>(g), npen, tws, out + row0);
    return;
  }
  C* res = fft_run<T, true>(bufA, bufB, plan_code_of<T>(g), npen, tws);
  for (int e = tid; e < R * n; e += nt) {
    const int r = e >> lg, x = e & (n - 1);
    const C v = res[(r >> 1) * PS + padi(x)];
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

// Weight t of axis c of point i in T (W[c][t * m + i]).
template <typename T>
__device__ __forceinline__ T interp_w(const PointData& p, int c, int t, int i, int m) {
  return wtab<T>(p, c)[t * m + i];
}

// Grid load of the interpolation: around L1 (ld.global.cg) where another
// block of the same launch wrote the grid, through the read-only cache when
// an earlier launch did (neighbouring points then share cached lines).
template <typename T, bool CACHED>
__device__ __forceinline__ T grid_load(const T* p) {
  return CACHED ? __ldg(p) : __ldcg(p);
}

// sum over the 4^d taps of grid * prod_c W[c][t]  (S* u at X_i, Sec. 5.2)
template <typename T, int D, bool CACHED = false>
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
      for (int tx = 0; tx < 4; ++tx) r += grid_load<T, CACHED>(row + col[tx]) * wx[tx];
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
        for (int tx = 0; tx < 4; ++tx) r += grid_load<T, CACHED>(row + col[tx]) * wx[tx];
        pz += r * wy[ty];
      }
      acc += pz * wz;
    }
  }
  return acc;
}

}  // namespace ibdl
