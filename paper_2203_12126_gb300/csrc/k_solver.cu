// Persistent GMRES solver: one cooperative launch runs whole IBDL solves
// (Sec. 5.3: unpreconditioned GMRES on the second-kind boundary system) for
// one or many instances, with no host round trip between iterations.
//
// Each instance runs rounds; in a round it does one action of its state
// machine as a sequence of phases, each a set of independent work items:
//
//   A   rows_fwd   spread-divergence of the matvec input + x FFT   (matvec)
//   B   pencils    y (and z) FFT passes with the symbol            (matvec)
//   C   rows_inv   x inverse FFT to the real grid                  (matvec)
//   D   interp     w = S* grid +- input/2, then the first-pass dot products
//   E   reduce, w1 = w - V h1 (CGS pass 1), second-pass dots h2 and ||w1||^2
//   F   reduce, w2 = w1 - V h2 (CGS pass 2), ||w2|| = sqrt(||w1||^2 - |h2|^2)
//       (Pythagoras: V is orthonormal), normalise; Givens rotation; control
//
// An Arnoldi step is D, E, F; a residual round D, E (E normalises r and runs
// control); FINISH D, E (back substitution, x += V y, control); the Neumann
// right-hand side D alone.  (Small instances in large batches do the vector
// work of a round as one item on one block.)
// Actions: RHS (Neumann right-hand side), RESID_ZERO (r = b at x = 0),
// MV_RESIDUAL (r = b - A64 x), MV_ARNOLDI (Arnoldi step j with the float64
// or float32 operator), FINISH (back substitution, x += V y), DONE.  The
// float64 mode restarts with the true residual after every cycle; the
// float32-refined mode runs one float32 GMRES cycle per refinement step
// between float64 residuals.
//
// Blocks take items of any instance dynamically (see "dynamic scheduling"),
// so instances of different sizes and precisions overlap instead of moving
// in lock step.  Every wait is bounded; on timeout an error flag is raised
// and every block leaves the kernel.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "ibdl_device.cuh"
#include "ibdl_solver.cuh"

namespace ibdl {

constexpr unsigned kSpinLimit = 1u << 27;  // x >= 20 ns sleeps: a few seconds

// Acquire-release fence at GPU scope: orders this thread's earlier memory
// operations (and, after a block barrier, its block's) before its later
// ones for every observer on the GPU.  The scheduler's message passing (data,
// then a counter or claim word; a counter or claim word, then data) needs no
// more than that, and it is cheaper than a sequentially consistent fence.
__device__ __forceinline__ void fence_acq_rel() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Counting barrier among `parties` blocks on ctr[0] (arrivals) and ctr[1]
// (generation).  The spin is bounded (`limit` polls): on timeout it raises
// *err, which every later barrier sees, and all blocks leave the kernel.
__device__ bool counted_barrier(unsigned* ctr, unsigned parties, unsigned* err,
                                unsigned limit = kSpinLimit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = ctr + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(ctr, 1u);
    if (arrived == parties - 1) {
      atomicExch(ctr, 0u);
      __threadfence();
      atomicAdd(ctr + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*vgen == gen) {
        if (++spins > limit) {
          atomicExch(err, 1u);
          break;
        }
        if (*(volatile unsigned*)err) break;
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile unsigned*)err == 0u;
}

// Self-test of the bounded wait: a barrier of two parties that only this
// one block joins, so its wait must give up after `limit` polls and raise
// bar[2].
__global__ void k_barrier_selftest(unsigned* bar, unsigned limit) {
  counted_barrier(bar, 2u, bar + 2, limit);
}

cudaError_t launch_barrier_selftest(unsigned* bar, unsigned limit, cudaStream_t st) {
  k_barrier_selftest<<<1, 32, 0, st>>>(bar, limit);
  return cudaGetLastError();
}

// bar[0..1]: the start-up grid barrier, bar[2]: error flag, bar[3]: count of
// instances done (or paused) in this launch, bar[4 + kSchedWords k ..]:
// instance k's scheduler words.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  return counted_barrier(bar, nblocks, bar + 2);
}

struct RoundView {
  int action, prec, j, kdim;
};

constexpr int kMaxCols = 66;  // restart (<= 64) + 2

struct BlockRed;
__device__ void control(const SolveInst& I, SolveState* S, const RoundView& v, double hn,
                        double beta, double bnorm2, BlockRed& R,
                        const SolveState* pre = nullptr);

// The instance state as the control step reads it: written by other blocks
// in earlier rounds, so read around L1.
__device__ __forceinline__ SolveState load_state(const SolveState* S) {
  SolveState s;
  volatile const SolveState* vs = S;
  s.action = vs->action;
  s.prec = vs->prec;
  s.j = vs->j;
  s.kdim = vs->kdim;
  s.iters = vs->iters;
  s.outer = vs->outer;
  s.status = vs->status;
  s.matvecs = vs->matvecs;
  s.nhist = vs->nhist;
  s.xinit = vs->xinit;
  s.nupd = vs->nupd;
  s.beta = vs->beta;
  s.bnorm = vs->bnorm;
  s.tol_abs = vs->tol_abs;
  s.rel = vs->rel;
  s.rerr = vs->rerr;
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of ncols products per thread: vals(c) for c < ncols -> out[c]
// (thread 0 of the block holds nothing special; results land in shared red).
struct BlockRed {
  double red[kMaxCols][kSolverThreads / 32];
  double h[kMaxCols];
  double col[kMaxCols];  // staged H column / Givens vectors for the control step
  double cs[kMaxCols];
  double sn[kMaxCols];
  int fin;  // k > 0: the control step just chose FINISH with k columns
};

// out[c] = sum over chunks of part[ch * pstride + c0 + c], c < ncols: one
// warp per column, lanes over chunks (one L2 round trip, then shuffles).
__device__ void reduce_parts(const double* part, int nchunk, int pstride, int c0, int ncols,
                             double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < ncols; c += nw) {
    double s = 0;
    for (int ch = lane; ch < nchunk; ch += 32) s += __ldcg(part + (size_t)ch * pstride + c0 + c);
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
  __syncthreads();
}

// Writes, for c < ncols, the block sum of x_i * V_c[i] over this chunk, and
// optionally the sum of x_i^2 as column ncols, to part[chunk][.].
// Basis columns are read kColBatch at a time, all loads of a batch in
// flight together (one L2 round trip per batch, not per column).
constexpr int kColBatch = 8;

__device__ void chunk_dots(const SolveInst& I, double xi, bool valid, int i, int ncols,
                           bool with_norm, double* part, int chunk, BlockRed& R) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < ncols; c0 += kColBatch) {
    double vc[kColBatch];
#pragma unroll
    for (int u = 0; u < kColBatch; ++u)
      vc[u] = (valid && c0 + u < ncols) ? __ldcg(I.V + (size_t)(c0 + u) * I.ld + i) : 0.0;
#pragma unroll
    for (int u = 0; u < kColBatch; ++u) {
      if (c0 + u < ncols) {
        const double sm = warp_sum(xi * vc[u]);
        if (lane == 0) R.red[c0 + u][wid] = sm;
      }
    }
  }
  if (with_norm) {
    const double s = warp_sum(valid ? xi * xi : 0.0);
    if (lane == 0) R.red[ncols][wid] = s;
  }
  __syncthreads();
  const int tot = ncols + (with_norm ? 1 : 0);
  for (int c = threadIdx.x; c < tot; c += blockDim.x) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += R.red[c][w];
    part[(size_t)chunk * I.pstride + c] = s;
  }
  __syncthreads();
}

// w - sum_{c < ncols} h[c] V_c[i]
__device__ __forceinline__ double sub_projection(const SolveInst& I, double w, int i, int ncols,
                                                 const double* h) {
  for (int c0 = 0; c0 < ncols; c0 += kColBatch) {
    double vc[kColBatch];
#pragma unroll
    for (int u = 0; u < kColBatch; ++u)
      vc[u] = c0 + u < ncols ? __ldcg(I.V + (size_t)(c0 + u) * I.ld + i) : 0.0;
#pragma unroll
    for (int u = 0; u < kColBatch; ++u)
      if (c0 + u < ncols) w -= h[c0 + u] * vc[u];
  }
  return w;
}

template <typename T>
__device__ __forceinline__ SpectralWs<T> ws_of(const SolveInst& I);
template <>
__device__ __forceinline__ SpectralWs<double> ws_of<double>(const SolveInst& I) {
  return I.w64;
}
template <>
__device__ __forceinline__ SpectralWs<float> ws_of<float>(const SolveInst& I) {
  return I.w32;
}
template <>
__device__ __forceinline__ SpectralWs<dd> ws_of<dd>(const SolveInst& I) {
  return I.wdd;
}

__device__ __forceinline__ bool is_mv(int a) {
  return a == ACT_MV_ARNOLDI || a == ACT_MV_RESIDUAL || a == ACT_RHS || a == ACT_MV_UPDATE;
}

__device__ __forceinline__ const double* mv_input(const SolveInst& I, const RoundView& v) {
  if (v.action == ACT_RHS) return nullptr;
  if (v.action == ACT_MV_UPDATE) return I.dvec;
  return v.action == ACT_MV_ARNOLDI ? I.V + (size_t)v.j * I.ld : I.x;
}

template <typename T>
__host__ __device__ int mv_items(const SolveInst& I, int phase) {
  const int d = I.g.dim, n = I.g.n;
  if (phase == 0 || phase == 4) return I.b.ntiles;
  PencilLayout L;
  if (d == 2) {
    if (phase != 2) return 0;
    L = solver_layout<T>(I.g, 1);
  } else {
    L = solver_layout<T>(I.g, phase == 2 ? 1 : 0);
  }
  return (L.npencils + L.c - 1) / L.c;
}

// The solver's pencil items follow the fixed rule of pencil_layout, not the
// autotuner's pencils per item: the tuner times launch-based matvecs, where
// more, smaller items help a lone instance, while in the persistent launch
// the instances share the blocks (the C2 pair took 1.55 ms with the tuned
// one-pencil float32 items against 1.41 ms with the rule's two).
//
// Each matvec phase is called through a non-inlined wrapper, so that every
// phase gets its own register allocation inside this one large kernel.  The
// wrappers take the instance by reference to its global-memory descriptor.
template <typename T, int D>
__device__ __noinline__ void solver_rows_fwd(const SolveInst& I, const double* q, bool with_rhs,
                                             int item, unsigned char* smem) {
  SpreadSrc src;
  src.skip_empty_planes = true;  // the grid feeds only the interpolation
  if (q) {
    src.q_div = q;
    src.coef_div = 1.0;
    if (with_rhs) {
      // residual of a solve whose b is not stored: the spread of S V_b
      // joins S~ x (linearity of the Helmholtz solve and of S*)
      src.v_plain = I.vdata;
      src.coef_plain = 1.0;
    }
  } else {
    src.v_plain = I.vdata;  // right-hand side: -S V_b
    src.coef_plain = -1.0;
  }
  const SpectralWs<T> ws = ws_of<T>(I);
  phase_rows_fwd<T, D>(I.g, I.p, I.b, src, ws.spec, ws.tw, nullptr, item, smem);
}

// 2D Arnoldi step, after x-inverse tile `tile` has written its R grid rows:
// the tile's share of w = S* grid + jump v_j (Sec. 5.2, eq. (ibdl 2)), for
// every point of its bin whose 4-row stencil meets the tile, added to
// w = V[j+1] (zeroed by the phase before; a stencil meets at most two
// tiles), the jump term by the tile holding the stencil's first row; and
// the tile's share of the first CGS dot products V_c . w, c <= j, as the
// tile's row of partial sums (linear in the shares).  Replaces phase D of
// the step.  The grid rows were written by this block: read them plainly.
template <typename G>
__device__ void fused_interp_tile(const SolveInst& I, const RoundView& v, const G* grid,
                                  int tile, unsigned char* smem) {
  const GridDesc& g = I.g;
  const PointData& p = I.p;
  const int n = g.n, mask = n - 1, R = I.b.rows, y0 = tile * R, m = p.m;
  const int lo = I.b.start[tile], hi = I.b.start[tile + 1];
  const double jump = I.bc == IBDL_DIRICHLET ? 0.5 : -0.5;
  const int ncols = v.j + 1;
  double* w = I.V + (size_t)(v.j + 1) * I.ld;
  const double* vin = I.V + (size_t)v.j * I.ld;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* red = reinterpret_cast<double*>(smem);  // [ncols][nw], the FFT is done with smem
  for (int c = threadIdx.x; c < ncols * nw; c += blockDim.x) red[c] = 0.0;
  __syncthreads();
  for (int e0 = lo; e0 < hi; e0 += blockDim.x) {
    const int e = e0 + threadIdx.x;
    double contrib = 0.0;
    int i = 0;
    bool any = false;
    if (e < hi) {
      i = __ldg(I.b.pts + e);
      const int bx = p.base[0][i], by = p.base[1][i];
      G acc = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int row = (by + t) & mask;
        if ((unsigned)(row - y0) < (unsigned)R) {
          const G* rp = grid + (size_t)row * n;
          G r = 0;
#pragma unroll
          for (int tx = 0; tx < 4; ++tx) r += rp[(bx + tx) & mask] * interp_w<G>(p, 0, tx, i, m);
          acc += r * interp_w<G>(p, 1, t, i, m);
          any = true;
        }
      }
      contrib = (double)acc;
      if ((unsigned)((by & mask) - y0) < (unsigned)R) {
        contrib += jump * __ldcg(vin + i);
        any = true;
      }
      if (any) atomicAdd(w + i, contrib);
    }
    for (int c0 = 0; c0 < ncols; c0 += kColBatch) {
      double vc[kColBatch];
#pragma unroll
      for (int u = 0; u < kColBatch; ++u)
        vc[u] = (any && c0 + u < ncols) ? __ldcg(I.V + (size_t)(c0 + u) * I.ld + i) : 0.0;
#pragma unroll
      for (int u = 0; u < kColBatch; ++u) {
        if (c0 + u < ncols) {
          const double sm = warp_sum(contrib * vc[u]);
          if (lane == 0) red[(c0 + u) * nw + wid] += sm;
        }
      }
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double sm = 0;
    for (int q = 0; q < nw; ++q) sm += red[c * nw + q];
    I.part[(size_t)tile * I.pstride + c] = sm;
  }
  __syncthreads();
}

// Whether an Arnoldi step of this precision interpolates in its x-inverse
// tiles (I.fuse_interp: 1 float32 steps, 2 all steps).
__device__ __forceinline__ bool fused_step(const SolveInst& I, int action, int prec) {
  return action == ACT_MV_ARNOLDI && (I.fuse_interp == 2 || (I.fuse_interp == 1 && prec == 1));
}

// A float32 Arnoldi step that interpolates in phase D (not in its x-inverse
// tiles) may orthogonalise in one pass: phase D adds ||w||^2 to the dot
// products V_c . w, and phase E takes h = V^T w, ||w - V h||^2 = ||w||^2 -
// |h|^2 (V orthonormal), w <- (w - V h) / ||w - V h||, Givens and control --
// one vector phase fewer per step.  Inner solves stop at a 1e-5 reduction
// within a few steps, where one pass loses little orthogonality (the loss
// grows with ||w|| / ||w - V h||) and the subtraction loses about
// eps64 ||w||^2 / ||w - V h||^2 of the new norm; the benchmark's solves keep
// their iteration counts and errors.  Float64 steps (tolerances to 1e-12,
// longer cycles) keep two passes.
__device__ __forceinline__ bool single_pass(const SolveInst& I, int action, int prec) {
  return I.cgs1 && action == ACT_MV_ARNOLDI && prec == 1 && !fused_step(I, action, prec);
}

template <typename T, int D>
__device__ __noinline__ void solver_rows_inv(const SolveInst& I, const RoundView& v, int item,
                                             unsigned char* smem) {
  const SpectralWs<T> ws = ws_of<T>(I);
  if constexpr (std::is_same<T, dd>::value) {  // double-float writes the float64 grid
    phase_rows_inv<T, D, double>(I.g, I.b, ws.spec, ws.tw, I.w64.grid, item, smem, true);
    if (D == 2 && fused_step(I, v.action, v.prec))
      fused_interp_tile<double>(I, v, I.w64.grid, item, smem);
  } else {
    phase_rows_inv<T, D, T>(I.g, I.b, ws.spec, ws.tw, ws.grid, item, smem, true);
    if (D == 2 && fused_step(I, v.action, v.prec))
      fused_interp_tile<T>(I, v, ws.grid, item, smem);
  }
}

template <typename T, int MODE>
__device__ __noinline__ void solver_pencils(const SolveInst& I, int which, int item,
                                            unsigned char* smem) {
  const SpectralWs<T> ws = ws_of<T>(I);
  const GridDesc& g = I.g;
  const T cfac = (T)symbol_cfac(g);
  const T scale0 = (T)symbol_scale0(g);
  // the matvec's grid feeds only the interpolation and has no grid source:
  // 3D y-pass items of planes without points are skipped (both directions)
  const int* zskip = (g.dim == 3 && MODE != 2) ? I.b.start : nullptr;
  phase_pencils<T, MODE>(g, solver_layout<T>(g, which), ws.spec, ws.tw, ws.s2, cfac,
                         scale0, item, smem, zskip, g.n / I.b.rows,
                         (g.dim == 3 && MODE == 2) ? I.b.zempty : nullptr);
}

// phase: 0 rows_fwd, 1 y forward (3D), 2 solve pass, 3 y inverse (3D), 4 rows_inv
template <typename T>
__device__ void mv_item(const SolveInst& I, const RoundView& v, int phase, int item,
                        unsigned char* smem) {
  const int d = I.g.dim;
  if (phase == 0) {
    const bool with_rhs = v.action == ACT_MV_RESIDUAL && I.rhs_resid;
    if (d == 2)
      solver_rows_fwd<T, 2>(I, mv_input(I, v), with_rhs, item, smem);
    else
      solver_rows_fwd<T, 3>(I, mv_input(I, v), with_rhs, item, smem);
  } else if (phase == 4) {
    if (d == 2)
      solver_rows_inv<T, 2>(I, v, item, smem);
    else
      solver_rows_inv<T, 3>(I, v, item, smem);
  } else if (d == 2 || phase == 2) {
    solver_pencils<T, 2>(I, 1, item, smem);
  } else if (phase == 1) {
    solver_pencils<T, 0>(I, 0, item, smem);
  } else {
    solver_pencils<T, 1>(I, 0, item, smem);
  }
}


// ---- vector phases ------------------------------------------------------------

// Back substitution R y = g (R: the rotated Hessenberg's k x k upper
// triangle, column l at H + l ldh), by the whole block; y goes to I.ysol,
// which the next phase reads (released with the item's done count).  The
// block stages R and g in shared memory in one round of loads (up to
// kMaxCols (kSolverThreads / 32) entries; larger k read them as they go),
// then one thread solves.
__device__ void back_substitute(const SolveInst& I, int k, BlockRed& R) {
  const int ldh = I.restart + 1;
  const bool staged = k * (k + 1) / 2 <= kMaxCols * (kSolverThreads / 32);
  double* tri = &R.red[0][0];  // entry (r, l), r <= l, at l (l + 1) / 2 + r
  if (staged) {
    for (int e = threadIdx.x; e < k * (k + 1) / 2; e += blockDim.x) {
      int l = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while (l * (l + 1) / 2 > e) --l;
      while ((l + 1) * (l + 2) / 2 <= e) ++l;
      const int r = e - l * (l + 1) / 2;
      tri[e] = __ldcg(I.H + (size_t)l * ldh + r);
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) R.h[r] = __ldcg(I.gv + r);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int r = k - 1; r >= 0; --r) {
      double sacc = staged ? R.h[r] : __ldcg(I.gv + r);
      for (int l = r + 1; l < k; ++l)
        sacc -= (staged ? tri[l * (l + 1) / 2 + r] : __ldcg(I.H + (size_t)l * ldh + r)) *
                R.col[l];
      const double dgn = staged ? tri[r * (r + 1) / 2 + r] : __ldcg(I.H + (size_t)r * ldh + r);
      R.col[r] = dgn != 0.0 ? sacc / dgn : 0.0;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) I.ysol[r] = R.col[r];
}

template <int D>
__device__ void phase_D(const SolveInst& I, SolveState* S, const RoundView& v, int chunk,
                        BlockRed& R) {
  const int i = chunk * blockDim.x + threadIdx.x;
  const bool valid = i < I.p.m;
  double* part1 = I.part;
  if (v.action == ACT_FINISH) {
    // (the control step that chose FINISH solved for y already, phase_F;
    // a round that starts here solves now)
    if (chunk == 0) back_substitute(I, v.kdim, R);
    return;
  }
  if (v.action == ACT_RHS) {
    // b = S* grid, grid = -kappa L'^{-1} S V_b (the Neumann right-hand side;
    // in float32 when the residuals carry the S V_b term); the round ends
    // here, so chunk 0 also picks the next action
    if (valid)
      I.bvec[i] = v.prec ? (double)interp_point<float, D>(I.g, I.p, I.w32.grid, i)
                         : interp_point<double, D>(I.g, I.p, I.w64.grid, i);
    if (chunk == 0 && threadIdx.x == 0) control(I, S, v, 0, 0, 0, R);
    if (!I.rhs_r0) return;
    // the solve starts from x = 0 (RESID_ZERO next): this phase also does
    // that round's phase D, r = b and its partial sums (below), so the round
    // starts at phase E
  }
  const double jump = I.bc == IBDL_DIRICHLET ? 0.5 : -0.5;
  if (v.action == ACT_MV_ARNOLDI) {
    double w = 0;
    if (valid) {
      const double* vin = I.V + (size_t)v.j * I.ld;
      const double acc = v.prec ? (double)interp_point<float, D>(I.g, I.p, I.w32.grid, i)
                                : interp_point<double, D>(I.g, I.p, I.w64.grid, i);
      w = acc + jump * __ldcg(vin + i);
      I.V[(size_t)(v.j + 1) * I.ld + i] = w;
    }
    chunk_dots(I, w, valid, i, v.j + 1, single_pass(I, v.action, v.prec), part1, chunk, R);
    return;
  }
  // residual actions: r = b - A x (or r = b), partial ||r||^2 and ||b||^2
  double r = 0, bi = 0;
  if (valid) {
    bi = __ldcg(I.bvec + i);
    if (v.action == ACT_MV_RESIDUAL) {
      const double t = interp_point<double, D>(I.g, I.p, I.w64.grid, i) + jump * __ldcg(I.x + i);
      r = I.rhs_resid ? -t : bi - t;  // rhs_resid: t = A x - b
    } else if (v.action == ACT_MV_UPDATE) {
      // r <- r - A32 d: x moved by d since r was formed
      const double t =
          (double)interp_point<float, D>(I.g, I.p, I.w32.grid, i) + jump * __ldcg(I.dvec + i);
      r = __ldcg(I.r + i) - t;
    } else {
      r = bi;
    }
    I.r[i] = r;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double s0 = warp_sum(valid ? r * r : 0.0);
  const double s1 = warp_sum(valid ? bi * bi : 0.0);
  if (lane == 0) {
    R.red[0][wid] = s0;
    R.red[1][wid] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += R.red[threadIdx.x][w];
    part1[(size_t)chunk * I.pstride + threadIdx.x] = s;
  }
  __syncthreads();
}

// First CGS pass of an Arnoldi step: h1 = sum of the partials (section
// `in`), H[:, j] = h1 (chunk 0), w1 = w - V h1; then the dots of w1 with V
// and ||w1||^2 (column j + 1) into `out`, for phase F.
__device__ void cgs_pass(const SolveInst& I, const RoundView& v, int chunk, BlockRed& R,
                         const double* in, double* out) {
  const int ncols = v.j + 1;
  const int ldh = I.restart + 1;
  // the first pass's partial sums: one row per x tile when the x-inverse
  // tiles interpolated (2D), else one per vector chunk (phase D)
  reduce_parts(in, fused_step(I, v.action, v.prec) ? I.b.ntiles : I.nchunk, I.pstride, 0, ncols,
               R.h);
  if (chunk == 0) {
    double* Hcol = I.H + (size_t)v.j * ldh;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) Hcol[c] = R.h[c];
  }
  const int i = chunk * blockDim.x + threadIdx.x;
  const bool valid = i < I.p.m;
  double w = 0;
  double* wp = I.V + (size_t)(v.j + 1) * I.ld;
  if (valid) {
    w = sub_projection(I, __ldcg(wp + i), i, ncols, R.h);
    wp[i] = w;
  }
  __syncthreads();
  chunk_dots(I, w, valid, i, ncols, true, out, chunk, R);
}

__device__ void phase_F(const SolveInst& I, SolveState* S, const RoundView& v, int chunk,
                        BlockRed& R, bool single = false);

__device__ void phase_E(const SolveInst& I, SolveState* S, const RoundView& v, int chunk,
                        BlockRed& R) {
  double* part1 = I.part;
  double* part2 = I.part + (size_t)I.nsec * I.pstride;
  if (v.action == ACT_MV_ARNOLDI) {
    if (single_pass(I, v.action, v.prec))
      phase_F(I, S, v, chunk, R, true);  // the one pass: F's work on D's sums
    else
      cgs_pass(I, v, chunk, R, part1, part2);
    return;
  }
  // item nchunk runs the round's control step beside the vector work of
  // items 0 .. nchunk - 1 (it reads the same reduced sums and nothing they
  // write), so the step's serial float64 work is off the phase's longest item
  if (chunk == I.nchunk) {
    SolveState st;
    if (threadIdx.x == 0) st = load_state(S);
    if (v.action == ACT_FINISH) {
      if (threadIdx.x == 0) {
        // ||d|| = ||V y|| = ||y|| (V orthonormal): the update residual's bound
        double yy = 0;
        if (I.upd_resid)
          for (int c = 0; c < v.kdim; ++c) {
            const double yc = __ldcg(I.ysol + c);
            yy += yc * yc;
          }
        control(I, S, v, 0, sqrt(yy), 0, R, &st);
      }
    } else {
      reduce_parts(part1, I.nchunk, I.pstride, 0, 2, R.h);
      if (threadIdx.x == 0) control(I, S, v, 0, sqrt(R.h[0]), R.h[1], R, &st);
    }
    __syncthreads();
    return;
  }
  const int i = chunk * blockDim.x + threadIdx.x;
  const bool valid = i < I.p.m;
  if (v.action == ACT_FINISH) {
    // x += V y: stage -y in shared memory, then one batched pass over V
    for (int c = threadIdx.x; c < v.kdim; c += blockDim.x) R.h[c] = -__ldcg(I.ysol + c);
    __syncthreads();
    if (valid) {
      if (I.upd_resid) {
        // the correction d = V y (R.h holds -y) is kept for an update of
        // the residual
        const double d = sub_projection(I, 0.0, i, v.kdim, R.h);
        I.dvec[i] = d;
        I.x[i] = __ldcg(I.x + i) + d;
      } else {
        I.x[i] = sub_projection(I, __ldcg(I.x + i), i, v.kdim, R.h);
      }
    }
    __syncthreads();
    return;
  }
  // residual actions: V0 = r / ||r|| (and V1 cleared for the x-inverse
  // tiles' interpolation of the first Arnoldi step)
  const double ri = valid ? __ldcg(I.r + i) : 0.0;
  reduce_parts(part1, I.nchunk, I.pstride, 0, 2, R.h);
  const double beta = sqrt(R.h[0]);
  const double inv = (beta > 0 && isfinite(beta)) ? 1.0 / beta : 0.0;
  if (valid) {
    I.V[i] = ri * inv;
    if (I.fuse_interp && I.restart >= 1) I.V[(size_t)I.ld + i] = 0.0;
  }
  __syncthreads();
}

// Control of one instance (one thread).  hn: new subdiagonal, beta: residual
// norm of a residual action, bnorm2: ||b||^2 partial sum; pre: the state,
// when the caller loaded it ahead (it cannot change during the phase).  Its
// writes reach the other blocks through the block's release of its done
// count at the end of the item.
__device__ void control(const SolveInst& I, SolveState* S, const RoundView& v, double hn,
                        double beta, double bnorm2, BlockRed& R, const SolveState* pre) {
  const int ldh = I.restart + 1;
  SolveState s;
  if (pre) {
    s = *pre;
  } else {
    // written by other blocks in earlier rounds: read around L1
    volatile const SolveState* vs = S;
    s.action = vs->action;
    s.prec = vs->prec;
    s.j = vs->j;
    s.kdim = vs->kdim;
    s.iters = vs->iters;
    s.outer = vs->outer;
    s.status = vs->status;
    s.matvecs = vs->matvecs;
    s.nhist = vs->nhist;
    s.xinit = vs->xinit;
    s.nupd = vs->nupd;
    s.beta = vs->beta;
    s.bnorm = vs->bnorm;
    s.tol_abs = vs->tol_abs;
    s.rel = vs->rel;
    s.rerr = vs->rerr;
  }
  if (v.action == ACT_MV_ARNOLDI) {
    const int j = v.j;
    double* col = I.H + (size_t)j * ldh;
    double* cj = R.col;  // staged by the block: H[0..j, j], cs, sn, gv[j]
    cj[j + 1] = hn;
    for (int r = 0; r < j; ++r) {
      const double cr = R.cs[r], sr = R.sn[r];
      const double t = cr * cj[r] + sr * cj[r + 1];
      cj[r + 1] = -sr * cj[r] + cr * cj[r + 1];
      cj[r] = t;
    }
    // the rotation zeroing b against a; the Hessenberg entries of this
    // second-kind operator are O(1), far from where the plain
    // sqrt(a^2 + b^2) could overflow, and one reciprocal serves both ratios
    // (float64 is slow on this part, and this sits on every step's path)
    const double a = cj[j], b = cj[j + 1];
    const double den = sqrt(fma(a, a, b * b));
    double c = 1.0, sn = 0.0;
    if (den > 0) {
      const double inv = 1.0 / den;
      c = a * inv;
      sn = b * inv;
    }
    cj[j] = den;
    cj[j + 1] = 0.0;
    for (int r = 0; r <= j + 1; ++r) col[r] = cj[r];
    I.cs[j] = c;
    I.sn[j] = sn;
    const double gj = R.h[0];
    I.gv[j + 1] = -sn * gj;
    I.gv[j] = c * gj;
    const double est = fabs(sn * gj);
    s.iters++;
    s.matvecs++;
    if (s.nhist < I.hist_cap) I.hist[s.nhist++] = est / s.bnorm;
    if (!isfinite(est) || !isfinite(hn)) {
      s.status = IBDL_ERR_NONFINITE;
      s.action = ACT_DONE;
    } else if (est <= s.tol_abs || hn == 0.0 || j + 1 == I.restart || s.iters >= I.maxit) {
      s.kdim = j + 1;
      s.action = ACT_FINISH;
    } else {
      s.j = j + 1;
    }
  } else if (v.action == ACT_FINISH) {
    // beta carries ||d||, the norm of this inner solve's correction.  A small
    // correction updates the residual with a float32 matvec, r -= A32 d,
    // whose error is at most kF32OpErr ||d|| (x_new = x + d, so
    // b - A x_new = r - A d); the errors of the updates since the last
    // float64-grade residual may add up to a tenth of the tolerance
    const double bound = kF32OpErr * beta;
    if (I.upd_resid && s.bnorm > 0 && s.rerr + bound <= 0.1 * I.tol * s.bnorm) {
      s.rerr += bound;
      s.nupd++;
      s.action = ACT_MV_UPDATE;
      s.prec = 1;
    } else {
      s.action = ACT_MV_RESIDUAL;
      s.prec = 0;
    }
  } else if (v.action == ACT_RHS) {
    s.action = s.xinit ? ACT_MV_RESIDUAL : ACT_RESID_ZERO;
    s.prec = 0;
  } else {
    if (v.action == ACT_MV_RESIDUAL || v.action == ACT_MV_UPDATE) s.matvecs++;
    // the stored residual's error bound (the update added its own share
    // when it was chosen); r = b32 is no float64-grade residual at all
    if (v.action == ACT_MV_RESIDUAL) s.rerr = 0.0;
    if (v.action == ACT_RESID_ZERO) s.rerr = I.rhs_resid ? __longlong_as_double(0x7ff0000000000000LL) : 0.0;
    if (s.bnorm < 0) s.bnorm = sqrt(bnorm2);
    s.beta = beta;
    s.rel = s.bnorm > 0 ? beta / s.bnorm : 0.0;
    if (s.bnorm == 0.0) {
      s.status = IBDL_OK;
      s.action = ACT_DONE;
    } else if (!isfinite(beta)) {
      s.status = IBDL_ERR_NONFINITE;
      s.action = ACT_DONE;
    } else if ((beta + s.rerr) / s.bnorm <= I.tol) {
      s.status = IBDL_OK;
      s.action = ACT_DONE;
    } else if (s.iters >= I.maxit || (I.refined && s.outer >= I.max_refine)) {
      s.status = IBDL_ERR_NOT_CONVERGED;
      s.action = ACT_DONE;
    } else {
      I.gv[0] = beta;
      for (int k = 1; k <= I.restart; ++k) I.gv[k] = 0.0;
      s.j = 0;
      s.action = ACT_MV_ARNOLDI;
      if (I.refined) {
        s.prec = 1;
        s.outer++;
        s.tol_abs = fmax(I.inner_tol * beta, 0.5 * I.tol * s.bnorm);
      } else {
        s.prec = 0;
        s.tol_abs = I.tol * s.bnorm;
      }
    }
  }
  *S = s;
}

// Second CGS pass of an Arnoldi step, normalisation and control: h2 and
// ||w1||^2 come from phase E's partials; ||w2||^2 = ||w1||^2 - |h2|^2 since
// w2 = w1 - V h2 with V orthonormal and h2 = V^T w1 (the second pass's
// correction is small, so the difference does not cancel).
// single: a one-pass step (single_pass), run as phase E on phase D's sums
// (h1 and ||w||^2; the Hessenberg column is h1 alone)
__device__ void phase_F(const SolveInst& I, SolveState* S, const RoundView& v, int chunk,
                        BlockRed& R, bool single) {
  const int j = v.j, ncols = j + 1, ldh = I.restart + 1;
  double* part2 = single ? I.part : I.part + (size_t)I.nsec * I.pstride;
  // item nchunk runs the control step beside the normalisation of items
  // 0 .. nchunk - 1; its inputs (the state, the Hessenberg column's first
  // pass, the earlier rotations, g_j) go out beside the partial sums' loads
  const bool ctl_item = chunk == I.nchunk;
  double hcol = 0, csr = 0, snr = 0, gj = 0;
  SolveState st;
  if (ctl_item) {
    const int r = threadIdx.x;
    if (r <= j && !single) hcol = __ldcg(I.H + (size_t)j * ldh + r);
    if (r < j) {
      csr = __ldcg(I.cs + r);
      snr = __ldcg(I.sn + r);
    }
    if (r == 0) {
      gj = __ldcg(I.gv + j);
      st = load_state(S);
    }
  }
  reduce_parts(part2, I.nchunk, I.pstride, 0, ncols + 1, R.h);
  double ss = 0;
  for (int c = 0; c < ncols; ++c) ss += R.h[c] * R.h[c];
  const double d2 = R.h[ncols] - ss;
  const double hn = sqrt(d2 > 0.0 ? d2 : 0.0);
  if (ctl_item) {
    // stage the Hessenberg column (h1 from phase E plus h2), the earlier
    // rotations and g_j for the control step (j < restart <= blockDim)
    const int r = threadIdx.x;
    if (r <= j) R.col[r] = hcol + R.h[r];
    if (r < j) {
      R.cs[r] = csr;
      R.sn[r] = snr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      R.h[0] = gj;
      control(I, S, v, hn, 0, 0, R, &st);
      // its own writes (state, H column, g): the FINISH round's back
      // substitution runs here, so that round starts at phase E
      const volatile SolveState* vs = S;
      R.fin = vs->action == ACT_FINISH ? vs->kdim : 0;
    }
    __syncthreads();
    if (R.fin > 0) back_substitute(I, R.fin, R);
    return;
  }
  const double inv = (hn > 0 && isfinite(hn)) ? 1.0 / hn : 0.0;
  const int i = chunk * blockDim.x + threadIdx.x;
  if (i < I.p.m) {
    double* wp = I.V + (size_t)(j + 1) * I.ld;
    const double w = sub_projection(I, __ldcg(wp + i), i, ncols, R.h);
    wp[i] = inv != 0.0 ? w * inv : w;
    // the next step's w, accumulated by its x-inverse tiles
    if (I.fuse_interp && j + 2 <= I.restart) wp[I.ld + i] = 0.0;
  }
  __syncthreads();
}

// ---- single-block vector step (instances with few points) ------------------
// For m <= kSingleMax in batches of >= kSingleMinBatch the whole post-matvec
// work of an action (interpolation, both CGS passes, norm, Givens, control)
// is one work item run by one block with block-level synchronisation.  The
// block that takes it may differ from round to round, so everything another
// round wrote is read around L1 (ld.global.cg).

__device__ double block_sum_all(double v, BlockRed& R) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) R.red[0][wid] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < nw; ++w) s += R.red[0][w];
  __syncthreads();
  return s;
}

template <int D>
__device__ double interp_any(const SolveInst& I, int prec, int i) {
  return prec ? (double)interp_point<float, D>(I.g, I.p, I.w32.grid, i)
              : interp_point<double, D>(I.g, I.p, I.w64.grid, i);
}

constexpr int kSingleK = kSingleMax / kSolverThreads;  // elements per thread

__device__ void vec_single(const SolveInst& I, SolveState* S, const RoundView& v, BlockRed& R) {
  const int m = I.p.m, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const double jump = I.bc == IBDL_DIRICHLET ? 0.5 : -0.5;
  const bool d3 = I.g.dim == 3;
  // element k of this thread: i = tid + k * nt (m <= kSingleK * nt)
  if (v.action == ACT_RHS) {
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      if (i < m) I.bvec[i] = d3 ? interp_any<3>(I, v.prec, i) : interp_any<2>(I, v.prec, i);
    }
    __syncthreads();
    if (tid == 0) control(I, S, v, 0, 0, 0, R);
    __syncthreads();
    return;
  }
  if (v.action == ACT_FINISH) {
    if (tid == 0) {
      const int k = v.kdim, ldh = I.restart + 1;
      for (int r = k - 1; r >= 0; --r) {
        double sacc = __ldcg(I.gv + r);
        for (int l = r + 1; l < k; ++l) sacc -= __ldcg(I.H + (size_t)l * ldh + r) * R.h[l];
        const double dgn = __ldcg(I.H + (size_t)r * ldh + r);
        R.h[r] = dgn != 0.0 ? sacc / dgn : 0.0;
      }
    }
    __syncthreads();
    // x += V y; with upd_resid the correction d = V y is summed on its own
    // and kept for an update of the residual
    const bool upd = I.upd_resid;
    double xk[kSingleK];
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      xk[k] = (i < m && !upd) ? __ldcg(I.x + i) : 0.0;
    }
    for (int c = 0; c < v.kdim; ++c) {
      const double yc = R.h[c];
      const double* vc = I.V + (size_t)c * I.ld;
#pragma unroll
      for (int k = 0; k < kSingleK; ++k) {
        const int i = tid + k * nt;
        if (i < m) xk[k] += yc * __ldcg(vc + i);
      }
    }
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      if (i < m) {
        if (upd) {
          I.dvec[i] = xk[k];
          I.x[i] = __ldcg(I.x + i) + xk[k];
        } else {
          I.x[i] = xk[k];
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      double yy = 0;  // ||d|| = ||y|| (V orthonormal)
      if (upd)
        for (int c = 0; c < v.kdim; ++c) yy += R.h[c] * R.h[c];
      control(I, S, v, 0, sqrt(yy), 0, R);
    }
    __syncthreads();
    return;
  }
  if (v.action == ACT_MV_ARNOLDI) {
    const int j = v.j, ncols = j + 1;
    double* w = I.V + (size_t)(j + 1) * I.ld;
    const double* vin = I.V + (size_t)j * I.ld;
    double wk[kSingleK];
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      wk[k] = 0.0;
      if (i < m) {
        const double acc = d3 ? interp_any<3>(I, v.prec, i) : interp_any<2>(I, v.prec, i);
        wk[k] = acc + jump * __ldcg(vin + i);
      }
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int c = 0; c < ncols; ++c) {
        const double* vc = I.V + (size_t)c * I.ld;
        double sacc = 0;
#pragma unroll
        for (int k = 0; k < kSingleK; ++k) {
          const int i = tid + k * nt;
          if (i < m) sacc += wk[k] * __ldcg(vc + i);
        }
        sacc = warp_sum(sacc);
        if (lane == 0) R.red[c][wid] = sacc;
      }
      __syncthreads();
      if (tid < ncols) {
        double t = 0;
        for (int q = 0; q < nw; ++q) t += R.red[tid][q];
        R.h[tid] = t;
        R.col[tid] = pass == 0 ? t : R.col[tid] + t;
      }
      __syncthreads();
      for (int c = 0; c < ncols; ++c) {
        const double hc = R.h[c];
        const double* vc = I.V + (size_t)c * I.ld;
#pragma unroll
        for (int k = 0; k < kSingleK; ++k) {
          const int i = tid + k * nt;
          if (i < m) wk[k] -= hc * __ldcg(vc + i);
        }
      }
      __syncthreads();
    }
    double nrm = 0;
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) nrm += wk[k] * wk[k];
    const double hn = sqrt(block_sum_all(nrm, R));
    const double inv = (hn > 0 && isfinite(hn)) ? 1.0 / hn : 0.0;
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      if (i < m) w[i] = inv != 0.0 ? wk[k] * inv : wk[k];
    }
    for (int r = tid; r < j; r += nt) {
      R.cs[r] = __ldcg(I.cs + r);
      R.sn[r] = __ldcg(I.sn + r);
    }
    if (tid == 0) R.h[0] = __ldcg(I.gv + j);
    __syncthreads();
    if (tid == 0) control(I, S, v, hn, 0, 0, R);
    __syncthreads();
    return;
  }
  // residual actions: r = b - A x (or b); V0 = r / ||r||; control
  double rk[kSingleK];
  double rr = 0, bb = 0;
#pragma unroll
  for (int k = 0; k < kSingleK; ++k) {
    const int i = tid + k * nt;
    rk[k] = 0.0;
    if (i < m) {
      const double bi = __ldcg(I.bvec + i);
      double r = bi;
      if (v.action == ACT_MV_RESIDUAL) {
        const double acc = d3 ? interp_point<double, 3>(I.g, I.p, I.w64.grid, i)
                              : interp_point<double, 2>(I.g, I.p, I.w64.grid, i);
        const double t = acc + jump * __ldcg(I.x + i);
        r = I.rhs_resid ? -t : bi - t;  // rhs_resid: t = A x - b
      } else if (v.action == ACT_MV_UPDATE) {
        const double t = (d3 ? interp_any<3>(I, 1, i) : interp_any<2>(I, 1, i)) +
                         jump * __ldcg(I.dvec + i);
        r = __ldcg(I.r + i) - t;
      }
      I.r[i] = r;
      rk[k] = r;
      rr += r * r;
      bb += bi * bi;
    }
  }
  rr = block_sum_all(rr, R);
  bb = block_sum_all(bb, R);
  const double beta = sqrt(rr);
  const double inv = (beta > 0 && isfinite(beta)) ? 1.0 / beta : 0.0;
#pragma unroll
  for (int k = 0; k < kSingleK; ++k) {
    const int i = tid + k * nt;
    if (i < m) I.V[i] = rk[k] * inv;
  }
  __syncthreads();
  if (tid == 0) control(I, S, v, 0, beta, bb, R);
  __syncthreads();
}

// ---- the persistent kernel ----------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- dynamic scheduling -------------------------------------------------------
//
// Each instance walks its own phase sequence; no phase of one instance waits
// for another instance.  Per instance (scheduler words in `bar`):
//   claim : 64-bit  (epoch << 32) | next item index, taken with atomicAdd
//   done  : items finished in the current epoch
//   desc  : the current phase, its item count and the round's view of the
//           solver state, written before the epoch is published
// A block looking for work takes an item of any instance whose current phase
// has items left; the block that finishes an instance's last item advances
// that instance to its next phase (or, after the vector phases, to the next
// round from the state its control step wrote).  Items of one phase are
// independent, so no block ever waits for another block's item: an idle
// block only spins (bounded) until new items are published.

struct PhaseDesc {
  int epoch, phase, nitems, round;
  int action, prec, j, kdim;
};

constexpr int kPhaseD = 5, kPhaseE = 6, kPhaseF = 7, kPhaseSingle = 9;

// claim word: bits 63..48 the phase epoch (mod 2^16), 47..32 the phase's
// item count, 31..0 the next item index.  A claim is valid exactly when the
// index it took is below the count it carries, so neither the scan nor the
// claim needs the descriptor; a valid claim then reads the descriptor, which
// was written before the claim word was published and cannot change until
// the claimed item is done.
__device__ __forceinline__ unsigned long long claim_value(int epoch, int nitems) {
  return ((unsigned long long)(epoch & 0xffff) << 48) |
         ((unsigned long long)(nitems & 0xffff) << 32);
}
__device__ __forceinline__ bool claim_open(unsigned long long w) {
  return (unsigned)(w & 0xffffffffu) < (unsigned)((w >> 32) & 0xffffu);
}

__device__ __forceinline__ unsigned long long* claim_word(unsigned* bar, int k) {
  return reinterpret_cast<unsigned long long*>(bar + 4 + kSchedWords * k);
}
__device__ __forceinline__ unsigned* done_word(unsigned* bar, int k) {
  return bar + 4 + kSchedWords * k + 2;
}
__device__ __forceinline__ PhaseDesc* desc_of(unsigned* bar, int k) {
  return reinterpret_cast<PhaseDesc*>(bar + 4 + kSchedWords * k + 4);
}

// Descriptor reads go around L1 in two 16-byte loads.
__device__ PhaseDesc load_desc(const PhaseDesc* p) {
  const int4 a = __ldcg(reinterpret_cast<const int4*>(p));
  const int4 b = __ldcg(reinterpret_cast<const int4*>(p) + 1);
  PhaseDesc d;
  d.epoch = a.x;
  d.phase = a.y;
  d.nitems = a.z;
  d.round = a.w;
  d.action = b.x;
  d.prec = b.y;
  d.j = b.z;
  d.kdim = b.w;
  return d;
}

__device__ void store_desc(PhaseDesc* p, const PhaseDesc& d) {
  int4* q = reinterpret_cast<int4*>(p);
  __stcg(q, make_int4(d.epoch, d.phase, d.nitems, d.round));
  __stcg(q + 1, make_int4(d.action, d.prec, d.j, d.kdim));
}

__device__ int first_phase(const SolveInst& I, int action) {
  if (is_mv(action)) return 0;
  if (I.single) return kPhaseSingle;
  // r = b and its partial sums came with the right-hand side's phase D
  if (action == ACT_RESID_ZERO && I.rhs_r0) return kPhaseE;
  // y was solved for by the control step that chose FINISH (phase_F)
  return action == ACT_FINISH ? kPhaseE : kPhaseD;
}

// -1: the round ends after `phase` (of a round doing `action`)
__device__ int next_phase(const SolveInst& I, int phase, int action, int prec) {
  const bool d3 = I.g.dim == 3;
  switch (phase) {
    case 0: return d3 ? 1 : 2;
    case 1: return 2;
    case 2: return d3 ? 3 : 4;
    case 3: return 4;
    case 4:
      if (I.single) return kPhaseSingle;
      return fused_step(I, action, prec) ? kPhaseE : kPhaseD;
    case kPhaseD: return action == ACT_RHS ? -1 : kPhaseE;
    case kPhaseE:
      return action == ACT_MV_ARNOLDI && !single_pass(I, action, prec) ? kPhaseF : -1;
    default: return -1;
  }
}

__device__ int items_of(const SolveInst& I, const PhaseDesc& d) {
  if (d.phase < 5) return I.mv_nitems[d.phase][d.prec ? 1 : 0];
  if (d.phase == kPhaseSingle) return 1;
  // the control step is an item of its own in F, and in E when the round
  // ends there (phase_E, phase_F)
  if (d.phase == kPhaseF ||
      (d.phase == kPhaseE &&
       (d.action != ACT_MV_ARNOLDI || single_pass(I, d.action, d.prec))))
    return I.nchunk + 1;
  return I.nchunk;
}

// each element type's own pencil layout (run_item dispatches the same way)
void solver_fill_items(SolveInst& I) {
  for (int ph = 0; ph < 5; ++ph) {
    I.mv_nitems[ph][0] = I.dd64 ? mv_items<dd>(I, ph) : mv_items<double>(I, ph);
    I.mv_nitems[ph][1] = mv_items<float>(I, ph);
  }
}

// The round view of the state; `active` is false when the instance is done.
__device__ bool view_from_state(const SolveState* S, PhaseDesc& d) {
  const volatile SolveState* vs = S;
  d.action = vs->action;
  d.prec = vs->prec;
  d.j = vs->j;
  d.kdim = vs->kdim;
  return d.action != ACT_DONE;
}

// Publishes instance k's next phase (one thread).  `finished` counts
// instances that are done or have used their rounds for this launch.
// `cur` is the descriptor of the phase whose last item the caller finished:
// the stored one, which nobody else can change now.
// With take_first the caller keeps item 0 of the new phase for itself (the
// claim word is published with item 1 next): returns true and the new
// descriptor in *out when there is such an item.
__device__ bool advance(const SolveInst& I, const SolveState* S, unsigned* bar, int k,
                        int max_rounds, const PhaseDesc& cur, bool take_first,
                        PhaseDesc* out) {
  PhaseDesc d = cur;
  int np = next_phase(I, d.phase, d.action, d.prec);
  if (np < 0) {
    d.round++;
    const bool active = view_from_state(S, d);
    if (!active || (max_rounds > 0 && d.round >= max_rounds)) {
      d.nitems = 0;
      d.epoch++;
      store_desc(desc_of(bar, k), d);
      fence_acq_rel();
      atomicExch(claim_word(bar, k), claim_value(d.epoch, 0));
      atomicAdd(bar + 3, 1u);
      return false;
    }
    np = first_phase(I, d.action);
  }
  d.phase = np;
  d.nitems = items_of(I, d);
  d.epoch++;
  store_desc(desc_of(bar, k), d);
  *(volatile unsigned*)done_word(bar, k) = 0u;
  fence_acq_rel();
  const bool take = take_first && d.nitems > 0;
  atomicExch(claim_word(bar, k), claim_value(d.epoch, d.nitems) + (take ? 1ull : 0ull));
  *out = d;
  return take;
}

__device__ void run_item(const SolveInst& I, SolveState* S, const PhaseDesc& d, int item,
                         unsigned char* smem, BlockRed& R) {
  RoundView v;
  v.action = d.action;
  v.prec = d.prec;
  v.j = d.j;
  v.kdim = d.kdim;
  if (d.phase < 5) {
    if (v.prec)
      mv_item<float>(I, v, d.phase, item, smem);
    else if (I.dd64)
      mv_item<dd>(I, v, d.phase, item, smem);
    else
      mv_item<double>(I, v, d.phase, item, smem);
  } else if (d.phase == kPhaseD) {
    if (I.g.dim == 2)
      phase_D<2>(I, S, v, item, R);
    else
      phase_D<3>(I, S, v, item, R);
  } else if (d.phase == kPhaseE) {
    phase_E(I, S, v, item, R);
  } else if (d.phase == kPhaseF) {
    phase_F(I, S, v, item, R);
  } else {
    vec_single(I, S, v, R);
  }
}

// Item timing (optional): the executing block's thread 0 adds each item's
// duration to ptimes[2*id] and counts it in ptimes[2*id+1].  Ids: 0..4
// matvec phases in float64 (rows_fwd, y fwd, solve, y inv, rows_inv), 5..9
// the same in float32, 10 the vector phases D..G (and the one-block step),
// 14 idle block time spent looking for work.
__device__ __forceinline__ void add_time(unsigned long long* ptimes, int id,
                                         unsigned long long dt) {
  atomicAdd(ptimes + 2 * id, dt);
  atomicAdd(ptimes + 2 * id + 1, 1ull);
}

// One record of the item trace (thread 0, while the trace is on): block b
// owns records [b * per_block, (b + 1) * per_block) of the trace and counts
// its own in *n, so a record costs three stores and no atomic.
__device__ __forceinline__ void trace_item(unsigned long long* ptimes, int* n,
                                           unsigned long long t0, unsigned long long t1, int k,
                                           int phase, int prec, int item) {
  const int per_block = kTraceCap / (int)gridDim.x;
  if (*n >= per_block) return;
  const size_t r = (size_t)blockIdx.x * per_block + (*n)++;
  unsigned long long* rec = ptimes + kTraceFlag + 2 + 3 * r;
  rec[0] = t0;
  rec[1] = t1;
  rec[2] = ((unsigned long long)blockIdx.x << 40) | ((unsigned long long)(k & 0xffff) << 24) |
           ((unsigned long long)(phase & 15) << 20) | ((unsigned long long)(prec & 3) << 18) |
           (unsigned long long)(item & 0x3ffff);
}

struct ItemSlot {
  int k, item, have;
  PhaseDesc d;
};

__global__ void __launch_bounds__(kSolverThreads, 2)
    k_persistent_solve(const SolveInst* __restrict__ insts, SolveState* states, int ninst,
                       unsigned* bar, unsigned long long* ptimes, int max_rounds) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BlockRed R;
  __shared__ ItemSlot slot;
  const unsigned nblocks = gridDim.x;
  const int bid = blockIdx.x;

  // block 0 publishes every instance's first phase
  if (bid == 0) {
    for (int k = threadIdx.x; k < ninst; k += blockDim.x) {
      PhaseDesc d;
      d.round = 0;
      d.epoch = 1;
      if (view_from_state(states + k, d)) {
        d.phase = first_phase(insts[k], d.action);
        d.nitems = items_of(insts[k], d);
      } else {
        d.phase = 0;
        d.nitems = 0;
        atomicAdd(bar + 3, 1u);
      }
      store_desc(desc_of(bar, k), d);
      *(volatile unsigned*)done_word(bar, k) = 0u;
      __threadfence();
      atomicExch(claim_word(bar, k), claim_value(d.epoch, d.nitems));
    }
  }
  if (!grid_barrier(bar, nblocks)) return;

  unsigned spins = 0;
  unsigned long long idle0 = 0;
  int rot = bid % (ninst > 0 ? ninst : 1);
  const int lane = threadIdx.x & 31;
  // thread 0: the slot already holds an item this block claimed when it
  // finished its last one (the next item of the same phase, or item 0 of the
  // phase it handed off to)
  int preclaimed = 0;
  // the item trace: switched on for the whole launch, or not at all
  const bool tracing =
      ptimes && threadIdx.x == 0 && *(volatile unsigned long long*)(ptimes + kTraceFlag) != 0ull;
  int ntrace = 0;
  for (;;) {
    // warp 0 looks for an item: its lanes probe 32 instances at a time (the
    // descriptor's epoch and item count and the claim word, read around L1)
    if (threadIdx.x < 32) {
      // a block with an item in hand runs it; one without first checks the
      // error word (set when a wait gave up: then every block leaves)
      int have = 0;
      if (lane == 0) {
        if (preclaimed)
          have = 1;
        else if (*(volatile unsigned*)(bar + 2) != 0u)
          have = -1;
      }
      preclaimed = 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      for (int base = 0; base < ninst && have == 0; base += 32) {
        const int t = base + lane;
        const int k = (rot + t) % ninst;
        const bool avail = t < ninst && claim_open(__ldcg(claim_word(bar, k)));
        unsigned cand = __ballot_sync(0xffffffffu, avail);
        while (cand && have == 0) {
          const int l = __ffs(cand) - 1;
          cand &= cand - 1;
          const int kk = __shfl_sync(0xffffffffu, k, l);
          int got = 0;
          if (lane == 0) {
            const unsigned long long w = atomicAdd(claim_word(bar, kk), 1ull);
            if (claim_open(w)) {
              fence_acq_rel();
              slot.k = kk;
              slot.item = (int)(w & 0xffffffffu);
              slot.d = load_desc(desc_of(bar, kk));
              got = 1;
            }
          }
          got = __shfl_sync(0xffffffffu, got, 0);
          if (got) {
            have = 1;
            rot = kk;  // stay on this instance while it has items
          }
        }
      }
      if (lane == 0) {
        if (have == 0) {
          if (*(volatile unsigned*)(bar + 3) >= (unsigned)ninst) {
            have = -1;  // every instance is done (or paused)
          } else {
            if (ptimes && spins == 0) idle0 = global_ns();
            if (++spins > kSpinLimit) {
              atomicExch(bar + 2, 1u);
              have = -1;
            } else {
              __nanosleep(20);
            }
          }
        } else if (have > 0 && spins) {
          if (ptimes) add_time(ptimes, 14, global_ns() - idle0);
          spins = 0;
        }
        slot.have = have;
      }
      rot = __shfl_sync(0xffffffffu, rot, 0);
    }
    __syncthreads();
    const int have = slot.have;
    if (have < 0) break;
    if (have == 0) {
      __syncthreads();
      continue;
    }
    const int k = slot.k, item = slot.item;
    const PhaseDesc d = slot.d;
    __syncthreads();  // slot is rewritten by thread 0 in the next iteration
    unsigned long long ta = 0;
    if (ptimes && threadIdx.x == 0) ta = global_ns();
    run_item(insts[k], states + k, d, item, smem, R);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tb = 0;
      if (ptimes) {
        tb = global_ns();
        add_time(ptimes, d.phase < 5 ? d.phase + 5 * d.prec : 10, tb - ta);
        if (tracing) trace_item(ptimes, &ntrace, ta, tb, k, d.phase, d.prec, item);
      }
      fence_acq_rel();  // the item's writes before its done count
      // the next item of the same phase is claimed together with the done
      // count (both atomics in flight at once): a block that stays on one
      // phase needs no scan and no descriptor read between its items
      const unsigned long long w = atomicAdd(claim_word(bar, k), 1ull);
      const unsigned prior = atomicAdd(done_word(bar, k), 1u);
      if (claim_open(w)) {
        slot.k = k;
        slot.item = (int)(w & 0xffffffffu);
        if ((unsigned)(w >> 48) == ((unsigned)d.epoch & 0xffffu)) {
          slot.d = d;
        } else {
          // another block advanced the phase between the two atomics
          fence_acq_rel();
          slot.d = load_desc(desc_of(bar, k));
        }
        preclaimed = 1;
      }
      if ((int)prior == d.nitems - 1) {
        // every item of the phase is done: see their writes (the state of
        // the control step included) before choosing the next phase; the
        // claim above found the phase exhausted, so this block takes item 0
        // of the next one
        fence_acq_rel();
        PhaseDesc nd = d;
        const bool took = advance(insts[k], states + k, bar, k, max_rounds, d,
                                  !preclaimed, &nd);
        if (took) {
          slot.k = k;
          slot.item = 0;
          slot.d = nd;
          preclaimed = 1;
        }
        if (tracing)
          trace_item(ptimes, &ntrace, tb, global_ns(), k, 15, nd.prec, took ? nd.phase : 15);
      }
    }
  }
}

// Dynamic shared memory of one matvec work item of element type T: the row
// tiles of the x passes and the pencil items of each pencil layout (2D: the
// y solve; 3D: the z solve and the y passes).  out[0] row tile, out[1..2]
// the pencil layouts (out[2] = 0 in 2D).
template <typename T>
static void item_smem(const GridDesc& g, int rows, size_t out[3]) {
  out[0] = rows_smem_bytes<T>(g.n, rows);
  out[1] = pencil_smem_bytes<T>(solver_layout<T>(g, 1), g.n);
  out[2] = g.dim == 3 ? pencil_smem_bytes<T>(solver_layout<T>(g, 0), g.n) : 0;
}

void solver_item_smem(const GridDesc& g, int rows, int elem, size_t out[3]) {
  if (elem == 1)
    item_smem<float>(g, rows, out);
  else if (elem == 2)
    item_smem<dd>(g, rows, out);
  else
    item_smem<double>(g, rows, out);
}

// The launch reserves the largest need of every element type a solve of this
// geometry may run: float64 (plain solves, and the float64-grade matvecs of
// large batches), double-float (those of small refined launches) and float32
// (the refined inner operator) -- each from its own plan and layout.
int solver_smem_bytes(const GridDesc& g, int rows, int need32) {
  size_t s = 0;
  for (int elem = 0; elem < 3; ++elem) {
    if (elem == 1 && !need32) continue;
    size_t need[3];
    solver_item_smem(g, rows, elem, need);
    for (int k = 0; k < 3; ++k)
      if (need[k] > s) s = need[k];
  }
  return s > (size_t)INT32_MAX ? -1 : (int)s;
}

// Before a cooperative launch: every item the instances can run fits in the
// dynamic shared memory the launch reserves.  A shortfall would let an item
// address past its block's shared window, so the launch is refused instead.
bool solver_smem_fits(const SolveInst* h_insts, int ninst, int smem, char* why, size_t why_len) {
  for (int k = 0; k < ninst; ++k) {
    const SolveInst& I = h_insts[k];
    const int elems[2] = {I.dd64 ? 2 : 0, I.refined ? 1 : -1};
    for (int e : elems) {
      if (e < 0) continue;
      size_t need[3];
      solver_item_smem(I.g, I.b.rows, e, need);
      for (int c = 0; c < 3; ++c)
        if (need[c] > (size_t)(smem < 0 ? 0 : smem)) {
          snprintf(why, why_len,
                   "persistent solver: instance %d (dim %d, n %d, element type %d, item kind %d) "
                   "needs %zu bytes of shared memory, the launch reserves %d",
                   k, I.g.dim, I.g.n, e, c, need[c], smem);
          return false;
        }
    }
  }
  return true;
}

cudaError_t launch_persistent_solve(const SolveInst* d_insts, SolveState* d_states, int ninst,
                                    unsigned* d_bar, int smem, cudaStream_t st, int max_rounds,
                                    int reserve_sms) {
  unsigned long long* ptimes = prof_phase_buffer();
  // per device: SM count and the shared-memory limit already raised
  static std::mutex mu;
  static int sm_counts[kMaxDevices] = {};
  static int configured_smem[kMaxDevices] = {};
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (smem < 0) return cudaErrorInvalidValue;
  int sm_count = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!sm_counts[dev]) {
      if ((e = cudaDeviceGetAttribute(&sm_counts[dev], cudaDevAttrMultiProcessorCount, dev)))
        return e;
    }
    sm_count = sm_counts[dev];
    if (smem > configured_smem[dev]) {
      if ((e = cudaFuncSetAttribute((const void*)k_persistent_solve,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
      configured_smem[dev] = smem;
    }
  }
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent_solve,
                                                         kSolverThreads, smem)))
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > 2) per_sm = 2;
  int sms = sm_count - (reserve_sms > 0 ? reserve_sms : 0);
  if (sms < 1) sms = 1;
  const int blocks = per_sm * sms;
  if ((e = cudaMemsetAsync(d_bar, 0, (4 + kSchedWords * (size_t)ninst) * sizeof(unsigned),
                           st)))
    return e;
  void* args[] = {(void*)&d_insts, (void*)&d_states, (void*)&ninst, (void*)&d_bar,
                  (void*)&ptimes, (void*)&max_rounds};
  prof_begin(st);
  e = cudaLaunchCooperativeKernel((const void*)k_persistent_solve, dim3(blocks),
                                  dim3(kSolverThreads), args, (size_t)smem, st);
  count_launch("persistent_solve", st);
  return e;
}

}  // namespace ibdl
