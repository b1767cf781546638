// Persistent GMRES solver: one cooperative launch runs whole IBDL solves
// (Sec. 5.3: unpreconditioned GMRES on the second-kind boundary system) for
// one or many instances, with no host round trip between iterations.
//
// Every block loops over "rounds".  In a round each active instance does one
// action of its state machine, split into phases separated by grid barriers:
//
//   A   rows_fwd   spread-divergence of the matvec input + x FFT   (matvec)
//   B   pencils    y (and z) FFT passes with the symbol            (matvec)
//   C   rows_inv   x inverse FFT to the real grid                  (matvec)
//   D   interp     w = S* grid +- input/2, then the first-pass dot products
//   E   reduce, w -= V h (CGS pass 1), second-pass dots / residual norm
//   F   reduce, w -= V h (CGS pass 2), norm partial / x update
//   G   normalise w; Givens rotation; control (next action)
//
// Actions: RESID_ZERO (r = b at x = 0), MV_RESIDUAL (r = b - A64 x),
// MV_ARNOLDI (Arnoldi step j with the float64 or float32 operator),
// FINISH (back substitution, x += V y), DONE.  The float64 mode restarts with
// the true residual after every cycle; the float32-refined mode runs one
// float32 GMRES cycle per refinement step between float64 residuals.
//
// Work items of all instances are concatenated per phase and dealt to blocks
// round-robin.  The grid barrier spins a bounded number of times; on timeout
// it sets an error flag and every block leaves the kernel.
#include <math.h>

#include "ibdl_device.cuh"
#include "ibdl_solver.cuh"

namespace ibdl {

constexpr unsigned kSpinLimit = 1u << 27;  // x >= 20 ns sleeps: a few seconds

// Counting barrier among `parties` blocks on ctr[0] (arrivals) and ctr[1]
// (generation).  The spin is bounded: on timeout it raises *err, which every
// later barrier sees, and all blocks leave the kernel.
__device__ bool counted_barrier(unsigned* ctr, unsigned parties, unsigned* err) {
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
        if (++spins > kSpinLimit) {
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

// bar[0..1]: grid barrier, bar[2]: error flag, bar[4 + 4k ..]: barrier of the
// blocks that hold instance k's vector chunks.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  return counted_barrier(bar, nblocks, bar + 2);
}

struct RoundView {
  int action, prec, j, kdim;
};

constexpr int kMaxCols = 66;  // restart (<= 64) + 2

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
__device__ void chunk_dots(const SolveInst& I, double xi, bool valid, int i, int ncols,
                           bool with_norm, double* part, int chunk, BlockRed& R) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < ncols; ++c) {
    const double v = valid ? xi * __ldcg(I.V + (size_t)c * I.ld + i) : 0.0;
    const double s = warp_sum(v);
    if (lane == 0) R.red[c][wid] = s;
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
  for (int c = 0; c < ncols; ++c) w -= h[c] * __ldcg(I.V + (size_t)c * I.ld + i);
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

__device__ __forceinline__ bool is_mv(int a) {
  return a == ACT_MV_ARNOLDI || a == ACT_MV_RESIDUAL || a == ACT_RHS;
}

__device__ __forceinline__ const double* mv_input(const SolveInst& I, const RoundView& v) {
  if (v.action == ACT_RHS) return nullptr;
  return v.action == ACT_MV_ARNOLDI ? I.V + (size_t)v.j * I.ld : I.x;
}

template <typename T>
__device__ int mv_items(const SolveInst& I, int phase) {
  const int d = I.g.dim, n = I.g.n;
  if (phase == 0 || phase == 4) return I.b.ntiles;
  PencilLayout L;
  if (d == 2) {
    if (phase != 2) return 0;
    L = solve_layout<T>(2, n, 1);
  } else {
    L = solve_layout<T>(3, n, phase == 2 ? 1 : 0);
  }
  return (L.npencils + L.c - 1) / L.c;
}

// Each matvec phase is called through a non-inlined wrapper, so that every
// phase gets its own register allocation inside this one large kernel.  The
// wrappers take the instance by reference to its global-memory descriptor.
template <typename T, int D>
__device__ __noinline__ void solver_rows_fwd(const SolveInst& I, const double* q, int item,
                                             unsigned char* smem) {
  SpreadSrc src;
  src.skip_empty_planes = true;  // the grid feeds only the interpolation
  if (q) {
    src.q_div = q;
    src.coef_div = 1.0;
  } else {
    src.v_plain = I.vdata;  // right-hand side: -S V_b
    src.coef_plain = -1.0;
  }
  const SpectralWs<T> ws = ws_of<T>(I);
  phase_rows_fwd<T, D>(I.g, I.p, I.b, src, ws.spec, ws.tw, nullptr, item, smem);
}

template <typename T, int D>
__device__ __noinline__ void solver_rows_inv(const SolveInst& I, int item, unsigned char* smem) {
  const SpectralWs<T> ws = ws_of<T>(I);
  phase_rows_inv<T, D, T>(I.g, I.b, ws.spec, ws.tw, ws.grid, item, smem, true);
}

template <typename T, int MODE>
__device__ __noinline__ void solver_pencils(const SolveInst& I, int which, int item,
                                            unsigned char* smem) {
  const SpectralWs<T> ws = ws_of<T>(I);
  const GridDesc& g = I.g;
  const double nd = g.dim == 3 ? (double)g.n * g.n * g.n : (double)g.n * g.n;
  const T cfac = (T)(4.0 * g.kappa / (g.h * g.h));
  const T scale0 = (T)(g.kappa / nd);
  // the matvec's grid feeds only the interpolation and has no grid source:
  // 3D y-pass items of planes without points are skipped (both directions)
  const int* zskip = (g.dim == 3 && MODE != 2) ? I.b.start : nullptr;
  phase_pencils<T, MODE>(g, solve_layout<T>(g.dim, g.n, which), ws.spec, ws.tw, ws.s2, cfac,
                         scale0, item, smem, zskip, g.n / I.b.rows,
                         (g.dim == 3 && MODE == 2) ? I.b.zempty : nullptr);
}

// phase: 0 rows_fwd, 1 y forward (3D), 2 solve pass, 3 y inverse (3D), 4 rows_inv
template <typename T>
__device__ void mv_item(const SolveInst& I, const RoundView& v, int phase, int item,
                        unsigned char* smem) {
  const int d = I.g.dim;
  if (phase == 0) {
    if (d == 2)
      solver_rows_fwd<T, 2>(I, mv_input(I, v), item, smem);
    else
      solver_rows_fwd<T, 3>(I, mv_input(I, v), item, smem);
  } else if (phase == 4) {
    if (d == 2)
      solver_rows_inv<T, 2>(I, item, smem);
    else
      solver_rows_inv<T, 3>(I, item, smem);
  } else if (d == 2 || phase == 2) {
    solver_pencils<T, 2>(I, 1, item, smem);
  } else if (phase == 1) {
    solver_pencils<T, 0>(I, 0, item, smem);
  } else {
    solver_pencils<T, 1>(I, 0, item, smem);
  }
}

__device__ int phase_items(const SolveInst& I, const RoundView& v, int phase) {
  if (phase < 5) {
    if (!is_mv(v.action)) return 0;
    return v.prec ? mv_items<float>(I, phase) : mv_items<double>(I, phase);
  }
  if (v.action == ACT_DONE) return 0;
  if (I.single) return 0;  // handled by vec_single on its own block
  return I.nchunk;
}

// ---- vector phases ------------------------------------------------------------

template <int D>
__device__ void phase_D(const SolveInst& I, const RoundView& v, int chunk, BlockRed& R) {
  const int i = chunk * blockDim.x + threadIdx.x;
  const bool valid = i < I.p.m;
  double* part1 = I.part;
  if (v.action == ACT_FINISH) {
    if (chunk == 0 && threadIdx.x == 0) {
      const int k = v.kdim, ldh = I.restart + 1;
      for (int r = k - 1; r >= 0; --r) {
        double s = __ldcg(I.gv + r);
        for (int l = r + 1; l < k; ++l) s -= __ldcg(I.H + (size_t)l * ldh + r) * I.ysol[l];
        const double dgn = __ldcg(I.H + (size_t)r * ldh + r);
        I.ysol[r] = dgn != 0.0 ? s / dgn : 0.0;
      }
      __threadfence();
    }
    return;
  }
  if (v.action == ACT_RHS) {
    // b = S* grid, grid = -kappa L'^{-1} S V_b (the Neumann right-hand side)
    if (valid) I.bvec[i] = interp_point<double, D>(I.g, I.p, I.w64.grid, i);
    return;
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
    chunk_dots(I, w, valid, i, v.j + 1, false, part1, chunk, R);
    return;
  }
  // residual actions: r = b - A x (or r = b), partial ||r||^2 and ||b||^2
  double r = 0, bi = 0;
  if (valid) {
    bi = __ldcg(I.bvec + i);
    if (v.action == ACT_MV_RESIDUAL) {
      const double t = interp_point<double, D>(I.g, I.p, I.w64.grid, i) + jump * __ldcg(I.x + i);
      r = bi - t;
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

// CGS pass: h = sum of partials (section `in`), Hcol (+)= h (chunk 0),
// w -= V h; then dots of w with V (pass 1) or ||w||^2 (pass 2) into `out`.
__device__ void cgs_pass(const SolveInst& I, const RoundView& v, int chunk, BlockRed& R,
                         const double* in, double* out, bool first) {
  const int ncols = v.j + 1;
  const int ldh = I.restart + 1;
  reduce_parts(in, I.nchunk, I.pstride, 0, ncols, R.h);
  if (chunk == 0) {
    double* Hcol = I.H + (size_t)v.j * ldh;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x)
      Hcol[c] = first ? R.h[c] : __ldcg(Hcol + c) + R.h[c];
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
  if (first) {
    chunk_dots(I, w, valid, i, ncols, false, out, chunk, R);
  } else {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double s = warp_sum(valid ? w * w : 0.0);
    if (lane == 0) R.red[0][wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int k = 0; k < nw; ++k) t += R.red[0][k];
      out[(size_t)chunk * I.pstride] = t;
    }
    __syncthreads();
  }
}

__device__ void phase_E(const SolveInst& I, const RoundView& v, int chunk, BlockRed& R) {
  double* part1 = I.part;
  double* part2 = I.part + (size_t)I.nchunk * I.pstride;
  if (v.action == ACT_MV_ARNOLDI) {
    cgs_pass(I, v, chunk, R, part1, part2, true);
    return;
  }
  if (v.action == ACT_RHS) return;
  const int i = chunk * blockDim.x + threadIdx.x;
  const bool valid = i < I.p.m;
  if (v.action == ACT_FINISH) {
    // x += V y: stage -y in shared memory, then one batched pass over V
    for (int c = threadIdx.x; c < v.kdim; c += blockDim.x) R.h[c] = -__ldcg(I.ysol + c);
    __syncthreads();
    if (valid) I.x[i] = sub_projection(I, __ldcg(I.x + i), i, v.kdim, R.h);
    __syncthreads();
    return;
  }
  // residual actions: V0 = r / ||r||
  reduce_parts(part1, I.nchunk, I.pstride, 0, 1, R.h);
  const double beta = sqrt(R.h[0]);
  const double inv = (beta > 0 && isfinite(beta)) ? 1.0 / beta : 0.0;
  if (valid) I.V[i] = __ldcg(I.r + i) * inv;
  __syncthreads();
}

__device__ void phase_F(const SolveInst& I, const RoundView& v, int chunk, BlockRed& R) {
  if (v.action != ACT_MV_ARNOLDI) return;
  double* part2 = I.part + (size_t)I.nchunk * I.pstride;
  double* part3 = I.part + 2 * (size_t)I.nchunk * I.pstride;
  cgs_pass(I, v, chunk, R, part2, part3, false);
}

// Control of one instance (one thread).  hn: new subdiagonal, beta: residual
// norm of a residual action, bnorm2: ||b||^2 partial sum.
__device__ void control(const SolveInst& I, SolveState* S, const RoundView& v, double hn,
                        double beta, double bnorm2, BlockRed& R) {
  const int ldh = I.restart + 1;
  SolveState s;
  {
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
    s.beta = vs->beta;
    s.bnorm = vs->bnorm;
    s.tol_abs = vs->tol_abs;
    s.rel = vs->rel;
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
    const double a = cj[j], b = cj[j + 1];
    const double den = hypot(a, b);
    double c = 1.0, sn = 0.0;
    if (den > 0) {
      c = a / den;
      sn = b / den;
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
    s.action = ACT_MV_RESIDUAL;
    s.prec = 0;
  } else if (v.action == ACT_RHS) {
    s.action = s.xinit ? ACT_MV_RESIDUAL : ACT_RESID_ZERO;
    s.prec = 0;
  } else {
    if (v.action == ACT_MV_RESIDUAL) s.matvecs++;
    if (s.bnorm < 0) s.bnorm = sqrt(bnorm2);
    s.beta = beta;
    s.rel = s.bnorm > 0 ? beta / s.bnorm : 0.0;
    if (s.bnorm == 0.0) {
      s.status = IBDL_OK;
      s.action = ACT_DONE;
    } else if (!isfinite(beta)) {
      s.status = IBDL_ERR_NONFINITE;
      s.action = ACT_DONE;
    } else if (s.rel <= I.tol) {
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
  __threadfence();
}

__device__ void phase_G(const SolveInst& I, SolveState* S, const RoundView& v, int chunk,
                        BlockRed& R) {
  if (v.action == ACT_MV_ARNOLDI) {
    double* part3 = I.part + 2 * (size_t)I.nchunk * I.pstride;
    reduce_parts(part3, I.nchunk, I.pstride, 0, 1, R.h);
    const double hn = sqrt(R.h[0]);
    const double inv = (hn > 0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    const int i = chunk * blockDim.x + threadIdx.x;
    if (i < I.p.m && inv != 0.0) {
      double* wp = I.V + (size_t)(v.j + 1) * I.ld;
      wp[i] = __ldcg(wp + i) * inv;
    }
    if (chunk == 0) {
      const int j = v.j, ldh = I.restart + 1;
      __syncthreads();
      for (int r = threadIdx.x; r <= j; r += blockDim.x) {
        R.col[r] = __ldcg(I.H + (size_t)j * ldh + r);
        if (r < j) {
          R.cs[r] = __ldcg(I.cs + r);
          R.sn[r] = __ldcg(I.sn + r);
        }
      }
      if (threadIdx.x == 0) R.h[0] = __ldcg(I.gv + j);
      __syncthreads();
      if (threadIdx.x == 0) control(I, S, v, hn, 0, 0, R);
    }
    __syncthreads();
    return;
  }
  if (chunk != 0) return;
  double beta = 0, b2 = 0;
  if (v.action != ACT_FINISH && v.action != ACT_RHS) {
    reduce_parts(I.part, I.nchunk, I.pstride, 0, 2, R.h);
    beta = sqrt(R.h[0]);
    b2 = R.h[1];
  }
  if (threadIdx.x == 0) control(I, S, v, 0, beta, b2, R);
  __syncthreads();
}

// ---- single-block vector step (instances with few points) ------------------
// For m <= kSingleMax the whole post-matvec work of an action (interpolation,
// both CGS passes, norm, Givens, control) runs in one block with block-level
// synchronisation: one grid barrier per round instead of four.  The block is
// fixed per instance (instance k -> block k mod gridDim), so every Krylov
// vector, x and r of the instance is produced and consumed on the same SM
// and is read back with ordinary (L1-coherent) loads; only the grid, written
// by other blocks, is read around L1.

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
      if (i < m)
        I.bvec[i] = d3 ? interp_point<double, 3>(I.g, I.p, I.w64.grid, i)
                       : interp_point<double, 2>(I.g, I.p, I.w64.grid, i);
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
    double xk[kSingleK];
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      xk[k] = i < m ? I.x[i] : 0.0;
    }
    for (int c = 0; c < v.kdim; ++c) {
      const double yc = R.h[c];
      const double* vc = I.V + (size_t)c * I.ld;
#pragma unroll
      for (int k = 0; k < kSingleK; ++k) {
        const int i = tid + k * nt;
        if (i < m) xk[k] += yc * vc[i];
      }
    }
#pragma unroll
    for (int k = 0; k < kSingleK; ++k) {
      const int i = tid + k * nt;
      if (i < m) I.x[i] = xk[k];
    }
    __syncthreads();
    if (tid == 0) control(I, S, v, 0, 0, 0, R);
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
        wk[k] = acc + jump * vin[i];
      }
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int c = 0; c < ncols; ++c) {
        const double* vc = I.V + (size_t)c * I.ld;
        double sacc = 0;
#pragma unroll
        for (int k = 0; k < kSingleK; ++k) {
          const int i = tid + k * nt;
          if (i < m) sacc += wk[k] * vc[i];
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
          if (i < m) wk[k] -= hc * vc[i];
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
        r = bi - (acc + jump * I.x[i]);
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

// Phase timing (optional): block 0, thread 0 adds the wall time between
// consecutive grid-barrier exits to ptimes[2*id] and counts in ptimes[2*id+1].
// Ids: 0..4 matvec phases in float64 (rows_fwd, y fwd, solve, y inv,
// rows_inv), 5..9 the same in float32, 10 the vector phases D..G, 14 round
// bookkeeping.
__device__ __forceinline__ void phase_tick(unsigned long long* ptimes, int id,
                                           unsigned long long& t0) {
  if (ptimes && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long t = global_ns();
    ptimes[2 * id] += t - t0;
    ptimes[2 * id + 1] += 1;
    t0 = t;
  }
}

__global__ void __launch_bounds__(kSolverThreads, 2)
    k_persistent_solve(const SolveInst* __restrict__ insts, SolveState* states, int ninst,
                       unsigned* bar, unsigned long long* ptimes, int max_rounds) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RoundView rv[kMaxBatch];
  __shared__ BlockRed R;
  __shared__ int flags[4];
  const unsigned nblocks = gridDim.x;
  const int G = gridDim.x, bid = blockIdx.x;
  unsigned long long t0 = 0;
  if (ptimes && bid == 0 && threadIdx.x == 0) t0 = global_ns();

  for (int round = 0;; ++round) {
    // a bounded slice stops between rounds; the states stay in global memory
    // and the next launch resumes them
    if (max_rounds > 0 && round >= max_rounds) break;
    if (threadIdx.x == 0) {
      flags[0] = 0;
      flags[1] = 0;
      flags[2] = 0;
      flags[3] = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ninst; k += blockDim.x) {
      volatile SolveState* s = states + k;
      RoundView v;
      v.action = s->action;
      v.prec = s->prec;
      v.j = s->j;
      v.kdim = s->kdim;
      rv[k] = v;
      if (v.action != ACT_DONE) {
        atomicOr(&flags[0], 1);
        if (!insts[k].single) atomicOr(&flags[3], 1);
      }
      if (is_mv(v.action)) {
        atomicOr(&flags[1], 1);
        if (insts[k].g.dim == 3) atomicOr(&flags[2], 1);
      }
    }
    __syncthreads();
    if (!flags[0]) break;
    const bool any_mv = flags[1] != 0, any3d = flags[2] != 0, any_multi = flags[3] != 0;
    phase_tick(ptimes, 14, t0);
    const int prec0 = rv[0].prec;

    // matvec phases
    for (int phase = 0; phase < 5 && any_mv; ++phase) {
      if ((phase == 1 || phase == 3) && !any3d) continue;
      int base = 0;
      for (int k = 0; k < ninst; ++k) {
        const RoundView v = rv[k];
        const int cnt = phase_items(insts[k], v, phase);
        if (cnt == 0) continue;
        const int first = ((bid - base) % G + G) % G;
        for (int it = first; it < cnt; it += G) {
          if (v.prec)
            mv_item<float>(insts[k], v, phase, it, smem);
          else
            mv_item<double>(insts[k], v, phase, it, smem);
        }
        base += cnt;
      }
      if (!grid_barrier(bar, nblocks)) return;
      phase_tick(ptimes, phase + 5 * prec0, t0);
    }
    // vector phases D..G.  Single-block instances finish in one block; the
    // others run D, E, F, G on the blocks that hold their chunks, separated
    // by a barrier among those blocks only, and one grid barrier closes the
    // round.
    for (int k = bid; k < ninst; k += G) {
      const RoundView v = rv[k];
      if (insts[k].single && v.action != ACT_DONE) vec_single(insts[k], states + k, v, R);
    }
    if (any_multi) {
      int base = 0;
      for (int k = 0; k < ninst; ++k) {
        const RoundView v = rv[k];
        const SolveInst& I = insts[k];
        const int cnt = phase_items(I, v, 5);
        if (cnt == 0) continue;
        const int first = ((bid - base) % G + G) % G;
        base += cnt;
        if (first >= cnt) continue;
        const unsigned parties = cnt < G ? (unsigned)cnt : (unsigned)G;
        unsigned* ib = bar + 4 + 4 * k;
        for (int it = first; it < cnt; it += G) {
          if (I.g.dim == 2)
            phase_D<2>(I, v, it, R);
          else
            phase_D<3>(I, v, it, R);
        }
        if (!counted_barrier(ib, parties, bar + 2)) return;
        for (int it = first; it < cnt; it += G) phase_E(I, v, it, R);
        if (!counted_barrier(ib, parties, bar + 2)) return;
        for (int it = first; it < cnt; it += G) phase_F(I, v, it, R);
        if (!counted_barrier(ib, parties, bar + 2)) return;
        for (int it = first; it < cnt; it += G) phase_G(I, states + k, v, it, R);
      }
    }
    if (!grid_barrier(bar, nblocks)) return;
    phase_tick(ptimes, 10, t0);
  }
}

int solver_smem_bytes(const GridDesc& g, int need32) {
  size_t s = rows_smem_bytes<double>(g.n, rows_per_tile(g.dim, g.n));
  const int nl = g.dim == 2 ? 1 : 2;
  for (int w = 0; w < nl; ++w) {
    const PencilLayout L = solve_layout<double>(g.dim, g.n, w == 0 ? 1 : 0);
    const size_t ps = pencil_smem_bytes<double>(L, g.n);
    if (ps > s) s = ps;
    if (need32) {
      const PencilLayout L32 = solve_layout<float>(g.dim, g.n, w == 0 ? 1 : 0);
      const size_t p32 = pencil_smem_bytes<float>(L32, g.n);
      if (p32 > s) s = p32;
    }
  }
  return (int)s;
}

cudaError_t launch_persistent_solve(const SolveInst* d_insts, SolveState* d_states, int ninst,
                                    unsigned* d_bar, int smem, cudaStream_t st, int max_rounds,
                                    int reserve_sms) {
  unsigned long long* ptimes = prof_phase_buffer();
  static int sm_count = 0;
  static int configured_smem = -1;
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if (!sm_count) {
    if ((e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev))) return e;
  }
  if (smem > configured_smem) {
    if ((e = cudaFuncSetAttribute((const void*)k_persistent_solve,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
      return e;
    configured_smem = smem;
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
  if ((e = cudaMemsetAsync(d_bar, 0, (4 + 4 * (size_t)ninst) * sizeof(unsigned), st)))
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
