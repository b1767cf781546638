// Descriptors of the persistent GMRES solver (k_solver.cu).
#pragma once

#include "ibdl_internal.cuh"

namespace ibdl {

constexpr int kSolverThreads = 256;  // threads per block; also the vector chunk
constexpr int kMaxBatch = 512;       // instances per persistent launch
constexpr int kSingleMax = 4096;     // points up to which one block does the vector work
constexpr int kSingleMinBatch = 8;   // ... when at least this many instances share a launch
// Largest launch whose float64-grade matvecs transform in double-float: in a
// few-instance launch they sit on the critical path and the float64 pipe's
// latency dominates; a saturated batch is bound by issue slots, where
// double-float's extra float32 instructions cost more than they save.
constexpr int kDdMaxBatch = 16;
// Scheduler words per instance in the solver's barrier buffer (4 + this many
// per instance, 32-bit words): claim counter, done counter, phase descriptor.
constexpr int kSchedWords = 12;

enum SolveAction {
  ACT_DONE = 0,
  ACT_RESID_ZERO = 1,   // r = b (x = 0)
  ACT_MV_RESIDUAL = 2,  // r = b - A64 x
  ACT_MV_ARNOLDI = 3,   // Arnoldi step j
  ACT_FINISH = 4,       // back substitution, x += V y
  ACT_RHS = 5,          // Neumann right-hand side b = -kappa S* L'^{-1} S V_b
  ACT_MV_UPDATE = 6     // r -= A32 d, d = V y the last correction (refined solves)
};

// Bound on the float32 operator's error relative to its argument,
// ||A32 v - A v|| <= kF32OpErr ||v||, used to bound the error of a residual
// updated by a float32 matvec of the last correction (ACT_MV_UPDATE).  The
// parity tests hold every float32 matvec within 1e-5 of the float64 oracle
// (2-norm and element-wise); measured on GB300: 0.6e-8 - 6e-8 (C1, C2, C3).
constexpr double kF32OpErr = 1e-5;

// Read-only during a launch.
struct SolveInst {
  GridDesc g;
  PointData p;
  Bins b;
  SpectralWs<double> w64;
  SpectralWs<float> w32;
  SpectralWs<dd> wdd;  // double-float view of w64's buffers
  int dd64;            // 1: the float64-grade matvecs transform in double-float
  double* V;        // (restart + 1) x ld
  int ld;
  int restart;
  double* H;        // column j at H + j * (restart + 1)
  double* cs;
  double* sn;
  double* gv;       // restart + 1
  double* ysol;     // restart
  double* part;     // partial sums: three sections of nsec x pstride
  int nchunk;
  int pstride;
  int nsec;         // rows per section: max(nchunk, the 2D x tiles)
  // 2D Arnoldi steps that interpolate in their x-inverse tiles (no phase D;
  // their first dot products come as per-tile partial sums): 0 none, 1 the
  // float32 steps, 2 all steps
  int fuse_interp;
  double* bvec;         // right-hand side (written by ACT_RHS)
  const double* vdata;  // V_b for ACT_RHS
  // 1 (float32-refined Neumann solves whose right-hand side the solver
  // builds): ACT_RHS runs in float32 and gives only the inner solves' first
  // right-hand side; every float64-grade residual spreads S~ x + S V_b into
  // one Helmholtz solve, r = -(S* kappa L'^{-1} (S~ x + S V_b) - x / 2)
  // = b - A x, so b itself is never needed to float64 accuracy
  int rhs_resid;
  // 1: ACT_RHS is followed by RESID_ZERO (x = 0); its phase D also writes
  // r = b and the partial sums of ||r||^2, ||b||^2, and RESID_ZERO starts at E
  int rhs_r0;
  // 1 (float32-refined solves): after an inner solve whose correction d is
  // small, the residual is updated, r <- r - A32 d (ACT_MV_UPDATE), instead
  // of recomputed with a float64-grade matvec; its error grows by at most
  // kF32OpErr ||d|| (SolveState::rerr), which is allowed up to a tenth of
  // the tolerance and counted against it
  int upd_resid;
  double* dvec;         // the last inner solve's correction d = V y
  // 1: float32 Arnoldi steps that interpolate in phase D orthogonalise in
  // one classical Gram-Schmidt pass, the new norm by Pythagoras from the
  // same reduction (phases D and E; float64 steps keep two passes)
  int cgs1;
  double* x;
  double* r;
  int bc;
  int refined;
  int maxit;
  int max_refine;
  double tol;
  double inner_tol;
  double* hist;
  int hist_cap;
  int single;       // 1: all vector work of a round on one block (m <= kSingleMax)
  // work items of matvec phase 0..4 in the float64-grade (float64 or
  // double-float, [.][0]) and float32 ([.][1]) operator; filled on the host
  // (solver_fill_items), so that a phase hand-off reads them
  int mv_nitems[5][2];
};

// Mutable; written by the instance's control thread.
struct SolveState {
  int action, prec, j, kdim;
  int iters, outer, status, matvecs;
  int nhist, xinit;  // xinit: the solve starts from a caller-given x
  int nupd;          // residuals updated by a float32 matvec (ACT_MV_UPDATE)
  double beta, bnorm, tol_abs, rel;
  // bound on ||r - (b - A x)|| of the stored residual r: 0 after a
  // float64-grade residual, + kF32OpErr ||d|| per update, infinite while r
  // is a right-hand side built in float32
  double rerr;
};

int solver_smem_bytes(const GridDesc& g, int rows, int need32);
// Fills I.mv_nitems from the instance's grid, tiling and element types.
void solver_fill_items(SolveInst& I);
// Dynamic shared memory of one matvec work item per kind (row tile, pencil
// layouts) for element type elem (0 float64, 1 float32, 2 double-float).
void solver_item_smem(const GridDesc& g, int rows, int elem, size_t out[3]);
// True when every item of every instance fits in `smem` bytes; else a
// message in why.
bool solver_smem_fits(const SolveInst* h_insts, int ninst, int smem, char* why, size_t why_len);
// One block joins a two-party barrier: its bounded wait gives up after
// `limit` polls and sets bar[2] (bar: 4 zeroed words).
cudaError_t launch_barrier_selftest(unsigned* bar, unsigned limit, cudaStream_t st);
// max_rounds > 0 stops the launch after that many rounds (states persist for
// the next launch); reserve_sms SMs are left without solver blocks.
cudaError_t launch_persistent_solve(const SolveInst* d_insts, SolveState* d_states, int ninst,
                                    unsigned* d_bar, int smem, cudaStream_t st,
                                    int max_rounds = 0, int reserve_sms = 0);

}  // namespace ibdl
