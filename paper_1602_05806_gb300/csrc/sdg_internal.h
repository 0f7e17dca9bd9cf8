// Internal declarations shared by the CUDA translation units of libsdg.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/sdg.h"
#include "sdg_basis.h"

namespace sdg {

// Device-resident control block of one iterative solve.  Written only by
// the last block of a reducing kernel, read by every block of the next
// kernel on the same stream (kernel boundaries order the accesses).
struct SolverState {
  double rr;        // current ||r||^2 (recursive)
  double rr_old;    // previous ||r||^2
  double pAp;       // p^T A p of the current iteration
  double alpha;     // rr / pAp (set by the operator kernel's last block)
  double beta;      // rr / rr_old (set by the update kernel's last block)
  float alpha_f, beta_f;  // the same in FP32, read by every thread of FP32 kernels
  double bnorm2;    // ||b||^2
  double tol2;      // (rtol ||b||)^2
  double mean;      // mixed: mean of the FP64 residual (removed: periodic kernel)
  double sigma;     // mixed: FP32 vectors hold sigma * (FP64 quantities), sigma = 1/||b||
  double maxrr;     // mixed: largest recursive ||r||^2 since the last reliable update
  double delta2;    // mixed: reliable update when rr < delta2 * maxrr
  double red[4];    // results of plain reductions
  int iter;         // iterations done
  int maxit;
  int done;         // 1 once converged / failed / capped
  int status;       // sdg_status of this solve
  int reliable;     // 1: FP32 iterations pause for FP64 residual replacement
  int pause;        // set by the update kernel when a reliable update is due
  int updates;      // reliable updates done
  int xpend;        // two-launch form: 1 while x lacks alpha p of the last operator launch
                    // (the next operator launch adds it, or the CG loop when it returns)
  int nop;          // two-launch form: blocks of the last operator launch (their p.Ap totals
                    // wait in the partials for the update launch)
  unsigned int counter;  // last-block ticket counter (reset by the last block)
};

// Geometry of a field: element-major blocks of n1^dim nodes.
struct Geo {
  int dim, n1, npe;
  int n[3];
  long long ncell, ndof;
};

// Offsets (in doubles) of the 1D matrices inside the device matrix table;
// every matrix occupies kMaxN1*kMaxN1 slots, indexed [p*n1 + q].
enum MatId { kW = 0, kWinv, kPhi0, kPhi1, kM, kRt, kLt, kRb, kLb, kML, kMR, kHR, kHL, kHC, kDn, kNumMats };
constexpr int kMatStride = kMaxN1 * kMaxN1;
constexpr int kMatTable = kNumMats * kMatStride;

constexpr int kMaxStates = 8;
constexpr int kKernelBlocks = 512;     // grid of the per-local-node element sum
constexpr int kDeflateBlocks = 304;    // grid of the deflated FP32 CG update
constexpr int kPartialSlots = 4;       // doubles per block in a partials array
constexpr int kReduceBlocks = 152 * 8; // grid of the vector / reduction kernels

enum StateId { kStP64 = 0, kStP32 = 1, kStV64 = 2, kStV32 = 3, kStMisc = 4, kStTrue = 5 };

constexpr int kProfEvents = 64;  // event pairs per CG batch when profiling

}  // namespace sdg

struct sdg_handle {
  int device;
  int nsm;                       // streaming multiprocessors of the device
  sdg::Geo g;
  int dim;
  double L[3], dx[3];
  double nu, theta, dt;
  int nsub;                      // SSP-RK3 sub-steps of the explicit convection per dt
  int tile32;                    // tile shape variant of the 2D FP32 operator
  int form;                      // CG iteration form: 0 one launch, 1 / 2 operator + update launches
  int precision;
  double rtol_p, rtol_v;
  double delta;     // mixed: reliable-update factor
  int maxit, max_updates;
  sdg::Basis1D basis;
  sdg::CoefSet coef64, coef32;   // stored operator blocks per precision
  int deflate;                   // mixed: deflate the kernel in FP32 iterations
  int verbose;                   // SDG_VERBOSE=1: log every reliable update to stderr

  // state
  double* U[3];
  double* P;
  // step work
  double* Vm[3];    // main-grid velocity
  double* S1[3];    // RK stage 1
  double* S2[3];    // RK stage 2
  double* Lc[3];    // convection operator, accumulated over the directions
  double* F[3];     // RK3 result Fu
  double* Vh[3];    // viscous solution U^{n+1/2} on the main grid
  double* Us[3];    // U* on the dual grids
  double* b;        // right-hand side
  double* Pn;       // new pressure
  double* tmp;      // scratch field
  double* adj;      // adjoint work arena (allocated by the first sdg_step_adjoint)
  long long adj_fields;  // fields of ndof doubles in adj
  // solver vectors
  // p is double-buffered: the fused apply reads p_old with its halo while
  // other CTAs write p_new, so the two must not alias; with one launch per
  // iteration r and Ap are read with their halo too and alternate likewise
  // (r64 / r64b, Ap64 / Ap64b, r32 / r32b, Ap32 / Ap32b).
  double *r64, *r64b, *p64[2], *Ap64, *Ap64b;
  float *x32, *r32, *r32b, *p32[2], *Ap32, *Ap32b;
  sdg::SolverState* st;   // kMaxStates device states
  sdg::SolverState* st_host;  // pinned mirror
  double* partials;       // kMaxStates * max_blocks * kPartialSlots
  long long max_blocks;
  double* mats;           // device matrix table (kMatTable doubles)
  // kernel restoration of mixed pressure solves (see kernel_projector)
  double* x0buf;          // copy of x0 (ndof)
  double* kpart;          // per-block partial element sums (kKernelBlocks * npe)
  double* kcorr;          // correction pattern (npe)
  double* kproj;          // 1D kernel projector (n1 * n1)
  int kdim;               // dimension of the 1D kernel
  double* kbasis;         // local kernel patterns (kdim^dim x npe), orthonormal
  int kd;                 // kdim^dim
  float* kdpart;          // deflation partial sums (kDeflateBlocks * npe)
  float* kc;              // deflation correction pattern (npe)
  cudaEvent_t ev0, ev1, ev2, ev3;
  // instrumentation
  long long launches;     // kernels launched by this handle
  int profile;            // time every fused CG operator launch with events
  cudaEvent_t pev[2 * sdg::kProfEvents];
  double prof_ms[2];      // [0] FP64, [1] FP32 fused-apply device time
  long long prof_n[2];    // launches timed
};

namespace sdg {

// Record the text returned by sdg_last_error (this thread).
void set_last_error(const char* msg);

// ---- launchers (sdg_apply_*.cu) -------------------------------------------
// y = cmass * W x + sum_d s[d] M^{perp d} (H^L x_{i-1} + H^C x_i + H^R x_{i+1})_d
// If fuse != 0: the input is p = r + beta p_old (beta from `st`, p = r on the
// first iteration), p is written to p_out, and p^T y is reduced into
// st->pAp / st->alpha (the CG step-length); the kernel exits at once when
// st->done is set.
// Deflation of the kernel of the periodic pressure operator in the FP32
// iterations (odd N: the per-cell sawtooth patterns, which FP32 rounding of
// the stored blocks turns into spurious small eigenvalues).  The update kernel
// reduces per-local-node sums of the new residual, projects them on the
// orthonormal local kernel patterns and leaves in kc the kernel part of r
// (one value per local node, the same in every element); the next fused
// operator forms p from r - kc.
struct Deflate {
  float* kpart;          // per-block, per-local-node partial sums (grid * npe); null = off
  const double* kbasis;  // kd x npe orthonormal local kernel patterns
  float* kc;             // npe: kernel part of r per local node
  int npe, kd;
  long long ncell;
};

template <typename T>
struct ApplyArgs {
  const T* x;      // input (fuse = 0) or r (fuse = 1)
  const T* p_old;  // fuse = 1
  T* p_out;        // fuse = 1
  // fuse = 1 with xsol set: the operator launch of iteration k also adds
  // alpha_{k-1} p_{k-1} to xsol (state flag xpend), so that the update launch
  // reads and writes only r and Ap
  T* y;
  double s[3];
  double cmass;
  int fuse;
  SolverState* st;
  double* partials;
  const float* kc;  // fuse = 1, FP32: subtract kc (per local node) from r; null = off
  int accurate;     // FP64: use the accurate contraction (FP32 always does)
  int tile;         // 2D FP32: tile shape variant (0 base, 1 wide in x, 2 wide in y)
  int pdl;          // launch with programmatic stream serialisation (CG loop)
  // fuse = 2: one launch per CG iteration k.  x is r_{k-1}, p_old p_{k-1},
  // ap_old A p_{k-1}; the kernel writes r_k = r_{k-1} - alpha Ap_{k-1} to
  // r_out, adds alpha p_{k-1} to xsol, forms p_k = r_k + beta p_{k-1} (to
  // p_out) and Ap_k (to y), and reduces p.Ap, r.r, r.Ap, Ap.Ap into the state
  // (alpha_k, beta_{k+1}, stopping decisions).  Iteration 0 takes p_0 = r_0.
  const T* ap_old;
  T* r_out;
  T* xsol;
};

cudaError_t launch_apply_f64(const sdg_handle* h, const ApplyArgs<double>& a, cudaStream_t s);
cudaError_t launch_apply_f32(const sdg_handle* h, const ApplyArgs<float>& a, cudaStream_t s);

// per-(dim, n1) dispatch entry points, one per translation unit
cudaError_t apply_dispatch_2d(const sdg_handle* h, const ApplyArgs<double>& a, cudaStream_t s);
cudaError_t apply_dispatch_2d(const sdg_handle* h, const ApplyArgs<float>& a, cudaStream_t s);
cudaError_t apply_dispatch_3d(const sdg_handle* h, const ApplyArgs<double>& a, cudaStream_t s);
cudaError_t apply_dispatch_3d(const sdg_handle* h, const ApplyArgs<float>& a, cudaStream_t s);

// ---- vector / step kernels (sdg_kernels.cu) --------------------------------
// Update launch of a two-launch CG iteration: alpha from the operator
// blocks' p.Ap totals (slot kOpSlot of partials), r -= alpha Ap, r.r, and
// the iteration's decisions; x += alpha p too unless x is null (then the next
// operator launch adds it).  nsm: SMs of the device (grid of one wave).
cudaError_t cg_update_f64(double* x, double* r, const double* p, const double* Ap, long long n,
                          SolverState* st, double* partials, int nsm, cudaStream_t s);
cudaError_t cg_update_f32(float* x, float* r, const float* p, const float* Ap, long long n,
                          SolverState* st, double* partials, const Deflate& df, int nsm, cudaStream_t s);
// FP32 CG with FP64 reliable updates:
//   rel_accumulate: x64 += x32 / sigma, x32 = 0
//   rel_residual:   r64 = b - Ax (FP64), mean and ||r - mean|| reduced in FP64;
//                   the last block replaces the recursive residual norm by the
//                   true one (scaled by sigma^2) and decides convergence.  With
//                   init = 1 it also starts the solve (sigma = 1/||b||, or 1
//                   when unscaled = 1, iter = 0).  project = 1 removes the mean
//                   from the norm and from r64 (singular pressure system).
//   rel_convert:    r32 = sigma r64
cudaError_t rel_accumulate(double* x64, float* x32, long long n, const SolverState* st, cudaStream_t s);
// mode: 1 starts the solve; 2 replaces the residual of a running iteration
// (alpha and beta kept: the direction continues); 0 replaces it and
// restarts the direction from its norm (beta = r.r new / r.r old)
cudaError_t rel_residual(const double* b, const double* Ax, double* r64, long long n, SolverState* st,
                         double* partials, double rtol, int maxit, double delta, int mode, int project,
                         int unscaled, cudaStream_t s);
cudaError_t rel_convert(const double* r64, float* r32, long long n, const SolverState* st, cudaStream_t s);
// st->red[0..2] = sum(r), sum(r^2), sum(b^2) of r = b - Ax (b may be NULL:
// zero; nothing written but the state): the true residual of a finished solve
cudaError_t resid_norms(const double* b, const double* Ax, long long n, SolverState* st, double* partials,
                        cudaStream_t s);
// u_i = s_i ulp(x_i) / (2 sqrt 3), s_i = +-1 from a hash of i: the spread of
// rounding x to FP64, whose image under the operator estimates the residual
// floor of FP64 solutions
cudaError_t rounding_perturbation(const double* x, double* u, long long n, cudaStream_t s);
// After the range projection of a replaced residual r (singular system):
// rr = sigma^2 ||r||^2 and the stopping / direction decisions of
// rel_residual (same mode) taken again on it
cudaError_t rel_renorm(const double* r, long long n, SolverState* st, double* partials, int mode, cudaStream_t s);
// x += alpha p (state's alpha): the pending update of a one-launch CG
// iteration stopped at maxit
cudaError_t pending_update(double* x, const double* p, long long n, const SolverState* st, cudaStream_t s);
cudaError_t pending_update(float* x, const float* p, long long n, const SolverState* st, cudaStream_t s);
// x += alpha p if the state's xpend is set (the two-launch form's last step
// when its CG loop returns), then xpend = 0
cudaError_t pending_x(double* x, const double* p, long long n, SolverState* st, cudaStream_t s);
cudaError_t pending_x(float* x, const float* p, long long n, SolverState* st, cudaStream_t s);

// Restore the component of x in the kernel of the periodic pressure operator
// to that of x0: c = (1/ncell) (P1 (x) ... (x) P1) sum_e (x - x0)[e], then
// x[e] -= c for every element (P1: 1D kernel projector, kproj).  x0 = NULL
// removes the kernel component of x (projection onto the range).
cudaError_t kernel_restore(const sdg_handle* h, double* x, const double* x0, cudaStream_t s, int* launches);

// step stages
cudaError_t k_dual_to_main(const sdg_handle* h, int d, const double* in, double* out, cudaStream_t s);
cudaError_t k_main_to_dual(const sdg_handle* h, int d, const double* in, double* out, cudaStream_t s);
// out_c = a * V0_c + b * (V_c + dt L(V)_c) for every component c (out may
// alias V0, not V); one launch per direction, L accumulated in h->Lc
cudaError_t k_convect_stage(const sdg_handle* h, const double* const* V0, const double* const* V,
                            double* const* out, double a, double b, double dt, cudaStream_t s);
// b = W F, x0 = F
cudaError_t k_mass_rhs(const sdg_handle* h, const double* F, double* b, double* x0, cudaStream_t s);
// out = base + scale * sum_d (1/dx_d) M^{perp d} (Rb U_d - Lb U_d,shift)  ; reduces sum(out) into st->red[0]
cudaError_t k_divergence(const sdg_handle* h, const double* const* U, const double* base, double scale,
                         double* out, SolverState* st, double* partials, cudaStream_t s);
// x -= st->red[slot] * factor
cudaError_t k_shift(double* x, long long n, const SolverState* st, int slot, double factor, cudaStream_t s);
cudaError_t k_velocity_update(const sdg_handle* h, const double* const* Ustar, const double* Pn,
                              const double* Po, double* const* U, cudaStream_t s);
// st->red[slot] = sum W x (y == NULL) or sum W x y
cudaError_t k_weighted_sum(const sdg_handle* h, const double* x, const double* y, SolverState* st,
                           int slot, double* partials, cudaStream_t s);
// st->red[slot] = sum x*x
cudaError_t k_norm2(const double* x, long long n, SolverState* st, int slot, double* partials, cudaStream_t s);

// adjoint of the step (transposed stages, FP64)
cudaError_t adj_project_T(const sdg_handle* h, bool dual_to_main, int d, const double* lam, double* out,
                          cudaStream_t s);
cudaError_t adj_velocity_T(const sdg_handle* h, const double* const* lamU, const double* lamP, double* lx,
                           double* lPo, cudaStream_t s);
cudaError_t adj_divergence_T(const sdg_handle* h, const double* const* lamU, const double* lb, double* const* out,
                             cudaStream_t s);
cudaError_t adj_convect_T(const sdg_handle* h, const double* const* X, const double* const* lam,
                          const double* const* base, double* const* out, double a, double b, double k,
                          cudaStream_t s);
cudaError_t adj_axpby(double* out, double a, const double* x, double b, const double* y, long long n,
                      cudaStream_t s);
cudaError_t adj_dot(const double* x, const double* y, long long n, SolverState* st, int slot, double* partials,
                    cudaStream_t s);
cudaError_t adj_sub_weighted(const sdg_handle* h, double* x, const SolverState* st, int slot, double factor,
                             cudaStream_t s);

}  // namespace sdg
