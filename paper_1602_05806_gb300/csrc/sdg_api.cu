// C ABI of libsdg: handle life cycle, operators, CG drivers (FP64 and
// FP32-inner / FP64-refined) and the fractional time step of Sec. 2.3.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sdg_internal.h"

using namespace sdg;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, const char* a = "", int line = 0) {
  std::snprintf(g_err, sizeof(g_err), fmt, a, line);
}

#define SDG_CK(call)                                                         \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_err("CUDA error %s at sdg_api.cu:%d", cudaGetErrorString(e_), __LINE__); \
      return SDG_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

#define SDG_ARG(cond, msg)             \
  do {                                 \
    if (!(cond)) {                     \
      set_err("invalid argument: %s", msg); \
      return SDG_ERR_INVALID_ARG;      \
    }                                  \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline SolverState* st_dev(sdg_handle* h, int id) { return h->st + id; }
inline double* parts(sdg_handle* h, int id) {
  return h->partials + (size_t)id * (size_t)h->max_blocks * kPartialSlots;
}

struct Op {
  double s[3];
  double cmass;
};

Op pressure_op(const sdg_handle* h) {
  Op o{};
  for (int d = 0; d < h->dim; ++d) o.s[d] = h->theta * h->dt / (h->dx[d] * h->dx[d]);
  o.cmass = 0.0;
  return o;
}

Op viscous_op(const sdg_handle* h) {
  Op o{};
  for (int d = 0; d < h->dim; ++d) o.s[d] = h->nu * h->dt / (h->dx[d] * h->dx[d]);
  o.cmass = 1.0;
  return o;
}

}  // namespace

namespace sdg {

void set_last_error(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

cudaError_t launch_apply_f64(const sdg_handle* h, const ApplyArgs<double>& a, cudaStream_t s) {
  return h->dim == 2 ? apply_dispatch_2d(h, a, s) : apply_dispatch_3d(h, a, s);
}
cudaError_t launch_apply_f32(const sdg_handle* h, const ApplyArgs<float>& a, cudaStream_t s) {
  return h->dim == 2 ? apply_dispatch_2d(h, a, s) : apply_dispatch_3d(h, a, s);
}

}  // namespace sdg

extern "C" const char* sdg_strerror(int status);

namespace {

template <typename T>
cudaError_t apply_plain(const sdg_handle* h, const Op& op, const T* x, T* y, cudaStream_t s,
                        int accurate = 0) {
  ApplyArgs<T> a{};
  a.accurate = accurate;
  a.x = x;
  a.y = y;
  for (int d = 0; d < 3; ++d) a.s[d] = op.s[d];
  a.cmass = op.cmass;
  a.fuse = 0;
  a.tile = h->tile32;
  if constexpr (sizeof(T) == 8)
    return launch_apply_f64(h, a, s);
  else
    return launch_apply_f32(h, a, s);
}

#define SDG_K(call)     \
  do {                  \
    ++h->launches;      \
    SDG_CK(call);       \
  } while (0)

// Host loop of one CG solve in precision T on vectors x (in/out), r, p[2], Ap.
// fused: one launch per iteration (r[2] and Ap[2] alternate with the
// iteration like p: iteration j reads r[j&1], p[j&1], Ap[j&1] and writes the
// other three, so after j iterations the current residual is r[j&1]);
// otherwise the operator launch and the update launch of a two-launch form
// (r[0], Ap[0]; the kernel deflation of the FP32 iteration runs in the
// update launch).  Form 2 (default): the operator launch of iteration k adds
// alpha_{k-1} p_{k-1} to x, so the update launch moves only r and Ap, and the
// last step's alpha p is added when the loop returns; form 1: the update
// launch adds alpha p to x.
// Convergence (and, in reliable mode, the need for an FP64 residual
// replacement) is decided on the device; the host reads the state after each
// batch of iterations.  Returns with h->st_host[sid] current.
template <typename T>
int cg_loop(sdg_handle* h, const Op& op, T* x, T* const* r, T* const* p, T* const* Ap, int sid, cudaStream_t s,
            bool fused, bool deflate = false, long long segment_cap = 0) {
  const int iter_start = h->st_host[sid].iter;
  Deflate df{};
  if (deflate) {
    df.kpart = h->kdpart;
    df.kbasis = h->kbasis;
    df.kc = h->kc;
    df.npe = h->g.npe;
    df.kd = h->kd;
    df.ncell = h->g.ncell;
  }
  SolverState* st = st_dev(h, sid);
  double* pa = parts(h, sid);
  const long long n = h->g.ndof;
  // two-launch forms: x += alpha p in the operator launch (form 2) or in the
  // update launch (form 1, and always with the FP32 kernel deflation)
  const bool xop = !fused && h->form == 2 && !deflate;
  // buffers alternate with the executed iteration; launches skipped after a
  // pause or convergence do not count, so j restarts from the device count
  long long launched = h->st_host[sid].iter;
  int batch = 4;
  const int pk = sizeof(T) == 8 ? 0 : 1;
  int iter_before = h->st_host[sid].iter;
  long long batches_run = 0;
  for (;;) {
    const bool prof = h->profile != 0;
    const int nb = prof && batch > kProfEvents ? kProfEvents : batch;
    for (int k = 0; k < nb; ++k) {
      const int j0 = (int)(launched & 1), j1 = (int)((launched + 1) & 1);
      ApplyArgs<T> a{};
      a.p_old = p[j0];
      a.p_out = p[j1];
      for (int d = 0; d < 3; ++d) a.s[d] = op.s[d];
      a.cmass = op.cmass;
      a.st = st;
      a.partials = pa;
      a.tile = h->tile32;
      a.accurate = 1;  // FP64: kernel-exact contraction (FP32 always uses it)
      a.pdl = prof ? 0 : 1;
      if (fused) {
        a.fuse = 2;
        a.x = r[j0];
        a.r_out = r[j1];
        a.ap_old = Ap[j0];
        a.y = Ap[j1];
        a.xsol = x;
      } else {
        // the operator launch also adds the previous step alpha p to x
        a.fuse = 1;
        a.x = r[0];
        a.y = Ap[0];
        a.xsol = xop ? x : nullptr;
        a.kc = deflate ? h->kc : nullptr;
      }
      if (prof) SDG_CK(cudaEventRecord(h->pev[2 * k], s));
      if constexpr (sizeof(T) == 8) {
        SDG_K(launch_apply_f64(h, a, s));
        if (prof) SDG_CK(cudaEventRecord(h->pev[2 * k + 1], s));
        if (!fused) SDG_K(cg_update_f64(xop ? nullptr : x, r[0], p[j1], Ap[0], n, st, pa, h->nsm, s));
      } else {
        SDG_K(launch_apply_f32(h, a, s));
        if (prof) SDG_CK(cudaEventRecord(h->pev[2 * k + 1], s));
        if (!fused) SDG_K(cg_update_f32(xop ? nullptr : x, r[0], p[j1], Ap[0], n, st, pa, df, h->nsm, s));
      }
      ++launched;
    }
    SDG_CK(cudaMemcpyAsync(h->st_host + sid, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    SDG_CK(cudaStreamSynchronize(s));
    const SolverState& hs = h->st_host[sid];
    if (prof) {
      // the operator ran in iterations iter_before .. hs.iter-1 of this batch
      const int ran = hs.iter - iter_before;
      for (int k = 0; k < ran && k < nb; ++k) {
        float ms = 0.f;
        SDG_CK(cudaEventElapsedTime(&ms, h->pev[2 * k], h->pev[2 * k + 1]));
        h->prof_ms[pk] += ms;
        h->prof_n[pk] += 1;
      }
    }
    iter_before = hs.iter;
    launched = hs.iter;
    if (hs.done || hs.pause) break;
    if (++batches_run > (long long)h->maxit / 4 + 64) {  // the device caps at maxit; never spin past it
      set_err("CG host loop ran past maxit without a device stop%s", "");
      return SDG_ERR_CUDA;
    }
    if (segment_cap > 0 && hs.iter - iter_start >= segment_cap) break;  // caller replaces the residual
    if (batch < 32) batch *= 2;
  }
  if (xop) {
    // the last operator launch (iteration iter - 1) wrote p[iter & 1]; its
    // alpha p is still to be added to x (no-op after a breakdown: alpha 0)
    SDG_K(pending_x(x, p[h->st_host[sid].iter & 1], n, st, s));
    h->st_host[sid].xpend = 0;
  }
  return SDG_OK;
}

void fill_info(sdg_cg_info* info, const SolverState& hs, int outer, int a64, int a32, int status,
               double true_res, double floor_res, double eval_res) {
  if (status != SDG_OK) {
    std::snprintf(g_err, sizeof(g_err),
                  "%s: iter %d, true ||r||/||b|| %.3e, floor %.3e, eval %.3e, rr %.3e, rr_old %.3e, pAp %.3e, "
                  "tol2 %.3e, updates %d",
                  sdg_strerror(status), hs.iter, true_res, floor_res, eval_res, hs.rr, hs.rr_old, hs.pAp, hs.tol2,
                  hs.updates);
  }
  if (!info) return;
  info->iters = hs.iter;
  info->outer_iters = outer;
  info->applies_fp64 = a64;
  info->applies_fp32 = a32;
  // the state keeps rr scaled by sigma^2 (sigma = 1/||b|| for FP32 iterations, 1 for FP64)
  info->rel_res = hs.bnorm2 == 0.0 ? 0.0 : std::sqrt(hs.rr) / (hs.sigma * std::sqrt(hs.bnorm2));
  info->status = status;
  info->true_res = true_res;
  info->floor_res = floor_res;
  info->eval_res = eval_res;
}

// Residual floor of FP64 solutions near x, relative to ||b|| (bnorm2 =
// ||b||^2): ||A u|| / ||b|| for u = random-sign ulp(x) / (2 sqrt 3) (the
// spread of rounding x to FP64), with the accurate FP64 operator.  Uses
// h->tmp and Ap64.
int floor_residual(sdg_handle* h, const Op& op, const double* x, double bnorm2, bool singular, cudaStream_t s,
                   double* out) {
  const long long n = h->g.ndof;
  SDG_K(rounding_perturbation(x, h->tmp, n, s));
  SDG_K(apply_plain<double>(h, op, h->tmp, h->Ap64, s, 1));
  SDG_K(resid_norms(nullptr, h->Ap64, n, st_dev(h, kStTrue), parts(h, kStTrue), s));
  SDG_CK(cudaMemcpyAsync(h->st_host + kStTrue, st_dev(h, kStTrue), sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SDG_CK(cudaStreamSynchronize(s));
  const SolverState& t = h->st_host[kStTrue];
  const double mean = singular ? t.red[0] / (double)n : 0.0;
  double rr = t.red[1] - (double)n * mean * mean;
  if (rr < 0.0) rr = 0.0;
  *out = bnorm2 > 0.0 ? std::sqrt(rr / bnorm2) : 0.0;
  return SDG_OK;
}

// Rounding of A x itself, relative to ||b||: ||A x - A~ x|| / ||b|| for the
// accurate (A) and the direct (A~) FP64 contraction, the same operator in
// exact arithmetic.  Uses h->tmp and Ap64.
int eval_residual(sdg_handle* h, const Op& op, const double* x, double bnorm2, cudaStream_t s, double* out) {
  const long long n = h->g.ndof;
  SDG_K(apply_plain<double>(h, op, x, h->tmp, s, 1));
  SDG_K(apply_plain<double>(h, op, x, h->Ap64, s, 0));
  SDG_K(resid_norms(h->tmp, h->Ap64, n, st_dev(h, kStTrue), parts(h, kStTrue), s));
  SDG_CK(cudaMemcpyAsync(h->st_host + kStTrue, st_dev(h, kStTrue), sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SDG_CK(cudaStreamSynchronize(s));
  const double rr = h->st_host[kStTrue].red[1];
  *out = bnorm2 > 0.0 ? std::sqrt((rr > 0.0 ? rr : 0.0) / bnorm2) : 0.0;
  return SDG_OK;
}

// CG with reliable updates (residual replacement that keeps the Krylov
// direction), in FP64 (fp32 = false) or with FP32 iterations (fp32 = true).
//   FP64:  the iteration updates x and r in FP64; whenever the recursive
//          residual has dropped by `delta` since the last replacement (or
//          reached the tolerance) the true residual b - A x is recomputed in
//          FP64 and replaces it.  Without the replacements the recursive
//          residual of a long FP64 CG drifts from the true one (on 256^2
//          cells at N = 7: true 7e-10 when the recursion reports 1e-12) and
//          the iteration diverges once it is asked for less.
//   FP32:  the iteration runs on the sigma-scaled residual in FP32 and
//          accumulates its correction in x32; at each replacement the
//          correction is folded into the FP64 x first.
// Converged when the true residual satisfies ||b - A x|| <= tol ||b|| with
// tol = max(rtol, 3 floor), floor the residual that rounding the starting
// vector to FP64 leaves (floor_residual): no FP64 vector has a smaller one
// (the solves measured here level off at 2.2-2.3 times it), or when the
// true residual stops improving within 10 floor (evaluation error of A x).
// The FP32 iteration is replaced whenever its residual has dropped by delta
// (or after a segment cap); the FP64 one only when its recursion reports the
// tolerance: its recursive residual stays accurate far longer, and frequent
// replacements cost it more conjugacy than they save.  For the singular
// pressure system every replaced residual is projected onto the range of the
// operator (its kernel part is round-off of b and of A x, which no iteration
// can reduce and which, left in, ends near-kernel directions in breakdown).
int solve_reliable(sdg_handle* h, const Op& op, const double* b, double* x, double rtol, int sid,
                   sdg_cg_info* info, cudaStream_t s, bool singular, bool fp32, int sid64 = -1) {
  const long long n = h->g.ndof;
  // deflate the kernel in the FP32 iterations when it is more than the
  // constants (the constants are annihilated exactly by the operator kernel)
  const bool deflate = fp32 && singular && h->kd > 1 && h->deflate;
  SolverState* st = st_dev(h, sid);
  double* pa = parts(h, sid);
  const double delta = h->delta;
  const int unscaled = fp32 ? 0 : 1;
  // one launch per iteration unless asked otherwise or the FP32 iteration
  // deflates the kernel
  const bool fused = !deflate && h->form == 0;
  double* r64v[2] = {h->r64, fused ? h->r64b : h->r64};
  double* Ap64v[2] = {h->Ap64, fused ? h->Ap64b : h->Ap64};
  float* r32v[2] = {h->r32, fused ? h->r32b : h->r32};
  float* Ap32v[2] = {h->Ap32, fused ? h->Ap32b : h->Ap32};
  int a64 = 0, updates = 0;
  if (singular) SDG_CK(cudaMemcpyAsync(h->x0buf, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // start: r = b - A x0 (x32 = 0)
  if (fp32) SDG_CK(cudaMemsetAsync(h->x32, 0, n * sizeof(float), s));
  SDG_K(apply_plain<double>(h, op, x, h->Ap64, s, 1));
  ++a64;
  SDG_K(rel_residual(b, h->Ap64, h->r64, n, st, pa, rtol, h->maxit, fp32 ? delta : 0.0, 1, singular, unscaled, s));
  if (singular) {
    int nl = 0;
    SDG_CK(kernel_restore(h, h->r64, nullptr, s, &nl));
    h->launches += nl;
    SDG_K(rel_renorm(h->r64, n, st, pa, 1, s));
  }
  SDG_CK(cudaMemcpyAsync(h->st_host + sid, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SDG_CK(cudaStreamSynchronize(s));
  // the reachable tolerance: three times the FP64 residual floor near x0
  double floor_res = 0.0;
  if (!h->st_host[sid].done) {
    const int rc = floor_residual(h, op, x, h->st_host[sid].bnorm2, singular, s, &floor_res);
    if (rc != SDG_OK) return rc;
    ++a64;
    if (3.0 * floor_res > rtol) {
      SolverState& hs = h->st_host[sid];
      const double tol = 3.0 * floor_res;
      hs.tol2 = tol * tol * hs.bnorm2 * hs.sigma * hs.sigma;
      if (hs.rr <= hs.tol2) hs.done = 1;
      SDG_CK(cudaMemcpyAsync(st, h->st_host + sid, sizeof(SolverState), cudaMemcpyHostToDevice, s));
    }
  }
  if (fp32) SDG_K(rel_convert(h->r64, h->r32, n, st, s));
  h->st_host[sid].iter = 0;
  int status = SDG_OK;
  // FP32 iterations: the replacement factor adapts to the segment lengths.
  // A replacement costs an FP64 operator application (about ten FP32
  // iterations on GB300); where the residual halves within a few
  // iterations (short solves, e.g. 3D at N = 4: about 435 iterations for
  // 12 decades) delta is squared until segments last kMinSeg iterations, and
  // it returns toward the configured value where they run long.
  constexpr int kMinSeg = 64;
  double delta_cur = delta;
  int it_last = 0;
  bool stalled = false;  // FP32 iterations stopped improving above the tolerance
  double eval_res = 0.0;  // rounding of A x itself (computed when the residual stalls)
  double best = -1.0;   // best true residual so far
  int stagnant = 0;     // consecutive replacements without a 1.25x improvement of it
  for (;;) {
    SDG_CK(cudaMemcpyAsync(h->st_host + sid, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    SDG_CK(cudaStreamSynchronize(s));
    if (h->st_host[sid].done) break;
    {
      // a true residual that has stopped improving long before reaching the
      // tolerance (evaluation error above the representation floor): give up
      const double cur = std::sqrt(h->st_host[sid].rr);
      if (best < 0.0 || cur < 0.8 * best) stagnant = 0; else ++stagnant;
      if (best < 0.0 || cur < best) best = cur;
      if (stagnant >= (fp32 ? 30 : 2)) {
        // A x is itself evaluated in FP64, so the true residual can level
        // off a few times above the representation floor (estimated again
        // at the current x): within 10x of it the solve has the accuracy
        // FP64 allows
        int rc = floor_residual(h, op, x, h->st_host[sid].bnorm2, singular, s, &floor_res);
        if (rc == SDG_OK) rc = eval_residual(h, op, x, h->st_host[sid].bnorm2, s, &eval_res);
        if (rc != SDG_OK) return rc;
        a64 += 3;
        const double rel = cur / (h->st_host[sid].sigma * std::sqrt(h->st_host[sid].bnorm2));
        status = rel <= 10.0 * std::max(floor_res, eval_res) ? SDG_OK : SDG_ERR_NOT_CONVERGED;
        stalled = status != SDG_OK;
        break;
      }
    }
    if (fp32 && updates > 0) {
      const int seg = h->st_host[sid].iter - it_last;
      double d = delta_cur;
      if (seg < kMinSeg) d = std::max(d * d, 1e-4);
      else if (seg > 4 * kMinSeg) d = std::min(std::sqrt(d), delta);
      if (d != delta_cur) {
        delta_cur = d;
        h->st_host[sid].delta2 = d * d;
        SDG_CK(cudaMemcpyAsync(&st->delta2, &h->st_host[sid].delta2, sizeof(double), cudaMemcpyHostToDevice, s));
      }
    }
    it_last = h->st_host[sid].iter;
    // the FP32 residual comes from the FP64 one: its kernel part is round-off
    if (deflate) SDG_CK(cudaMemsetAsync(h->kc, 0, h->g.npe * sizeof(float), s));
    // a segment that runs long without the residual dropping by delta is cut
    // short so that the true residual is checked
    const long long it_now = h->st_host[sid].iter;
    // (FP64: a segment may at most double the iteration count, FP32: 1/8)
    const long long cap = !fp32 ? (it_now > 5000 ? it_now : 5000) : (it_now / 8 > 2000 ? it_now / 8 : 2000);
    int rc = fp32 ? cg_loop<float>(h, op, h->x32, r32v, h->p32, Ap32v, sid, s, fused, deflate, cap)
                  : cg_loop<double>(h, op, x, r64v, h->p64, Ap64v, sid, s, fused, false, cap);
    if (rc != SDG_OK) return rc;
    const SolverState hs = h->st_host[sid];
    // replace the residual (also after a cap or a breakdown, so that x and
    // the reported residual are current): the current residual buffer is
    // r[iter & 1]; A x goes to tmp (Ap[iter & 1] holds A p of the last
    // iteration, which the next one-launch iteration reads)
    const int cur = fused ? (hs.iter & 1) : 0;
    // stopped at maxit: the one-launch form has not yet applied the last
    // step x += alpha p (the next iteration would), so apply it here
    if (fused && hs.done && hs.status == SDG_ERR_NOT_CONVERGED) {
      if (fp32) SDG_K(pending_update(h->x32, h->p32[cur], n, st, s));
      else SDG_K(pending_update(x, h->p64[cur], n, st, s));
    }
    if (fp32) SDG_K(rel_accumulate(x, h->x32, n, st, s));
    SDG_K(apply_plain<double>(h, op, x, h->tmp, s, 1));
    ++a64;
    double* rdst = fp32 ? h->r64 : r64v[cur];
    // the direction continues with the recursion's alpha and beta (measured
    // on 256 x 256, N = 7, FP32: 30,000 iterations, against 40,100 when the
    // direction restarts from the replaced norm, beta = r.r true / r.r old)
    const int mode = 2;
    SDG_K(rel_residual(b, h->tmp, rdst, n, st, pa, rtol, h->maxit, fp32 ? delta : 0.0, mode, singular, unscaled,
                       s));
    if (singular) {
      int nl = 0;
      SDG_CK(kernel_restore(h, rdst, nullptr, s, &nl));
      h->launches += nl;
      SDG_K(rel_renorm(rdst, n, st, pa, mode, s));
    }
    ++updates;
    if (h->verbose) {
      SDG_CK(cudaMemcpyAsync(h->st_host + sid, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      SDG_CK(cudaStreamSynchronize(s));
      const SolverState& v = h->st_host[sid];
      std::fprintf(stderr, "sdg: reliable update %d at %s iteration %d: true ||r||/||b|| = %.3e\n", updates,
                   fp32 ? "FP32" : "FP64", v.iter, std::sqrt(v.rr) / (v.sigma * std::sqrt(v.bnorm2)));
    }
    if (hs.done || updates >= h->max_updates) {
      // the iteration hit maxit or broke down, or the update cap is
      // reached: report the true residual of the final x
      SDG_CK(cudaMemcpyAsync(h->st_host + sid, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      SDG_CK(cudaStreamSynchronize(s));
      const SolverState& f = h->st_host[sid];
      status = f.rr <= f.tol2 ? SDG_OK : (hs.done ? hs.status : SDG_ERR_NOT_CONVERGED);
      if (status == SDG_OK && hs.status != SDG_OK && f.rr > f.tol2) status = hs.status;
      break;
    }
    if (fp32) SDG_K(rel_convert(h->r64, r32v[cur], n, st, s));
  }
  // CG in exact arithmetic never changes the kernel component of x (every
  // update lies in the range of the operator); rounding does, so put it back
  // to that of x0 (Sec. 2.1: P is defined up to weak solutions of grad p = 0)
  if (singular) {
    int nl = 0;
    SDG_CK(kernel_restore(h, x, h->x0buf, s, &nl));
    h->launches += nl;
  }
  const SolverState& hs = h->st_host[sid];
  if (status == SDG_OK && hs.done) status = hs.status;
  // the state's residual is the true FP64 one of the final x
  const double tr = hs.bnorm2 > 0.0 ? std::sqrt(hs.rr) / (hs.sigma * std::sqrt(hs.bnorm2)) : 0.0;
  if (fp32 && stalled && sid64 >= 0) {
    // the FP32 iterations cannot resolve what is left (for odd N, smoothly
    // modulated kernel patterns with tiny eigenvalues that FP32 rounding of
    // the operator blurs): finish with FP64 iterations from the current x
    // (a budget of 1/8 of the FP32 iterations: where the FP32 iterations
    // only crawled, FP64 ones crawl too)
    const int it32 = hs.iter;
    sdg_cg_info i64{};
    const int maxit_saved = h->maxit;
    h->maxit = std::min(maxit_saved, std::max(2000, it32 / 8));
    const int st64 = solve_reliable(h, op, b, x, rtol, sid64, &i64, s, singular, false);
    h->maxit = maxit_saved;
    if (st64 == SDG_ERR_CUDA || st64 == SDG_ERR_INVALID_ARG) return st64;
    if (info) {
      *info = i64;
      info->iters = it32;
      info->outer_iters = updates + i64.outer_iters;
      info->applies_fp64 = a64 + i64.applies_fp64;
      info->applies_fp32 = it32;
    }
    return st64;
  }
  fill_info(info, hs, updates, fp32 ? a64 : a64 + hs.iter, fp32 ? hs.iter : 0, status, tr, floor_res, eval_res);
  return status;
}

int solve(sdg_handle* h, bool pressure, const double* b, double* x, sdg_cg_info* info, cudaStream_t s) {
  const Op op = pressure ? pressure_op(h) : viscous_op(h);
  const double rtol = pressure ? h->rtol_p : h->rtol_v;
  const bool fp32 = h->precision == SDG_MIXED;
  const int sid64 = pressure ? kStP64 : kStV64;
  return solve_reliable(h, op, b, x, rtol, fp32 ? (pressure ? kStP32 : kStV32) : sid64, info, s, pressure, fp32,
                        sid64);
}

int pressure_rhs(sdg_handle* h, const double* const* Us, const double* Pold, double* b, cudaStream_t s) {
  Op op{};
  for (int d = 0; d < h->dim; ++d) op.s[d] = -(1.0 - h->theta) * h->dt / (h->dx[d] * h->dx[d]);
  SDG_K(apply_plain<double>(h, op, Pold, h->tmp, s));
  SDG_K(k_divergence(h, Us, h->tmp, -1.0, b, st_dev(h, kStMisc), parts(h, kStMisc), s));
  SDG_K(k_shift(b, h->g.ndof, st_dev(h, kStMisc), 0, 1.0 / (double)h->g.ndof, s));
  return SDG_OK;
}

template <typename P>
int alloc(P** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(P));
  if (e != cudaSuccess) {
    set_err("cudaMalloc failed: %s", cudaGetErrorString(e));
    return SDG_ERR_CUDA;
  }
  *p = static_cast<P*>(v);
  return SDG_OK;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

const char* sdg_strerror(int status) {
  switch (status) {
    case SDG_OK: return "ok";
    case SDG_ERR_INVALID_ARG: return "invalid argument";
    case SDG_ERR_CUDA: return "CUDA error";
    case SDG_ERR_NOT_CONVERGED: return "CG did not converge within maxit";
    case SDG_ERR_BREAKDOWN: return "CG breakdown (p^T A p <= 0 or not finite)";
    case SDG_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* sdg_last_error(void) { return g_err; }

int sdg_nodes(int N, double* xi, double* w) {
  SDG_ARG(N >= 0 && N <= kMaxN, "N must be in [0, 11]");
  SDG_ARG(xi && w, "NULL output");
  gauss_legendre(N + 1, xi, w);
  return SDG_OK;
}

int sdg_matrices(int N, double* out) {
  SDG_ARG(N >= 0 && N <= kMaxN, "N must be in [0, 11]");
  SDG_ARG(out, "NULL output");
  Basis1D b;
  build_basis(N, &b);
  const int m = (N + 1) * (N + 1);
  const double* src[10] = {b.M, b.Rt, b.Lt, b.Rb, b.Lb, b.ML, b.MR, b.HR, b.HL, b.HC};
  for (int k = 0; k < 10; ++k) std::memcpy(out + k * m, src[k], m * sizeof(double));
  return SDG_OK;
}

int sdg_kernel_projector(int N, double* proj, int* dim) {
  SDG_ARG(N >= 0 && N <= kMaxN, "N must be in [0, 11]");
  SDG_ARG(proj, "NULL output");
  Basis1D b;
  build_basis(N, &b);
  const int d = kernel_projector(b, proj);
  if (dim) *dim = d;
  return SDG_OK;
}

int sdg_line_operator(int N, int fp32, double* HL, double* Mc, double* HR) {
  SDG_ARG(N >= 0 && N <= kMaxN, "N must be in [0, 11]");
  SDG_ARG(HL && Mc && HR, "NULL output");
  Basis1D b;
  build_basis(N, &b);
  CoefSet c;
  build_coefs(b, fp32 ? 1 : 0, &c);
  line_operator(c, HL, Mc, HR);
  return SDG_OK;
}

int sdg_create(const sdg_grid* grid, int N, double nu, double theta, double dt, sdg_handle** out) {
  SDG_ARG(grid && out, "NULL argument");
  SDG_ARG(grid->dim == 2 || grid->dim == 3, "dim must be 2 or 3");
  SDG_ARG(N >= 0 && N <= kMaxN, "N must be in [0, 11]");
  SDG_ARG(nu >= 0.0 && std::isfinite(nu), "nu must be >= 0");
  SDG_ARG(theta >= 0.5 && theta <= 1.0, "theta must be in [1/2, 1]");
  SDG_ARG(dt > 0.0 && std::isfinite(dt), "dt must be > 0");
  for (int d = 0; d < grid->dim; ++d) {
    SDG_ARG(grid->n[d] >= 1, "cells per direction must be >= 1");
    SDG_ARG(grid->L[d] > 0.0, "box lengths must be > 0");
  }
  sdg_handle* h = new (std::nothrow) sdg_handle();
  if (!h) return SDG_ERR_CUDA;
  std::memset(h, 0, sizeof(*h));
  SDG_CK(cudaGetDevice(&h->device));
  SDG_CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
  h->dim = grid->dim;
  h->g.dim = grid->dim;
  h->g.n1 = N + 1;
  h->g.npe = 1;
  for (int d = 0; d < grid->dim; ++d) h->g.npe *= (N + 1);
  h->g.ncell = 1;
  for (int d = 0; d < 3; ++d) {
    h->g.n[d] = d < grid->dim ? grid->n[d] : 1;
    h->L[d] = d < grid->dim ? grid->L[d] : 1.0;
    h->dx[d] = h->L[d] / h->g.n[d];
    h->g.ncell *= h->g.n[d];
  }
  h->g.ndof = h->g.ncell * h->g.npe;
  h->nu = nu;
  h->theta = theta;
  h->dt = dt;
  h->precision = SDG_FP64;
  h->rtol_p = h->rtol_v = 1e-12;
  h->delta = 0.5;
  h->nsub = 1;
  h->tile32 = 0;
  h->form = 2;  // measured faster than the other forms (2D and 3D)
  h->maxit = 1000000;
  h->max_updates = 10000;
  build_basis(N, &h->basis);
  build_coefs(h->basis, 0, &h->coef64);
  build_coefs(h->basis, 1, &h->coef32);
  h->deflate = 0;
  {
    const char* v = std::getenv("SDG_VERBOSE");
    h->verbose = (v && v[0] == '1') ? 1 : 0;
  }

  const long long n = h->g.ndof;
  // the operator kernel has one CTA per element box; the smallest box is one
  // element, so ncell bounds every grid (and the reduction grid is capped)
  h->max_blocks = h->g.ncell > kReduceBlocks ? h->g.ncell : kReduceBlocks;
  int rc = SDG_OK;
#define A_(p, c) if (rc == SDG_OK) rc = alloc(&(p), (size_t)(c))
  for (int d = 0; d < h->dim; ++d) {
    A_(h->U[d], n); A_(h->Vm[d], n); A_(h->S1[d], n); A_(h->S2[d], n);
    A_(h->F[d], n); A_(h->Vh[d], n); A_(h->Us[d], n); A_(h->Lc[d], n);
  }
  A_(h->P, n); A_(h->b, n); A_(h->Pn, n); A_(h->tmp, n);
  A_(h->r64, n); A_(h->r64b, n); A_(h->p64[0], n); A_(h->p64[1], n); A_(h->Ap64, n); A_(h->Ap64b, n);
  A_(h->x32, n); A_(h->r32, n); A_(h->r32b, n); A_(h->p32[0], n); A_(h->p32[1], n); A_(h->Ap32, n);
  A_(h->Ap32b, n);
  A_(h->st, kMaxStates);
  A_(h->partials, (size_t)kMaxStates * h->max_blocks * kPartialSlots);
  A_(h->mats, kMatTable);
  A_(h->x0buf, n);
  A_(h->kpart, (size_t)kKernelBlocks * h->g.npe);
  A_(h->kcorr, h->g.npe);
  A_(h->kproj, h->g.n1 * h->g.n1);
  A_(h->kdpart, (size_t)kDeflateBlocks * h->g.npe);
  A_(h->kc, h->g.npe);
#undef A_
  if (rc != SDG_OK) { sdg_destroy(h); return rc; }
  if (cudaMallocHost(&h->st_host, kMaxStates * sizeof(SolverState)) != cudaSuccess) {
    sdg_destroy(h);
    set_err("cudaMallocHost failed%s", "");
    return SDG_ERR_CUDA;
  }
  // device matrix table
  double table[kMatTable];
  std::memset(table, 0, sizeof(table));
  const Basis1D& B = h->basis;
  const int n1 = h->g.n1;
  for (int i = 0; i < n1; ++i) {
    table[kW * kMatStride + i] = B.w[i];
    table[kWinv * kMatStride + i] = 1.0 / B.w[i];
    table[kPhi0 * kMatStride + i] = B.phi0[i];
    table[kPhi1 * kMatStride + i] = B.phi1[i];
  }
  const double* mats[] = {B.M, B.Rt, B.Lt, B.Rb, B.Lb, B.ML, B.MR, B.HR, B.HL, B.HC, B.Dn};
  const int ids[] = {kM, kRt, kLt, kRb, kLb, kML, kMR, kHR, kHL, kHC, kDn};
  for (int k = 0; k < 11; ++k) std::memcpy(table + ids[k] * kMatStride, mats[k], n1 * n1 * sizeof(double));
  cudaError_t e = cudaMemcpy(h->mats, table, sizeof(table), cudaMemcpyHostToDevice);
  {
    double proj[kMaxN1 * kMaxN1], b1[kMaxN1 * kMaxN1];
    h->kdim = kernel_projector(h->basis, proj);
    if (e == cudaSuccess) e = cudaMemcpy(h->kproj, proj, n1 * n1 * sizeof(double), cudaMemcpyHostToDevice);
    // local kernel patterns: tensor products of the 1D basis vectors
    const int kd1 = kernel_basis(h->basis, b1);
    const int npe = h->g.npe;
    h->kd = 1;
    for (int d = 0; d < h->dim; ++d) h->kd *= kd1;
    std::vector<double> kb((size_t)h->kd * npe);
    for (int j = 0; j < h->kd; ++j) {
      int jj = j, idx[3] = {0, 0, 0};
      for (int d = 0; d < h->dim; ++d) { idx[d] = jj % kd1; jj /= kd1; }
      for (int l = 0; l < npe; ++l) {
        int ll = l;
        double v = 1.0;
        for (int d = 0; d < h->dim; ++d) { v *= b1[idx[d] * n1 + ll % n1]; ll /= n1; }
        kb[(size_t)j * npe + l] = v;
      }
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->kbasis, kb.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(h->kbasis, kb.data(), kb.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->kc, 0, npe * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMemset(h->st, 0, kMaxStates * sizeof(SolverState));
  for (int d = 0; d < h->dim && e == cudaSuccess; ++d) e = cudaMemset(h->U[d], 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->P, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->p64[0], 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->p32[0], 0, n * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev2);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev3);
  for (int k = 0; k < 2 * kProfEvents && e == cudaSuccess; ++k) e = cudaEventCreate(&h->pev[k]);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_err("CUDA error %s in sdg_create", cudaGetErrorString(e));
    sdg_destroy(h);
    return SDG_ERR_CUDA;
  }
  *out = h;
  return SDG_OK;
}

int sdg_destroy(sdg_handle* h) {
  if (!h) return SDG_OK;
  for (int d = 0; d < 3; ++d) {
    cudaFree(h->U[d]); cudaFree(h->Vm[d]); cudaFree(h->S1[d]); cudaFree(h->S2[d]);
    cudaFree(h->F[d]); cudaFree(h->Vh[d]); cudaFree(h->Us[d]); cudaFree(h->Lc[d]);
  }
  cudaFree(h->P); cudaFree(h->b); cudaFree(h->Pn); cudaFree(h->tmp);
  cudaFree(h->r64); cudaFree(h->r64b); cudaFree(h->p64[0]); cudaFree(h->p64[1]); cudaFree(h->Ap64);
  cudaFree(h->Ap64b);
  cudaFree(h->x32); cudaFree(h->r32); cudaFree(h->r32b); cudaFree(h->p32[0]); cudaFree(h->p32[1]);
  cudaFree(h->Ap32); cudaFree(h->Ap32b);
  cudaFree(h->st); cudaFree(h->partials); cudaFree(h->mats);
  cudaFree(h->x0buf); cudaFree(h->kpart); cudaFree(h->kcorr); cudaFree(h->kproj);
  cudaFree(h->kbasis); cudaFree(h->kdpart); cudaFree(h->kc); cudaFree(h->adj);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->ev3) cudaEventDestroy(h->ev3);
  for (int k = 0; k < 2 * kProfEvents; ++k)
    if (h->pev[k]) cudaEventDestroy(h->pev[k]);
  delete h;
  return SDG_OK;
}

int sdg_set_options(sdg_handle* h, int precision, double rtol_p, double rtol_v, int maxit) {
  SDG_ARG(h, "NULL handle");
  SDG_ARG(precision == SDG_FP64 || precision == SDG_MIXED, "precision must be SDG_FP64 or SDG_MIXED");
  SDG_ARG(rtol_p > 0.0 && rtol_v > 0.0, "tolerances must be > 0");
  SDG_ARG(maxit >= 1, "maxit must be >= 1");
  h->precision = precision;
  h->rtol_p = rtol_p;
  h->rtol_v = rtol_v;
  h->maxit = maxit;
  return SDG_OK;
}

int sdg_set_mixed_options(sdg_handle* h, double delta, int max_updates, int deflate) {
  SDG_ARG(h, "NULL handle");
  SDG_ARG(delta > 0.0 && delta < 1.0, "delta must be in (0, 1)");
  SDG_ARG(max_updates >= 1, "max_updates must be >= 1");
  h->delta = delta;
  h->max_updates = max_updates;
  h->deflate = deflate ? 1 : 0;
  return SDG_OK;
}

int sdg_set_convection_substeps(sdg_handle* h, int nsub) {
  SDG_ARG(h, "NULL handle");
  SDG_ARG(nsub >= 1 && nsub <= 1000, "nsub must be in [1, 1000]");
  h->nsub = nsub;
  return SDG_OK;
}

int sdg_set_iteration_form(sdg_handle* h, int form) {
  SDG_ARG(h, "NULL handle");
  SDG_ARG(form >= 0 && form <= 2, "iteration form must be 0, 1 or 2");
  h->form = form;
  return SDG_OK;
}

int sdg_set_tile(sdg_handle* h, int variant) {
  SDG_ARG(h, "NULL handle");
  SDG_ARG(variant >= 0 && variant <= 2, "tile variant must be 0, 1 or 2");
  h->tile32 = h->dim == 2 ? variant : (variant ? 1 : 0);
  return SDG_OK;
}

int sdg_autotune(sdg_handle* h, int* variant, double* us, void* stream) {
  SDG_ARG(h, "NULL handle");
  cudaStream_t s = S(stream);
  const int nv = h->dim == 2 ? 3 : 2;
  Op op = pressure_op(h);
  double best = 1e300;
  int pick = 0;
  for (int v = 0; v < nv; ++v) {
    h->tile32 = v;
    for (int k = 0; k < 3; ++k) SDG_K(apply_plain<float>(h, op, h->p32[0], h->Ap32, s));
    SDG_CK(cudaEventRecord(h->ev0, s));
    constexpr int kReps = 10;
    for (int k = 0; k < kReps; ++k) SDG_K(apply_plain<float>(h, op, h->p32[0], h->Ap32, s));
    SDG_CK(cudaEventRecord(h->ev1, s));
    SDG_CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    SDG_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    const double t = 1e3 * ms / kReps;
    if (us) us[v] = t;
    if (t < best) {
      best = t;
      pick = v;
    }
  }
  h->tile32 = pick;
  if (variant) *variant = pick;
  return SDG_OK;
}

long long sdg_ndof(const sdg_handle* h) { return h ? h->g.ndof : 0; }

int sdg_set_state(sdg_handle* h, const double* u, const double* v, const double* w, const double* p,
                  void* stream) {
  SDG_ARG(h && u && v && p, "NULL argument");
  SDG_ARG(h->dim == 2 || w, "w required in 3D");
  const size_t bytes = (size_t)h->g.ndof * sizeof(double);
  const double* src[3] = {u, v, w};
  for (int d = 0; d < h->dim; ++d) SDG_CK(cudaMemcpyAsync(h->U[d], src[d], bytes, cudaMemcpyDefault, S(stream)));
  SDG_CK(cudaMemcpyAsync(h->P, p, bytes, cudaMemcpyDefault, S(stream)));
  SDG_CK(cudaStreamSynchronize(S(stream)));
  return SDG_OK;
}

int sdg_get_state(sdg_handle* h, double* u, double* v, double* w, double* p, void* stream) {
  SDG_ARG(h, "NULL handle");
  const size_t bytes = (size_t)h->g.ndof * sizeof(double);
  double* dst[3] = {u, v, w};
  for (int d = 0; d < h->dim; ++d)
    if (dst[d]) SDG_CK(cudaMemcpyAsync(dst[d], h->U[d], bytes, cudaMemcpyDefault, S(stream)));
  if (p) SDG_CK(cudaMemcpyAsync(p, h->P, bytes, cudaMemcpyDefault, S(stream)));
  SDG_CK(cudaStreamSynchronize(S(stream)));
  return SDG_OK;
}

int sdg_pressure_apply(sdg_handle* h, const void* x, void* y, int fp32, void* stream) {
  SDG_ARG(h && x && y && x != y, "bad arguments");
  const Op op = pressure_op(h);
  if (fp32)
    SDG_K(apply_plain<float>(h, op, static_cast<const float*>(x), static_cast<float*>(y), S(stream)));
  else
    SDG_K(apply_plain<double>(h, op, static_cast<const double*>(x), static_cast<double*>(y), S(stream)));
  return SDG_OK;
}

int sdg_viscous_apply(sdg_handle* h, const void* x, void* y, int fp32, void* stream) {
  SDG_ARG(h && x && y && x != y, "bad arguments");
  const Op op = viscous_op(h);
  if (fp32)
    SDG_K(apply_plain<float>(h, op, static_cast<const float*>(x), static_cast<float*>(y), S(stream)));
  else
    SDG_K(apply_plain<double>(h, op, static_cast<const double*>(x), static_cast<double*>(y), S(stream)));
  return SDG_OK;
}

int sdg_pressure_cg(sdg_handle* h, const double* b, double* x, sdg_cg_info* info, void* stream) {
  SDG_ARG(h && b && x && b != x, "bad arguments");
  return solve(h, true, b, x, info, S(stream));
}

int sdg_viscous_cg(sdg_handle* h, const double* b, double* x, sdg_cg_info* info, void* stream) {
  SDG_ARG(h && b && x && b != x, "bad arguments");
  return solve(h, false, b, x, info, S(stream));
}

int sdg_dual_to_main(sdg_handle* h, int d, const double* in, double* out, void* stream) {
  SDG_ARG(h && in && out && in != out, "bad arguments");
  SDG_ARG(d >= 0 && d < h->dim, "direction out of range");
  SDG_K(k_dual_to_main(h, d, in, out, S(stream)));
  return SDG_OK;
}

int sdg_main_to_dual(sdg_handle* h, int d, const double* in, double* out, void* stream) {
  SDG_ARG(h && in && out && in != out, "bad arguments");
  SDG_ARG(d >= 0 && d < h->dim, "direction out of range");
  SDG_K(k_main_to_dual(h, d, in, out, S(stream)));
  return SDG_OK;
}

// SSP-RK3 (Shu-Osher form) of the explicit convection over one dt, in
// h->nsub equal sub-steps: W <- W/3 + 2/3 (W2 + k L(W2)) with
// W1 = W + k L(W), W2 = 3/4 W + 1/4 (W1 + k L(W1)), k = dt / nsub.  The first
// sub-step reads V; later ones update F in place (out may alias V0).
static int convect_rk3(sdg_handle* h, const double* const* V, double* const* F, cudaStream_t s) {
  const double k = h->dt / h->nsub;
  for (int sub = 0; sub < h->nsub; ++sub) {
    const double* const* W = sub == 0 ? V : F;
    SDG_K(k_convect_stage(h, nullptr, W, h->S1, 0.0, 1.0, k, s));
    SDG_K(k_convect_stage(h, W, h->S1, h->S2, 0.75, 0.25, k, s));
    SDG_K(k_convect_stage(h, W, h->S2, F, 1.0 / 3.0, 2.0 / 3.0, k, s));
    h->launches += 3 * (h->dim - 1);  // a stage is one launch per direction
  }
  return SDG_OK;
}

int sdg_convect(sdg_handle* h, const double* const* V, double* const* F, void* stream) {
  SDG_ARG(h && V && F, "bad arguments");
  for (int d = 0; d < h->dim; ++d) SDG_ARG(V[d] && F[d], "NULL component");
  return convect_rk3(h, V, F, S(stream));
}

int sdg_pressure_rhs(sdg_handle* h, const double* const* Ustar, const double* P_old, double* b, void* stream) {
  SDG_ARG(h && Ustar && P_old && b, "bad arguments");
  return pressure_rhs(h, Ustar, P_old, b, S(stream));
}

int sdg_velocity_update(sdg_handle* h, const double* const* Ustar, const double* P_new, const double* P_old,
                        double* const* U, void* stream) {
  SDG_ARG(h && Ustar && P_new && P_old && U, "bad arguments");
  SDG_K(k_velocity_update(h, Ustar, P_new, P_old, U, S(stream)));
  return SDG_OK;
}

int sdg_step(sdg_handle* h, int nsteps, sdg_step_info* info, void* stream) {
  SDG_ARG(h && nsteps >= 0, "bad arguments");
  cudaStream_t s = S(stream);
  const long long n = h->g.ndof;
  double p_ms = 0.0;
  long long p_applies = 0;
  int first_bad = SDG_OK;
  sdg_cg_info pinfo{}, vinfo[3]{};
  const long long launches0 = h->launches;
  SDG_CK(cudaEventRecord(h->ev2, s));
  for (int step = 0; step < nsteps; ++step) {
    // 1. dual -> main (Eq. l2forward)
    for (int d = 0; d < h->dim; ++d) SDG_K(k_dual_to_main(h, d, h->U[d], h->Vm[d], s));
    // 2. SSP-RK3 of the explicit convection (Eqs. Fu-Fw)
    {
      const int rc = convect_rk3(h, h->Vm, h->F, s);
      if (rc != SDG_OK) return rc;
    }
    // 3. implicit viscosity per component (Eq. LOdiffusionU-W)
    for (int c = 0; c < h->dim; ++c) {
      SDG_K(k_mass_rhs(h, h->F[c], h->b, h->Vh[c], s));
      int rc = solve(h, false, h->b, h->Vh[c], &vinfo[c], s);
      if (rc == SDG_ERR_CUDA || rc == SDG_ERR_INVALID_ARG) return rc;
      if (rc != SDG_OK && first_bad == SDG_OK) first_bad = rc;
    }
    // 4. main -> dual (Eq. l2backward)
    for (int d = 0; d < h->dim; ++d) SDG_K(k_main_to_dual(h, d, h->Vh[d], h->Us[d], s));
    // 5. pressure system (Eqs. pSyst, LOpressure), x0 = P^n
    {
      int rc = pressure_rhs(h, h->Us, h->P, h->b, s);
      if (rc != SDG_OK) return rc;
    }
    SDG_CK(cudaMemcpyAsync(h->Pn, h->P, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SDG_CK(cudaEventRecord(h->ev0, s));
    {
      int rc = solve(h, true, h->b, h->Pn, &pinfo, s);
      if (rc == SDG_ERR_CUDA || rc == SDG_ERR_INVALID_ARG) return rc;
      if (rc != SDG_OK && first_bad == SDG_OK) first_bad = rc;
    }
    SDG_CK(cudaEventRecord(h->ev1, s));
    SDG_CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    SDG_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    p_ms += ms;
    p_applies += pinfo.applies_fp64 + pinfo.applies_fp32;
    // 6. gauge: zero physical mean of P^{n+1}
    SDG_K(k_weighted_sum(h, h->Pn, nullptr, st_dev(h, kStMisc), 1, parts(h, kStMisc), s));
    SDG_K(k_shift(h->Pn, n, st_dev(h, kStMisc), 1, 1.0 / (double)h->g.ncell, s));
    // 7. velocity update with q = theta P^{n+1} + (1-theta) P^n (Eq. LOvelocityU-W)
    SDG_K(k_velocity_update(h, h->Us, h->Pn, h->P, h->U, s));
    double* t = h->P;
    h->P = h->Pn;
    h->Pn = t;
  }
  SDG_CK(cudaEventRecord(h->ev3, s));
  SDG_CK(cudaEventSynchronize(h->ev3));
  float total = 0.f;
  SDG_CK(cudaEventElapsedTime(&total, h->ev2, h->ev3));
  if (info) {
    info->pressure = pinfo;
    for (int c = 0; c < 3; ++c) info->viscous[c] = vinfo[c];
    info->pressure_ms = p_ms;
    info->step_ms = total;
    info->pressure_applies = p_applies;
    info->kernel_launches = h->launches - launches0;
  }
  return first_bad;
}

int sdg_step_adjoint(sdg_handle* h, const double* const* U, double* const* lamU, double* lamP, double* dnu,
                     void* stream) {
  SDG_ARG(h && U && lamU && lamP && dnu, "NULL argument");
  for (int d = 0; d < h->dim; ++d) SDG_ARG(U[d] && lamU[d], "NULL component");
  cudaStream_t s = S(stream);
  const int D = h->dim, K = h->nsub;
  const long long n = h->g.ndof;
  const long long need = 3LL * K * D + 7LL * D + 5;
  if (h->adj_fields < need) {
    SDG_CK(cudaStreamSynchronize(s));
    SDG_CK(cudaFree(h->adj));
    h->adj = nullptr;
    h->adj_fields = 0;
    if (alloc(&h->adj, (size_t)(need * n)) != SDG_OK) return SDG_ERR_CUDA;
    h->adj_fields = need;
  }
  long long next = 0;
  auto field = [&]() { return h->adj + (next++) * n; };
  std::vector<double*> stW(K * D), stS1(K * D), stS2(K * D);
  for (int k = 0; k < K * D; ++k) {
    stW[k] = field();
    stS1[k] = field();
    stS2[k] = field();
  }
  double *lx = field(), *kx = field(), *zero = field(), *lPo = field(), *mup = field();
  double *lUs[3] = {nullptr, nullptr, nullptr}, *lVh[3] = {nullptr, nullptr, nullptr};
  double *mu[3] = {nullptr, nullptr, nullptr}, *lam[3] = {nullptr, nullptr, nullptr};
  double *lamW[3] = {nullptr, nullptr, nullptr}, *lamS1[3] = {nullptr, nullptr, nullptr};
  double *lamS2[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < D; ++d) {
    lUs[d] = field();
    lVh[d] = field();
    mu[d] = field();
    lam[d] = field();
    lamW[d] = field();
    lamS1[d] = field();
    lamS2[d] = field();
  }
  const size_t bytes = (size_t)n * sizeof(double);
  const double kdt = h->dt / K;
  int first_bad = SDG_OK;
  auto note = [&](int rc) {
    if (rc != SDG_OK && first_bad == SDG_OK) first_bad = rc;
  };
  SolverState* stm = st_dev(h, kStMisc);
  double* pm = parts(h, kStMisc);

  // ---- forward recompute of the step's convection stages and viscous solves
  for (int d = 0; d < D; ++d) SDG_K(k_dual_to_main(h, d, U[d], stW[d], s));
  for (int k = 0; k < K; ++k) {
    const double* W[3] = {stW[k * D], D > 1 ? stW[k * D + 1] : nullptr, D > 2 ? stW[k * D + 2] : nullptr};
    double* S1[3] = {stS1[k * D], D > 1 ? stS1[k * D + 1] : nullptr, D > 2 ? stS1[k * D + 2] : nullptr};
    double* S2[3] = {stS2[k * D], D > 1 ? stS2[k * D + 1] : nullptr, D > 2 ? stS2[k * D + 2] : nullptr};
    double* out[3];
    for (int d = 0; d < 3; ++d) out[d] = (k + 1 < K) ? (d < D ? stW[(k + 1) * D + d] : nullptr) : h->F[d];
    SDG_K(k_convect_stage(h, nullptr, W, S1, 0.0, 1.0, kdt, s));
    SDG_K(k_convect_stage(h, W, S1, S2, 0.75, 0.25, kdt, s));
    SDG_K(k_convect_stage(h, W, S2, out, 1.0 / 3.0, 2.0 / 3.0, kdt, s));
    h->launches += 3 * (h->dim - 1);  // a stage is one launch per direction
  }
  sdg_cg_info info{};
  for (int c = 0; c < D; ++c) {
    SDG_K(k_mass_rhs(h, h->F[c], h->b, h->Vh[c], s));
    const int rc = solve(h, false, h->b, h->Vh[c], &info, s);
    if (rc == SDG_ERR_CUDA || rc == SDG_ERR_INVALID_ARG) return rc;
    note(rc);
  }

  // ---- velocity update and pressure (Eqs. LOvelocityU-W, LOpressure, gauge)
  SDG_K(adj_velocity_T(h, lamU, lamP, lx, lPo, s));
  SDG_K(adj_dot(lx, nullptr, n, stm, 0, pm, s));
  SDG_K(adj_sub_weighted(h, lx, stm, 0, 1.0 / (double)h->g.ncell, s));
  SDG_CK(cudaMemcpyAsync(kx, lx, bytes, cudaMemcpyDeviceToDevice, s));
  SDG_CK(cudaMemsetAsync(zero, 0, bytes, s));
  {
    int nl = 0;
    SDG_CK(kernel_restore(h, lx, zero, s, &nl));  // lx <- range part
    h->launches += nl;
  }
  SDG_K(adj_axpby(kx, 1.0, kx, -1.0, lx, n, s));  // kernel part passes to P^n
  SDG_K(adj_axpby(lPo, 1.0, lPo, 1.0, kx, n, s));
  SDG_CK(cudaMemsetAsync(mup, 0, bytes, s));
  {
    const int rc = solve(h, true, lx, mup, &info, s);
    if (rc == SDG_ERR_CUDA || rc == SDG_ERR_INVALID_ARG) return rc;
    note(rc);
  }
  SDG_K(adj_dot(mup, nullptr, n, stm, 0, pm, s));
  SDG_K(k_shift(mup, n, stm, 0, 1.0 / (double)n, s));  // lambda_b (zero mean)
  SDG_K(adj_divergence_T(h, lamU, mup, lUs, s));
  {
    Op op{};
    for (int d = 0; d < D; ++d) op.s[d] = (1.0 - h->theta) * h->dt / (h->dx[d] * h->dx[d]);
    SDG_K(apply_plain<double>(h, op, mup, h->tmp, s));
    SDG_K(adj_axpby(lPo, 1.0, lPo, -1.0, h->tmp, n, s));
  }
  // ---- projections back and the viscous solves (symmetric operator)
  for (int d = 0; d < D; ++d) SDG_K(adj_project_T(h, false, d, lUs[d], lVh[d], s));
  for (int c = 0; c < D; ++c) {
    SDG_CK(cudaMemsetAsync(mu[c], 0, bytes, s));
    const int rc = solve(h, false, lVh[c], mu[c], &info, s);
    if (rc == SDG_ERR_CUDA || rc == SDG_ERR_INVALID_ARG) return rc;
    note(rc);
  }
  // d/dnu: Vh = (M + nu A')^-1 M F  =>  - mu . A' Vh
  {
    Op op{};
    for (int d = 0; d < D; ++d) op.s[d] = h->dt / (h->dx[d] * h->dx[d]);
    double acc = 0.0;
    for (int c = 0; c < D; ++c) {
      SDG_K(apply_plain<double>(h, op, h->Vh[c], h->tmp, s));
      SDG_K(adj_dot(mu[c], h->tmp, n, stm, 1, pm, s));
      SDG_CK(cudaMemcpyAsync(h->st_host + kStMisc, stm, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      SDG_CK(cudaStreamSynchronize(s));
      acc += h->st_host[kStMisc].red[1];
    }
    *dnu -= acc;
  }
  for (int c = 0; c < D; ++c) SDG_K(k_mass_rhs(h, mu[c], lam[c], nullptr, s));  // lambda_F = M mu
  // ---- SSP-RK3 sub-steps in reverse
  for (int k = K - 1; k >= 0; --k) {
    const double* W[3] = {stW[k * D], D > 1 ? stW[k * D + 1] : nullptr, D > 2 ? stW[k * D + 2] : nullptr};
    const double* S1[3] = {stS1[k * D], D > 1 ? stS1[k * D + 1] : nullptr, D > 2 ? stS1[k * D + 2] : nullptr};
    const double* S2[3] = {stS2[k * D], D > 1 ? stS2[k * D + 1] : nullptr, D > 2 ? stS2[k * D + 2] : nullptr};
    const double* lamc[3] = {lam[0], lam[1], lam[2]};
    const double* ls2[3] = {lamS2[0], lamS2[1], lamS2[2]};
    const double* ls1[3] = {lamS1[0], lamS1[1], lamS1[2]};
    const double* lw[3] = {lamW[0], lamW[1], lamW[2]};
    SDG_K(adj_convect_T(h, S2, lamc, nullptr, lamS2, 0.0, 2.0 / 3.0, kdt, s));
    for (int c = 0; c < D; ++c) SDG_K(adj_axpby(lamW[c], 1.0 / 3.0, lam[c], 0.75, lamS2[c], n, s));
    SDG_K(adj_convect_T(h, S1, ls2, nullptr, lamS1, 0.0, 0.25, kdt, s));
    SDG_K(adj_convect_T(h, W, ls1, lw, lam, 1.0, 1.0, kdt, s));
  }
  for (int d = 0; d < D; ++d) SDG_K(adj_project_T(h, true, d, lam[d], lamU[d], s));
  SDG_CK(cudaMemcpyAsync(lamP, lPo, bytes, cudaMemcpyDeviceToDevice, s));
  return first_bad;
}

int sdg_set_profiling(sdg_handle* h, int enable) {
  SDG_ARG(h, "NULL handle");
  h->profile = enable ? 1 : 0;
  h->launches = 0;
  h->prof_ms[0] = h->prof_ms[1] = 0.0;
  h->prof_n[0] = h->prof_n[1] = 0;
  return SDG_OK;
}

int sdg_counters(const sdg_handle* h, long long* launches, double* apply_ms, long long* apply_launches) {
  SDG_ARG(h, "NULL handle");
  if (launches) *launches = h->launches;
  if (apply_ms) { apply_ms[0] = h->prof_ms[0]; apply_ms[1] = h->prof_ms[1]; }
  if (apply_launches) { apply_launches[0] = h->prof_n[0]; apply_launches[1] = h->prof_n[1]; }
  return SDG_OK;
}

int sdg_diagnostics(sdg_handle* h, double* kinetic_energy, double* div_norm, void* stream) {
  SDG_ARG(h, "NULL handle");
  cudaStream_t s = S(stream);
  SolverState* st = st_dev(h, kStMisc);
  double* pa = parts(h, kStMisc);
  double ke = 0.0;
  if (kinetic_energy) {
    for (int d = 0; d < h->dim; ++d) {
      SDG_K(k_weighted_sum(h, h->U[d], h->U[d], st, 2, pa, s));
      SDG_CK(cudaMemcpyAsync(h->st_host + kStMisc, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      SDG_CK(cudaStreamSynchronize(s));
      ke += h->st_host[kStMisc].red[2];
    }
    double cellvol = 1.0, vol = 1.0;
    for (int d = 0; d < h->dim; ++d) { cellvol *= h->dx[d]; vol *= h->L[d]; }
    *kinetic_energy = 0.5 * cellvol * ke / vol;
  }
  if (div_norm) {
    SDG_K(k_divergence(h, h->U, nullptr, 1.0, h->tmp, st, pa, s));
    SDG_K(k_norm2(h->tmp, h->g.ndof, st, 3, pa, s));
    SDG_CK(cudaMemcpyAsync(h->st_host + kStMisc, st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    SDG_CK(cudaStreamSynchronize(s));
    *div_norm = std::sqrt(h->st_host[kStMisc].red[3]);
  }
  return SDG_OK;
}

}  // extern "C"
