// Vector kernels of the CG solvers and the per-node kernels of the time step
// (L2 projections, Rusanov convection stage, pressure right-hand side,
// velocity update, reductions).
#include "sdg_device.cuh"

namespace sdg {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > kReduceBlocks) b = kReduceBlocks;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Launch with programmatic stream serialisation (the kernel may start while
// the previous kernel of the stream finishes; see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// grid of the vectorised CG update: enough blocks to fill the machine
inline unsigned grid_vec(long long n, int w) {
  long long b = (n / w + kThreads - 1) / kThreads;
  if (b > kReduceBlocks) b = kReduceBlocks;
  if (b < 1) b = 1;
  return (unsigned)b;
}

inline unsigned grid_full(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ CG vectors
template <typename T>
struct V4;
template <>
struct V4<float> { using V = float4; static constexpr int W = 4; };
template <>
struct V4<double> { using V = double2; static constexpr int W = 2; };

// Per-thread accumulator of a dot product: FP64 for FP64 data; for FP32 data
// a compensated (Kahan) FP32 sum, so that no FP64 arithmetic runs per element
// (GB300 issues FP64 at 1/64 of the FP32 rate).  Blocks reduce in FP64.
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T v) { s = fma((double)v, 1.0, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
  __device__ __forceinline__ F2 pair() const { return F2{s, -c}; }
};

template <typename T>
__device__ __forceinline__ void upd1(T& x, T& r, T p, T Ap, T alpha, DotAcc<T>& rr) {
  x = fma(alpha, p, x);
  r = fma(-alpha, Ap, r);
  rr.add(r * r);
}

// x += alpha p ; r -= alpha Ap ; rr = r.r  (vectorised, scalar tail).  With
// x null only r and Ap move (the operator launch adds alpha p to x).
// With deflation (FP32, df.kpart != null) the kernel part of the new r is
// reduced too, removed from rr, and left in df.kc for the next direction.
// Compiled per use (deflation, x in this launch); without deflation for
// four 256-thread blocks per SM (64 registers, no spills).
template <typename T, bool DEFL, bool WITHX>
__global__ void __launch_bounds__(kThreads, DEFL ? 1 : 4)
    k_cg_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ Ap,
                long long n, SolverState* st, double* partials, Deflate df) {
  pdl_trigger();
  pdl_wait();  // the p.Ap totals and Ap come from the operator kernel just before
  if (st->done || st->pause) return;
  using V = typename V4<T>::V;
  constexpr int W = V4<T>::W;
  const long long nv = n / W;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  // U vectors per thread and pass, all loads issued before the arithmetic
  // (the update is bound by memory latency, not bandwidth, at one vector);
  // the first pass's loads go out before alpha is formed
  constexpr int U = 2;
  constexpr bool withx = WITHX;
  V xv[U], rv[U], pv[U], av[U];
  auto issue = [&](long long i0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * nth;
      if (i < nv) {
        if (withx) {
          xv[u] = reinterpret_cast<V*>(x)[i];
          pv[u] = reinterpret_cast<const V*>(p)[i];
        }
        rv[u] = reinterpret_cast<V*>(r)[i];
        av[u] = reinterpret_cast<const V*>(Ap)[i];
      }
    }
  };
  issue(tid);
  // alpha = r.r / p.Ap from the operator blocks' totals (every block forms the
  // same value; one FP64 division per block)
  __shared__ double s_opr[32];
  __shared__ double s_alpha;
  const double pAp = sizeof(T) == 4 ? sum_op_partials_f2(partials, st->nop, s_opr)
                                    : sum_op_partials_f64(partials, st->nop, s_opr);
  const bool breakdown = !(pAp > 0.0) || !isfinite(pAp);
  if (threadIdx.x == 0) s_alpha = breakdown ? 0.0 : st->rr / pAp;
  __syncthreads();
  extern __shared__ double s_dyn[];  // (deflation only)
  float* s_k = reinterpret_cast<float*>(s_dyn);  // npe floats (deflation)
  constexpr bool defl = DEFL;
  if (defl) {
    for (int l = threadIdx.x; l < df.npe; l += blockDim.x) s_k[l] = 0.0f;
    __syncthreads();
  }
  const T alpha = sizeof(T) == 4 ? (T)(float)s_alpha : (T)s_alpha;
  DotAcc<T> rr;
  for (long long i0 = tid; i0 < nv; i0 += U * nth) {
    if (i0 != tid) issue(i0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * nth;
      if (i >= nv) break;
      T* xs = reinterpret_cast<T*>(&xv[u]);
      T* rs = reinterpret_cast<T*>(&rv[u]);
      const T* ps = reinterpret_cast<const T*>(&pv[u]);
      const T* as = reinterpret_cast<const T*>(&av[u]);
      if (withx) {
#pragma unroll
        for (int k = 0; k < W; ++k) upd1(xs[k], rs[k], ps[k], as[k], alpha, rr);
        reinterpret_cast<V*>(x)[i] = xv[u];
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          rs[k] = fma(-alpha, as[k], rs[k]);
          rr.add(rs[k] * rs[k]);
        }
      }
      reinterpret_cast<V*>(r)[i] = rv[u];
      if (defl) {
        const unsigned l0 = (unsigned)((unsigned long long)(i * W) % (unsigned)df.npe);
#pragma unroll
        for (int k = 0; k < W; ++k) {
          unsigned l = l0 + k;
          if (l >= (unsigned)df.npe) l -= df.npe;
          atomicAdd(&s_k[l], (float)rs[k]);
        }
      }
    }
  }
  for (long long i = nv * W + tid; i < n; i += nth) {
    if (withx) {
      upd1(x[i], r[i], p[i], Ap[i], alpha, rr);
    } else {
      r[i] = fma(-alpha, Ap[i], r[i]);
      rr.add(r[i] * r[i]);
    }
    if (defl) atomicAdd(&s_k[(unsigned)((unsigned long long)i % (unsigned)df.npe)], (float)r[i]);
  }
  if (defl) {
    __syncthreads();
    for (int l = threadIdx.x; l < df.npe; l += blockDim.x)
      df.kpart[(size_t)blockIdx.x * df.npe + l] = s_k[l];
    __threadfence();
  }
  double tot[1];
  bool last;
  if constexpr (sizeof(T) == 4) {
    F2 v[1] = {rr.pair()};
    last = grid_sum_f2<1>(v, partials, &st->counter, tot);
  } else {
    double v[1] = {rr.value()};
    last = grid_sum<1>(v, partials, &st->counter, tot);
  }
  if (last) {
    double rK2 = 0.0;
    if (defl) {
      // S[l] = sum over blocks of the partial sums, in FP64, by G thread groups
      const int npe = df.npe;
      const int G = blockDim.x >= 2 * npe ? blockDim.x / npe : 1;
      double* S = s_dyn;               // npe
      double* Gp = s_dyn + npe;        // G * npe
      __shared__ double s_a[8];
      __syncthreads();
      if (G > 1) {
        const int l = threadIdx.x % npe, g = threadIdx.x / npe;
        if (g < G) {
          double acc = 0.0;
          for (unsigned b = g; b < gridDim.x; b += G) acc += (double)__ldcg(&df.kpart[(size_t)b * npe + l]);
          Gp[g * npe + l] = acc;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < npe; q += blockDim.x) {
          double acc = 0.0;
          for (int g2 = 0; g2 < G; ++g2) acc += Gp[g2 * npe + q];
          S[q] = acc;
        }
      } else {
        for (int q = threadIdx.x; q < npe; q += blockDim.x) {
          double acc = 0.0;
          for (unsigned b = 0; b < gridDim.x; ++b) acc += (double)__ldcg(&df.kpart[(size_t)b * npe + q]);
          S[q] = acc;
        }
      }
      __syncthreads();
      if ((int)threadIdx.x < df.kd) {
        double a = 0.0;
        for (int q = 0; q < npe; ++q) a += df.kbasis[threadIdx.x * npe + q] * S[q];
        s_a[threadIdx.x] = a;
      }
      __syncthreads();
      const double inv = 1.0 / (double)df.ncell;
      for (int q = threadIdx.x; q < npe; q += blockDim.x) {
        double c = 0.0;
        for (int j = 0; j < df.kd; ++j) c += s_a[j] * df.kbasis[j * npe + q];
        df.kc[q] = (float)(c * inv);
      }
      for (int j = 0; j < df.kd; ++j) rK2 += s_a[j] * s_a[j] * inv;
    }
    if (threadIdx.x == 0) {
      st->pAp = pAp;
      st->alpha = s_alpha;
      st->alpha_f = (float)s_alpha;
      if (!WITHX) st->xpend = 1;  // x lacks alpha_k p_k (the next operator launch adds it)
      double rr = tot[0] - rK2;  // residual norm in the range of the operator
      if (rr < 0.0) rr = 0.0;
      st->rr_old = st->rr;
      st->rr = rr;
      st->beta = st->rr_old > 0.0 ? rr / st->rr_old : 0.0;  // for the next direction
      st->beta_f = (float)st->beta;
      st->iter += 1;
      if (rr > st->maxrr) st->maxrr = rr;
      if (breakdown || !isfinite(rr)) {
        st->done = 1;
        st->status = SDG_ERR_BREAKDOWN;
      } else if (rr <= st->tol2) {
        // plain CG stops here; reliable mode confirms with the FP64 residual
        if (st->reliable) st->pause = 1;
        else { st->done = 1; st->status = SDG_OK; }
      } else if (st->reliable && rr < st->delta2 * st->maxrr) {
        st->pause = 1;
      } else if (st->iter >= st->maxit) {
        st->done = 1;
        st->status = SDG_ERR_NOT_CONVERGED;
      }
    }
  }
}

// ------------------------------------------------------------------ mixed precision
// x64 += x32 / sigma ; x32 = 0
__global__ void __launch_bounds__(kThreads)
    k_rel_accumulate(double* __restrict__ x64, float* __restrict__ x32, long long n, const SolverState* st) {
  const double inv = 1.0 / st->sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x64[i] += (double)x32[i] * inv;
    x32[i] = 0.0f;
  }
}

// r = b - Ax in FP64 with sum(r), sum(r^2), sum(b^2).  The last block
// replaces the recursive residual by the true one (mean removed, scaled by
// sigma^2) and decides convergence.
__global__ void __launch_bounds__(kThreads)
    k_rel_residual(const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
                   long long n, SolverState* st, double* partials, double rtol, int maxit, double delta,
                   int mode, int project, int unscaled) {
  const bool init = mode == 1;
  double s = 0.0, ss = 0.0, bb = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - Ax[i];
    r[i] = ri;
    s += ri;
    ss += ri * ri;
    bb += bi * bi;
  }
  double v[3] = {s, ss, bb}, tot[3];
  if (grid_sum<3>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
    // singular (periodic pressure) system: the constant part of r is round-off
    const double mean = project ? tot[0] / (double)n : 0.0;
    double rrp = tot[1] - (double)n * mean * mean;
    if (rrp < 0.0) rrp = 0.0;
    if (init) {
      st->bnorm2 = tot[2];
      // FP32 iterations run on sigma-scaled vectors (||b|| -> 1); FP64
      // iterations replace their own residual vector, unscaled
      st->sigma = (unscaled || !(tot[2] > 0.0)) ? 1.0 : 1.0 / sqrt(tot[2]);
      st->tol2 = rtol * rtol * tot[2] * st->sigma * st->sigma;
      st->iter = 0;
      st->maxit = maxit;
      st->updates = 0;
      st->reliable = 1;
      st->delta2 = delta * delta;
      st->status = SDG_OK;
      st->alpha = 0.0;
      st->pAp = 0.0;
      st->xpend = 0;
    } else {
      st->updates += 1;
    }
    const double rr = rrp * st->sigma * st->sigma;
    st->mean = mean;
    if (mode != 2) {
      // the next direction: p = r_true + (rr_true / rr_old) p_old
      st->beta = (!init && st->rr_old > 0.0) ? rr / st->rr_old : 0.0;
      st->beta_f = (float)st->beta;
    }
    // the next direction uses beta = rr_true / rr_k, rr_k being the residual
    // norm of the iteration before the one that triggered the update
    if (init) st->rr_old = rr;
    st->rr = rr;
    st->maxrr = rr;
    st->pause = 0;
    st->done = (tot[2] == 0.0 || rr <= st->tol2) ? 1 : 0;
    if (!isfinite(rr)) {
      st->done = 1;
      st->status = SDG_ERR_BREAKDOWN;
    }
  }
}

// red[0..2] = sum(r), sum(r^2), sum(b^2) of r = b - Ax
__global__ void __launch_bounds__(kThreads)
    k_resid_norms(const double* __restrict__ b, const double* __restrict__ Ax, long long n, SolverState* st,
                  double* partials) {
  double s = 0.0, ss = 0.0, bb = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double bi = b ? b[i] : 0.0;
    const double ri = bi - Ax[i];
    s += ri;
    ss += ri * ri;
    bb += bi * bi;
  }
  double v[3] = {s, ss, bb}, tot[3];
  if (grid_sum<3>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
    st->red[0] = tot[0];
    st->red[1] = tot[1];
    st->red[2] = tot[2];
  }
}

// u_i = s_i ulp(x_i) / (2 sqrt 3): ulp from the exponent bits of x_i (0 for
// zero and subnormal x_i), s_i the top bit of an integer hash of i
__global__ void __launch_bounds__(kThreads)
    k_rounding_perturbation(const double* __restrict__ x, double* __restrict__ u, long long n) {
  const double scale = 0.5 / 1.7320508075688772 / 4503599627370496.0;  // 1 / (2 sqrt 3) / 2^52
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    // 2^floor(log2 |x|): the exponent field alone
    const double pw = __longlong_as_double(__double_as_longlong(x[i]) & 0x7FF0000000000000LL);
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    u[i] = ((z >> 63) ? -scale : scale) * pw;
  }
}

// Norm and decisions of a replaced residual after its projection onto the
// range (singular pressure system): rr = sigma^2 ||r||^2 of the projected
// r, and the decisions k_rel_residual took on the unprojected norm taken
// again (the iteration's alpha = rr / pAp must see the norm of the vector it
// iterates on).
__global__ void __launch_bounds__(kThreads)
    k_rel_renorm(const double* __restrict__ r, long long n, SolverState* st, double* partials, int mode) {
  double ss = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    ss += r[i] * r[i];
  double v[1] = {ss}, tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
    const double rr = tot[0] * st->sigma * st->sigma;
    if (mode == 1) st->rr_old = rr;
    if (mode == 0) {
      st->beta = st->rr_old > 0.0 ? rr / st->rr_old : 0.0;
      st->beta_f = (float)st->beta;
    }
    st->rr = rr;
    st->maxrr = rr;
    if (!isfinite(rr)) {
      st->done = 1;
      st->status = SDG_ERR_BREAKDOWN;
    } else {
      st->done = (st->bnorm2 == 0.0 || rr <= st->tol2) ? 1 : 0;
    }
  }
}

// x += alpha p with the state's alpha: the update the next one-launch CG
// iteration would have applied, when the iteration stops at maxit
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pending_update(T* __restrict__ x, const T* __restrict__ p, long long n, const SolverState* st) {
  const T alpha = sizeof(T) == 4 ? (T)st->alpha_f : (T)st->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(alpha, p[i], x[i]);
}

// x += alpha p when the state's xpend is set (the step the next operator
// launch of the two-launch form would have added); the flag is cleared by a
// separate copy after this kernel
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pending_x(T* __restrict__ x, const T* __restrict__ p, long long n, const SolverState* st) {
  if (!st->xpend) return;
  const T alpha = sizeof(T) == 4 ? (T)st->alpha_f : (T)st->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(alpha, p[i], x[i]);
}

// r -= mean (the round-off constant part of a replaced FP64 residual)
__global__ void __launch_bounds__(kThreads)
    k_sub_mean(double* __restrict__ r, long long n, const SolverState* st) {
  const double mean = st->mean;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    r[i] -= mean;
}

// r32 = sigma r64 (r64 already has its kernel part removed)
__global__ void __launch_bounds__(kThreads)
    k_rel_convert(const double* __restrict__ r64, float* __restrict__ r32, long long n, const SolverState* st) {
  const double sigma = st->sigma;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    r32[i] = (float)(r64[i] * sigma);
}

// ------------------------------------------------------------------ step stages
// Per-node kernels: one thread per output node; the 1D matrices are staged
// in shared memory because the row index varies across the warp.
struct StepParams {
  Geo g;
  double invdx[3];
};

__device__ __forceinline__ void load_mats(const double* mats, double* s_m, const int* ids, int nid) {
  for (int k = 0; k < nid; ++k)
    for (int i = threadIdx.x; i < kMatStride; i += blockDim.x) s_m[k * kMatStride + i] = mats[ids[k] * kMatStride + i];
  __syncthreads();
}

// out[e] = M^-1 (M^L in[e-1] + M^R in[e]) along d   (Eq. l2forward)
// out[e] = M^-1 (M^L in[e] + M^R in[e+1]) along d   (Eq. l2backward)
template <bool TO_MAIN>
__global__ void __launch_bounds__(kThreads)
    k_project(Geo g, int d, const double* __restrict__ in, double* __restrict__ out, const double* mats) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kML, kMR, kWinv};
  load_mats(mats, s_m, ids, 3);
  const double* ML = s_m;
  const double* MR = s_m + kMatStride;
  const double* winv = s_m + 2 * kMatStride;
  const int n1 = g.n1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    const long long ec = elem_of(g, e);
    const long long en = elem_shift(g, e, d, TO_MAIN ? -1 : +1);
    const int m = l[d];
    int l0[3] = {l[0], l[1], l[2]};
    l0[d] = 0;
    const int lb = local_of(g, l0), st = lstride(g, d);
    const double* a = in + (TO_MAIN ? en : ec) * g.npe + lb;  // multiplied by M^L
    const double* b = in + (TO_MAIN ? ec : en) * g.npe + lb;  // multiplied by M^R
    double acc = 0.0;
    for (int q = 0; q < n1; ++q) acc += ML[m * n1 + q] * a[q * st] + MR[m * n1 + q] * b[q * st];
    out[idx] = acc * winv[m];
  }
}

// Trace of field X of element el at xi = side along d, at the face node given
// by the other local indices (lb = local base with l_d = 0).
__device__ __forceinline__ double trace(const double* X, long long el, int npe, int lb, int st, int n1,
                                        const double* phis) {
  const double* p = X + el * npe + lb;
  double s = 0.0;
  for (int q = 0; q < n1; ++q) s += phis[q] * p[q * st];
  return s;
}

// out_c = a V0_c + b (V_c + dt L(V)_c), with the collocated Rusanov DG operator
//   L(q) = - sum_d (1/dx_d) M_d^-1 [phi(1) F^_{e+1/2} - phi(0) F^_{e-1/2} - Dn^T W (q v_d)]
// F^ = (q^- v^- + q^+ v^+)/2 - s (q^+ - q^-)/2,  s = 2 max(|v_d^-|, |v_d^+|).
// Applied by lines: one thread per (element, line along d) forms the four
// traces and two face fluxes of its line once and the n1 outputs of every
// component.  Directions run as successive launches: the first writes L, the
// next add to it, the last writes out_c = a V0_c + b (V_c + dt L_c) instead.
struct ConvLineParams {
  Geo g;
  int d, first, last;
  double invdx;
  const double* V0[3];
  const double* V[3];
  double* L[3];
  double* out[3];
  double a, b, dt;
};

__global__ void __launch_bounds__(kThreads) k_convect_line(ConvLineParams p, const double* mats) {
  __shared__ double s_m[5 * kMatStride];
  const int ids[5] = {kW, kWinv, kPhi0, kPhi1, kDn};
  load_mats(mats, s_m, ids, 5);
  const double* w = s_m;
  const double* winv = s_m + kMatStride;
  const double* phi0 = s_m + 2 * kMatStride;
  const double* phi1 = s_m + 3 * kMatStride;
  const double* Dn = s_m + 4 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1, dim = g.dim, d = p.d;
  const int lpe = g.npe / n1;  // lines per element along d
  const long long nlines = g.ncell * (long long)lpe;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nlines;
       t += (long long)gridDim.x * blockDim.x) {
    const long long el = t / lpe;
    const int lam = (int)(t - el * lpe);
    int e[3];
    e[0] = (int)(el % g.n[0]);
    const long long rest = el / g.n[0];
    e[1] = (int)(rest % g.n[1]);
    e[2] = (int)(rest / g.n[1]);
    if (dim == 2) e[2] = 0;
    // the other local indices of the line, in increasing direction order
    int l0[3] = {0, 0, 0};
    {
      int r = lam;
      for (int d2 = 0; d2 < dim; ++d2) {
        if (d2 == d) continue;
        l0[d2] = r % n1;
        r /= n1;
      }
    }
    const int lb = local_of(g, l0), st = lstride(g, d);
    const long long ec = elem_of(g, e);
    const long long em = elem_shift(g, e, d, -1), ep = elem_shift(g, e, d, +1);
    const double* Vd = p.V[d];
    const double vd_l_m = trace(Vd, em, g.npe, lb, st, n1, phi1);
    const double vd_l_p = trace(Vd, ec, g.npe, lb, st, n1, phi0);
    const double vd_r_m = trace(Vd, ec, g.npe, lb, st, n1, phi1);
    const double vd_r_p = trace(Vd, ep, g.npe, lb, st, n1, phi0);
    const double s_l = 2.0 * fmax(fabs(vd_l_m), fabs(vd_l_p));
    const double s_r = 2.0 * fmax(fabs(vd_r_m), fabs(vd_r_p));
    const double* vdc = Vd + ec * g.npe + lb;
    for (int c = 0; c < dim; ++c) {
      const double* Q = p.V[c];
      const double q_l_m = trace(Q, em, g.npe, lb, st, n1, phi1);
      const double q_l_p = trace(Q, ec, g.npe, lb, st, n1, phi0);
      const double q_r_m = trace(Q, ec, g.npe, lb, st, n1, phi1);
      const double q_r_p = trace(Q, ep, g.npe, lb, st, n1, phi0);
      const double f_l = 0.5 * (q_l_m * vd_l_m + q_l_p * vd_l_p) - 0.5 * s_l * (q_l_p - q_l_m);
      const double f_r = 0.5 * (q_r_m * vd_r_m + q_r_p * vd_r_p) - 0.5 * s_r * (q_r_p - q_r_m);
      const double* qc = Q + ec * g.npe + lb;
      for (int m = 0; m < n1; ++m) {
        double vol = 0.0;
        for (int k = 0; k < n1; ++k) vol += w[k] * Dn[k * n1 + m] * qc[k * st] * vdc[k * st];
        const double surf = phi1[m] * f_r - phi0[m] * f_l;
        const long long idx = ec * g.npe + lb + (long long)m * st;
        const double Lv = (p.first ? 0.0 : p.L[c][idx]) - p.invdx * winv[m] * (surf - vol);
        if (p.last) {
          const double v0 = p.a != 0.0 ? p.V0[c][idx] : 0.0;
          p.out[c][idx] = p.a * v0 + p.b * (Q[idx] + p.dt * Lv);
        } else {
          p.L[c][idx] = Lv;
        }
      }
    }
  }
}


__global__ void __launch_bounds__(kThreads)
    k_mass(Geo g, const double* __restrict__ F, double* __restrict__ b, double* __restrict__ x0,
           const double* mats) {
  __shared__ double s_w[kMaxN1];
  if (threadIdx.x < kMaxN1) s_w[threadIdx.x] = mats[kW * kMatStride + threadIdx.x];
  __syncthreads();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    double W = s_w[l[0]] * s_w[l[1]];
    if (g.dim == 3) W *= s_w[l[2]];
    const double f = F[idx];
    b[idx] = W * f;
    if (x0) x0[idx] = f;
  }
}

// out = base + scale * sum_d (1/dx_d) M^{perp d} (Rb U_d[e] - Lb U_d[e-1])   (Eq. pSDG1)
struct DivParams {
  Geo g;
  double invdx[3];
  const double* U[3];
  const double* base;
  double scale;
  double* out;
};

__global__ void __launch_bounds__(kThreads) k_div(DivParams p, const double* mats, SolverState* st,
                                                  double* partials) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kRb, kLb, kW};
  load_mats(mats, s_m, ids, 3);
  const double* Rb = s_m;
  const double* Lb = s_m + kMatStride;
  const double* w = s_m + 2 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1;
  double sum = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    const long long ec = elem_of(g, e);
    double acc = 0.0;
    for (int d = 0; d < g.dim; ++d) {
      const long long em = elem_shift(g, e, d, -1);
      const int m = l[d];
      int l0[3] = {l[0], l[1], l[2]};
      l0[d] = 0;
      const int lb = local_of(g, l0), stp = lstride(g, d);
      const double* uc = p.U[d] + ec * g.npe + lb;
      const double* um = p.U[d] + em * g.npe + lb;
      double t = 0.0;
      for (int q = 0; q < n1; ++q) t += Rb[m * n1 + q] * uc[q * stp] - Lb[m * n1 + q] * um[q * stp];
      double wp = 1.0;
      for (int d2 = 0; d2 < g.dim; ++d2)
        if (d2 != d) wp *= w[l[d2]];
      acc += p.invdx[d] * wp * t;
    }
    const double v = (p.base ? p.base[idx] : 0.0) + p.scale * acc;
    p.out[idx] = v;
    sum += v;
  }
  double v1[1] = {sum}, tot[1];
  if (grid_sum<1>(v1, partials, &st->counter, tot) && threadIdx.x == 0) st->red[0] = tot[0];
}

__global__ void __launch_bounds__(kThreads)
    k_shift_kernel(double* __restrict__ x, long long n, const SolverState* st, int slot, double factor) {
  const double c = st->red[slot] * factor;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] -= c;
}

// U_d = U*_d - (dt/dx_d) M^-1 (R~ q[e+1] - L~ q[e]),  q = theta Pn + (1-theta) Po   (Eq. LOvelocityU)
struct VelParams {
  Geo g;
  double coef[3];  // dt / dx_d
  double theta;
  const double* Us[3];
  const double* Pn;
  const double* Po;
  double* U[3];
};

__global__ void __launch_bounds__(kThreads) k_velocity(VelParams p, const double* mats) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kRt, kLt, kWinv};
  load_mats(mats, s_m, ids, 3);
  const double* Rt = s_m;
  const double* Lt = s_m + kMatStride;
  const double* winv = s_m + 2 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1;
  const double th = p.theta, th1 = 1.0 - p.theta;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    const long long ec = elem_of(g, e);
    for (int d = 0; d < g.dim; ++d) {
      const long long ep = elem_shift(g, e, d, +1);
      const int m = l[d];
      int l0[3] = {l[0], l[1], l[2]};
      l0[d] = 0;
      const int lb = local_of(g, l0), stp = lstride(g, d);
      double t = 0.0;
      for (int q = 0; q < n1; ++q) {
        const long long ic = ec * g.npe + lb + q * stp, ip = ep * g.npe + lb + q * stp;
        const double qc = th * p.Pn[ic] + th1 * p.Po[ic];
        const double qp = th * p.Pn[ip] + th1 * p.Po[ip];
        t += Rt[m * n1 + q] * qp - Lt[m * n1 + q] * qc;
      }
      p.U[d][idx] = p.Us[d][idx] - p.coef[d] * winv[m] * t;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    k_wsum(Geo g, const double* __restrict__ x, const double* __restrict__ y, SolverState* st, int slot,
           double* partials, const double* mats) {
  __shared__ double s_w[kMaxN1];
  if (threadIdx.x < kMaxN1) s_w[threadIdx.x] = mats[kW * kMatStride + threadIdx.x];
  __syncthreads();
  double sum = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    double W = s_w[l[0]] * s_w[l[1]];
    if (g.dim == 3) W *= s_w[l[2]];
    sum += W * x[idx] * (y ? y[idx] : 1.0);
  }
  double v1[1] = {sum}, tot[1];
  if (grid_sum<1>(v1, partials, &st->counter, tot) && threadIdx.x == 0) st->red[slot] = tot[0];
}

__global__ void __launch_bounds__(kThreads)
    k_norm2_kernel(const double* __restrict__ x, long long n, SolverState* st, int slot, double* partials) {
  double sum = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    sum += x[i] * x[i];
  double v1[1] = {sum}, tot[1];
  if (grid_sum<1>(v1, partials, &st->counter, tot) && threadIdx.x == 0) st->red[slot] = tot[0];
}

// ------------------------------------------------------------------ kernel restoration
// part[b][l] = sum over elements e = b, b + G, ... of (x - x0)[e][l]
__global__ void __launch_bounds__(kThreads)
    k_kernel_partial(Geo g, const double* __restrict__ x, const double* __restrict__ x0, double* part) {
  const int G = gridDim.x;
  for (int l = threadIdx.x; l < g.npe; l += blockDim.x) {
    double acc = 0.0;
    for (long long e = blockIdx.x; e < g.ncell; e += G) {
      const long long i = e * g.npe + l;
      acc += x0 ? x[i] - x0[i] : x[i];
    }
    part[(size_t)blockIdx.x * g.npe + l] = acc;
  }
}

// One block: S = sum_b part[b]; corr = (1/ncell) (P1 (x) P1 (x) P1) S
__global__ void __launch_bounds__(kThreads)
    k_kernel_finalize(Geo g, const double* part, int G, const double* proj, double* corr) {
  extern __shared__ double sm[];
  double* A = sm;            // npe
  double* B = sm + g.npe;    // npe
  __shared__ double P1[kMaxN1 * kMaxN1];
  const int n1 = g.n1;
  for (int i = threadIdx.x; i < n1 * n1; i += blockDim.x) P1[i] = proj[i];
  for (int l = threadIdx.x; l < g.npe; l += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += part[(size_t)b * g.npe + l];
    A[l] = s;
  }
  __syncthreads();
  for (int d = 0; d < g.dim; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n1 : n1 * n1);
    for (int l = threadIdx.x; l < g.npe; l += blockDim.x) {
      const int m = (l / st) % n1;
      const int base = l - m * st;
      double t = 0.0;
      for (int q = 0; q < n1; ++q) t += P1[m * n1 + q] * A[base + q * st];
      B[l] = t;
    }
    __syncthreads();
    double* T = A;
    A = B;
    B = T;
  }
  for (int l = threadIdx.x; l < g.npe; l += blockDim.x) corr[l] = A[l] / (double)g.ncell;
}

__global__ void __launch_bounds__(kThreads)
    k_kernel_subtract(Geo g, double* __restrict__ x, const double* __restrict__ corr) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.ndof;
       i += (long long)gridDim.x * blockDim.x)
    x[i] -= corr[i % g.npe];
}

}  // namespace

cudaError_t kernel_restore(const sdg_handle* h, double* x, const double* x0, cudaStream_t s, int* launches) {
  const Geo& g = h->g;
  const int G = (int)(g.ncell < kKernelBlocks ? g.ncell : kKernelBlocks);
  k_kernel_partial<<<G, kThreads, 0, s>>>(g, x, x0, h->kpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = 2 * (size_t)g.npe * sizeof(double);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_kernel_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_kernel_finalize<<<1, kThreads, smem, s>>>(g, h->kpart, G, h->kproj, h->kcorr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_kernel_subtract<<<grid_for(g.ndof), kThreads, 0, s>>>(g, x, h->kcorr);
  *launches += 3;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
// Grid of the update launch: one wave of the four resident blocks per SM
// (a grid-wide finish costs a few ns per block; measured 10.3 against 12.3 us
// per launch for 4,194,304 FP32 values at 608 against 1216 blocks)
inline unsigned grid_update(long long n, int w, int nsm) {
  unsigned g = grid_vec(n, w);
  const unsigned cap = nsm > 0 ? 4u * (unsigned)nsm : g;
  return g < cap ? g : cap;
}
cudaError_t cg_update_f64(double* x, double* r, const double* p, const double* Ap, long long n,
                          SolverState* st, double* partials, int nsm, cudaStream_t s) {
  const unsigned g = grid_update(n, 2, nsm);
  if (x == nullptr)
    return launch_pdl(k_cg_update<double, false, false>, g, kThreads, 0, s, x, r, p, Ap, n, st, partials,
                      Deflate{});
  return launch_pdl(k_cg_update<double, false, true>, g, kThreads, 0, s, x, r, p, Ap, n, st, partials, Deflate{});
}
cudaError_t cg_update_f32(float* x, float* r, const float* p, const float* Ap, long long n,
                          SolverState* st, double* partials, const Deflate& df, int nsm, cudaStream_t s) {
  if (df.kpart == nullptr) {
    const unsigned g = grid_update(n, 4, nsm);
    if (x == nullptr)
      return launch_pdl(k_cg_update<float, false, false>, g, kThreads, 0, s, x, r, p, Ap, n, st, partials, df);
    return launch_pdl(k_cg_update<float, false, true>, g, kThreads, 0, s, x, r, p, Ap, n, st, partials, df);
  }
  // deflation: x += alpha p in the update launch (form 1 is forced)
  if (x == nullptr) return cudaErrorInvalidValue;
  const int npe = df.npe;
  const int G = kThreads >= 2 * npe ? kThreads / npe : 1;
  size_t smem = (size_t)(G + 1) * npe * sizeof(double);
  if (smem < npe * sizeof(float)) smem = npe * sizeof(float);
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_cg_update<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  unsigned g = grid_vec(n, 4);
  if (g > (unsigned)kDeflateBlocks) g = kDeflateBlocks;
  k_cg_update<float, true, true><<<g, kThreads, smem, s>>>(x, r, p, Ap, n, st, partials, df);
  return cudaGetLastError();
}
cudaError_t rel_accumulate(double* x64, float* x32, long long n, const SolverState* st, cudaStream_t s) {
  k_rel_accumulate<<<grid_for(n), kThreads, 0, s>>>(x64, x32, n, st);
  return cudaGetLastError();
}
cudaError_t rel_residual(const double* b, const double* Ax, double* r64, long long n, SolverState* st,
                         double* partials, double rtol, int maxit, double delta, int mode, int project,
                         int unscaled, cudaStream_t s) {
  k_rel_residual<<<grid_for(n), kThreads, 0, s>>>(b, Ax, r64, n, st, partials, rtol, maxit, delta, mode,
                                                  project, unscaled);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !project) return e;
  k_sub_mean<<<grid_for(n), kThreads, 0, s>>>(r64, n, st);
  return cudaGetLastError();
}
cudaError_t resid_norms(const double* b, const double* Ax, long long n, SolverState* st, double* partials,
                        cudaStream_t s) {
  k_resid_norms<<<grid_for(n), kThreads, 0, s>>>(b, Ax, n, st, partials);
  return cudaGetLastError();
}
cudaError_t rel_renorm(const double* r, long long n, SolverState* st, double* partials, int mode, cudaStream_t s) {
  k_rel_renorm<<<grid_for(n), kThreads, 0, s>>>(r, n, st, partials, mode);
  return cudaGetLastError();
}
cudaError_t pending_update(double* x, const double* p, long long n, const SolverState* st, cudaStream_t s) {
  k_pending_update<double><<<grid_for(n), kThreads, 0, s>>>(x, p, n, st);
  return cudaGetLastError();
}
cudaError_t pending_update(float* x, const float* p, long long n, const SolverState* st, cudaStream_t s) {
  k_pending_update<float><<<grid_for(n), kThreads, 0, s>>>(x, p, n, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t pending_x_t(T* x, const T* p, long long n, SolverState* st, cudaStream_t s) {
  k_pending_x<T><<<grid_for(n), kThreads, 0, s>>>(x, p, n, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&st->xpend, 0, sizeof(int), s);
}
cudaError_t pending_x(double* x, const double* p, long long n, SolverState* st, cudaStream_t s) {
  return pending_x_t(x, p, n, st, s);
}
cudaError_t pending_x(float* x, const float* p, long long n, SolverState* st, cudaStream_t s) {
  return pending_x_t(x, p, n, st, s);
}
cudaError_t rounding_perturbation(const double* x, double* u, long long n, cudaStream_t s) {
  k_rounding_perturbation<<<grid_for(n), kThreads, 0, s>>>(x, u, n);
  return cudaGetLastError();
}
cudaError_t rel_convert(const double* r64, float* r32, long long n, const SolverState* st, cudaStream_t s) {
  k_rel_convert<<<grid_for(n), kThreads, 0, s>>>(r64, r32, n, st);
  return cudaGetLastError();
}

cudaError_t k_dual_to_main(const sdg_handle* h, int d, const double* in, double* out, cudaStream_t s) {
  k_project<true><<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, d, in, out, h->mats);
  return cudaGetLastError();
}
cudaError_t k_main_to_dual(const sdg_handle* h, int d, const double* in, double* out, cudaStream_t s) {
  k_project<false><<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, d, in, out, h->mats);
  return cudaGetLastError();
}
cudaError_t k_convect_stage(const sdg_handle* h, const double* const* V0, const double* const* V,
                            double* const* out, double a, double b, double dt, cudaStream_t s) {
  const long long nlines = h->g.ndof / h->g.n1;
  for (int d = 0; d < h->dim; ++d) {
    ConvLineParams q;
    q.g = h->g;
    q.d = d;
    q.first = d == 0;
    q.last = d == h->dim - 1;
    q.invdx = 1.0 / h->dx[d];
    for (int c = 0; c < 3; ++c) {
      const bool on = c < h->dim;
      q.V0[c] = on && V0 ? V0[c] : nullptr;
      q.V[c] = on ? V[c] : nullptr;
      q.L[c] = on ? h->Lc[c] : nullptr;
      q.out[c] = on ? out[c] : nullptr;
    }
    q.a = a;
    q.b = b;
    q.dt = dt;
    k_convect_line<<<grid_full(nlines), kThreads, 0, s>>>(q, h->mats);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t k_mass_rhs(const sdg_handle* h, const double* F, double* b, double* x0, cudaStream_t s) {
  k_mass<<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, F, b, x0, h->mats);
  return cudaGetLastError();
}
cudaError_t k_divergence(const sdg_handle* h, const double* const* U, const double* base, double scale,
                         double* out, SolverState* st, double* partials, cudaStream_t s) {
  DivParams p;
  p.g = h->g;
  for (int d = 0; d < 3; ++d) {
    p.invdx[d] = d < h->dim ? 1.0 / h->dx[d] : 0.0;
    p.U[d] = d < h->dim ? U[d] : nullptr;
  }
  p.base = base;
  p.scale = scale;
  p.out = out;
  k_div<<<grid_for(h->g.ndof), kThreads, 0, s>>>(p, h->mats, st, partials);
  return cudaGetLastError();
}
cudaError_t k_shift(double* x, long long n, const SolverState* st, int slot, double factor, cudaStream_t s) {
  k_shift_kernel<<<grid_for(n), kThreads, 0, s>>>(x, n, st, slot, factor);
  return cudaGetLastError();
}
cudaError_t k_velocity_update(const sdg_handle* h, const double* const* Ustar, const double* Pn,
                              const double* Po, double* const* U, cudaStream_t s) {
  VelParams p;
  p.g = h->g;
  for (int d = 0; d < 3; ++d) {
    p.coef[d] = d < h->dim ? h->dt / h->dx[d] : 0.0;
    p.Us[d] = d < h->dim ? Ustar[d] : nullptr;
    p.U[d] = d < h->dim ? U[d] : nullptr;
  }
  p.theta = h->theta;
  p.Pn = Pn;
  p.Po = Po;
  k_velocity<<<grid_full(h->g.ndof), kThreads, 0, s>>>(p, h->mats);
  return cudaGetLastError();
}
cudaError_t k_weighted_sum(const sdg_handle* h, const double* x, const double* y, SolverState* st, int slot,
                           double* partials, cudaStream_t s) {
  k_wsum<<<grid_for(h->g.ndof), kThreads, 0, s>>>(h->g, x, y, st, slot, partials, h->mats);
  return cudaGetLastError();
}
cudaError_t k_norm2(const double* x, long long n, SolverState* st, int slot, double* partials, cudaStream_t s) {
  k_norm2_kernel<<<grid_for(n), kThreads, 0, s>>>(x, n, st, slot, partials);
  return cudaGetLastError();
}

}  // namespace sdg
