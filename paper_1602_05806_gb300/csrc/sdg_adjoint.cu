// Kernels of the adjoint (transposed linearisation) of one time step, FP64,
// one thread per output node in gather form: every output node sums the
// contributions of the inputs that the forward stage maps onto it, so no
// atomics are needed and the result is deterministic.  Transposes are with
// respect to the Euclidean inner product of the DOF arrays.
//
// Forward stages (Sec. 2.2 - 2.3) and their transposes:
//   Eq. l2forward   V[e]  = M^-1 (M^L U[e-1] + M^R U[e])
//                   U'[j] = M^Lt M^-1 V'[j+1] + M^Rt M^-1 V'[j]
//   Eq. l2backward  U[j]  = M^-1 (M^L F[j] + M^R F[j+1])
//                   F'[i] = M^Lt M^-1 U'[i] + M^Rt M^-1 U'[i-1]
//   Eq. LOvelocityU U_d   = U*_d - (dt/dx_d) M^-1 (R~ q[e+1] - L~ q[e])
//                   q'[e] = -sum_d (dt/dx_d) (R~t M^-1 U'_d[e-1] - L~t M^-1 U'_d[e])
//   Eq. pSDG1       b     = sum_d (1/dx_d) M^perp (R-bar U_d[e] - L-bar U_d[e-1])
//                   U'_d[j] = (1/dx_d) M^perp (R-bar^t b'[j] - L-bar^t b'[j+1])
//   Eqs. Fu-Fw      the Rusanov DG convection, linearised at a state X with
//                   the sub-gradient of the larger side of s = 2 max(|v-|, |v+|)
#include "sdg_device.cuh"

namespace sdg {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_full(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : b);
}

inline unsigned grid_red(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > kReduceBlocks) b = kReduceBlocks;
  return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void stage_mats(const double* mats, double* s_m, const int* ids, int nid) {
  for (int k = 0; k < nid; ++k)
    for (int i = threadIdx.x; i < kMatStride; i += blockDim.x) s_m[k * kMatStride + i] = mats[ids[k] * kMatStride + i];
  __syncthreads();
}

struct Line {
  long long ec, em, ep;  // element, its left and right neighbour along d
  int m, lb, st;         // node index along d, line base offset, stride
};

__device__ __forceinline__ Line line_of(const Geo& g, const int e[3], const int l[3], int d) {
  Line L;
  L.ec = elem_of(g, e);
  L.em = elem_shift(g, e, d, -1);
  L.ep = elem_shift(g, e, d, +1);
  L.m = l[d];
  int l0[3] = {l[0], l[1], l[2]};
  l0[d] = 0;
  L.lb = local_of(g, l0);
  L.st = lstride(g, d);
  return L;
}

// transposed L2 projections along d
template <bool DUAL_TO_MAIN>
__global__ void __launch_bounds__(kThreads)
    k_project_T(Geo g, int d, const double* __restrict__ lam, double* __restrict__ out, const double* mats) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kML, kMR, kWinv};
  stage_mats(mats, s_m, ids, 3);
  const double* ML = s_m;
  const double* MR = s_m + kMatStride;
  const double* winv = s_m + 2 * kMatStride;
  const int n1 = g.n1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    const Line L = line_of(g, e, l, d);
    // DUAL_TO_MAIN: MR^t on lam[e], ML^t on lam[e+1]; else ML^t on lam[e], MR^t on lam[e-1]
    const double* A = DUAL_TO_MAIN ? MR : ML;
    const double* B = DUAL_TO_MAIN ? ML : MR;
    const double* lc = lam + L.ec * g.npe + L.lb;
    const double* ln = lam + (DUAL_TO_MAIN ? L.ep : L.em) * g.npe + L.lb;
    double t = 0.0;
    for (int q = 0; q < n1; ++q)
      t += winv[q] * (A[q * n1 + L.m] * lc[q * L.st] + B[q * n1 + L.m] * ln[q * L.st]);
    out[idx] = t;
  }
}

// q' of the velocity update; lx = lamP + theta q', lPo = (1 - theta) q'
struct VelTParams {
  Geo g;
  double coef[3];  // dt / dx_d
  double theta;
  const double* lamU[3];
  const double* lamP;
  double* lx;
  double* lPo;
};

__global__ void __launch_bounds__(kThreads) k_velocity_T(VelTParams p, const double* mats) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kRt, kLt, kWinv};
  stage_mats(mats, s_m, ids, 3);
  const double* Rt = s_m;
  const double* Lt = s_m + kMatStride;
  const double* winv = s_m + 2 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    double q = 0.0;
    for (int d = 0; d < g.dim; ++d) {
      const Line L = line_of(g, e, l, d);
      const double* um = p.lamU[d] + L.em * g.npe + L.lb;
      const double* uc = p.lamU[d] + L.ec * g.npe + L.lb;
      double t = 0.0;
      for (int k = 0; k < n1; ++k)
        t += winv[k] * (Rt[k * n1 + L.m] * um[k * L.st] - Lt[k * n1 + L.m] * uc[k * L.st]);
      q -= p.coef[d] * t;
    }
    p.lx[idx] = p.lamP[idx] + p.theta * q;
    p.lPo[idx] = (1.0 - p.theta) * q;
  }
}

// out_d = lamU_d - (1/dx_d) M^perp (R-bar^t lb[e] - L-bar^t lb[e+1])
struct DivTParams {
  Geo g;
  double invdx[3];
  const double* lamU[3];
  const double* lb;
  double* out[3];
};

__global__ void __launch_bounds__(kThreads) k_div_T(DivTParams p, const double* mats) {
  __shared__ double s_m[3 * kMatStride];
  const int ids[3] = {kRb, kLb, kW};
  stage_mats(mats, s_m, ids, 3);
  const double* Rb = s_m;
  const double* Lb = s_m + kMatStride;
  const double* w = s_m + 2 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    for (int d = 0; d < g.dim; ++d) {
      const Line L = line_of(g, e, l, d);
      const double* bc = p.lb + L.ec * g.npe + L.lb;
      const double* bp = p.lb + L.ep * g.npe + L.lb;
      double t = 0.0;
      for (int k = 0; k < n1; ++k) t += Rb[k * n1 + L.m] * bc[k * L.st] - Lb[k * n1 + L.m] * bp[k * L.st];
      double wp = 1.0;
      for (int d2 = 0; d2 < g.dim; ++d2)
        if (d2 != d) wp *= w[l[d2]];
      p.out[d][idx] = p.lamU[d][idx] - p.invdx[d] * wp * t;
    }
  }
}

// out_c = a base_c + b (lam_c + k J(X)^t lam),  J the Jacobian of the
// convection operator L at X (every component c)
struct ConvTParams {
  Geo g;
  double invdx[3];
  const double* X[3];
  const double* lam[3];
  const double* base[3];
  double* out[3];
  double a, b, k;
};

__device__ __forceinline__ double trace_line(const double* p, int st, int n1, const double* phi) {
  double s = 0.0;
  for (int q = 0; q < n1; ++q) s += phi[q] * p[q * st];
  return s;
}

__global__ void __launch_bounds__(kThreads) k_convect_T(ConvTParams p, const double* mats) {
  __shared__ double s_m[5 * kMatStride];
  const int ids[5] = {kW, kWinv, kPhi0, kPhi1, kDn};
  stage_mats(mats, s_m, ids, 5);
  const double* w = s_m;
  const double* winv = s_m + kMatStride;
  const double* phi0 = s_m + 2 * kMatStride;
  const double* phi1 = s_m + 3 * kMatStride;
  const double* Dn = s_m + 4 * kMatStride;
  const Geo& g = p.g;
  const int n1 = g.n1, dim = g.dim, npe = g.npe;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    double gr[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < dim; ++d) {
      const Line L = line_of(g, e, l, d);
      const int m = L.m, st = L.st;
      const double* Xd = p.X[d];
      // normal velocity traces at the faces e-1/2 (l) and e+1/2 (r)
      const double vR_l = trace_line(Xd + L.em * npe + L.lb, st, n1, phi1);
      const double vLp_l = trace_line(Xd + L.ec * npe + L.lb, st, n1, phi0);
      const double vR_r = trace_line(Xd + L.ec * npe + L.lb, st, n1, phi1);
      const double vLp_r = trace_line(Xd + L.ep * npe + L.lb, st, n1, phi0);
      const bool left_l = fabs(vR_l) >= fabs(vLp_l), left_r = fabs(vR_r) >= fabs(vLp_r);
      const double s_l = 2.0 * fmax(fabs(vR_l), fabs(vLp_l));
      const double s_r = 2.0 * fmax(fabs(vR_r), fabs(vLp_r));
      auto sgn = [](double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); };
      const double sL_l = left_l ? 0.0 : 2.0 * sgn(vLp_l);   // ds/dv+ at the left face
      const double sR_r = left_r ? 2.0 * sgn(vR_r) : 0.0;    // ds/dv- at the right face
      const double xd_node = Xd[idx];
      for (int c = 0; c < dim; ++c) {
        const double* Xc = p.X[c];
        const double* lamc = p.lam[c];
        // Z = -(1/dx_d) M^-1 lam_c on the lines of e-1, e, e+1
        double fm1 = 0.0, f0c = 0.0, f1c = 0.0, fp0 = 0.0, vol = 0.0;
        for (int q = 0; q < n1; ++q) {
          const double zm = winv[q] * lamc[L.em * npe + L.lb + q * st];
          const double zc = winv[q] * lamc[L.ec * npe + L.lb + q * st];
          const double zp = winv[q] * lamc[L.ep * npe + L.lb + q * st];
          fm1 += phi1[q] * zm;
          f0c += phi0[q] * zc;
          f1c += phi1[q] * zc;
          fp0 += phi0[q] * zp;
          vol += Dn[m * n1 + q] * w[m] * zc;  // (DW)^t row m: DW[q][m] = Dn[m][q] w[m]
        }
        const double sc = -p.invdx[d];
        // lambda of the flux at the faces: lf = face(Z[e-1], 1) - face(Z[e], 0) (left),
        // face(Z[e], 1) - face(Z[e+1], 0) (right)
        const double lf_l = sc * (fm1 - f0c), lf_r = sc * (f1c - fp0);
        const double lprod = -sc * vol;
        gr[c] += lprod * xd_node;
        gr[d] += lprod * Xc[idx];
        // right face: this element is the "-" side (phi(1))
        const double qm_r = trace_line(Xc + L.ec * npe + L.lb, st, n1, phi1);
        const double qp_r = trace_line(Xc + L.ep * npe + L.lb, st, n1, phi0);
        gr[c] += phi1[m] * lf_r * (0.5 * vR_r + 0.5 * s_r);
        gr[d] += phi1[m] * (lf_r * 0.5 * qm_r - lf_r * 0.5 * (qp_r - qm_r) * sR_r);
        // left face: this element is the "+" side (phi(0))
        const double qm_l = trace_line(Xc + L.em * npe + L.lb, st, n1, phi1);
        const double qp_l = trace_line(Xc + L.ec * npe + L.lb, st, n1, phi0);
        gr[c] += phi0[m] * lf_l * (0.5 * vLp_l - 0.5 * s_l);
        gr[d] += phi0[m] * (lf_l * 0.5 * qp_l - lf_l * 0.5 * (qp_l - qm_l) * sL_l);
      }
    }
    for (int c = 0; c < dim; ++c) {
      const double bse = (p.a != 0.0) ? p.a * p.base[c][idx] : 0.0;
      p.out[c][idx] = bse + p.b * (p.lam[c][idx] + p.k * gr[c]);
    }
  }
}

// out = a x + b y (y may be null)
__global__ void __launch_bounds__(kThreads)
    k_axpby(double* __restrict__ out, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
            long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// st->red[slot] = sum_i x_i (y_i or 1)
__global__ void __launch_bounds__(kThreads)
    k_dot(const double* __restrict__ x, const double* __restrict__ y, long long n, SolverState* st, int slot,
          double* partials) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * (y ? y[i] : 1.0);
  double v[1] = {s}, tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st->red[slot] = tot[0];
}

// x -= (M^{xyz} weight of the node) * factor * st->red[slot]
__global__ void __launch_bounds__(kThreads)
    k_sub_weighted(Geo g, double* __restrict__ x, const SolverState* st, int slot, double factor, const double* mats) {
  __shared__ double s_w[kMaxN1];
  if (threadIdx.x < kMaxN1) s_w[threadIdx.x] = mats[kW * kMatStride + threadIdx.x];
  __syncthreads();
  const double c = st->red[slot] * factor;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.ndof;
       idx += (long long)gridDim.x * blockDim.x) {
    int e[3], l[3];
    split_index(g, idx, e, l);
    double W = s_w[l[0]] * s_w[l[1]];
    if (g.dim == 3) W *= s_w[l[2]];
    x[idx] -= W * c;
  }
}

}  // namespace

cudaError_t adj_project_T(const sdg_handle* h, bool dual_to_main, int d, const double* lam, double* out,
                          cudaStream_t s) {
  if (dual_to_main)
    k_project_T<true><<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, d, lam, out, h->mats);
  else
    k_project_T<false><<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, d, lam, out, h->mats);
  return cudaGetLastError();
}

cudaError_t adj_velocity_T(const sdg_handle* h, const double* const* lamU, const double* lamP, double* lx,
                           double* lPo, cudaStream_t s) {
  VelTParams p{};
  p.g = h->g;
  for (int d = 0; d < 3; ++d) {
    p.coef[d] = d < h->dim ? h->dt / h->dx[d] : 0.0;
    p.lamU[d] = d < h->dim ? lamU[d] : nullptr;
  }
  p.theta = h->theta;
  p.lamP = lamP;
  p.lx = lx;
  p.lPo = lPo;
  k_velocity_T<<<grid_full(h->g.ndof), kThreads, 0, s>>>(p, h->mats);
  return cudaGetLastError();
}

cudaError_t adj_divergence_T(const sdg_handle* h, const double* const* lamU, const double* lb, double* const* out,
                             cudaStream_t s) {
  DivTParams p{};
  p.g = h->g;
  for (int d = 0; d < 3; ++d) {
    p.invdx[d] = d < h->dim ? 1.0 / h->dx[d] : 0.0;
    p.lamU[d] = d < h->dim ? lamU[d] : nullptr;
    p.out[d] = d < h->dim ? out[d] : nullptr;
  }
  p.lb = lb;
  k_div_T<<<grid_full(h->g.ndof), kThreads, 0, s>>>(p, h->mats);
  return cudaGetLastError();
}

cudaError_t adj_convect_T(const sdg_handle* h, const double* const* X, const double* const* lam,
                          const double* const* base, double* const* out, double a, double b, double k,
                          cudaStream_t s) {
  ConvTParams p{};
  p.g = h->g;
  for (int d = 0; d < 3; ++d) {
    const bool on = d < h->dim;
    p.invdx[d] = on ? 1.0 / h->dx[d] : 0.0;
    p.X[d] = on ? X[d] : nullptr;
    p.lam[d] = on ? lam[d] : nullptr;
    p.base[d] = (on && base) ? base[d] : nullptr;
    p.out[d] = on ? out[d] : nullptr;
  }
  p.a = base ? a : 0.0;
  p.b = b;
  p.k = k;
  k_convect_T<<<grid_full(h->g.ndof), kThreads, 0, s>>>(p, h->mats);
  return cudaGetLastError();
}

cudaError_t adj_axpby(double* out, double a, const double* x, double b, const double* y, long long n,
                      cudaStream_t s) {
  k_axpby<<<grid_full(n), kThreads, 0, s>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t adj_dot(const double* x, const double* y, long long n, SolverState* st, int slot, double* partials,
                    cudaStream_t s) {
  k_dot<<<grid_red(n), kThreads, 0, s>>>(x, y, n, st, slot, partials);
  return cudaGetLastError();
}

cudaError_t adj_sub_weighted(const sdg_handle* h, double* x, const SolverState* st, int slot, double factor,
                             cudaStream_t s) {
  k_sub_weighted<<<grid_full(h->g.ndof), kThreads, 0, s>>>(h->g, x, st, slot, factor, h->mats);
  return cudaGetLastError();
}

}  // namespace sdg
