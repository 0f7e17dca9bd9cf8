// Element-tile kernel of the block penta- (2D) / hepta- (3D) diagonal
// staggered DG operator (Eq. pSyst):
//   y = cmass * W x + sum_d s_d M^{perp d} (H^L x_{i-1} + H^C x_i + H^R x_{i+1})_d
// applied dimension by dimension as 1D n1 x n1 contractions (Eq. tensorP1).
//
// One CTA owns a TX x TY (x TZ) box of elements.  It stages the box plus the
// one-element face halo in each direction (corners are never needed) in
// shared memory with coalesced vector loads, then runs one pass per
// direction in which every thread owns one 1D line of one element: it holds
// the 3 n1 line values (left neighbour, centre, right neighbour) in
// registers and forms the n1 outputs with the 1D blocks.  All threads of a
// warp use the same matrix entry at the same instruction, so the blocks are
// read straight from the kernel-parameter constant bank.  Partial results of
// the passes meet in a shared-memory accumulator; the last step stores the
// box with vector stores and (CG mode) leaves the block's p^T A p total for
// the update launch, which forms alpha (no grid-wide finish here).
#pragma once

#include <atomic>
#include <type_traits>

#include "sdg_device.cuh"

namespace sdg {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Element box per CTA for each (dim, n1): about 200-300 threads (one per
// line) for the base shape V = 0; in 2D, V = 1 doubles the box along x and
// V = 2 along y (fewer halo loads per element, twice the threads).
template <int DIM, int N1, int V = 0>
struct Tile {
  static constexpr int BX = DIM == 2 ? (N1 <= 1 ? 16 : N1 <= 2 ? 16 : N1 <= 4 ? 8 : N1 <= 8 ? 8 : 4)
                                     : (N1 <= 1 ? 8 : N1 <= 2 ? 4 : N1 <= 3 ? 4 : N1 <= 4 ? 4 : N1 <= 10 ? 2 : 1);
  static constexpr int BY = DIM == 2 ? (N1 <= 1 ? 16 : N1 <= 2 ? 8 : N1 <= 4 ? 8 : N1 <= 8 ? 4 : 4)
                                     : (N1 <= 1 ? 8 : N1 <= 2 ? 4 : N1 <= 3 ? 4 : N1 <= 4 ? 2 : N1 <= 8 ? 2 : 1);
  static constexpr int TX = BX * ((DIM == 2 && V == 1) ? 2 : 1);
  static constexpr int TY = BY * ((DIM == 2 && V == 2) ? 2 : 1);
  static constexpr int TZ = DIM == 2 ? 1
                                     : (N1 <= 1 ? 4 : N1 <= 2 ? 4 : N1 <= 3 ? 2 : N1 <= 4 ? 2 : N1 <= 5 ? 2 : 1);
  static constexpr int TE = TX * TY * TZ;
  static constexpr int NPE = ipow(N1, DIM);
  static constexpr int LINES = ipow(N1, DIM - 1);
  static constexpr int THREADS = TE * LINES;
  static constexpr int NSLOT = TE + 2 * TY * TZ + 2 * TX * TZ + (DIM == 3 ? 2 * TX * TY : 0);
  // shared-memory layout of one element: rows of N1 values padded to RS so
  // that the row-wise (x) and the strided (y, z) line reads of a warp hit
  // distinct banks
  static constexpr int RS = N1 + 1;
  static constexpr int PS = N1 * RS;
  static constexpr int ES = DIM == 2 ? PS : N1 * PS;
};

// Stored line operator in the compute precision, in the even/odd basis of
// the line (see CoefSet): H^R = [[A, B], [-B^T, D]], H^L = [[A, -B], [B^T, D]],
// H^C = diag(CE, CO); kernel correction rho (even N) or the fit and
// S0 / S1 correction (odd N).
template <typename T, int N1>
struct Coef {
  static constexpr int H = N1 / 2, HE = (N1 + 1) / 2, HO = H > 0 ? H : 1;
  T A[HE * HE], B[HE * HO], D[HO * HO], CE[HE * HE], CO[HO * HO];
  T rho_e[HE], rho_o[HO];
  T zn[HO], z2[HO], S0[HO], S1[HO], k1[HO];
  T k0, inv_n;
};

template <typename T, int DIM, int N1>
struct ApplyParams {
  Coef<T, N1> c;
  T w[N1];
  const T* x;
  const T* p_old;
  T* p_out;
  T* y;
  T s[3];
  T cmass;
  int n[3];
  int ntile[3];
  int fuse;
  SolverState* st;
  double* partials;
  const float* kc;  // FP32 CG: kernel part of r per local node (null = off)
  // fuse = 2 (one launch per CG iteration): x is r_{k-1}; ap_old = A p_{k-1};
  // r_out receives r_k = r_{k-1} - alpha Ap_{k-1}; xsol += alpha p_{k-1}
  const T* ap_old;
  T* r_out;
  T* xsol;
  int zc;  // marching 3D kernel: planes per CTA
};

template <typename T>
struct VecOf;
template <>
struct VecOf<double> { using V = double2; static constexpr int W = 2; };
template <>
struct VecOf<float> { using V = float4; static constexpr int W = 4; };

template <typename T, int NPE>
struct Vec {
  static constexpr bool kOk = (NPE * (int)sizeof(T)) % 16 == 0;
  static constexpr int W = kOk ? VecOf<T>::W : 1;
};

// Shared-memory slot of tile-local element (lx,ly,lz), which may lie one
// step outside the valid box [0,V) along exactly one direction.
template <int TX, int TY, int TZ>
__device__ __forceinline__ int slot_of(int lx, int ly, int lz, int VX, int VY, int VZ) {
  constexpr int TE = TX * TY * TZ;
  constexpr int XF = TE, YF = XF + 2 * TY * TZ, ZF = YF + 2 * TX * TZ;
  if (lx < 0) return XF + lz * TY + ly;
  if (lx >= VX) return XF + TY * TZ + lz * TY + ly;
  if (ly < 0) return YF + lz * TX + lx;
  if (ly >= VY) return YF + TX * TZ + lz * TX + lx;
  if (lz < 0) return ZF + ly * TX + lx;
  if (lz >= VZ) return ZF + TX * TY + ly * TX + lx;
  return (lz * TY + ly) * TX + lx;
}

// Global element coordinates held by slot s; false if the slot is unused.
template <int DIM, int TX, int TY, int TZ>
__device__ __forceinline__ bool slot_elem(int s, const int o[3], int VX, int VY, int VZ, const int n[3],
                                          int g[3]) {
  constexpr int TE = TX * TY * TZ;
  int lx, ly, lz;
  if (s < TE) {
    lx = s % TX;
    ly = (s / TX) % TY;
    lz = s / (TX * TY);
    if (lx >= VX || ly >= VY || lz >= VZ) return false;
  } else if ((s -= TE) < 2 * TY * TZ) {
    const int side = s / (TY * TZ), r = s % (TY * TZ);
    ly = r % TY;
    lz = r / TY;
    if (ly >= VY || lz >= VZ) return false;
    lx = side ? VX : -1;
  } else if ((s -= 2 * TY * TZ) < 2 * TX * TZ) {
    const int side = s / (TX * TZ), r = s % (TX * TZ);
    lx = r % TX;
    lz = r / TX;
    if (lx >= VX || lz >= VZ) return false;
    ly = side ? VY : -1;
  } else {
    if (DIM != 3) return false;
    s -= 2 * TX * TZ;
    const int side = s / (TX * TY), r = s % (TX * TY);
    lx = r % TX;
    ly = r / TX;
    if (lx >= VX || ly >= VY) return false;
    lz = side ? VZ : -1;
  }
  int gx = o[0] + lx, gy = o[1] + ly, gz = o[2] + lz;
  gx = gx < 0 ? gx + n[0] : (gx >= n[0] ? gx - n[0] : gx);
  gy = gy < 0 ? gy + n[1] : (gy >= n[1] ? gy - n[1] : gy);
  gz = gz < 0 ? gz + n[2] : (gz >= n[2] ? gz - n[2] : gz);
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
  return true;
}

// Last block of a one-launch CG iteration k: p.Ap, r.r (of r_k), r.Ap and
// Ap.Ap of this iteration.  alpha_k = r.r / p.Ap; the next direction needs
// beta_{k+1} = ||r_{k+1}||^2 / ||r_k||^2 before r_{k+1} exists, so its norm
// is formed ahead from r_{k+1} = r_k - alpha_k Ap_k:
//   ||r_{k+1}||^2 = r.r - 2 alpha_k r.Ap + alpha_k^2 Ap.Ap
// (the next launch reduces ||r_{k+1}||^2 directly for its own alpha and for
// the stopping test).  Stopping decisions as in the two-launch update.
__device__ __forceinline__ void cg_iteration_finish(SolverState* st, double pAp, double rr, double rAp,
                                                    double ApAp) {
  st->pAp = pAp;
  st->rr_old = st->rr;
  st->rr = rr;
  st->iter += 1;
  if (rr > st->maxrr) st->maxrr = rr;
  if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(rr)) {
    st->done = 1;
    st->status = SDG_ERR_BREAKDOWN;
    st->alpha = 0.0;
    st->beta = 0.0;
  } else {
    const double al = rr / pAp;
    double next = rr - 2.0 * al * rAp + al * al * ApAp;
    if (!(next > 0.0)) next = 0.0;
    st->alpha = al;
    st->beta = rr > 0.0 ? next / rr : 0.0;
    if (rr <= st->tol2) {
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
  st->alpha_f = (float)st->alpha;
  st->beta_f = (float)st->beta;
}

// The 1D line operator of one direction applied to one line of nodes: the
// outputs val[m] = f (H^L xl + H^C xc + H^R xr)[m] of the block row of
// Eq. pSyst (f: the direction's scale times the perpendicular weight), in
// the even/odd basis of the line (see Coef), with the accurate contraction
// when ACC.
template <typename T, int N1, bool ACC>
__device__ __forceinline__ void line_apply(const Coef<T, N1>& c, const T (&xl)[N1], const T (&xc)[N1],
                                           const T (&xr)[N1], T f, T (&val)[N1]) {
  // Even/odd form of the three line segments (see Coef): the neighbour
  // segments enter only through sE = l^_E + r^_E, dE = l^_E - r^_E,
  // sO = l^_O + r^_O, dO = r^_O - l^_O, the centre through cE, cO.
  constexpr int H = N1 / 2, HE = (N1 + 1) / 2, HO = H > 0 ? H : 1;
  constexpr bool MID = (N1 % 2) == 1;
  // Accuracy of the contraction (it matters in FP32).  The operator
  // annihilates every line-repeated pattern q of its local kernel (the
  // constants; for odd N also the sawtooth z), so q may be removed from
  // the three segments first: a centre node value c0 (differences of
  // nearby values are exact), then for odd N the orthogonal fit onto
  // {1, z} of the centre segment.  The operands shrink to the local
  // variation of smooth fields, and the rounding of the products drops
  // by orders of magnitude on the smooth and sawtooth-modulated modes
  // with tiny eigenvalues.  The stored blocks annihilate q only up to
  // rounding, so a symmetric correction (-rho, or -k0 S0 - k1 S1) keeps
  // the applied operator exactly symmetric and exactly zero on q.
  constexpr bool KZ = ACC && (N1 % 2 == 0);
  T sE[HE], dE[HE], sO[HO], dO[HO], cE[HE], cO[HO];
  if constexpr (ACC) {
    const T c0 = xc[N1 / 2];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const T l0 = xl[k] - c0, l1 = xl[N1 - 1 - k] - c0;
      const T r0 = xr[k] - c0, r1 = xr[N1 - 1 - k] - c0;
      sE[k] = (l0 + l1) + (r0 + r1);
      dE[k] = (l0 - r0) + (l1 - r1);
      const T lO = l0 - l1, rO = r0 - r1;
      sO[k] = lO + rO;
      dO[k] = rO - lO;
      const T c0k = xc[k] - c0, c1k = xc[N1 - 1 - k] - c0;
      cE[k] = c0k + c1k;
      cO[k] = c0k - c1k;
    }
    if constexpr (MID) {
      const T l0 = xl[H] - c0, r0 = xr[H] - c0;
      sE[H] = l0 + r0;
      dE[H] = l0 - r0;
      cE[H] = xc[H] - c0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const T lE = xl[k] + xl[N1 - 1 - k], lO = xl[k] - xl[N1 - 1 - k];
      const T rE = xr[k] + xr[N1 - 1 - k], rO = xr[k] - xr[N1 - 1 - k];
      sE[k] = lE + rE;
      dE[k] = lE - rE;
      sO[k] = lO + rO;
      dO[k] = rO - lO;
      cE[k] = xc[k] + xc[N1 - 1 - k];
      cO[k] = xc[k] - xc[N1 - 1 - k];
    }
    if constexpr (MID) {
      sE[H] = xl[H] + xr[H];
      dE[H] = xl[H] - xr[H];
      cE[H] = xc[H];
    }
  }
  if constexpr (KZ) {
    // orthogonal fit mu 1 + dz z of the centre segment, removed from all three
    T sum = T(0), dz = T(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      sum += cE[k];
      dz = fma(c.zn[k], cO[k], dz);
    }
    const T mu2 = T(2) * (sum * c.inv_n);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      cE[k] -= mu2;
      sE[k] = fma(T(-2), mu2, sE[k]);
      cO[k] = fma(-dz, c.z2[k], cO[k]);
      sO[k] = fma(T(-2) * dz, c.z2[k], sO[k]);
    }
  }
  // contractions: yE = A sE + B dO + CE cE ; yO = B^T dE + D sO + CO cO
  T yE[HE], yO[HO];
#pragma unroll
  for (int m = 0; m < HE; ++m) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < HE; ++j) {
      acc = fma(c.A[m * HE + j], sE[j], acc);
      acc = fma(c.CE[m * HE + j], cE[j], acc);
    }
#pragma unroll
    for (int j = 0; j < H; ++j) acc = fma(c.B[m * HO + j], dO[j], acc);
    yE[m] = acc;
  }
#pragma unroll
  for (int m = 0; m < H; ++m) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < HE; ++j) acc = fma(c.B[j * HO + m], dE[j], acc);
#pragma unroll
    for (int j = 0; j < H; ++j) {
      acc = fma(c.D[m * HO + j], sO[j], acc);
      acc = fma(c.CO[m * HO + j], cO[j], acc);
    }
    yO[m] = acc;
  }
  if constexpr (KZ) {
    T al = T(0), be = T(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      al = fma(c.S0[k], cE[k], al);
      be = fma(c.S1[k], cO[k], be);
    }
    const T ak = al * c.k0;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      yE[m] -= ak;
      yO[m] = fma(-be, c.k1[m], yO[m]);
    }
  } else if constexpr (ACC) {
#pragma unroll
    for (int m = 0; m < HE; ++m) yE[m] = fma(-c.rho_e[m], cE[m], yE[m]);
#pragma unroll
    for (int m = 0; m < H; ++m) yO[m] = fma(-c.rho_o[m], cO[m], yO[m]);
  }
  // back to the nodes: out_k = yE + yO, out_{n-1-k} = yE - yO (scaled)
#pragma unroll
  for (int m = 0; m < H; ++m) {
    const T t = f * yE[m];
    val[m] = fma(f, yO[m], t);
    val[N1 - 1 - m] = fma(-f, yO[m], t);
  }
  if constexpr (MID) val[H] = f * yE[H];
}

// ACC: accurate contraction (local kernel removal + symmetric correction),
// used for every FP32 application and for the FP64 true residuals of the
// mixed solver; plain FP64 CG uses the direct contraction.
// Blocks per SM the kernel is compiled for (register cap).  2D FP32 with
// n1 = 8 fits 40 registers without spills, so six 256-thread blocks (three
// of the 512-thread shapes) share an SM, as the shared-memory tile allows;
// elsewhere the compiler chooses.
// The one-launch CG iteration (ONE) keeps more values live (its r_k and four
// sums), so it is compiled for five blocks per SM instead of six.
template <typename T, int DIM, int N1, int V, bool ONE>
constexpr int apply_min_blocks() {
  return (sizeof(T) == 4 && DIM == 2 && N1 == 8) ? (ONE ? 5 : (V == 0 ? 6 : 3)) : 1;
}

// ONE: compiled for the one-launch CG iteration (fuse = 2) only; otherwise
// for the plain apply (fuse = 0) and the two-launch operator (fuse = 1).
template <typename T, int DIM, int N1, bool ACC, int TV, bool ONE>
__global__ void __launch_bounds__(Tile<DIM, N1, TV>::THREADS, (apply_min_blocks<T, DIM, N1, TV, ONE>()))
    k_apply(const __grid_constant__ ApplyParams<T, DIM, N1> a) {
  using TS = Tile<DIM, N1, TV>;
  constexpr int TX = TS::TX, TY = TS::TY, TZ = TS::TZ, TE = TS::TE;
  constexpr int NPE = TS::NPE, LINES = TS::LINES, NSLOT = TS::NSLOT;
  // thread t works on element t / LINES: whole elements per warp when LINES
  // divides 32 (and the block is whole warps)
  constexpr bool WARP_ELEMS = (32 % LINES == 0) && (TS::THREADS % 32 == 0);
  constexpr int VW = Vec<T, NPE>::W;
  constexpr int NV = NPE / VW;  // vectors per element
  using V = typename std::conditional<VW == 1, T, typename VecOf<T>::V>::type;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RS = TS::RS, PS = TS::PS, ES = TS::ES;
  T* s_in = reinterpret_cast<T*>(smem_raw);  // NSLOT * ES
  T* s_out = s_in + NSLOT * ES;              // TE * ES
  __shared__ T s_w[N1];
  __shared__ T s_kc[sizeof(T) == 4 ? NPE : 1];
  __shared__ int s_gel[NSLOT];  // global element held by each slot (-1: unused)

  const bool fuse = ONE || a.fuse != 0;
  constexpr bool fuse2 = ONE;
  const bool defl = sizeof(T) == 4 && fuse && !fuse2 && a.kc != nullptr;
  pdl_trigger();

  // prologue that reads nothing earlier kernels write: tile origin and valid
  // extents, weights, slot table (overlaps the previous kernel's tail)
  const int bx = blockIdx.x % a.ntile[0];
  const int by = (blockIdx.x / a.ntile[0]) % a.ntile[1];
  const int bz = blockIdx.x / (a.ntile[0] * a.ntile[1]);
  const int o[3] = {bx * TX, by * TY, bz * TZ};
  const int VX = min(TX, a.n[0] - o[0]);
  const int VY = min(TY, a.n[1] - o[1]);
  const int VZ = DIM == 3 ? min(TZ, a.n[2] - o[2]) : 1;

  if (threadIdx.x < N1) s_w[threadIdx.x] = a.w[threadIdx.x];
  // 2D tile fully inside the grid, elements of whole vectors: staging and
  // store take the element of each vector from its position (no slot table)
  const bool fast2 = DIM == 2 && !fuse2 && !defl && VW > 1 && VX == TX && VY == TY;
  if (!fast2)
  for (int sl = threadIdx.x; sl < NSLOT; sl += blockDim.x) {
    int g[3];
    s_gel[sl] = slot_elem<DIM, TX, TY, TZ>(sl, o, VX, VY, VZ, a.n, g)
                    ? (int)(((long long)g[2] * a.n[1] + g[1]) * a.n[0] + g[0])
                    : -1;
  }

  pdl_wait();
  bool first = false, xupd = false;
  T beta = T(0), alpha = T(0);
  if (fuse) {
    if (a.st->done || a.st->pause) return;  // uniform: written by the previous kernel
    first = (a.st->iter == 0);
    // alpha and beta were formed once by the previous kernel (no FP64
    // division per thread)
    if (!first) {
      beta = sizeof(T) == 4 ? (T)a.st->beta_f : (T)a.st->beta;
      alpha = sizeof(T) == 4 ? (T)a.st->alpha_f : (T)a.st->alpha;
      // two-launch form: x += alpha_{k-1} p_{k-1} on the owned nodes
      xupd = !fuse2 && a.xsol != nullptr && a.st->xpend != 0;
    }
  }
  if (defl)
    for (int l = threadIdx.x; l < NPE; l += blockDim.x) s_kc[l] = (T)a.kc[l];
  __syncthreads();

  // ---- stage box + face halo (coalesced vector loads, padded rows) ----
  // fuse = 2: the box values come first, in a fixed thread mapping (v = tid +
  // i blockDim) that the store loop repeats, so that each thread keeps its
  // r_k values in registers for the reductions
  constexpr int NBOX = (TE * NV + TS::THREADS - 1) / TS::THREADS;
  V rkeep[NBOX];
  if constexpr (fuse2) {
#pragma unroll
    for (int i = 0; i < NBOX; ++i) {
      const int v = threadIdx.x + i * TS::THREADS;
      if (v >= TE * NV) break;
      const int s = v / NV, off = v - s * NV;
      const int ge = s_gel[s];
      if (ge < 0) continue;
      const size_t gi = (size_t)ge * NV + off;
      V r = reinterpret_cast<const V*>(a.x)[gi];
      V val;
      T* rp = reinterpret_cast<T*>(&r);
      T* vp = reinterpret_cast<T*>(&val);
      if (first) {
        val = r;
      } else {
        const V ao = reinterpret_cast<const V*>(a.ap_old)[gi];
        const V po = reinterpret_cast<const V*>(a.p_old)[gi];
        V xv = reinterpret_cast<const V*>(a.xsol)[gi];
        const T* ap = reinterpret_cast<const T*>(&ao);
        const T* pp = reinterpret_cast<const T*>(&po);
        T* xp = reinterpret_cast<T*>(&xv);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          rp[k] = fma(-alpha, ap[k], rp[k]);  // r_k = r_{k-1} - alpha Ap_{k-1}
          xp[k] = fma(alpha, pp[k], xp[k]);   // x_k = x_{k-1} + alpha p_{k-1}
          vp[k] = fma(beta, pp[k], rp[k]);    // p_k = r_k + beta p_{k-1}
        }
        reinterpret_cast<V*>(a.xsol)[gi] = xv;
      }
      reinterpret_cast<V*>(a.r_out)[gi] = r;
      reinterpret_cast<V*>(a.p_out)[gi] = val;
      rkeep[i] = r;
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        const int q = off * VW + k, row = q / N1, l1 = q - row * N1;
        s_in[s * ES + row * RS + l1] = vp[k];
      }
    }
  }
  if (fast2) {
    constexpr int RV = TX * NV;  // vectors in one box row of TX elements
    const int nx = a.n[0], ny = a.n[1];
    // one vector of the value the passes read: x (plain) or p = r + beta
    // p_old (CG; owned: stored, and x += alpha p_old), into slot at off
    auto stage2 = [&](size_t gi, bool owned, int slot, int off) {
      V val = reinterpret_cast<const V*>(a.x)[gi];
      if (fuse && !first) {
        const V po = reinterpret_cast<const V*>(a.p_old)[gi];
        T* vp = reinterpret_cast<T*>(&val);
        const T* pp = reinterpret_cast<const T*>(&po);
#pragma unroll
        for (int k = 0; k < VW; ++k) vp[k] = vp[k] + beta * pp[k];
        if (owned && xupd) {
          V xv = reinterpret_cast<const V*>(a.xsol)[gi];
          T* xp = reinterpret_cast<T*>(&xv);
#pragma unroll
          for (int k = 0; k < VW; ++k) xp[k] = fma(alpha, pp[k], xp[k]);
          reinterpret_cast<V*>(a.xsol)[gi] = xv;
        }
      }
      if (fuse && owned) reinterpret_cast<V*>(a.p_out)[gi] = val;
      const T* vp = reinterpret_cast<const T*>(&val);
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        const int q = off * VW + k, row = q / N1, l1 = q - row * N1;
        s_in[slot * ES + row * RS + l1] = vp[k];
      }
    };
    for (int v = threadIdx.x; v < TY * RV; v += TS::THREADS) {  // box rows
      const int row = v / RV, i = v - row * RV, e = i / NV;
      stage2(((size_t)(o[1] + row) * nx + o[0]) * NV + i, true, row * TX + e, i - e * NV);
    }
    for (int v = threadIdx.x; v < 2 * RV; v += TS::THREADS) {  // y = -1, y = TY rows
      const int side = v / RV, i = v - side * RV, e = i / NV;
      int gy = side ? o[1] + TY : o[1] - 1;
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      stage2(((size_t)gy * nx + o[0]) * NV + i, false, TE + 2 * TY + side * TX + e, i - e * NV);
    }
    for (int v = threadIdx.x; v < 2 * TY * NV; v += TS::THREADS) {  // x = -1, x = TX columns
      const int sl = v / NV, off = v - sl * NV, side = sl / TY, ly = sl - side * TY;
      int gx = side ? o[0] + TX : o[0] - 1;
      gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
      stage2(((size_t)(o[1] + ly) * nx + gx) * NV + off, false, TE + sl, off);
    }
  } else
  for (int v = threadIdx.x + (fuse2 ? TE * NV : 0); v < NSLOT * NV; v += blockDim.x) {
    const int s = v / NV, off = v - s * NV;
    const int ge = s_gel[s];
    if (ge < 0) continue;
    const size_t gi = (size_t)ge * NV + off;
    V val;
    if (fuse2) {
      // face halo: p_k of the neighbour, formed as its owner forms it
      V r = reinterpret_cast<const V*>(a.x)[gi];
      T* rp = reinterpret_cast<T*>(&r);
      T* vp = reinterpret_cast<T*>(&val);
      if (first) {
        val = r;
      } else {
        const V ao = reinterpret_cast<const V*>(a.ap_old)[gi];
        const V po = reinterpret_cast<const V*>(a.p_old)[gi];
        const T* ap = reinterpret_cast<const T*>(&ao);
        const T* pp = reinterpret_cast<const T*>(&po);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          rp[k] = fma(-alpha, ap[k], rp[k]);
          vp[k] = fma(beta, pp[k], rp[k]);
        }
      }
    } else if (!fuse) {
      val = reinterpret_cast<const V*>(a.x)[gi];
    } else {
      V r = reinterpret_cast<const V*>(a.x)[gi];
      if (defl) {  // the direction is built from the residual's range part
        T* rp = reinterpret_cast<T*>(&r);
#pragma unroll
        for (int k = 0; k < VW; ++k) rp[k] -= s_kc[off * VW + k];
      }
      if (first) {
        val = r;
      } else {
        V po = reinterpret_cast<const V*>(a.p_old)[gi];
        const T* rp = reinterpret_cast<const T*>(&r);
        const T* pp = reinterpret_cast<const T*>(&po);
        T* vp = reinterpret_cast<T*>(&val);
#pragma unroll
        for (int k = 0; k < VW; ++k) vp[k] = rp[k] + beta * pp[k];
        if (xupd && s < TE) {
          V xv = reinterpret_cast<const V*>(a.xsol)[gi];
          T* xp = reinterpret_cast<T*>(&xv);
#pragma unroll
          for (int k = 0; k < VW; ++k) xp[k] = fma(alpha, pp[k], xp[k]);
          reinterpret_cast<V*>(a.xsol)[gi] = xv;
        }
      }
      if (s < TE) reinterpret_cast<V*>(a.p_out)[gi] = val;
    }
    const T* vp = reinterpret_cast<const T*>(&val);
#pragma unroll
    for (int k = 0; k < VW; ++k) {
      const int q = off * VW + k, row = q / N1, l1 = q - row * N1;
      s_in[s * ES + row * RS + l1] = vp[k];
    }
  }
  __syncthreads();

  // ---- one pass per direction ----
  const int t = threadIdx.x;
  const int te = t / LINES, lam = t - te * LINES;
  const int lx = te % TX, ly = (te / TX) % TY, lz = te / (TX * TY);
  const bool active = (lx < VX) && (ly < VY) && (lz < VZ);

#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (active) {
      // fixed local indices of this line, its padded base offset and stride
      int base;
      const int stride = d == 0 ? 1 : (d == 1 ? RS : PS);
      T wp;
      if (DIM == 2) {
        // d = 0: lam = l2 (row), d = 1: lam = l1 (column)
        base = d == 0 ? lam * RS : lam;
        wp = s_w[lam];
      } else {
        const int q0 = lam % N1, q1 = lam / N1;
        if (d == 0) base = q0 * RS + q1 * PS;       // (l2, l3) = (q0, q1)
        else if (d == 1) base = q0 + q1 * PS;       // (l1, l3)
        else base = q0 + q1 * RS;                   // (l1, l2)
        wp = s_w[q0] * s_w[q1];
      }
      const int sc = (lz * TY + ly) * TX + lx;
      const int sl = slot_of<TX, TY, TZ>(lx - (d == 0), ly - (d == 1), lz - (d == 2), VX, VY, VZ);
      const int sr = slot_of<TX, TY, TZ>(lx + (d == 0), ly + (d == 1), lz + (d == 2), VX, VY, VZ);
      T xl[N1], xc[N1], xr[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        xl[k] = s_in[sl * ES + base + k * stride];
        xc[k] = s_in[sc * ES + base + k * stride];
        xr[k] = s_in[sr * ES + base + k * stride];
      }
      T val[N1];
      line_apply<T, N1, ACC>(a.c, xl, xc, xr, a.s[d] * wp, val);
      T* out = s_out + te * ES + base;
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        T v = val[m];
        if (d == 0) {
          if (a.cmass != T(0)) v = fma(a.cmass * wp * s_w[m], xc[m], v);
          out[m * stride] = v;
        } else {
          out[m * stride] += v;
        }
      }
    }
    // the passes of one element exchange data only through its own rows of
    // s_out; when whole elements fall in one warp, a warp barrier suffices
    if constexpr (WARP_ELEMS) __syncwarp();
    else __syncthreads();
  }

  if constexpr (fuse2) {
    // ---- one launch per CG iteration: store Ap_k and reduce, in the staging
    // thread mapping, p.Ap and r.r (compensated), r.Ap and Ap.Ap ----
    __syncthreads();
    T s_pa = T(0), c_pa = T(0), s_rr = T(0), c_rr = T(0), s_ra = T(0), s_aa = T(0);
#pragma unroll
    for (int i = 0; i < NBOX; ++i) {
      const int v = threadIdx.x + i * TS::THREADS;
      if (v >= TE * NV) break;
      const int e = v / NV, off = v - e * NV;
      const int ge = s_gel[e];
      if (ge < 0) continue;
      V yv;
      T* yp = reinterpret_cast<T*>(&yv);
      const T* rp = reinterpret_cast<const T*>(&rkeep[i]);
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        const int q = off * VW + k, row = q / N1, l1 = q - row * N1;
        const T y = s_out[e * ES + row * RS + l1];
        const T pv = s_in[e * ES + row * RS + l1];
        yp[k] = y;
        const T t1 = fma(pv, y, -c_pa);
        const T u1 = s_pa + t1;
        c_pa = (u1 - s_pa) - t1;
        s_pa = u1;
        const T t2 = fma(rp[k], rp[k], -c_rr);
        const T u2 = s_rr + t2;
        c_rr = (u2 - s_rr) - t2;
        s_rr = u2;
        s_ra = fma(rp[k], y, s_ra);
        s_aa = fma(y, y, s_aa);
      }
      reinterpret_cast<V*>(a.y)[(size_t)ge * NV + off] = yv;
    }
    double tot[4];
    bool last;
    if constexpr (sizeof(T) == 4) {
      F2 v4[4] = {F2{(float)s_pa, -(float)c_pa}, F2{(float)s_rr, -(float)c_rr}, F2{(float)s_ra, 0.0f},
                  F2{(float)s_aa, 0.0f}};
      last = grid_sum_f2<4>(v4, a.partials, &a.st->counter, tot);
    } else {
      double v4[4] = {(double)s_pa - (double)c_pa, (double)s_rr - (double)c_rr, (double)s_ra, (double)s_aa};
      last = grid_sum<4>(v4, a.partials, &a.st->counter, tot);
    }
    if (last && threadIdx.x == 0) cg_iteration_finish(a.st, tot[0], tot[1], tot[2], tot[3]);
    return;
  }

  // ---- store the box (vectorised) and reduce p^T A p ----
  // (WARP_ELEMS: every warp stores the elements it computed, with no block
  // barrier in between)
  T dsum = T(0), dcomp = T(0);  // compensated per-thread sum in T
  constexpr int EPW = WARP_ELEMS ? 32 / LINES : 1;  // elements per warp
  const int v0 = WARP_ELEMS ? (threadIdx.x >> 5) * EPW * NV + (threadIdx.x & 31) : threadIdx.x;
  const int v1 = WARP_ELEMS ? min(((threadIdx.x >> 5) + 1) * EPW, TE) * NV : TE * NV;
  const int vstep = WARP_ELEMS ? 32 : blockDim.x;
  for (int v = v0; v < v1; v += vstep) {
    const int e = v / NV, off = v - e * NV;
    const int ge = fast2 ? (o[1] + e / TX) * a.n[0] + o[0] + e % TX : s_gel[e];
    if (ge < 0) continue;
    V yv, pv;
    T* yp = reinterpret_cast<T*>(&yv);
    T* pp = reinterpret_cast<T*>(&pv);
#pragma unroll
    for (int k = 0; k < VW; ++k) {
      const int q = off * VW + k, row = q / N1, l1 = q - row * N1;
      yp[k] = s_out[e * ES + row * RS + l1];
      pp[k] = s_in[e * ES + row * RS + l1];
    }
    reinterpret_cast<V*>(a.y)[(size_t)ge * NV + off] = yv;
    if (fuse) {
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        const T yk = fma(pp[k], yp[k], -dcomp);
        const T tt = dsum + yk;
        dcomp = (tt - dsum) - yk;
        dsum = tt;
      }
    }
  }
  if (fuse) {
    // the block's p.Ap total for the update launch, which forms alpha
    __shared__ double s_opr[32];
    if constexpr (sizeof(T) == 4) op_partial_f2(F2{(float)dsum, -(float)dcomp}, a.partials, s_opr);
    else op_partial_f64((double)dsum - (double)dcomp, a.partials, s_opr);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->nop = (int)gridDim.x;
  }
}

// Kernel parameters from the handle and the launch arguments: the stored
// line operator in the compute precision, the weights, pointers, scales and
// grid size (the tile counts are set by each launcher).
template <typename T, int DIM, int N1>
void fill_apply_params(const sdg_handle* h, const ApplyArgs<T>& in, ApplyParams<T, DIM, N1>* pp) {
  ApplyParams<T, DIM, N1>& p = *pp;
  const Basis1D& b = h->basis;
  const CoefSet& cs = sizeof(T) == 4 ? h->coef32 : h->coef64;  // values exact in T
  constexpr int H = N1 / 2, HE = (N1 + 1) / 2, HO = H > 0 ? H : 1;
  p.c = Coef<T, N1>{};
  for (int i = 0; i < HE; ++i)
    for (int j = 0; j < HE; ++j) {
      p.c.A[i * HE + j] = (T)cs.A[i * HE + j];
      p.c.CE[i * HE + j] = (T)cs.CE[i * HE + j];
    }
  for (int i = 0; i < HE; ++i)
    for (int j = 0; j < H; ++j) p.c.B[i * HO + j] = (T)cs.B[i * H + j];
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < H; ++j) {
      p.c.D[i * HO + j] = (T)cs.D[i * H + j];
      p.c.CO[i * HO + j] = (T)cs.CO[i * H + j];
    }
  for (int i = 0; i < HE; ++i) p.c.rho_e[i] = (T)cs.rho_e[i];
  for (int i = 0; i < H; ++i) {
    p.c.rho_o[i] = (T)cs.rho_o[i];
    p.c.zn[i] = (T)cs.zn[i];
    p.c.z2[i] = (T)cs.z2[i];
    p.c.S0[i] = (T)cs.S0[i];
    p.c.S1[i] = (T)cs.S1[i];
    p.c.k1[i] = (T)cs.k1[i];
  }
  p.c.k0 = (T)cs.k0;
  p.c.inv_n = (T)cs.inv_n;
  for (int i = 0; i < N1; ++i) p.w[i] = (T)b.w[i];
  p.x = in.x;
  p.p_old = in.p_old;
  p.p_out = in.p_out;
  p.y = in.y;
  for (int d = 0; d < 3; ++d) p.s[d] = (T)in.s[d];
  p.cmass = (T)in.cmass;
  p.n[0] = h->g.n[0];
  p.n[1] = h->g.n[1];
  p.n[2] = DIM == 3 ? h->g.n[2] : 1;
  p.fuse = in.fuse;
  p.st = in.st;
  p.partials = in.partials;
  p.kc = in.kc;
  p.ap_old = in.ap_old;
  p.r_out = in.r_out;
  p.xsol = in.xsol;
  p.zc = 0;
}

template <typename T, int DIM, int N1, bool ACC, int V, bool ONE = false>
cudaError_t launch_apply_acc(const sdg_handle* h, const ApplyArgs<T>& in, cudaStream_t stream) {
  using TS = Tile<DIM, N1, V>;
  ApplyParams<T, DIM, N1> p;
  fill_apply_params<T, DIM, N1>(h, in, &p);
  p.ntile[0] = (p.n[0] + TS::TX - 1) / TS::TX;
  p.ntile[1] = (p.n[1] + TS::TY - 1) / TS::TY;
  p.ntile[2] = (p.n[2] + TS::TZ - 1) / TS::TZ;
  const long long nblk = (long long)p.ntile[0] * p.ntile[1] * p.ntile[2];
  if (nblk > h->max_blocks) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)(TS::NSLOT + TS::TE) * TS::ES * sizeof(T);
  // per instantiation (its shared-memory need is fixed); handles of a batch
  // launch from several host threads, and setting the attribute twice is
  // harmless
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_apply<T, DIM, N1, ACC, V, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(TS::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = in.pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_apply<T, DIM, N1, ACC, V, ONE>, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Tile shape variants exist for the 2D FP32 operator only (the FP64 one is
// bound by the FP64 pipe, not by the tile).
template <typename T, int DIM, int N1>
cudaError_t launch_apply_t(const sdg_handle* h, const ApplyArgs<T>& in, cudaStream_t stream) {
  // the one-launch CG iteration: base tile, accurate contraction
  if (in.fuse == 2) return launch_apply_acc<T, DIM, N1, true, 0, true>(h, in, stream);
  if constexpr (sizeof(T) == 4) {
    if constexpr (DIM == 2) {
      if (in.tile == 1) return launch_apply_acc<T, DIM, N1, true, 1>(h, in, stream);
      if (in.tile == 2) return launch_apply_acc<T, DIM, N1, true, 2>(h, in, stream);
    }
    return launch_apply_acc<T, DIM, N1, true, 0>(h, in, stream);
  } else {
    if (in.accurate) return launch_apply_acc<T, DIM, N1, true, 0>(h, in, stream);
    return launch_apply_acc<T, DIM, N1, false, 0>(h, in, stream);
  }
}

}  // namespace sdg
