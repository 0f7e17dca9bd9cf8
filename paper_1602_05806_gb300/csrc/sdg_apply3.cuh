// 3D operator kernel that marches through z (block hepta-diagonal system of
// Eq. pSyst, applied dimension by dimension as 1D contractions, Eq. tensorP1).
//
// One CTA owns a column of TX x TY elements in x and y and a run of zc planes
// in z.  It keeps three planes of the column (z-1, z, z+1) in a shared-memory
// ring and, per step, loads one new plane plus the x/y face halo of the plane
// it computes: every element is read about 1 + 2 (TX + TY) / (TX TY) + 2 / zc
// times (about 2.2 for 4 x 4 and zc = 12) instead of once per face
// neighbour.  Each thread owns one 1D line of one element of the plane per
// direction and applies the line operator (line_apply: the same accurate
// contraction as the element-tile kernel).  Each direction writes its own
// shared-memory accumulator (no barrier between the passes); the store adds
// them, and each plane is stored as it is finished.
//
// Modes as in k_apply: plain apply (fuse 0), the operator of the two-launch
// CG iteration (fuse 1: p = r + beta p_old, x += alpha p_old when the state
// asks for it, and the block's p.Ap total for the update launch) and the one-launch CG
// iteration (ONE: r -= alpha Ap_old, x += alpha p_old, p = r + beta p_old,
// Ap, and p.Ap, r.r, r.Ap, Ap.Ap).  Planes z0 - 1 and z0 + zc belong to the
// neighbouring runs: this CTA forms their values but writes nothing there.
#pragma once

#include "sdg_apply.cuh"

namespace sdg {

template <int N1>
struct March3 {
  static constexpr int TX = 4, TY = 4;
  static constexpr int PE = TX * TY;           // elements of one plane of the column
  static constexpr int NPE = N1 * N1 * N1;
  static constexpr int LINES = N1 * N1;        // lines of an element per direction
  static constexpr int THREADS = PE * LINES;
  // rows of N1 values, padded for even N1 only: for odd N1 the strided line
  // reads of a warp already fall on distinct banks, and the unpadded layout
  // makes staging a plain copy
  static constexpr int RS = (N1 % 2) ? N1 : N1 + 1;
  static constexpr int PS = N1 * RS;
  static constexpr int ES = N1 * PS;
  static constexpr int HALO = 2 * TX + 2 * TY;  // x and y face halo of a plane
};

// shared-memory offset of element-local node q (x fastest)
template <int N1>
__device__ __forceinline__ int m3_sidx(int q) {
  using M = March3<N1>;
  if constexpr (M::RS == N1) return q;
  const int row = q / N1;
  return row * M::RS + (q - row * N1);
}

// x-face halo slot of the marching kernel: an element rounded up to whole
// vectors of T
template <typename T, int N1>
__host__ __device__ constexpr int m3_halo_slot() {
  return (March3<N1>::ES + VecOf<T>::W - 1) / VecOf<T>::W * VecOf<T>::W;
}

// Resident CTAs per SM the kernel is compiled for (a register cap: without
// barriers between the passes the compiler keeps more values live): three
// in FP32 (48 registers per thread), two in FP64
template <typename T, bool ONE>
constexpr int march3_min_blocks() {
  return sizeof(T) == 4 ? 3 : 2;
}

template <typename T, int N1, bool ACC, bool ONE>
__global__ void __launch_bounds__(March3<N1>::THREADS, (march3_min_blocks<T, ONE>()))
    k_apply3m(const __grid_constant__ ApplyParams<T, 3, N1> a) {
  using M = March3<N1>;
  constexpr int TX = M::TX, TY = M::TY, PE = M::PE, NPE = M::NPE, LINES = M::LINES;
  constexpr int RS = M::RS, PS = M::PS, ES = M::ES, HALO = M::HALO, THREADS = M::THREADS;
  using VT = typename VecOf<T>::V;
  constexpr int VW = VecOf<T>::W;
  constexpr int HS = m3_halo_slot<T, N1>();  // x-halo slot: ES rounded up to whole vectors
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);  // 3 planes: 3 * PE * ES
  T* xhalo = ring + 3 * PE * ES;             // x = -1, x = VX faces: 2 TY * HS
  T* yhalo = xhalo + 2 * TY * HS;            // y = -1, y = VY faces (rows): 2 TX * ES
  T* s_out = yhalo + 2 * TX * ES;            // one accumulator per direction: 3 * PE * ES
  T* rring = s_out + 3 * PE * ES;            // ONE: r_k of the owned planes by ring slot, 3 * PE * ES
  __shared__ T s_w[N1];

  const bool fuse = ONE || a.fuse != 0;
  pdl_trigger();
  const int bx = blockIdx.x % a.ntile[0];
  const int by = (blockIdx.x / a.ntile[0]) % a.ntile[1];
  const int bz = blockIdx.x / (a.ntile[0] * a.ntile[1]);
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int ox = bx * TX, oy = by * TY, z0 = bz * a.zc;
  const int VX = min(TX, nx - ox), VY = min(TY, ny - oy);
  const int NZ = min(a.zc, nz - z0);  // planes owned by this CTA
  if (threadIdx.x < N1) s_w[threadIdx.x] = a.w[threadIdx.x];

  pdl_wait();
  bool first = false, xupd = false;
  T beta = T(0), alpha = T(0);
  if (fuse) {
    if (a.st->done || a.st->pause) return;  // uniform: written by the previous kernel
    first = (a.st->iter == 0);
    if (!first) {
      beta = sizeof(T) == 4 ? (T)a.st->beta_f : (T)a.st->beta;
      alpha = sizeof(T) == 4 ? (T)a.st->alpha_f : (T)a.st->alpha;
      // two-launch form: x += alpha_{k-1} p_{k-1} on the owned nodes
      xupd = !ONE && a.xsol != nullptr && a.st->xpend != 0;
    }
  }

  // the value of node gi that the passes read: x (plain), p = r + beta p_old
  // (CG); for an owned node also the CG writes (kept r_k in *rk)
  auto stage = [&](size_t gi, bool owned, T* rk) -> T {
    if (!fuse) return a.x[gi];
    T r = a.x[gi];
    if constexpr (ONE) {
      if (!first) {
        const T po = a.p_old[gi];
        r = fma(-alpha, a.ap_old[gi], r);
        const T p = fma(beta, po, r);
        if (owned) {
          a.xsol[gi] = fma(alpha, po, a.xsol[gi]);
          a.r_out[gi] = r;
          a.p_out[gi] = p;
          *rk = r;
        }
        return p;
      }
      if (owned) {
        a.r_out[gi] = r;
        a.p_out[gi] = r;
        *rk = r;
      }
      return r;
    } else {
      if (first) {
        if (owned) a.p_out[gi] = r;
        return r;
      }
      const T po = a.p_old[gi];
      const T p = fma(beta, po, r);
      if (owned) {
        a.p_out[gi] = p;
        if (xupd) a.xsol[gi] = fma(alpha, po, a.xsol[gi]);
      }
      return p;
    }
  };
  auto wrapz = [nz](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
  auto ring_slot = [](int iz) { return (iz + 3) % 3; };  // iz >= -1

  // Rows of the column (TX elements along x) are contiguous runs of TX NPE
  // values in global memory and, with unpadded rows, in shared memory; when
  // the column is full in x and nx is a multiple of the vector width they
  // start on 16-byte boundaries, and box planes, y-face halo and stores move
  // as float4 / double2 with one index computation per vector.
  constexpr int RV = TX * NPE / VW;  // vectors per row
  const size_t plane = (size_t)nx * ny * NPE;
  // (offsets within a plane are 32-bit in the vector path)
  const bool vec = (RS == N1) && (TX * NPE) % VW == 0 && VX == TX && nx % VW == 0 && plane < (size_t(1) << 31);
  // x-face halo elements in the vector path: element ox - 1 ends and element
  // ox + VX starts on a vector boundary (both neighbour a full, aligned row
  // of the column, or wrap to a row end / start), so each moves as the HS / VW
  // vectors that end (x = -1) or start (x = VX) there; the x = -1 element then
  // sits LOFF values into its slot, the few values before it are unused
  constexpr int LOFF = (VW - NPE % VW) % VW;
  const int loff = vec ? LOFF : 0;
  // stage() on the VW values of one vector
  auto stage_vec = [&](size_t gi, bool owned, VT* rk) -> VT {
    VT out, rv;
    T* o = reinterpret_cast<T*>(&out);
    T* rr = reinterpret_cast<T*>(&rv);
    if (!fuse) return *reinterpret_cast<const VT*>(a.x + gi);
    VT r = *reinterpret_cast<const VT*>(a.x + gi);
    T* rp = reinterpret_cast<T*>(&r);
    if constexpr (ONE) {
      if (!first) {
        const VT po = *reinterpret_cast<const VT*>(a.p_old + gi);
        const VT ao = *reinterpret_cast<const VT*>(a.ap_old + gi);
        const T* pp = reinterpret_cast<const T*>(&po);
        const T* ap = reinterpret_cast<const T*>(&ao);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          rp[k] = fma(-alpha, ap[k], rp[k]);
          o[k] = fma(beta, pp[k], rp[k]);
        }
        if (owned) {
          VT xv = *reinterpret_cast<const VT*>(a.xsol + gi);
          T* xp = reinterpret_cast<T*>(&xv);
#pragma unroll
          for (int k = 0; k < VW; ++k) xp[k] = fma(alpha, pp[k], xp[k]);
          *reinterpret_cast<VT*>(a.xsol + gi) = xv;
        }
      } else {
        out = r;
      }
      if (owned) {
        *reinterpret_cast<VT*>(a.r_out + gi) = r;
        *reinterpret_cast<VT*>(a.p_out + gi) = out;
        *rk = r;
      }
      (void)rr;
      return out;
    } else {
      if (first) {
        out = r;
      } else {
        const VT po = *reinterpret_cast<const VT*>(a.p_old + gi);
        const T* pp = reinterpret_cast<const T*>(&po);
#pragma unroll
        for (int k = 0; k < VW; ++k) o[k] = fma(beta, pp[k], rp[k]);
        if (owned && xupd) {
          VT xv = *reinterpret_cast<const VT*>(a.xsol + gi);
          T* xp = reinterpret_cast<T*>(&xv);
#pragma unroll
          for (int k = 0; k < VW; ++k) xp[k] = fma(alpha, pp[k], xp[k]);
          *reinterpret_cast<VT*>(a.xsol + gi) = xv;
        }
      }
      if (owned) *reinterpret_cast<VT*>(a.p_out + gi) = out;
      (void)rr;
      return out;
    }
  };

  // Per-thread vectors of the vector path, fixed over the march: box rows
  // (boff: offset in a plane of the global arrays, bsi: in a ring slot), the
  // y-face rows (yoff, ysi) and the x-face elements (xoff, xsi); -1 = none.
  constexpr int HV = HS / VW;                                  // vectors per x-face element
  constexpr int NBV = (PE * NPE) / VW;                         // box vectors of a plane
  constexpr int KP = (NBV + THREADS - 1) / THREADS;
  constexpr int KY = (2 * RV + THREADS - 1) / THREADS;
  constexpr int KX = (2 * TY * HV + THREADS - 1) / THREADS;
  int boff[KP], bsi[KP], yoff[KY], ysi[KY], xoff[KX], xsi[KX];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int v = threadIdx.x + k * THREADS;
    boff[k] = -1;
    bsi[k] = 0;
    if (vec && v < VY * RV) {
      const int row = v / RV, i = v - row * RV;
      boff[k] = ((oy + row) * nx + ox) * NPE + i * VW;
      bsi[k] = row * TX * ES + i * VW;
    }
  }
#pragma unroll
  for (int k = 0; k < KY; ++k) {
    const int v = threadIdx.x + k * THREADS;
    yoff[k] = -1;
    ysi[k] = 0;
    if (vec && v < 2 * RV) {
      const int side = v / RV, i = v - side * RV;
      int gy = side ? oy + VY : oy - 1;
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      yoff[k] = (gy * nx + ox) * NPE + i * VW;
      ysi[k] = side * TX * ES + i * VW;
    }
  }
#pragma unroll
  for (int k = 0; k < KX; ++k) {
    const int v = threadIdx.x + k * THREADS;
    xoff[k] = -1;
    xsi[k] = 0;
    if (vec && v < 2 * TY * HV) {
      const int s = v / HV, j = v - s * HV;
      const int sy = s < TY ? s : s - TY;
      if (sy < VY) {
        int gx = s < TY ? ox - 1 : ox + VX;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        const int ge = (oy + sy) * nx + gx;
        xoff[k] = (s < TY ? (ge + 1) * NPE - HS : ge * NPE) + j * VW;
        xsi[k] = s * HS + j * VW;
      }
    }
  }

  // box of plane iz (relative to z0) into its ring slot; owned iff 0 <= iz < NZ
  auto load_plane = [&](int iz) {
    const int z = wrapz(z0 + iz);
    const bool owned = iz >= 0 && iz < NZ;
    T* dst = ring + ring_slot(iz) * PE * ES;
    T* rdst = rring + ring_slot(iz) * PE * ES;
    if (vec) {
      const size_t zb = (size_t)z * plane;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        if (boff[k] < 0) continue;
        VT rk;
        *reinterpret_cast<VT*>(dst + bsi[k]) = stage_vec(zb + boff[k], owned, &rk);
        if constexpr (ONE) {
          if (owned) *reinterpret_cast<VT*>(rdst + bsi[k]) = rk;
        }
      }
      return;
    }
    for (int v = threadIdx.x; v < PE * NPE; v += THREADS) {
      const int s = v / NPE, q = v - s * NPE;
      const int sx = s % TX, sy = s / TX;
      if (sx >= VX || sy >= VY) continue;
      const long long ge = ((long long)z * ny + (oy + sy)) * nx + (ox + sx);
      T rk = T(0);
      const int si = s * ES + m3_sidx<N1>(q);
      dst[si] = stage((size_t)ge * NPE + q, owned, &rk);
      if constexpr (ONE) {
        if (owned) rdst[si] = rk;
      }
    }
  };
  // x and y face halo of plane iz: x-halo slots [0, TY) x = -1, [TY, 2 TY)
  // x = VX; y-halo slots [0, TX) y = -1, [TX, 2 TX) y = VY
  auto load_halo = [&](int iz) {
    const int z = wrapz(z0 + iz);
    if (vec) {
      const size_t zb = (size_t)z * plane;
      VT rk;
#pragma unroll
      for (int k = 0; k < KY; ++k)
        if (yoff[k] >= 0) *reinterpret_cast<VT*>(yhalo + ysi[k]) = stage_vec(zb + yoff[k], false, &rk);
#pragma unroll
      for (int k = 0; k < KX; ++k)
        if (xoff[k] >= 0) *reinterpret_cast<VT*>(xhalo + xsi[k]) = stage_vec(zb + xoff[k], false, &rk);
      return;
    }
    for (int v = threadIdx.x; v < HALO * NPE; v += THREADS) {
      const int s = v / NPE, q = v - s * NPE;
      int sx, sy;
      T* dst;
      if (s < 2 * TY) {
        sy = s < TY ? s : s - TY;
        sx = s < TY ? -1 : VX;
        if (sy >= VY) continue;
        dst = xhalo + s * HS;
      } else {
        const int u = s - 2 * TY;
        sx = u < TX ? u : u - TX;
        sy = u < TX ? -1 : VY;
        if (sx >= VX) continue;
        dst = yhalo + u * ES;
      }
      int gx = ox + sx, gy = oy + sy;
      gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      const long long ge = ((long long)z * ny + gy) * nx + gx;
      T rk;
      dst[m3_sidx<N1>(q)] = stage((size_t)ge * NPE + q, false, &rk);
    }
  };

  // reductions: p.Ap (fuse 1, compensated); ONE: p.Ap, r.r (compensated), r.Ap, Ap.Ap
  T s_pa = T(0), c_pa = T(0), s_rr = T(0), c_rr = T(0), s_ra = T(0), s_aa = T(0);
  auto reduce = [&](T y, T pv, T r) {
    const T t1 = fma(pv, y, -c_pa);
    const T u1 = s_pa + t1;
    c_pa = (u1 - s_pa) - t1;
    s_pa = u1;
    if constexpr (ONE) {
      const T t2 = fma(r, r, -c_rr);
      const T u2 = s_rr + t2;
      c_rr = (u2 - s_rr) - t2;
      s_rr = u2;
      s_ra = fma(r, y, s_ra);
      s_aa = fma(y, y, s_aa);
    }
  };
  // y = sum of the three direction accumulators of plane iz, stored; reduced in CG modes
  auto store_plane = [&](int iz) {
    const int z = z0 + iz;
    const T* cur = ring + ring_slot(iz) * PE * ES;
    const T* rk = rring + ring_slot(iz) * PE * ES;
    if (vec) {
      const size_t zb = (size_t)z * plane;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        if (boff[k] < 0) continue;
        const int si = bsi[k];
        VT yv = *reinterpret_cast<const VT*>(s_out + si);
        const VT y1 = *reinterpret_cast<const VT*>(s_out + PE * ES + si);
        const VT y2 = *reinterpret_cast<const VT*>(s_out + 2 * PE * ES + si);
        T* yw = reinterpret_cast<T*>(&yv);
        const T* a1 = reinterpret_cast<const T*>(&y1);
        const T* a2 = reinterpret_cast<const T*>(&y2);
#pragma unroll
        for (int m = 0; m < VW; ++m) yw[m] = (yw[m] + a1[m]) + a2[m];
        *reinterpret_cast<VT*>(a.y + zb + boff[k]) = yv;
        if (fuse) {
          const VT pv4 = *reinterpret_cast<const VT*>(cur + si);
          const T* pp = reinterpret_cast<const T*>(&pv4);
          VT rv4;
          if constexpr (ONE) rv4 = *reinterpret_cast<const VT*>(rk + si);
          const T* rp = reinterpret_cast<const T*>(&rv4);
#pragma unroll
          for (int m = 0; m < VW; ++m) reduce(yw[m], pp[m], ONE ? rp[m] : T(0));
        }
      }
      return;
    }
    for (int v = threadIdx.x; v < PE * NPE; v += THREADS) {
      const int s = v / NPE, q = v - s * NPE;
      const int sx = s % TX, sy = s / TX;
      if (sx >= VX || sy >= VY) continue;
      const long long ge = ((long long)z * ny + (oy + sy)) * nx + (ox + sx);
      const int si = s * ES + m3_sidx<N1>(q);
      const T y = (s_out[si] + s_out[PE * ES + si]) + s_out[2 * PE * ES + si];
      a.y[(size_t)ge * NPE + q] = y;
      if (fuse) reduce(y, cur[si], ONE ? rk[si] : T(0));
    }
  };

  // this thread's line in each direction
  const int t = threadIdx.x;
  const int te = t / LINES, lam = t - te * LINES;
  const int lx = te % TX, ly = te / TX;
  const bool active = lx < VX && ly < VY;
  const int q0 = lam % N1, q1 = lam / N1;

  // March: planes iz - 1, iz, iz + 1 are in the ring when plane iz is
  // computed.  Two barriers per plane: after the passes, and after storing
  // plane iz while loading plane iz + 2 (into the slot of iz - 1) and the
  // halo of iz + 1.
  load_plane(-1);
  load_plane(0);
  load_plane(1);
  load_halo(0);
  __syncthreads();
  for (int iz = 0; iz < NZ; ++iz) {
    const T* cur = ring + ring_slot(iz) * PE * ES;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (active) {
        int base, stride;
        const T* pl;
        const T* pr;
        if (d == 0) {  // lines along x: (l2, l3) = (q0, q1)
          base = q0 * RS + q1 * PS;
          stride = 1;
          pl = lx > 0 ? cur + (te - 1) * ES : xhalo + ly * HS + loff;
          pr = lx + 1 < VX ? cur + (te + 1) * ES : xhalo + (TY + ly) * HS;
        } else if (d == 1) {  // along y: (l1, l3)
          base = q0 + q1 * PS;
          stride = RS;
          pl = ly > 0 ? cur + (te - TX) * ES : yhalo + lx * ES;
          pr = ly + 1 < VY ? cur + (te + TX) * ES : yhalo + (TX + lx) * ES;
        } else {  // along z: (l1, l2)
          base = q0 + q1 * RS;
          stride = PS;
          pl = ring + ring_slot(iz - 1) * PE * ES + te * ES;
          pr = ring + ring_slot(iz + 1) * PE * ES + te * ES;
        }
        const T* pc = cur + te * ES;
        T xl[N1], xc[N1], xr[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          xl[k] = pl[base + k * stride];
          xc[k] = pc[base + k * stride];
          xr[k] = pr[base + k * stride];
        }
        T val[N1];
        const T wp = s_w[q0] * s_w[q1];
        line_apply<T, N1, ACC>(a.c, xl, xc, xr, a.s[d] * wp, val);
        // each direction has its own accumulator, so the passes need no
        // barrier between them (the store adds them in direction order)
        T* out = s_out + d * PE * ES + te * ES + base;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          T v = val[m];
          if (d == 0 && a.cmass != T(0)) v = fma(a.cmass * wp * s_w[m], xc[m], v);
          out[m * stride] = v;
        }
      }
    }
    __syncthreads();
    store_plane(iz);
    if (iz + 1 < NZ) {  // uniform over the CTA
      load_plane(iz + 2);
      load_halo(iz + 1);
      __syncthreads();
    }
  }

  if (!fuse) return;
  if constexpr (ONE) {
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
  } else {
    // the block's p.Ap total for the update launch, which forms alpha
    __shared__ double s_opr[32];
    if constexpr (sizeof(T) == 4) op_partial_f2(F2{(float)s_pa, -(float)c_pa}, a.partials, s_opr);
    else op_partial_f64((double)s_pa - (double)c_pa, a.partials, s_opr);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->nop = (int)gridDim.x;
  }
}

// z-run length: the shortest runs whose CTAs all fit on the GPU at once
// (slots = SMs x resident CTAs per SM), so that the launch is one wave; at
// least 2 planes per run (fewer only on grids with fewer planes)
inline int march3_zc(int ntx, int nty, int nz, long long slots) {
  const long long cols = (long long)ntx * nty;
  if (slots < 1) slots = 1;
  long long zc = (nz * cols + slots - 1) / slots;
  if (zc < 2) zc = 2;
  if (zc > nz) zc = nz;
  return (int)zc;
}

template <typename T, int N1, bool ACC, bool ONE>
cudaError_t launch_apply3m(const sdg_handle* h, const ApplyArgs<T>& in, cudaStream_t stream) {
  using M = March3<N1>;
  ApplyParams<T, 3, N1> p;
  fill_apply_params<T, 3, N1>(h, in, &p);
  const size_t smem = ((size_t)((3 + 3) * M::PE + 2 * M::TX + (ONE ? 3 * M::PE : 0)) * M::ES +
                       (size_t)2 * M::TY * m3_halo_slot<T, N1>()) * sizeof(T);
  // resident CTAs per SM of this instantiation (fixed: threads and shared
  // memory do not depend on the grid), measured once
  static std::atomic<int> occ{0};
  if (occ.load(std::memory_order_acquire) == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_apply3m<T, N1, ACC, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_apply3m<T, N1, ACC, ONE>, M::THREADS, smem);
    if (e != cudaSuccess) return e;
    occ.store(o > 0 ? o : 1, std::memory_order_release);
  }
  p.ntile[0] = (p.n[0] + M::TX - 1) / M::TX;
  p.ntile[1] = (p.n[1] + M::TY - 1) / M::TY;
  p.zc = march3_zc(p.ntile[0], p.ntile[1], p.n[2], (long long)h->nsm * occ.load(std::memory_order_acquire));
  p.ntile[2] = (p.n[2] + p.zc - 1) / p.zc;
  const long long nblk = (long long)p.ntile[0] * p.ntile[1] * p.ntile[2];
  if (nblk > h->max_blocks) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(M::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = in.pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_apply3m<T, N1, ACC, ONE>, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// 3D dispatch for small degrees: the marching kernel for every mode
template <typename T, int N1>
cudaError_t launch_apply3m_t(const sdg_handle* h, const ApplyArgs<T>& in, cudaStream_t stream) {
  if (in.fuse == 2) return launch_apply3m<T, N1, true, true>(h, in, stream);
  if (sizeof(T) == 8 && !in.accurate) return launch_apply3m<T, N1, false, false>(h, in, stream);
  return launch_apply3m<T, N1, true, false>(h, in, stream);
}

}  // namespace sdg
