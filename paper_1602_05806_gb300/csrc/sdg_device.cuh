// Device helpers: block / grid reductions with a deterministic last-block
// finish, and index arithmetic of the element-major field layout.
#pragma once

#include "sdg_internal.h"

namespace sdg {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum K values over the block; the totals end up in out[] of every thread.
// s_red: shared scratch of at least 32*K doubles.  Must be reached by all
// threads of the block.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* s_red, double (&out)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = warp_sum(v[k]);
    if (lane == 0) s_red[k * 32 + wid] = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = (lane < nw) ? s_red[k * 32 + lane] : 0.0;
    out[k] = warp_sum(t);  // every warp computes the same total
  }
  __syncthreads();
}

// Grid-wide sum with a deterministic finish: every block writes its partial
// sums to partials[block*kPartialSlots + k]; the last block to arrive adds
// them in block order and returns true (in all of its threads) with the
// totals in tot[].  Other blocks return false.  The ticket counter is reset
// by the last block, so the same counter serves the next launch.
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* partials, unsigned int* counter,
                                         double (&tot)[K]) {
  static_assert(K <= kPartialSlots, "too many reduction slots");
  __shared__ double s_red[32 * K];
  __shared__ int s_last;
  double b[K];
  block_sum<K>(v, s_red, b);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * kPartialSlots + k] = b[k];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(&partials[(size_t)i * kPartialSlots + k]);
  }
  block_sum<K>(acc, s_red, tot);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ---- FP32 reductions without FP64 arithmetic per thread -------------------
// GB300 issues FP64 at 1/64 of the FP32 rate, so FP32 kernels reduce their
// dot products as unevaluated float pairs (hi + lo) with the error-free
// TwoSum addition; FP64 is used only to add the per-warp pairs of a block.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return F2{s, a.lo + b.lo + e};
}

// Sum K float pairs over the block; totals (as doubles) in every thread.
// Warps and then warp 0 add pairs with TwoSum; only the block total is
// converted to FP64 (one thread).  s_red: at least 32*K doubles.
template <int K>
__device__ __forceinline__ void block_sum_f2(F2 (&v)[K], double* s_red, double (&out)[K]) {
  float2* s2 = reinterpret_cast<float2*>(s_red);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    F2 t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      F2 u{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
      t = f2_add(t, u);
    }
    if (lane == 0) s2[k * 32 + wid] = make_float2(t.hi, t.lo);
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      F2 t{0.0f, 0.0f};
      if (lane < nw) {
        const float2 q = s2[k * 32 + lane];
        t = F2{q.x, q.y};
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        F2 u{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
        t = f2_add(t, u);
      }
      // every lane of warp 0 has read its slot before the shuffles above
      if (lane == 0) s_red[k * 32] = (double)t.hi + (double)t.lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = s_red[k * 32];
  __syncthreads();
}

// grid_sum for float pairs: per-block totals in FP64, same deterministic
// last-block finish as grid_sum.
template <int K>
__device__ __forceinline__ bool grid_sum_f2(F2 (&v)[K], double* partials, unsigned int* counter,
                                            double (&tot)[K]) {
  static_assert(K <= kPartialSlots, "too many reduction slots");
  __shared__ double s_red2[32 * K];
  __shared__ int s_last2;
  double b[K];
  block_sum_f2<K>(v, s_red2, b);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * kPartialSlots + k] = b[k];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last2 = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last2) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(&partials[(size_t)i * kPartialSlots + k]);
  }
  double u[K];
  block_sum<K>(acc, s_red2, u);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = u[k];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ---- operator totals handed to the next launch ------------------------------
// The operator launch of a two-launch CG iteration ends without a grid-wide
// finish: each block leaves its p.Ap total in slot kOpSlot of its partials
// row (FP32 data: as a float pair), and every block of the update launch adds
// them in the same fixed order, so that no serial last-block step sits
// between the two launches.
constexpr int kOpSlot = 2;

// Block total of an FP32 operator block (float pair) into its partials row.
// All threads of the block must call it.
__device__ __forceinline__ void op_partial_f2(F2 v, double* partials, double* s_red) {
  F2 a[1] = {v};
  double b[1];
  block_sum_f2<1>(a, s_red, b);
  if (threadIdx.x == 0) {
    const float hi = (float)b[0];
    const float lo = (float)(b[0] - (double)hi);
    *reinterpret_cast<float2*>(partials + (size_t)blockIdx.x * kPartialSlots + kOpSlot) = make_float2(hi, lo);
  }
}
__device__ __forceinline__ void op_partial_f64(double v, double* partials, double* s_red) {
  double a[1] = {v}, b[1];
  block_sum<1>(a, s_red, b);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kPartialSlots + kOpSlot] = b[0];
}

// The sum of the n operator totals, the same in every thread of every block
// (fixed order: thread t adds totals t, t + blockDim, ..., then the block
// tree).  The loads go out in batches of eight, so that their latencies
// overlap.  All threads of the block must call it.
__device__ __forceinline__ double sum_op_partials_f2(const double* partials, int n, double* s_red) {
  constexpr int B = 8;
  F2 a{0.0f, 0.0f};
  for (int i0 = threadIdx.x; i0 < n; i0 += B * blockDim.x) {
    float2 q[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * blockDim.x;
      q[b] = i < n ? __ldcg(reinterpret_cast<const float2*>(partials + (size_t)i * kPartialSlots + kOpSlot))
                   : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) a = f2_add(a, F2{q[b].x, q[b].y});
  }
  F2 v[1] = {a};
  double out[1];
  block_sum_f2<1>(v, s_red, out);
  return out[0];
}
__device__ __forceinline__ double sum_op_partials_f64(const double* partials, int n, double* s_red) {
  constexpr int B = 8;
  double a = 0.0;
  for (int i0 = threadIdx.x; i0 < n; i0 += B * blockDim.x) {
    double q[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * blockDim.x;
      q[b] = i < n ? __ldcg(&partials[(size_t)i * kPartialSlots + kOpSlot]) : 0.0;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) a += q[b];
  }
  double v[1] = {a}, out[1];
  block_sum<1>(v, s_red, out);
  return out[0];
}

// ---- programmatic dependent launch -----------------------------------------
// A kernel launched with programmatic stream serialisation may start while
// the previous kernel of the stream finishes.  pdl_trigger lets the next
// kernel start (once every block of this one has called it); pdl_wait blocks
// until the previous kernel has completed and its memory is visible, and
// returns at once when the launch did not ask for the overlap.  Nothing that
// an earlier kernel writes may be read, and nothing written, before pdl_wait.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- layout ----------------------------------------------------------------
__device__ __forceinline__ void split_index(const Geo& g, long long idx, int e[3], int l[3]) {
  const long long el = idx / g.npe;
  int loc = (int)(idx - el * g.npe);
  l[0] = loc % g.n1;
  loc /= g.n1;
  l[1] = loc % g.n1;
  l[2] = loc / g.n1;
  e[0] = (int)(el % g.n[0]);
  const long long r = el / g.n[0];
  e[1] = (int)(r % g.n[1]);
  e[2] = (int)(r / g.n[1]);
  if (g.dim == 2) { l[2] = 0; e[2] = 0; }
}

__device__ __forceinline__ long long elem_of(const Geo& g, const int e[3]) {
  return ((long long)e[2] * g.n[1] + e[1]) * g.n[0] + e[0];
}

__device__ __forceinline__ int local_of(const Geo& g, const int l[3]) {
  return (l[2] * g.n1 + l[1]) * g.n1 + l[0];
}

// element index of e shifted by s (+-1) along d, periodic
__device__ __forceinline__ long long elem_shift(const Geo& g, const int e[3], int d, int s) {
  int f[3] = {e[0], e[1], e[2]};
  f[d] += s;
  if (f[d] < 0) f[d] += g.n[d];
  if (f[d] >= g.n[d]) f[d] -= g.n[d];
  return elem_of(g, f);
}

// local node stride of direction d
__device__ __forceinline__ int lstride(const Geo& g, int d) {
  return d == 0 ? 1 : (d == 1 ? g.n1 : g.n1 * g.n1);
}

}  // namespace sdg
