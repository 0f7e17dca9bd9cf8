// Allocation-free kinetic-energy reduction (sdg_kinetic_energy_noalloc).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator or pool that must not grow or fragment, and
// latency-critical loops where an allocation would stall the device.  For them this entry point needs no handle and allocates nothing:
// its scratch (the per-block partial sums and the ticket counter of the
// last-block reduction) is the file-scope array below, which every GPU that
// loads the library holds until the process exits.
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "sdg_device.cuh"

namespace {

// Largest grid of the reduction; each thread sums at most kPerThread nodes
// of every component, so one call handles at most
// kMaxBlocks * kThreads * kPerThread nodes per component.
constexpr int kThreads = 256;
constexpr int kPerThread = 64;
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxDof = (long long)kMaxBlocks * kThreads * kPerThread;  // 67,108,864

// kMaxBlocks partial sums, then one slot holding the ticket counter (32 KB).
static __device__ __align__(256) double g_scratch[kMaxBlocks + 32];

// Device address of g_scratch per device (host code may not use the symbol
// itself as a device pointer), looked up on the first call in each CUDA
// context of a device and keyed by that context's unique id, so that a
// replaced context (after cudaDeviceReset, or another driver context made
// current) triggers a fresh look-up instead of reusing a stale address.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id;
  double* addr;
};
ScratchSlot g_slot[kMaxDevices] = {};
std::mutex g_slot_mu;

// Driver entry points for the current context's id (taken through the
// runtime, so the library does not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
std::once_flag g_fn_once;

bool current_context_id(unsigned long long* id) {
  std::call_once(g_fn_once, [] {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess) {
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f0);
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
  });
  if (!g_ctx_current || !g_ctx_id) return false;
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

struct KeParams {
  sdg::Geo g;
  const double* U[3];
  double w[sdg::kMaxN1];
  double scale;  // 0.5 * cell volume / domain volume
  double* out;
  double* scratch;
};

// out = scale * sum_d sum_nodes W_l U_d^2  (Sec. 2.5: K = (1/|Omega|) int |v|^2 / 2)
__global__ void __launch_bounds__(kThreads) k_ke_noalloc(KeParams p) {
  __shared__ double s_red[32];
  __shared__ int s_last;
  const sdg::Geo& g = p.g;
  double sum = 0.0;
  const long long first = ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = first; idx < g.ndof; idx += stride) {
    const int loc = (int)(idx % g.npe);
    const int l0 = loc % g.n1, l1 = (loc / g.n1) % g.n1, l2 = loc / (g.n1 * g.n1);
    double W = p.w[l0] * p.w[l1];
    if (g.dim == 3) W *= p.w[l2];
    double s = 0.0;
    for (int d = 0; d < g.dim; ++d) s += p.U[d][idx] * p.U[d][idx];
    sum += W * s;
  }
  double v[1] = {sum}, b[1];
  sdg::block_sum<1>(v, s_red, b);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(p.scratch + kMaxBlocks);
  if (threadIdx.x == 0) {
    p.scratch[blockIdx.x] = b[0];
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc[1] = {0.0}, tot[1];
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) acc[0] += __ldcg(&p.scratch[i]);
  sdg::block_sum<1>(acc, s_red, tot);
  if (threadIdx.x == 0) {
    *p.out = p.scale * tot[0];
    *ticket = 0u;
  }
}

}  // namespace

extern "C" {

// See include/sdg.h.
int sdg_kinetic_energy_noalloc(const sdg_grid* grid, int N, const double* u, const double* v,
                               const double* w, double* ke, void* stream) {
  if (!grid || !u || !v || !ke || (grid->dim == 3 && !w) || (grid->dim != 2 && grid->dim != 3) ||
      N < 0 || N > sdg::kMaxN) {
    sdg::set_last_error("sdg_kinetic_energy_noalloc: invalid argument");
    return SDG_ERR_INVALID_ARG;
  }
  sdg::Geo g{};
  g.dim = grid->dim;
  g.n1 = N + 1;
  g.npe = 1;
  g.ncell = 1;
  double cellvol = 1.0, vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    if (d < g.dim) {
      if (grid->n[d] < 1 || !(grid->L[d] > 0.0)) {
        sdg::set_last_error("sdg_kinetic_energy_noalloc: cells must be >= 1 and lengths > 0");
        return SDG_ERR_INVALID_ARG;
      }
      g.n[d] = grid->n[d];
      g.npe *= g.n1;
      cellvol *= grid->L[d] / grid->n[d];
      vol *= grid->L[d];
    } else {
      g.n[d] = 1;
    }
    g.ncell *= g.n[d];
  }
  g.ndof = g.ncell * g.npe;
  if (g.ndof > kMaxDof) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "sdg_kinetic_energy_noalloc: %lld nodes per component exceed the fixed scratch limit of %lld",
                  g.ndof, kMaxDof);
    sdg::set_last_error(msg);
    return SDG_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    sdg::set_last_error("sdg_kinetic_energy_noalloc: no usable current device");
    return SDG_ERR_CUDA;
  }
  // id of the current context (none yet if this thread has not used the
  // runtime on this device: the symbol look-up below creates it)
  unsigned long long ctx_id = 0;
  const bool have_id = current_context_id(&ctx_id);
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_slot_mu);
    ScratchSlot& slot = g_slot[dev];
    if (!have_id || slot.addr == nullptr || slot.ctx_id != ctx_id) {
      // set-up, once per context of this device (the device is current):
      // the device address of the scratch array
      double* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_scratch);
      if (e != cudaSuccess || ptr == nullptr) {
        char msg[200];
        std::snprintf(msg, sizeof(msg), "sdg_kinetic_energy_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
        sdg::set_last_error(msg);
        return SDG_ERR_CUDA;
      }
      if (!have_id && !current_context_id(&ctx_id)) {
        sdg::set_last_error("sdg_kinetic_energy_noalloc: cannot identify the current CUDA context");
        return SDG_ERR_CUDA;
      }
      slot.addr = ptr;
      slot.ctx_id = ctx_id;
    }
    scratch = slot.addr;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KeParams p{};
  p.g = g;
  p.U[0] = u;
  p.U[1] = v;
  p.U[2] = g.dim == 3 ? w : nullptr;
  double xi[sdg::kMaxN1];
  sdg::gauss_legendre(g.n1, xi, p.w);
  p.scale = 0.5 * cellvol / vol;
  p.out = ke;
  p.scratch = scratch;
  long long blocks = (g.ndof + (long long)kThreads * kPerThread - 1) / ((long long)kThreads * kPerThread);
  if (blocks < 1) blocks = 1;
  // the ticket counter must start at zero (the last block also resets it)
  cudaError_t e = cudaMemsetAsync(p.scratch + kMaxBlocks, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    k_ke_noalloc<<<(unsigned)blocks, kThreads, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char msg[200];
    std::snprintf(msg, sizeof(msg), "sdg_kinetic_energy_noalloc: CUDA error %s", cudaGetErrorString(e));
    sdg::set_last_error(msg);
    return SDG_ERR_CUDA;
  }
  return SDG_OK;
}

}  // extern "C"
