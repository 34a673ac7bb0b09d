// Residual norms for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a host framework that
// hands out every byte of device memory from its own pool and treats any
// other allocation as an error, or a loop with a fixed time budget per
// iteration that cannot afford an allocation (which may synchronise the
// device) once it has started.  pf_residual_norms_noalloc serves them: the
// caller passes device inputs and the device output, and the kernel's scratch
// (one pair of partial results per block and a completion counter) lives in a
// fixed-size array of this file, kept by every GPU that loads the library
// until the process exits.
//
// It computes the same two numbers as the residual-norm step of
// pf_newton_iteration: the scaled max-norm used as the Newton convergence
// test and the 2-norm used by the forcing term, in one launch (the last block
// to finish reduces the per-block partials in a fixed order, so the result
// does not depend on block scheduling).
#include <math.h>

#include <mutex>
#include <string>
#include <vector>

#include "pf_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaCellsPerThread = 16;
constexpr int kNaMaxBlocks = 4096;
constexpr long long kNaMaxCells = (long long)kNaMaxBlocks * kNaThreads * kNaCellsPerThread;  // 16,777,216
constexpr int kNaMaxWells = 4096;
constexpr int kNaCounterSlot = 2 * kNaMaxBlocks;  // index of the completion counter (as a double slot)

// 2 partials per block + the counter word: 64 KiB + 256 B per device.
static __device__ __align__(256) double g_norm_scratch[2 * kNaMaxBlocks + 32];

thread_local std::string g_na_error;

std::mutex g_na_mutex;
std::vector<double*> g_na_addr;  // per device: device address of g_norm_scratch (nullptr until resolved)

__device__ __forceinline__ double na_nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ double na_wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = na_nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double na_wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kNaThreads) k_norms_noalloc(long long n, int nw, const double* __restrict__ R,
                                                               const double* __restrict__ inv_pv,
                                                               const double* __restrict__ well_denom, double rho_o,
                                                               double rho_w, double c_ref, double* __restrict__ out,
                                                               double* __restrict__ scratch) {
  const double io = 1.0 / rho_o, iw = 1.0 / rho_w, ic = 1.0 / c_ref;
  double mx = 0.0, ss = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ip = inv_pv[i];
    const double r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
    mx = na_nanmax(mx, fabs(r0) * ip * io);
    mx = na_nanmax(mx, fabs(r1) * ip * iw);
    mx = na_nanmax(mx, fabs(r2) * ip * ic);
    ss += r0 * r0 + r1 * r1 + r2 * r2;
  }
  __shared__ double smx[kNaThreads / 32], sss[kNaThreads / 32];
  __shared__ bool last;
  mx = na_wmax(mx);
  ss = na_wsum(ss);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { smx[wid] = mx; sss[wid] = ss; }
  __syncthreads();
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaCounterSlot);
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < kNaThreads / 32; ++t) { a = na_nanmax(a, smx[t]); b += sss[t]; }
    scratch[2 * blockIdx.x] = a;
    scratch[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || wid != 0) return;
  // last block, first warp: fixed-order reduction of the block partials, then the well rows
  __threadfence();
  double m2 = 0.0, s2 = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) {
    m2 = na_nanmax(m2, __ldcg(scratch + 2 * b));
    s2 += __ldcg(scratch + 2 * b + 1);
  }
  for (int w = lane; w < nw; w += 32) {
    const double r = R[3 * n + w];
    m2 = na_nanmax(m2, fabs(r) / well_denom[w]);
    s2 += r * r;
  }
  m2 = na_wmax(m2);
  s2 = na_wsum(s2);
  if (lane == 0) {
    out[0] = m2;
    out[1] = sqrt(s2);
    *counter = 0u;
  }
}

// Device address of g_norm_scratch on the current device: resolved once per
// device (a host-side symbol lookup that performs no allocation).
pf_status scratch_address(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_na_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PF_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if ((int)g_na_addr.size() <= dev) g_na_addr.resize(dev + 1, nullptr);
  if (!g_na_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_norm_scratch);
    if (e != cudaSuccess || !p) {
      g_na_error = std::string("cudaGetSymbolAddress(g_norm_scratch): ") + cudaGetErrorString(e);
      return PF_ECUDA;
    }
    g_na_addr[dev] = p;
  }
  *ptr = g_na_addr[dev];
  return PF_OK;
}

}  // namespace

extern "C" {

const char* pf_noalloc_last_error(void) { return g_na_error.c_str(); }

pf_status pf_residual_norms_noalloc(int64_t n_cells, int n_wells, const double* R, const double* inv_pv,
                                    const double* well_denom, double rho_o, double rho_w, double c_ref,
                                    double* out, void* stream) {
  if (n_cells < 0 || n_cells > kNaMaxCells) {
    g_na_error = "pf_residual_norms_noalloc: n_cells = " + std::to_string((long long)n_cells) +
                 " is outside [0, " + std::to_string(kNaMaxCells) + "], the size of its fixed scratch";
    return PF_EINVAL;
  }
  if (n_wells < 0 || n_wells > kNaMaxWells) {
    g_na_error = "pf_residual_norms_noalloc: n_wells = " + std::to_string(n_wells) + " is outside [0, " +
                 std::to_string(kNaMaxWells) + "]";
    return PF_EINVAL;
  }
  if ((n_cells + n_wells > 0 && !R) || (n_cells > 0 && !inv_pv) || (n_wells > 0 && !well_denom) || !out) {
    g_na_error = "pf_residual_norms_noalloc: NULL device pointer";
    return PF_EINVAL;
  }
  if (!(rho_o > 0.0) || !(rho_w > 0.0) || !(c_ref > 0.0)) {
    g_na_error = "pf_residual_norms_noalloc: reference densities and c_ref must be positive";
    return PF_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (st) {
    // the scratch address is the current device's; a stream of another
    // device would run the kernel against memory it does not own
    int cur = 0, sdev = 0;
    cudaError_t e0 = cudaGetDevice(&cur);
    if (e0 == cudaSuccess) e0 = cudaStreamGetDevice(st, &sdev);
    if (e0 != cudaSuccess) {
      g_na_error = std::string("pf_residual_norms_noalloc: stream device: ") + cudaGetErrorString(e0);
      return PF_EINVAL;
    }
    if (sdev != cur) {
      g_na_error = "pf_residual_norms_noalloc: the stream belongs to device " + std::to_string(sdev) +
                   ", the current device is " + std::to_string(cur);
      return PF_EINVAL;
    }
  }
  double* scratch = nullptr;
  pf_status rc = scratch_address(&scratch);
  if (rc != PF_OK) return rc;
  // the counter must start at zero even if an earlier call on this device was cut short
  cudaError_t e = cudaMemsetAsync(scratch + kNaCounterSlot, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    g_na_error = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
    return PF_ECUDA;
  }
  const long long per_block = (long long)kNaThreads * kNaCellsPerThread;
  int blocks = (int)((n_cells + per_block - 1) / per_block);
  if (blocks < 1) blocks = 1;
  k_norms_noalloc<<<blocks, kNaThreads, 0, st>>>(n_cells, n_wells, R, inv_pv, well_denom, rho_o, rho_w, c_ref, out,
                                                 scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_na_error = std::string("launch: ") + cudaGetErrorString(e);
    return PF_ECUDA;
  }
  return PF_OK;
}

}  // extern "C"
