// Block-sparse linear algebra of the Newton system (Sec. 3.4, block-wise
// ordering): 7-point 3x3-block SpMV on the structured grid with the bordered
// well rows and columns, block-Jacobi, and the FP64 vector kernels of the
// restarted Krylov solver (deterministic two-stage reductions).
#include <math.h>

#include "pf_internal.cuh"

namespace pf {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// y = J x  (cells), then the well border (one warp per well)
// ---------------------------------------------------------------------------

template <typename DT>
__global__ void __launch_bounds__(256) k_spmv_cells(Grid g, const DT* __restrict__ J, const double* __restrict__ x,
                                                    double* __restrict__ y) {
  const long long n = g.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / g.nxy;
    const long long rem = i - k * g.nxy;
    const long long j = rem / g.nx;
    const long long ii = rem - j * g.nx;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      long long c;
      bool has;
      switch (s) {
        case SL_D: c = i; has = true; break;
        case SL_XM: c = i - 1; has = ii > 0; break;
        case SL_XP: c = i + 1; has = ii + 1 < g.nx; break;
        case SL_YM: c = i - g.nx; has = j > 0; break;
        case SL_YP: c = i + g.nx; has = j + 1 < g.ny; break;
        case SL_ZM: c = i - g.nxy; has = k > 0; break;
        default: c = i + g.nxy; has = k + 1 < g.nz; break;
      }
      if (!has) continue;
      const DT* B = J + (size_t)s * 9 * n + i;
      const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      acc0 += (double)B[0] * x0 + (double)B[n] * x1 + (double)B[2 * n] * x2;
      acc1 += (double)B[3 * n] * x0 + (double)B[4 * n] * x1 + (double)B[5 * n] * x2;
      acc2 += (double)B[6 * n] * x0 + (double)B[7 * n] * x1 + (double)B[8 * n] * x2;
    }
    y[3 * i] = acc0;
    y[3 * i + 1] = acc1;
    y[3 * i + 2] = acc2;
  }
}

template <typename DT>
__global__ void k_spmv_wells(Grid g, Wells w, const DT* __restrict__ Bw, const DT* __restrict__ Cw,
                             const DT* __restrict__ Dw, const double* __restrict__ x, double* __restrict__ y) {
  const int wi = blockIdx.x;
  if (wi >= w.nw) return;
  const long long n = g.n, npf = w.npf;
  const double xw = x[3 * n + wi];
  double acc = 0.0;
  for (int m = w.ptr[wi] + threadIdx.x; m < w.ptr[wi + 1]; m += 32) {
    const long long c = w.cell[m];
    y[3 * c] += (double)Bw[m] * xw;
    y[3 * c + 1] += (double)Bw[npf + m] * xw;
    y[3 * c + 2] += (double)Bw[2 * npf + m] * xw;
    acc += (double)Cw[m] * x[3 * c] + (double)Cw[npf + m] * x[3 * c + 1] + (double)Cw[2 * npf + m] * x[3 * c + 2];
  }
  acc = wsum(acc);
  if (threadIdx.x == 0) y[3 * n + wi] = acc + (double)Dw[wi] * xw;
}

template <typename DT>
void launch_spmv(const Grid& g, const Wells& w, const DT* J, const DT* Bw, const DT* Cw, const DT* Dw,
                 const double* x, double* y, cudaStream_t st) {
  k_spmv_cells<DT><<<grid_for(g.n, 256), 256, 0, st>>>(g, J, x, y);
  if (w.nw > 0) k_spmv_wells<DT><<<w.nw, 32, 0, st>>>(g, w, Bw, Cw, Dw, x, y);
}

// ---------------------------------------------------------------------------
// block-Jacobi: inverse of each 3x3 diagonal block (adjugate / determinant)
// ---------------------------------------------------------------------------

template <typename DT, typename PT>
__global__ void __launch_bounds__(256) k_bjacobi_setup(long long n, const DT* __restrict__ J, PT* __restrict__ Dinv) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = (double)J[(size_t)e * n + i];
    const double c00 = a[4] * a[8] - a[5] * a[7];
    const double c01 = a[5] * a[6] - a[3] * a[8];
    const double c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double id = 1.0 / det;
    double inv[9];
    inv[0] = c00 * id;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    inv[3] = c01 * id;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    inv[6] = c02 * id;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) * id;
#pragma unroll
    for (int e = 0; e < 9; ++e) Dinv[(size_t)e * n + i] = (PT)inv[e];
  }
}

template <typename DT, typename PT>
__global__ void k_bjacobi_wells(int nw, const DT* __restrict__ Dw, PT* __restrict__ Dwinv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nw) Dwinv[t] = (PT)(1.0 / (double)Dw[t]);
}

template <typename DT, typename PT>
void launch_bjacobi_setup(const Grid& g, const Wells& w, const DT* J, const DT* Dw, PT* Dinv, PT* Dwinv,
                          cudaStream_t st) {
  k_bjacobi_setup<DT, PT><<<grid_for(g.n, 256), 256, 0, st>>>(g.n, J, Dinv);
  if (w.nw > 0) k_bjacobi_wells<DT, PT><<<grid_for(w.nw, 128), 128, 0, st>>>(w.nw, Dw, Dwinv);
}

template <typename PT>
__global__ void __launch_bounds__(256) k_bjacobi_apply(long long n, int nw, const PT* __restrict__ Dinv,
                                                       const PT* __restrict__ Dwinv, const double* __restrict__ r,
                                                       double* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n + nw;
       i += (long long)gridDim.x * blockDim.x) {
    if (i >= n) { z[3 * n + (i - n)] = (double)Dwinv[i - n] * r[3 * n + (i - n)]; continue; }
    const double r0 = r[3 * i], r1 = r[3 * i + 1], r2 = r[3 * i + 2];
    const PT* D = Dinv + i;
    z[3 * i] = (double)D[0] * r0 + (double)D[n] * r1 + (double)D[2 * n] * r2;
    z[3 * i + 1] = (double)D[3 * n] * r0 + (double)D[4 * n] * r1 + (double)D[5 * n] * r2;
    z[3 * i + 2] = (double)D[6 * n] * r0 + (double)D[7 * n] * r1 + (double)D[8 * n] * r2;
  }
}

template <typename PT>
void launch_bjacobi_apply(const Grid& g, int nw, const PT* Dinv, const PT* Dwinv, const double* r, double* z,
                          cudaStream_t st) {
  k_bjacobi_apply<PT><<<grid_for(g.n + nw, 256), 256, 0, st>>>(g.n, nw, Dinv, Dwinv, r, z);
}

// ---------------------------------------------------------------------------
// FP64 vector kernels
// ---------------------------------------------------------------------------

#define GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void k_copy(long long n, const double* __restrict__ a, double* __restrict__ b) { GRID_STRIDE(i, n) b[i] = a[i]; }
__global__ void k_fill(long long n, double v, double* __restrict__ a) { GRID_STRIDE(i, n) a[i] = v; }
__global__ void k_scale_dev(long long n, const double* a, const double* __restrict__ s, int inv_sqrt,
                            double* b) {
  const double f = inv_sqrt ? 1.0 / sqrt(s[0]) : s[0];
  GRID_STRIDE(i, n) b[i] = a[i] * f;
}
__global__ void k_axpy(long long n, double al, const double* __restrict__ x, double* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] += al * x[i];
}
__global__ void k_xpay(long long n, const double* __restrict__ x, double be, double* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = x[i] + be * y[i];
}
__global__ void k_sub(long long n, const double* a, const double* b, double* c) {
  GRID_STRIDE(i, n) c[i] = a[i] - b[i];
}

void launch_copy(long long n, const double* a, double* b, cudaStream_t st) {
  k_copy<<<grid_for(n, 256), 256, 0, st>>>(n, a, b);
}
void launch_fill(long long n, double v, double* a, cudaStream_t st) { k_fill<<<grid_for(n, 256), 256, 0, st>>>(n, v, a); }
void launch_scale_by_dev(long long n, const double* a, const double* s, int inv_sqrt, double* b, cudaStream_t st) {
  k_scale_dev<<<grid_for(n, 256), 256, 0, st>>>(n, a, s, inv_sqrt, b);
}
void launch_axpy(long long n, double al, const double* x, double* y, cudaStream_t st) {
  k_axpy<<<grid_for(n, 256), 256, 0, st>>>(n, al, x, y);
}
void launch_xpay(long long n, const double* x, double be, double* y, cudaStream_t st) {
  k_xpay<<<grid_for(n, 256), 256, 0, st>>>(n, x, be, y);
}
void launch_sub(long long n, const double* a, const double* b, double* c, cudaStream_t st) {
  k_sub<<<grid_for(n, 256), 256, 0, st>>>(n, a, b, c);
}

// Block reduction of KM partial sums held per thread; thread 0 writes them.
template <int KM>
__device__ __forceinline__ void block_reduce_write(double (&acc)[KM], int k, double* out_row) {
  __shared__ double sh[KM][8];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    if (j < k) {
      const double v = wsum(acc[j]);
      if (lane == 0) sh[j][wid] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) s += sh[threadIdx.x][t];
    out_row[threadIdx.x] = s;
  }
}

// The last block to finish sums the per-block rows in a fixed order (one warp
// per value, lanes over blocks, then a shuffle tree), so the result does not
// depend on which block came last; it then re-arms the counter.
__device__ __forceinline__ void last_block_reduce(const double* partial, int stride, int k, double* out,
                                                  unsigned int* counter, bool inv_norm = false) {
  __shared__ bool last;
  __threadfence();  // every thread that wrote a partial publishes it before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partial + (size_t)b * stride + j);
    s = wsum(s);
    if (lane == 0) {
      out[j] = s;
      // out[k] = 1 / sqrt(last value): one FP64 sqrt and divide for the whole
      // vector instead of one per thread of the scaling kernel
      if (inv_norm && j == k - 1) out[k] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

template <int KM>
__global__ void __launch_bounds__(256) k_multidot(long long n, int k, const double* __restrict__ V, long long ld,
                                                  const double* __restrict__ w, double* __restrict__ partial,
                                                  double* __restrict__ out, unsigned int* counter) {
  double acc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) acc[j] = 0.0;
  GRID_STRIDE(i, n) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) acc[j] += V[(size_t)j * ld + i] * wi;
  }
  block_reduce_write<KM>(acc, k, partial + (size_t)blockIdx.x * (KM + 1));
  last_block_reduce(partial, KM + 1, k, out, counter);
}

// w -= V h; partial dots of the updated w with V (j < k) and with itself (slot k)
template <int KM>
__global__ void __launch_bounds__(256) k_multi_axpy_dot(long long n, int k, const double* __restrict__ V, long long ld,
                                                        const double* __restrict__ h, double* __restrict__ w,
                                                        double* __restrict__ partial, double* __restrict__ out,
                                                        unsigned int* counter, int inv_norm) {
  __shared__ double hs[KM];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[KM + 1];
#pragma unroll
  for (int j = 0; j <= KM; ++j) acc[j] = 0.0;
  GRID_STRIDE(i, n) {
    double wi = w[i];
    for (int j = 0; j < k; ++j) wi -= V[(size_t)j * ld + i] * hs[j];
    w[i] = wi;
    // second read of the basis column hits L1: the same thread just loaded it
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) acc[j] += V[(size_t)j * ld + i] * wi;
    acc[KM] += wi * wi;
  }
  // move the norm into slot k before the block reduction
  double accr[KM + 1];
#pragma unroll
  for (int j = 0; j <= KM; ++j) accr[j] = (j < k) ? acc[j] : (j == k ? acc[KM] : 0.0);
  block_reduce_write<KM + 1>(accr, k + 1, partial + (size_t)blockIdx.x * (KM + 1));
  last_block_reduce(partial, KM + 1, k + 1, out, counter, inv_norm != 0);
}

void launch_multidot(long long n, int k, const double* V, long long ld, const double* w, double* partial, int nblocks,
                     double* out, unsigned int* counter, cudaStream_t st) {
  if (k <= 8) k_multidot<8><<<nblocks, 256, 0, st>>>(n, k, V, ld, w, partial, out, counter);
  else if (k <= 16) k_multidot<16><<<nblocks, 256, 0, st>>>(n, k, V, ld, w, partial, out, counter);
  else if (k <= 32) k_multidot<32><<<nblocks, 256, 0, st>>>(n, k, V, ld, w, partial, out, counter);
  else k_multidot<64><<<nblocks, 256, 0, st>>>(n, k, V, ld, w, partial, out, counter);
}

void launch_multi_axpy_dot(long long n, int k, const double* V, long long ld, const double* h, double* w,
                           double* partial, int nblocks, double* out, unsigned int* counter, cudaStream_t st,
                           int inv_norm) {
  if (k <= 8) k_multi_axpy_dot<8><<<nblocks, 256, 0, st>>>(n, k, V, ld, h, w, partial, out, counter, inv_norm);
  else if (k <= 16) k_multi_axpy_dot<16><<<nblocks, 256, 0, st>>>(n, k, V, ld, h, w, partial, out, counter, inv_norm);
  else if (k <= 32) k_multi_axpy_dot<32><<<nblocks, 256, 0, st>>>(n, k, V, ld, h, w, partial, out, counter, inv_norm);
  else k_multi_axpy_dot<64><<<nblocks, 256, 0, st>>>(n, k, V, ld, h, w, partial, out, counter, inv_norm);
}

__global__ void __launch_bounds__(256) k_multi_axpy_add(long long n, int k, const double* __restrict__ Z, long long ld,
                                                        const double* __restrict__ y, double* __restrict__ x) {
  __shared__ double ys[128];
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  GRID_STRIDE(i, n) {
    double s = x[i];
    for (int j = 0; j < k; ++j) s += Z[(size_t)j * ld + i] * ys[j];
    x[i] = s;
  }
}

void launch_multi_axpy_add(long long n, int k, const double* Z, long long ld, const double* y, double* x,
                           cudaStream_t st) {
  k_multi_axpy_add<<<grid_for(n, 256), 256, 0, st>>>(n, k, Z, ld, y, x);
}

void launch_dot(long long n, const double* a, const double* b, double* partial, int nblocks, double* out,
                unsigned int* counter, cudaStream_t st) {
  k_multidot<8><<<nblocks, 256, 0, st>>>(n, 1, a, 0, b, partial, out, counter);
}

// explicit instantiations
template void launch_spmv<double>(const Grid&, const Wells&, const double*, const double*, const double*,
                                  const double*, const double*, double*, cudaStream_t);
template void launch_spmv<float>(const Grid&, const Wells&, const float*, const float*, const float*, const float*,
                                 const double*, double*, cudaStream_t);
template void launch_bjacobi_setup<double, double>(const Grid&, const Wells&, const double*, const double*, double*,
                                                   double*, cudaStream_t);
template void launch_bjacobi_setup<float, float>(const Grid&, const Wells&, const float*, const float*, float*, float*,
                                                 cudaStream_t);
template void launch_bjacobi_apply<double>(const Grid&, int, const double*, const double*, const double*, double*,
                                           cudaStream_t);
template void launch_bjacobi_apply<float>(const Grid&, int, const float*, const float*, const double*, double*,
                                          cudaStream_t);

}  // namespace pf
