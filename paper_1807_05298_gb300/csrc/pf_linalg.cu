// Block-sparse linear algebra of the Newton system (Sec. 3.4, block-wise
// ordering): 7-point 3x3-block SpMV on the structured grid with the bordered
// well rows and columns, block-Jacobi, and the FP64 vector kernels of the
// restarted Krylov solver (deterministic two-stage reductions).
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "pf_internal.cuh"

namespace pf {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// y = J x with the bordered well rows and columns, one launch: the first
// cell_blocks blocks take the cells (a perforated cell adds its well column
// B x_w), the blocks after them take the well rows C x + D x_w, one warp per
// well.
// ---------------------------------------------------------------------------

// well rows, one warp per well (lanes stride the well's perforations, then a
// butterfly sum), by the warps of the blocks from cell_blocks on
template <typename DT, typename XT>
__device__ __forceinline__ void spmv_well_rows(const Grid& g, const Wells& w, const DT* __restrict__ Cw,
                                               const DT* __restrict__ Dw, const XT* __restrict__ x,
                                               double* __restrict__ y, int cell_blocks) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const long long n = g.n, npf = w.npf;
  for (int wi = (blockIdx.x - cell_blocks) * wpb + (threadIdx.x >> 5); wi < w.nw;
       wi += (gridDim.x - cell_blocks) * wpb) {
    double acc = 0.0;
    for (int m = w.ptr[wi] + lane; m < w.ptr[wi + 1]; m += 32) {
      const long long c = w.cell[m];
      acc = fma3((double)Cw[m], (double)Cw[npf + m], (double)Cw[2 * npf + m], (double)x[3 * c],
                 (double)x[3 * c + 1], (double)x[3 * c + 2], acc);
    }
    acc = wsum(acc);
    if (lane == 0) y[3 * n + wi] = acc + (double)Dw[wi] * (double)x[3 * n + wi];
  }
}

__device__ __forceinline__ void cell_coords(const Grid& g, long long i, long long& ii, long long& j, long long& k) {
  const unsigned int ui = (unsigned int)i, nxy = (unsigned int)g.nxy, nxu = (unsigned int)g.nx;
  k = ui / nxy;  // 32-bit division: fewer than 2^31 cells
  const unsigned int rem = ui - (unsigned int)k * nxy;
  j = rem / nxu;
  ii = rem - (unsigned int)j * nxu;
}

__device__ __forceinline__ bool stencil_nbr(const Grid& g, int s, long long i, long long ii, long long j,
                                            long long k, long long& c) {
  switch (s) {
    case SL_D: c = i; return true;
    case SL_XM: c = i - 1; return ii > 0;
    case SL_XP: c = i + 1; return ii + 1 < g.nx;
    case SL_YM: c = i - g.nx; return j > 0;
    case SL_YP: c = i + g.nx; return j + 1 < g.ny;
    case SL_ZM: c = i - g.nxy; return k > 0;
    default: c = i + g.nxy; return k + 1 < g.nz;
  }
}

template <typename DT>
__global__ void __launch_bounds__(256, 4) k_spmv_cells(Grid g, Wells w, const DT* __restrict__ J,
                                                    const DT* __restrict__ Bw, const DT* __restrict__ Cw,
                                                    const DT* __restrict__ Dw, const double* __restrict__ x,
                                                    double* __restrict__ y, int cell_blocks) {
  PF_PDL_ENTRY();
  if ((int)blockIdx.x >= cell_blocks) {
    spmv_well_rows(g, w, Cw, Dw, x, y, cell_blocks);
    return;
  }
  const long long n = g.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)cell_blocks * blockDim.x) {
    long long ii, j, k;
    cell_coords(g, i, ii, j, k);
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      long long c;
      if (!stencil_nbr(g, s, i, ii, j, k, c)) continue;
      const DT* B = J + (size_t)s * 9 * n + i;
      const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      acc0 = fma2((double)B[0], (double)B[n], x0, x1, acc0);  // oil row: no polymer column
      acc1 = fma3((double)B[3 * n], (double)B[4 * n], (double)B[5 * n], x0, x1, x2, acc1);
      acc2 = fma3((double)B[6 * n], (double)B[7 * n], (double)B[8 * n], x0, x1, x2, acc2);
    }
    if (w.nw > 0) {
      const int m = w.perf_of[i];
      if (m >= 0) {
        const double xw = x[3 * n + w.pwell[m]];
        acc0 = __fma_rn((double)Bw[m], xw, acc0);
        acc1 = __fma_rn((double)Bw[w.npf + m], xw, acc1);
        acc2 = __fma_rn((double)Bw[2 * w.npf + m], xw, acc2);
      }
    }
    y[3 * i] = acc0;
    y[3 * i + 1] = acc1;
    y[3 * i + 2] = acc2;
  }
}

// The same product with one thread per (cell, row): a block holds groups of
// three warps, one per block row, over the same 32 cells, so J streams
// coalesced per row and the three warps share the x loads in L1.  Three times
// the threads of k_spmv_cells fill the GPU at small N; each row's sum is
// taken in the same order, so the result is identical.
template <typename DT>
__global__ void __launch_bounds__(384, 2) k_spmv_rows(Grid g, Wells w, const DT* __restrict__ J,
                                                   const DT* __restrict__ Bw, const DT* __restrict__ Cw,
                                                   const DT* __restrict__ Dw, const double* __restrict__ x,
                                                   double* __restrict__ y, int cell_blocks) {
  PF_PDL_ENTRY();
  if ((int)blockIdx.x >= cell_blocks) {
    spmv_well_rows(g, w, Cw, Dw, x, y, cell_blocks);
    return;
  }
  const long long n = g.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = warp % 3;
  const int groups = blockDim.x / 96;
  const long long stride = (long long)cell_blocks * groups * 32;
  for (long long i = ((long long)blockIdx.x * groups + warp / 3) * 32 + lane; i < n; i += stride) {
    long long ii, j, k;
    cell_coords(g, i, ii, j, k);
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      long long c;
      if (!stencil_nbr(g, s, i, ii, j, k, c)) continue;
      const DT* B = J + ((size_t)s * 9 + 3 * r) * n + i;
      const double x0 = x[3 * c], x1 = x[3 * c + 1];
      if (r == 0) {  // oil row: no polymer column (r is the same for the whole warp)
        acc = fma2((double)B[0], (double)B[n], x0, x1, acc);
      } else {
        acc = fma3((double)B[0], (double)B[n], (double)B[2 * n], x0, x1, x[3 * c + 2], acc);
      }
    }
    if (w.nw > 0) {
      const int m = w.perf_of[i];
      if (m >= 0) acc = __fma_rn((double)Bw[r * w.npf + m], x[3 * n + w.pwell[m]], acc);
    }
    y[3 * i + r] = acc;
  }
}

// Mixed-precision operator: FP32 Jacobian times an FP32 copy of the vector,
// accumulated in FP32 per row, written as FP64 (no FP64 arithmetic in the
// cell rows; the well column is added to the FP64 value).
__global__ void __launch_bounds__(256, 4) k_spmv_cells_f32(Grid g, Wells w, const float* __restrict__ J,
                                                        const float* __restrict__ Bw, const float* __restrict__ Cw,
                                                        const float* __restrict__ Dw, const float* __restrict__ x,
                                                        double* __restrict__ y, int cell_blocks) {
  PF_PDL_ENTRY();
  if ((int)blockIdx.x >= cell_blocks) {
    spmv_well_rows(g, w, Cw, Dw, x, y, cell_blocks);
    return;
  }
  const long long n = g.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)cell_blocks * blockDim.x) {
    long long ii, j, k;
    cell_coords(g, i, ii, j, k);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      long long c;
      if (!stencil_nbr(g, s, i, ii, j, k, c)) continue;
      const float* B = J + (size_t)s * 9 * n + i;
      const float x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      acc0 = fma2(B[0], B[n], x0, x1, acc0);  // oil row: no polymer column
      acc1 = fma3(B[3 * n], B[4 * n], B[5 * n], x0, x1, x2, acc1);
      acc2 = fma3(B[6 * n], B[7 * n], B[8 * n], x0, x1, x2, acc2);
    }
    double y0 = (double)acc0, y1 = (double)acc1, y2 = (double)acc2;
    if (w.nw > 0) {
      const int m = w.perf_of[i];
      if (m >= 0) {
        const float xw = x[3 * n + w.pwell[m]];
        y0 += (double)(Bw[m] * xw);
        y1 += (double)(Bw[w.npf + m] * xw);
        y2 += (double)(Bw[2 * w.npf + m] * xw);
      }
    }
    y[3 * i] = y0;
    y[3 * i + 1] = y1;
    y[3 * i + 2] = y2;
  }
}

inline int well_blocks(const Wells& w, int block) {
  const int wpb = block / 32;
  return w.nw > 0 ? (w.nw + wpb - 1) / wpb : 0;
}

void launch_spmv_f32(const Grid& g, const Wells& w, const float* J, const float* Bw, const float* Cw,
                     const float* Dw, const float* x, double* y, cudaStream_t st, int block) {
  const int cb = grid_for(g.n, block);
  launch(k_spmv_cells_f32, cb + well_blocks(w, block), block, 0, st, g, w, J, Bw, Cw, Dw, x, y, cb);
}

template <typename DT>
void launch_spmv(const Grid& g, const Wells& w, const DT* J, const DT* Bw, const DT* Cw, const DT* Dw,
                 const double* x, double* y, cudaStream_t st, int block) {
  if (block < 0) {
    // row-split form: -block = threads per block, a multiple of 96 (<= 384)
    const int tb = -block, cb = grid_for(g.n, tb / 3);
    launch(k_spmv_rows<DT>, cb + well_blocks(w, tb), tb, 0, st, g, w, J, Bw, Cw, Dw, x, y, cb);
  } else {
    const int cb = grid_for(g.n, block);
    launch(k_spmv_cells<DT>, cb + well_blocks(w, block), block, 0, st, g, w, J, Bw, Cw, Dw, x, y, cb);
  }
}

// ---------------------------------------------------------------------------
// block-Jacobi: inverse of each 3x3 diagonal block (adjugate / determinant)
// ---------------------------------------------------------------------------

// (the inverse is formed in the storage precision PT: FP64 for the plain
// path, FP32 for the mixed one)
template <typename PT>
__device__ __forceinline__ PT det3(const PT a[9]) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) + a[1] * (a[5] * a[6] - a[3] * a[8]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

template <typename PT>
__device__ __forceinline__ void inverse3(const PT a[9], PT inv[9]) {
  const PT c00 = a[4] * a[8] - a[5] * a[7];
  const PT c01 = a[5] * a[6] - a[3] * a[8];
  const PT c02 = a[3] * a[7] - a[4] * a[6];
  const PT det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  const PT id = (PT)1 / det;
  inv[0] = c00 * id;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  inv[3] = c01 * id;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  inv[6] = c02 * id;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

template <typename DT, typename PT>
__global__ void __launch_bounds__(256) k_bjacobi_setup(long long n, const DT* __restrict__ J, PT* __restrict__ Dinv) {
  PF_PDL_ENTRY();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    PT a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = (PT)J[(size_t)e * n + i];
    PT inv[9];
    inverse3(a, inv);
#pragma unroll
    for (int e = 0; e < 9; ++e) Dinv[(size_t)e * n + i] = inv[e];
  }
}

template <typename DT, typename PT>
__global__ void k_bjacobi_wells(int nw, const DT* __restrict__ Dw, PT* __restrict__ Dwinv) {
  PF_PDL_ENTRY();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nw) Dwinv[t] = (PT)(1.0 / (double)Dw[t]);
}

template <typename DT, typename PT>
void launch_bjacobi_setup(const Grid& g, const Wells& w, const DT* J, const DT* Dw, PT* Dinv, PT* Dwinv,
                          cudaStream_t st) {
  launch(k_bjacobi_setup<DT, PT>, grid_for(g.n, 256), 256, 0, st, g.n, J, Dinv);
  if (w.nw > 0) launch(k_bjacobi_wells<DT, PT>, grid_for(w.nw, 128), 128, 0, st, w.nw, Dw, Dwinv);
}

template <typename PT>
__global__ void __launch_bounds__(256) k_bjacobi_apply(long long n, int nw, const PT* __restrict__ Dinv,
                                                       const PT* __restrict__ Dwinv, const double* __restrict__ r,
                                                       double* __restrict__ z) {
  PF_PDL_ENTRY();
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

// ---------------------------------------------------------------------------
// block ILU(0) in red-black order: the local solve of the restricted additive
// Schwarz stage of CPR-FP (Alg. 2) with one subdomain
// ---------------------------------------------------------------------------
// Colour of cell (i, j, k): (i + j + k) mod 2, red 0, black 1.  With the red
// cells ordered first, the 7-point block pattern couples no two cells of one
// colour, so ILU(0) keeps the red diagonal blocks D_r, replaces each black
// one by D_b - sum_j J_bj D_j^-1 J_jb (fill between black cells dropped), and
// its two triangular solves become sweeps over one colour each:
//   t_r = D_r^-1 f_r;   y_b = D'_b^-1 (f_b - sum_j J_bj t_j);
//   y_r = D_r^-1 (f_r - sum_k J_rk y_k)
// (two launches: the first line is formed inside the black sweep).
// Well rows keep their scalar inverse, as in block-Jacobi.

// The q-th cell of a colour: rows (j, k) of ceil(nx / 2) slots; in row (j, k)
// the colour's cells are x = ((j + k + colour) & 1) + 2m.  False for a slot
// past the row's end.  Consecutive threads take consecutive cells of a row.
__device__ __forceinline__ bool colour_cell(const Grid& g, int colour, long long q, long long& i, int& x, int& y,
                                            int& z) {
  const unsigned int hx = ((unsigned int)g.nx + 1u) >> 1;
  const unsigned int uq = (unsigned int)q;
  const unsigned int row = uq / hx, m = uq - row * hx;
  const unsigned int ny = (unsigned int)g.ny;
  z = (int)(row / ny);
  y = (int)(row - (unsigned int)z * ny);
  x = (int)(((unsigned int)(y + z + colour) & 1u) + 2u * m);
  if (x >= g.nx) return false;
  i = (long long)x + (long long)g.nx * row;
  return true;
}

__device__ __forceinline__ long long colour_slots(const Grid& g) {
  return (long long)((g.nx + 1) / 2) * g.ny * g.nz;
}

// neighbour of (x, y, z) through slot s (s != SL_D); false outside the grid
__device__ __forceinline__ bool slot_nbr(const Grid& g, int s, long long i, int x, int y, int z, long long& c) {
  switch (s) {
    case SL_XM: c = i - 1; return x > 0;
    case SL_XP: c = i + 1; return x + 1 < g.nx;
    case SL_YM: c = i - g.nx; return y > 0;
    case SL_YP: c = i + g.nx; return y + 1 < g.ny;
    case SL_ZM: c = i - g.nxy; return z > 0;
    default: c = i + g.nxy; return z + 1 < g.nz;
  }
}

// colour slot of the neighbour through slot s of the cell in colour slot q at
// column x (the neighbour has the other colour; its column is x -+ 1, or x)
__device__ __forceinline__ long long nbr_slot(const Grid& g, int s, long long q, int x) {
  const long long hx = (g.nx + 1) / 2;
  switch (s) {
    case SL_XM: return q - ((x & 1) ? 0 : 1);
    case SL_XP: return q + (x & 1);
    case SL_YM: return q - hx;
    case SL_YP: return q + hx;
    case SL_ZM: return q - hx * g.ny;
    default: return q + hx * g.ny;
  }
}

// storage conversions of the compact per-colour block copies (CT: the
// Jacobian's own type, or BF16)
__device__ __forceinline__ float to_ct(float v, float) { return v; }
__device__ __forceinline__ double to_ct(double v, double) { return v; }
__device__ __forceinline__ __nv_bfloat16 to_ct(float v, __nv_bfloat16) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __nv_bfloat16 to_ct(double v, __nv_bfloat16) { return __float2bfloat16_rn((float)v); }

// black diagonal blocks: D'_b = D_b - sum_j J_bj D_j^-1 J_jb, then inverted;
// the red blocks' inverses (from k_red_inverse) are read, not written.  With
// Dc (the block inverses per colour slot, red then black; null for none) the
// red inverses are read from it and the black ones written to it, else both
// go through Dinv by cell.
// With cred and cblack (the compact per-colour copies of the off-diagonal
// blocks; null for none) the kernel also writes the copies: a black cell's own
// six blocks into cblack, and each red neighbour's block that points back at it
// into cred (every red block points at exactly one black cell, so each is
// written once; blocks that leave the grid are never read).  It reads all of
// them for the Schur update anyway.  The oil row's polymer column is skipped
// (structurally zero, never read).  With pc (and pdg) it also writes the
// black row's pressure combination w_o (oil row) + w_w (water row) of each of
// its blocks for the CPR stage 2: pc [6 slots][3 columns][slots], pdg the
// diagonal block's [3 columns][slots] (from J, before the Schur update).
// Two blocks of 256 per SM (128 registers; FP64 spills up to 48 bytes a thread):
// at 27M cells FP64 0.9 ms per set-up faster than one block at 254 registers.
// With TF (with the copies), cblack receives T = J_bj D_j^-1 (all nine
// entries; the oil row's polymer column of T is not zero) in place of J_bj,
// and in FP64 the inverses go through Dc; otherwise Dc is ignored
// (compile-time choices, so that each form keeps its own register count).
template <typename DT, typename PT, typename CT, bool TF>
__global__ void __launch_bounds__(256, 2) k_ilu_setup_black(Grid g, const DT* __restrict__ J, PT* __restrict__ Dinv,
                                                          PT guard, CT* __restrict__ cred, CT* __restrict__ cblack,
                                                          CT* __restrict__ pc, PT* __restrict__ pdg, PT w_o,
                                                          PT w_w, PT* __restrict__ Dc) {
  PF_PDL_ENTRY();
  constexpr bool DS = TF && std::is_same<PT, double>::value;  // the inverses per colour slot (FP64)
  const long long n = g.n, nq = colour_slots(g);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
       q += (long long)gridDim.x * blockDim.x) {
    long long i;
    int x, y, z;
    if (!colour_cell(g, 1, q, i, x, y, z)) continue;
    PT a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = (PT)J[(size_t)e * n + i];
    if (pdg) {  // the oil row's polymer column is zero
      pdg[q] = w_o * a[0] + w_w * a[3];
      pdg[nq + q] = w_o * a[1] + w_w * a[4];
      pdg[2 * nq + q] = w_w * a[5];
    }
    const PT det0 = det3(a);
#pragma unroll
    for (int s = 1; s < SL_COUNT; ++s) {
      long long c;
      if (!slot_nbr(g, s, i, x, y, z, c)) continue;
      const int so = (s & 1) ? s + 1 : s - 1;  // the slot of row c that points back at i
      // the red neighbour's colour slot (for its compact copies)
      const long long qc = nbr_slot(g, s, q, x);
      const PT* Dj = DS ? Dc + qc : Dinv + c;  // D_j^-1
      const long long md = DS ? nq : n;
      CT* bl = cblack ? cblack + (size_t)(s - 1) * 9 * nq + q : nullptr;
      CT* rd = cred ? cred + (size_t)(so - 1) * 9 * nq + qc : nullptr;
      const CT zc{};
      PT T[9];  // J_bj D_j^-1 (the oil row of J_bj has no polymer column: fma2)
      PT po0 = 0, po1 = 0;  // the oil row (columns P, S) for the pressure combination
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const DT b0r = J[((size_t)s * 9 + 3 * r) * n + i], b1r = J[((size_t)s * 9 + 3 * r + 1) * n + i];
        const PT b0 = (PT)b0r, b1 = (PT)b1r;
        if (bl && !TF) {
          bl[(size_t)(3 * r) * nq] = to_ct(b0r, zc);
          bl[(size_t)(3 * r + 1) * nq] = to_ct(b1r, zc);
        }
        DT b2r = 0;
        if (r != 0) {
          b2r = J[((size_t)s * 9 + 3 * r + 2) * n + i];
          if (bl && !TF) bl[(size_t)(3 * r + 2) * nq] = to_ct(b2r, zc);
        }
        // the pressure combination w_o (oil row) + w_w (water row) of this block
        if (pc && r == 0) { po0 = b0; po1 = b1; }
        if (pc && r == 1) {
          CT* P3 = pc + (size_t)(s - 1) * 3 * nq + q;
          P3[0] = to_ct(w_o * po0 + w_w * b0, zc);
          P3[nq] = to_ct(w_o * po1 + w_w * b1, zc);
          P3[2 * nq] = to_ct(w_w * (PT)b2r, zc);
        }
#pragma unroll
        for (int col = 0; col < 3; ++col) {
          const PT d0 = Dj[col * md], d1 = Dj[(3 + col) * md];
          if (r == 0) {
            T[col] = fma2(b0, b1, d0, d1, (PT)0);
          } else {
            T[3 * r + col] = fma3(b0, b1, (PT)b2r, d0, d1, Dj[(6 + col) * md], (PT)0);
          }
        }
      }
      if (TF && bl) {
#pragma unroll
        for (int e = 0; e < 9; ++e) bl[(size_t)e * nq] = to_ct(T[e], zc);
      }
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        // column col of J_jb; its oil-row entry is zero in the polymer column
        const DT u1r = J[((size_t)so * 9 + 3 + col) * n + c], u2r = J[((size_t)so * 9 + 6 + col) * n + c];
        const PT u1 = (PT)u1r, u2 = (PT)u2r;
        if (rd) {
          rd[(size_t)(3 + col) * nq] = to_ct(u1r, zc);
          rd[(size_t)(6 + col) * nq] = to_ct(u2r, zc);
        }
        if (col == 2) {
#pragma unroll
          for (int r = 0; r < 3; ++r) a[3 * r + col] = fnms2(T[3 * r + 1], T[3 * r + 2], u1, u2, a[3 * r + col]);
        } else {
          const DT u0r = J[((size_t)so * 9 + col) * n + c];
          if (rd) rd[(size_t)col * nq] = to_ct(u0r, zc);
          const PT u0 = (PT)u0r;
#pragma unroll
          for (int r = 0; r < 3; ++r)
            a[3 * r + col] = fnms3(T[3 * r], T[3 * r + 1], T[3 * r + 2], u0, u1, u2, a[3 * r + col]);
        }
      }
    }
    // pivot guard: det(D'_b) / det(D_b) = det(I - D_b^-1 S) measures how much
    // closer to singular the Schur update made the block; below `guard` (or
    // of the other sign, or not finite) the cell keeps its own block D_b
    const PT ratio = det3(a) / det0;
    if (!(ratio > guard)) {
#pragma unroll
      for (int e = 0; e < 9; ++e) a[e] = (PT)J[(size_t)e * n + i];
    }
    PT inv[9];
    inverse3(a, inv);
    if (DS) {
#pragma unroll
      for (int e = 0; e < 9; ++e) Dc[(size_t)(9 + e) * nq + q] = inv[e];
    } else {
#pragma unroll
      for (int e = 0; e < 9; ++e) Dinv[(size_t)e * n + i] = inv[e];
    }
  }
}

// diagonal-only first sweep: t_r = D_r^-1 f_r on the red cells, into y
template <typename PT, typename OT, typename VT>
__global__ void __launch_bounds__(256) k_ilu_red_diag(Grid g, const PT* __restrict__ Dinv, const VT* __restrict__ f,
                                                      OT* __restrict__ y) {
  PF_PDL_ENTRY();
  const long long n = g.n, nq = colour_slots(g);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
       q += (long long)gridDim.x * blockDim.x) {
    long long i;
    int x, yy, z;
    if (!colour_cell(g, 0, q, i, x, yy, z)) continue;
    const PT f0 = (PT)f[3 * i], f1 = (PT)f[3 * i + 1], f2 = (PT)f[3 * i + 2];
    const PT* D = Dinv + i;
    y[3 * i] = (OT)(D[0] * f0 + D[n] * f1 + D[2 * n] * f2);
    y[3 * i + 1] = (OT)(D[3 * n] * f0 + D[4 * n] * f1 + D[5 * n] * f2);
    y[3 * i + 2] = (OT)(D[6 * n] * f0 + D[7 * n] * f1 + D[8 * n] * f2);
  }
}

// y_i = D_i^-1 (f_i - sum over neighbours J_ij t_j) on the cells of one
// colour (the neighbours all have the other colour).  Black sweep (colour 1):
// t_j = D_j^-1 f_j of the red neighbours, formed on the fly when fused (the
// diagonal-only red sweep folded in), else read from y where k_ilu_red_diag
// left it; red sweep (colour 0): t_j = y_j of the black neighbours, and the
// threads past the cells take the well rows y_w = f_w / D_w.
__device__ __forceinline__ float as_pt(float v, float) { return v; }
__device__ __forceinline__ float as_pt(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ double as_pt(double v, double) { return v; }
__device__ __forceinline__ double as_pt(float v, double) { return (double)v; }
__device__ __forceinline__ double as_pt(__nv_bfloat16 v, double) { return (double)__bfloat162float(v); }

// With COMPACT the off-diagonal blocks come from this colour's compact copy
// (written by k_ilu_setup_black: slot-major, indexed by the colour slot q, so a sweep reads
// only its own rows); otherwise from J itself, whose lines also carry the
// other colour's rows.  MODE: 0 the red sweep (t_j = y_j of the black
// neighbours, then the well rows), 1 the black sweep after k_ilu_red_diag
// (t_j = y_j of the red neighbours), 2 the black sweep with the red diagonal
// folded in (t_j = D_j^-1 f_j formed on the fly), 3 the black sweep through
// the set-up's products T = J_bj D_j^-1 (J_bj t_j = T f_j; J is then the
// by-slot array of T).  One instantiation per mode
// keeps each launch's code (and registers) to its own path.  In FP64 with
// COMPACT (modes 3 and 0) the diagonal block inverses come from Dc (both
// colours per colour slot, red then black), else from Dinv by cell.
template <typename BT, typename PT, typename OT, bool COMPACT, typename VT, int MODE>
__global__ void __launch_bounds__(256, 4) k_ilu_sweep(Grid g, int nw, const BT* __restrict__ J,
                                                   const PT* __restrict__ Dinv, const PT* __restrict__ Dc,
                                                   const PT* __restrict__ Dwinv, const VT* __restrict__ f,
                                                   OT* __restrict__ y) {
  PF_PDL_ENTRY();
  constexpr int colour = MODE == 0 ? 0 : 1;
  const long long n = g.n, nq = colour_slots(g);
  const long long nt = nq + (colour == 0 ? nw : 0);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nt;
       q += (long long)gridDim.x * blockDim.x) {
    if (colour == 0 && q >= nq) {
      const long long w = q - nq;
      y[3 * n + w] = (OT)((PT)Dwinv[w] * (PT)f[3 * n + w]);
      continue;
    }
    long long i;
    int x, yy, z;
    if (!colour_cell(g, colour, q, i, x, yy, z)) continue;
    PT r0 = (PT)f[3 * i], r1 = (PT)f[3 * i + 1], r2 = (PT)f[3 * i + 2];
#pragma unroll
    for (int s = 1; s < SL_COUNT; ++s) {
      long long c;
      if (!slot_nbr(g, s, i, x, yy, z, c)) continue;
      PT t0, t1, t2;
      if (MODE == 3) {
        t0 = (PT)f[3 * c];
        t1 = (PT)f[3 * c + 1];
        t2 = (PT)f[3 * c + 2];
      } else if (MODE == 2) {
        const PT f0 = (PT)f[3 * c], f1 = (PT)f[3 * c + 1], f2 = (PT)f[3 * c + 2];
        const PT* Dj = Dinv + c;
        t0 = Dj[0] * f0 + Dj[n] * f1 + Dj[2 * n] * f2;
        t1 = Dj[3 * n] * f0 + Dj[4 * n] * f1 + Dj[5 * n] * f2;
        t2 = Dj[6 * n] * f0 + Dj[7 * n] * f1 + Dj[8 * n] * f2;
      } else {
        t0 = (PT)y[3 * c];
        t1 = (PT)y[3 * c + 1];
        t2 = (PT)y[3 * c + 2];
      }
      const BT* B = COMPACT ? J + (size_t)(s - 1) * 9 * nq + q : J + (size_t)s * 9 * n + i;
      const long long m = COMPACT ? nq : n;
      const PT pz{};
      if (MODE == 3)  // T = J_bj D_j^-1: a full oil row
        r0 = fnms3(as_pt(B[0], pz), as_pt(B[m], pz), as_pt(B[2 * m], pz), t0, t1, t2, r0);
      else
        r0 = fnms2(as_pt(B[0], pz), as_pt(B[m], pz), t0, t1, r0);  // oil row: no polymer column
      r1 = fnms3(as_pt(B[3 * m], pz), as_pt(B[4 * m], pz), as_pt(B[5 * m], pz), t0, t1, t2, r1);
      r2 = fnms3(as_pt(B[6 * m], pz), as_pt(B[7 * m], pz), as_pt(B[8 * m], pz), t0, t1, t2, r2);
    }
    // FP64 with the copies: the inverses per colour slot
    constexpr bool dslot = COMPACT && std::is_same<PT, double>::value;
    const PT* D = dslot ? Dc + (size_t)colour * 9 * nq + q : Dinv + i;
    const long long md = dslot ? nq : n;
    y[3 * i] = (OT)(D[0] * r0 + D[md] * r1 + D[2 * md] * r2);
    y[3 * i + 1] = (OT)(D[3 * md] * r0 + D[4 * md] * r1 + D[5 * md] * r2);
    y[3 * i + 2] = (OT)(D[6 * md] * r0 + D[7 * md] * r1 + D[8 * md] * r2);
  }
}

// the red cells' diagonal block inverses (the black ones come from the
// Schur-updated blocks in k_ilu_setup_black), into Dinv by cell, or with the
// per-colour copies into Dr by red colour slot instead (Dinv is then not
// written: every reader takes the copy)
template <typename DT, typename PT>
__global__ void __launch_bounds__(256) k_red_inverse(Grid g, const DT* __restrict__ J, PT* __restrict__ Dinv,
                                                     PT* __restrict__ Dr) {
  PF_PDL_ENTRY();
  const long long n = g.n, nq = colour_slots(g);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
       q += (long long)gridDim.x * blockDim.x) {
    long long i;
    int x, y, z;
    if (!colour_cell(g, 0, q, i, x, y, z)) continue;
    PT a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = (PT)J[(size_t)e * n + i];
    PT inv[9];
    inverse3(a, inv);
    if (Dr) {
#pragma unroll
      for (int e = 0; e < 9; ++e) Dr[(size_t)e * nq + q] = inv[e];
    } else {
#pragma unroll
      for (int e = 0; e < 9; ++e) Dinv[(size_t)e * n + i] = inv[e];
    }
  }
}

template <typename DT, typename PT>
void launch_ilu_setup(const Grid& g, const Wells& w, const DT* J, const DT* Dw, PT* Dinv, PT* Dwinv,
                      double guard, const IluCompact& cp, cudaStream_t st, double w_o, double w_w) {
  launch(k_red_inverse<DT, PT>, grid_for(colour_slots_host(g), 256), 256, 0, st, g, J, Dinv, (PT*)cp.dr);
  if (w.nw > 0) launch(k_bjacobi_wells<DT, PT>, grid_for(w.nw, 128), 128, 0, st, w.nw, Dw, Dwinv);
  // the black set-up also writes the compact per-colour copies the sweeps read
  // and the pressure combination stage 2 reads
  const int grid = grid_for(colour_slots_host(g), 256);
  const PT wo = (PT)w_o, ww = (PT)w_w;
  if (cp.kind == 2)  // the copies: T = J_bj D_j^-1 into the black copy (FP64: the inverses per colour slot)
    launch(k_ilu_setup_black<DT, PT, __nv_bfloat16, true>, grid, 256, 0, st, g, J, Dinv, (PT)guard,
           (__nv_bfloat16*)cp.c[0], (__nv_bfloat16*)cp.c[1], (__nv_bfloat16*)cp.p, (PT*)cp.pd, wo, ww,
           (PT*)cp.dr);
  else if (cp.kind == 1)
    launch(k_ilu_setup_black<DT, PT, DT, true>, grid, 256, 0, st, g, J, Dinv, (PT)guard, (DT*)cp.c[0],
           (DT*)cp.c[1], (DT*)cp.p, (PT*)cp.pd, wo, ww, (PT*)cp.dr);
  else  // without the copies: the inverses by cell
    launch(k_ilu_setup_black<DT, PT, DT, false>, grid, 256, 0, st, g, J, Dinv, (PT)guard, (DT*)nullptr,
           (DT*)nullptr, (DT*)cp.p, (PT*)cp.pd, wo, ww, (PT*)nullptr);
}

template <typename DT, typename PT, typename OT, typename VT>
int launch_ilu_apply(const Grid& g, int nw, const DT* J, const PT* Dinv, const PT* Dwinv, const VT* f, OT* y,
                     int fused, const IluCompact& cp, cudaStream_t st) {
  const long long nq = colour_slots_host(g);
  const PT* Dc = (const PT*)cp.dr;  // the block inverses per colour slot (with the copies)
  const int grid1 = grid_for(nq, 256), grid0 = grid_for(nq + nw, 256);
  if (cp.kind == 2) {  // the copies: black sweep through T = J_bj D_j^-1, then the red sweep
    const __nv_bfloat16 *c0 = (const __nv_bfloat16*)cp.c[0], *c1 = (const __nv_bfloat16*)cp.c[1];
    launch(k_ilu_sweep<__nv_bfloat16, PT, OT, true, VT, 3>, grid1, 256, 0, st, g, nw, c1, Dinv, Dc, Dwinv, f, y);
    launch(k_ilu_sweep<__nv_bfloat16, PT, OT, true, VT, 0>, grid0, 256, 0, st, g, nw, c0, Dinv, Dc, Dwinv, f, y);
    return 2;
  }
  if (cp.kind == 1) {
    const DT *c0 = (const DT*)cp.c[0], *c1 = (const DT*)cp.c[1];
    launch(k_ilu_sweep<DT, PT, OT, true, VT, 3>, grid1, 256, 0, st, g, nw, c1, Dinv, Dc, Dwinv, f, y);
    launch(k_ilu_sweep<DT, PT, OT, true, VT, 0>, grid0, 256, 0, st, g, nw, c0, Dinv, Dc, Dwinv, f, y);
    return 2;
  }
  // without the copies, from J: the diagonal red sweep folded into the black one or on its own, then the red sweep
  const PT* none = nullptr;
  if (!fused) launch(k_ilu_red_diag<PT, OT, VT>, grid_for(nq, 256), 256, 0, st, g, Dinv, f, y);
  if (fused) launch(k_ilu_sweep<DT, PT, OT, false, VT, 2>, grid1, 256, 0, st, g, nw, J, Dinv, none, Dwinv, f, y);
  else launch(k_ilu_sweep<DT, PT, OT, false, VT, 1>, grid1, 256, 0, st, g, nw, J, Dinv, none, Dwinv, f, y);
  launch(k_ilu_sweep<DT, PT, OT, false, VT, 0>, grid0, 256, 0, st, g, nw, J, Dinv, none, Dwinv, f, y);
  return fused ? 2 : 3;
}

// CPR stage 2 after the red-black block ILU(0) first stage (Alg. 2):
// b0 = w_o (v - J y)_oil + w_w (v - J y)_water.  The red sweep, the last one,
// solved the red rows' cell part exactly, D_r y_r + sum_b J_rb y_b = v_r with
// the off-diagonal blocks it read, so a red row's residual is its well column
// alone, -B y_w (up to rounding).  The black rows are formed in full: with
// COMPACT from the pressure combination w_o (oil row) + w_w (water row) of
// each block, precomputed by the ILU(0) set-up per black colour slot (Pc, the
// off-diagonal blocks in the copy's type or J's; Pd, the diagonal block), so
// b0 = (w_o v_o + w_w v_w) - sum of the combined rows times y, three
// multiply-adds per block instead of five; otherwise from J's oil and water
// rows.  Threads [0, nq) take the black cells and [nq, 2 nq) the red ones, so
// the black threads of a warp run together.  With x0 the red threads also do
// the multigrid cycle's first pass on the finest pressure level, from its
// zero initial guess: x0 = b0 / a_ii (b0 times the stored 1 / diagonal, d0[q]
// of the red per-colour copy when d0_slot, else d0[i]).
template <typename T, typename BT, bool COMPACT, typename VT>
__global__ void __launch_bounds__(256, 4) k_stage2_ilu(Grid g, Wells w, const T* __restrict__ J,
                                                    const BT* __restrict__ Pc, const T* __restrict__ Pd,
                                                    const T* __restrict__ Bw, const T* __restrict__ y,
                                                    const VT* __restrict__ v, T w_o, T w_w, T* __restrict__ b0,
                                                    T* __restrict__ x0, const T* __restrict__ d0, int d0_slot) {
  PF_PDL_ENTRY();
  const long long n = g.n, nq = colour_slots(g);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * nq;
       t += (long long)gridDim.x * blockDim.x) {
    const int colour = t < nq ? 1 : 0;
    const long long q = colour ? t : t - nq;
    long long i;
    int x, yy, z;
    if (!colour_cell(g, colour, q, i, x, yy, z)) continue;
    T r = 0;
    if (colour == 1 && COMPACT) {
      const T d0 = y[3 * i], d1 = y[3 * i + 1], d2 = y[3 * i + 2];
      T t = fma3(Pd[q], Pd[nq + q], Pd[2 * nq + q], d0, d1, d2, (T)0);
      const T pz{};
#pragma unroll
      for (int s = 1; s < SL_COUNT; ++s) {
        long long c;
        if (!slot_nbr(g, s, i, x, yy, z, c)) continue;
        const BT* B = Pc + (size_t)(s - 1) * 3 * nq + q;
        t = fma3(as_pt(B[0], pz), as_pt(B[nq], pz), as_pt(B[2 * nq], pz), y[3 * c], y[3 * c + 1], y[3 * c + 2], t);
      }
      r = (w_o * (T)v[3 * i] + w_w * (T)v[3 * i + 1]) - t;
    } else if (colour == 1) {
      const T* D = J + i;
      const T d0 = y[3 * i], d1 = y[3 * i + 1], d2 = y[3 * i + 2];
      T t0 = fma2(D[0], D[n], d0, d1, (T)0);  // oil row: no polymer column
      T t1 = fma3(D[3 * n], D[4 * n], D[5 * n], d0, d1, d2, (T)0);
#pragma unroll
      for (int s = 1; s < SL_COUNT; ++s) {
        long long c;
        if (!slot_nbr(g, s, i, x, yy, z, c)) continue;
        const T* B = J + (size_t)s * 9 * n + i;
        const T x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
        t0 = fma2(B[0], B[n], x0, x1, t0);
        t1 = fma3(B[3 * n], B[4 * n], B[5 * n], x0, x1, x2, t1);
      }
      r = w_o * ((T)v[3 * i] - t0) + w_w * ((T)v[3 * i + 1] - t1);
    }
    if (w.nw > 0) {
      const int m = w.perf_of[i];
      if (m >= 0) r -= (w_o * Bw[m] + w_w * Bw[w.npf + m]) * y[3 * n + w.pwell[m]];
    }
    b0[i] = r;
    if (colour == 0 && x0) x0[i] = r * d0[d0_slot ? q : i];
  }
}

template <typename T, typename VT>
void launch_stage2_ilu(const Grid& g, const Wells& w, const T* J, const IluCompact& cp, const T* Bw, const T* y,
                       const VT* v, T w_o, T w_w, T* b0, T* x0, const T* d0, int d0_slot, int block,
                       cudaStream_t st) {
  const int grid = grid_for(2 * colour_slots_host(g), block);
  if (cp.kind != 2 && cp.p)
    launch(k_stage2_ilu<T, T, true, VT>, grid, block, 0, st, g, w, J, (const T*)cp.p, (const T*)cp.pd, Bw, y, v, w_o,
           w_w, b0, x0, d0, d0_slot);
  else if (cp.kind == 2 && cp.p)
    launch(k_stage2_ilu<T, __nv_bfloat16, true, VT>, grid, block, 0, st, g, w, J, (const __nv_bfloat16*)cp.p,
           (const T*)cp.pd, Bw, y, v, w_o, w_w, b0, x0, d0, d0_slot);
  else
    launch(k_stage2_ilu<T, T, false, VT>, grid, block, 0, st, g, w, J, (const T*)nullptr, (const T*)nullptr, Bw, y,
           v, w_o, w_w, b0, x0, d0, d0_slot);
}

template <typename PT>
void launch_bjacobi_apply(const Grid& g, int nw, const PT* Dinv, const PT* Dwinv, const double* r, double* z,
                          cudaStream_t st) {
  launch(k_bjacobi_apply<PT>, grid_for(g.n + nw, 256), 256, 0, st, g.n, nw, Dinv, Dwinv, r, z);
}

// ---------------------------------------------------------------------------
// FP64 vector kernels
// ---------------------------------------------------------------------------

#define GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void k_copy(long long n, const double* __restrict__ a, double* __restrict__ b) {
  PF_PDL_ENTRY(); GRID_STRIDE(i, n) b[i] = a[i]; }
__global__ void k_fill(long long n, double v, double* __restrict__ a) {
  PF_PDL_ENTRY(); GRID_STRIDE(i, n) a[i] = v; }
__global__ void k_scale_dev(long long n, const double* a, const double* __restrict__ s, int inv_sqrt,
                            double* b) {
  PF_PDL_ENTRY();
  const double f = inv_sqrt ? 1.0 / sqrt(s[0]) : s[0];
  GRID_STRIDE(i, n) b[i] = a[i] * f;
}

// the same, and an FP32 copy of b (the mixed-precision preconditioner's input)
__global__ void k_scale_dev_f32(long long n, const double* a, const double* __restrict__ s, int inv_sqrt, double* b,
                                float* __restrict__ bf) {
  PF_PDL_ENTRY();
  const double f = inv_sqrt ? 1.0 / sqrt(s[0]) : s[0];
  GRID_STRIDE(i, n) {
    const double v = a[i] * f;
    b[i] = v;
    bf[i] = (float)v;
  }
}
__global__ void k_axpy(long long n, double al, const double* __restrict__ x, double* __restrict__ y) {
  PF_PDL_ENTRY();
  GRID_STRIDE(i, n) y[i] += al * x[i];
}
__global__ void k_xpay(long long n, const double* __restrict__ x, double be, double* __restrict__ y) {
  PF_PDL_ENTRY();
  GRID_STRIDE(i, n) y[i] = x[i] + be * y[i];
}
__global__ void k_sub(long long n, const double* a, const double* b, double* c) {
  PF_PDL_ENTRY();
  GRID_STRIDE(i, n) c[i] = a[i] - b[i];
}

__global__ void k_to_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
  PF_PDL_ENTRY();
  GRID_STRIDE(i, n) b[i] = (float)a[i];
}
void launch_to_f32(long long n, const double* a, float* b, cudaStream_t st) {
  launch(k_to_f32, grid_for(n, 256), 256, 0, st, n, a, b);
}

void launch_copy(long long n, const double* a, double* b, cudaStream_t st) {
  launch(k_copy, grid_for(n, 256), 256, 0, st, n, a, b);
}
void launch_fill(long long n, double v, double* a, cudaStream_t st) { launch(k_fill, grid_for(n, 256), 256, 0, st, n, v, a); }
void launch_scale_by_dev(long long n, const double* a, const double* s, int inv_sqrt, double* b, cudaStream_t st,
                         float* bf) {
  if (bf) launch(k_scale_dev_f32, grid_for(n, 256), 256, 0, st, n, a, s, inv_sqrt, b, bf);
  else launch(k_scale_dev, grid_for(n, 256), 256, 0, st, n, a, s, inv_sqrt, b);
}
void launch_axpy(long long n, double al, const double* x, double* y, cudaStream_t st) {
  launch(k_axpy, grid_for(n, 256), 256, 0, st, n, al, x, y);
}
void launch_xpay(long long n, const double* x, double be, double* y, cudaStream_t st) {
  launch(k_xpay, grid_for(n, 256), 256, 0, st, n, x, be, y);
}
void launch_sub(long long n, const double* a, const double* b, double* c, cudaStream_t st) {
  launch(k_sub, grid_for(n, 256), 256, 0, st, n, a, b, c);
}

// Sum of p[b * stride] over b = lane, lane + 32, ... < nb, added in that order
// (the order of the plain strided loop), with the loads issued eight at a
// time so that a lane waits for one L2 round trip per eight values instead
// of one per value.
__device__ __forceinline__ double lane_sum_blocks(const double* p, size_t stride, int nb, int lane) {
  double s = 0.0;
  for (int b = lane; b < nb; b += 8 * 32) {
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = b + 32 * t < nb ? __ldcg(p + (size_t)(b + 32 * t) * stride) : 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (b + 32 * t < nb) s += v[t];
  }
  return s;
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
// scale (may be null): out[j] *= scale[j] for the first nscaled values.
// Returns true in the last block (whose threads then all see out).
__device__ __forceinline__ bool last_block_reduce(const double* partial, int stride, int k, double* out,
                                                  unsigned int* counter, bool inv_norm = false,
                                                  const double* norm0 = nullptr, int* decide = nullptr,
                                                  const double* scale = nullptr, int nscaled = 0) {
  __shared__ bool last;
  __threadfence();  // every thread that wrote a partial publishes it before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double s = lane_sum_blocks(partial + j, stride, (int)gridDim.x, lane);
    s = wsum(s);
    if (lane == 0) {
      out[j] = (scale && j < nscaled) ? s * scale[j] : s;
      // out[k] = 1 / sqrt(last value): one FP64 sqrt and divide for the whole
      // vector instead of one per thread of the scaling kernel
      if (inv_norm && j == k - 1) out[k] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
      // selective reorthogonalisation: a second pass is needed only if the
      // first removed more than half of |w|^2 (norm1^2 < norm0^2 / 2)
      if (decide && j == k - 1) *decide = (s > 0.5 * norm0[0]) ? 1 : 0;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// One tile of the multi-dot: NT columns of V (and <w, w> when SELF), with a
// compile-time width so that no FP64 FMA is issued for an unused slot (on
// this part a predicated-off FP64 instruction still costs its pipe cycles).
template <int NT, bool SELF>
__device__ __forceinline__ void md_tile(long long n, const double* __restrict__ V, long long ld,
                                        const double* __restrict__ w, int j0, double* partial_row) {
  constexpr int KM = NT + (SELF ? 1 : 0);
  constexpr int KA = KM > 0 ? KM : 1;  // storage (NT = 0 without SELF is never called)
  double acc[KA];
#pragma unroll
  for (int t = 0; t < KM; ++t) acc[t] = 0.0;
  GRID_STRIDE(i, n) {
    const double wi = w[i];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t] += V[(size_t)(j0 + t) * ld + i] * wi;
    if (SELF) acc[KM - 1] += wi * wi;
  }
  block_reduce_write<KA>(acc, KM, partial_row + j0);
  __syncthreads();
}

template <bool SELF>
__device__ __forceinline__ void md_dispatch(int nt, long long n, const double* V, long long ld, const double* w,
                                            int j0, double* row) {
  switch (nt) {
    case 0: md_tile<0, SELF>(n, V, ld, w, j0, row); break;
    case 1: md_tile<1, SELF>(n, V, ld, w, j0, row); break;
    case 2: md_tile<2, SELF>(n, V, ld, w, j0, row); break;
    case 3: md_tile<3, SELF>(n, V, ld, w, j0, row); break;
    case 4: md_tile<4, SELF>(n, V, ld, w, j0, row); break;
    case 5: md_tile<5, SELF>(n, V, ld, w, j0, row); break;
    case 6: md_tile<6, SELF>(n, V, ld, w, j0, row); break;
    case 7: md_tile<7, SELF>(n, V, ld, w, j0, row); break;
    default: md_tile<8, SELF>(n, V, ld, w, j0, row); break;
  }
}

// out[j] = <V_j, w> for j < k (times vs[j] when vs is given: V_j then holds
// the basis vector before its normalisation by vs[j]) and, with self_dot,
// out[k] = <w, w>; columns in tiles of up to 8 (few registers, high
// occupancy), w re-read per tile.  run_if (may be null): the kernel returns at
// once unless *run_if is set.
// pyth (may be null; needs self_dot and orthonormal v_j): the squared norm of
// w after the projection, by Pythagoras, |w - sum_j h_j v_j|^2 = |w|^2 -
// sum_j h_j^2 with h_j = out[j], into pyth[0] and its 1/sqrt into pyth[1] and
// *vs_next; *decide = 1 when it is below eta2 |w|^2 (a second Gram-Schmidt
// pass will follow and measure the norm directly).
__global__ void __launch_bounds__(256) k_multidot(long long n, int k, const double* __restrict__ V, long long ld,
                                                  const double* __restrict__ w, double* __restrict__ partial,
                                                  int stride, double* __restrict__ out, unsigned int* counter,
                                                  int self_dot, const int* run_if, const double* __restrict__ vs,
                                                  double* __restrict__ pyth, double* __restrict__ vs_next,
                                                  int* __restrict__ decide, double eta2) {
  PF_PDL_ENTRY();
  if (run_if && !*run_if) return;
  double* row = partial + (size_t)blockIdx.x * stride;
  int j0 = 0;
  for (; j0 + 8 < k || (j0 + 8 == k && self_dot); j0 += 8) md_dispatch<false>(8, n, V, ld, w, j0, row);
  const int nt = k - j0;  // 0..8 columns left
  if (self_dot) md_dispatch<true>(nt, n, V, ld, w, j0, row);
  else if (nt > 0) md_dispatch<false>(nt, n, V, ld, w, j0, row);
  if (!last_block_reduce(partial, stride, k + (self_dot ? 1 : 0), out, counter, false, nullptr, nullptr, vs, k))
    return;
  if (pyth && threadIdx.x < 32) {
    double q = 0.0;  // sum of h_j^2 in a fixed order (lanes over j, then a shuffle tree)
    for (int j = threadIdx.x; j < k; j += 32) q += __ldcg(out + j) * __ldcg(out + j);
    q = wsum(q);
    if (threadIdx.x == 0) {
      const double ww = __ldcg(out + k), e = ww - q;
      pyth[0] = e;
      pyth[1] = e > 0.0 ? 1.0 / sqrt(e) : 0.0;
      if (vs_next) *vs_next = pyth[1];
      if (decide) *decide = (e < eta2 * ww) ? 1 : 0;
    }
  }
}

// w -= sum_{j<k} v_j h[j] with v_j = vs[j] V_j (vs null: v_j = V_j), then
// (NORM) out[0] = |w|^2 and out[1] = 1 / |w| (also into *vs_next when given:
// w is kept as the next basis vector before its normalisation).  wf (may be
// null): an FP32 copy of the new w.  With norm0 and decide: *decide = 1 when
// |w_new|^2 < eta2 |w_old|^2, i.e. when the first pass cancelled so much of w
// that a second Gram-Schmidt pass is needed ("twice is enough").  run_if as in
// k_multidot.  Without NORM the kernel only projects (no sum of squares: no
// FP64 multiply-add per element, no reduction).
template <bool NORM>
__global__ void __launch_bounds__(256) k_axpy_norm(long long n, int k, const double* __restrict__ V, long long ld,
                                                   const double* __restrict__ h, double* __restrict__ w,
                                                   double* __restrict__ partial, int stride, double* __restrict__ out,
                                                   unsigned int* counter, const double* norm0, int* decide,
                                                   const int* run_if, double eta2, const double* __restrict__ vs,
                                                   float* __restrict__ wf, double* __restrict__ vs_next) {
  PF_PDL_ENTRY();
  if (run_if && !*run_if) return;
  __shared__ double hs[128];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = vs ? h[j] * vs[j] : h[j];
  __syncthreads();
  double acc[1] = {0.0};
  GRID_STRIDE(i, n) {
    double wi = w[i];
    for (int j = 0; j < k; ++j) wi -= V[(size_t)j * ld + i] * hs[j];
    w[i] = wi;
    if (wf) wf[i] = (float)wi;
    if (NORM) acc[0] += wi * wi;
  }
  if (!NORM) return;
  block_reduce_write<1>(acc, 1, partial + (size_t)blockIdx.x * stride);
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double sum = lane_sum_blocks(partial, stride, (int)gridDim.x, threadIdx.x);
    sum = wsum(sum);
    if (threadIdx.x == 0) {
      out[0] = sum;
      out[1] = sum > 0.0 ? 1.0 / sqrt(sum) : 0.0;
      if (vs_next) *vs_next = out[1];
      if (decide) *decide = (sum < eta2 * norm0[0]) ? 1 : 0;
      *counter = 0u;
    }
  }
}

void launch_multidot(long long n, int k, const double* V, long long ld, const double* w, double* partial, int nblocks,
                     double* out, unsigned int* counter, cudaStream_t st, int self_dot, const int* run_if,
                     const double* vs, double* pyth, double* vs_next, int* decide, double eta2) {
  launch(k_multidot, nblocks, 256, 0, st, n, k, V, ld, w, partial, 72, out, counter, self_dot, run_if, vs, pyth,
         vs_next, decide, eta2);
}

void launch_axpy_norm(long long n, int k, const double* V, long long ld, const double* h, double* w, double* partial,
                      int nblocks, double* out, unsigned int* counter, const double* norm0, int* decide,
                      const int* run_if, cudaStream_t st, double eta2, const double* vs, float* wf,
                      double* vs_next) {
  if (out)
    launch(k_axpy_norm<true>, nblocks, 256, 0, st, n, k, V, ld, h, w, partial, 72, out, counter, norm0, decide, run_if,
           eta2, vs, wf, vs_next);
  else
    launch(k_axpy_norm<false>, nblocks, 256, 0, st, n, k, V, ld, h, w, partial, 72, out, counter, norm0, decide,
           run_if, eta2, vs, wf, vs_next);
}

__global__ void __launch_bounds__(256) k_multi_axpy_add(long long n, int k, const double* __restrict__ Z, long long ld,
                                                        const double* __restrict__ y, double* __restrict__ x) {
  PF_PDL_ENTRY();
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
  launch(k_multi_axpy_add, grid_for(n, 256), 256, 0, st, n, k, Z, ld, y, x);
}

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b), for any a, b
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// x += sum_{j<k} Zf[j] y[j] with the preconditioned vectors held in FP32 (the
// mixed form computes them in FP32, so FP32 storage loses nothing).  The sum
// runs in two-float arithmetic on the FP32 pipe: each y_j is split as
// yh + yl (yh = y_j rounded to FP32, yl the FP32 rounding of the remainder);
// the product z yh is made exact by the FMA-based error of the product
// (p = z yh, e = fma(z, yh, -p)); the running sum (sh, sl) takes p by Knuth's
// TwoSum and is renormalised by a second TwoSum after each term.  That keeps
// about 47 significant bits (the FP64 sum keeps 53) and costs no FP64 unit
// time per term; one conversion pair per element joins the result to x.
// Where a split coefficient leaves the normal FP32 range the kernel sums in
// FP64 instead (conversions per term).  The intrinsics (_rn) keep the compiler
// from fusing the error-free steps into multiply-adds.
__global__ void __launch_bounds__(256) k_multi_axpy_add_f32(long long n, int k, const float* __restrict__ Zf,
                                                            long long ld, const double* __restrict__ y,
                                                            double* __restrict__ x) {
  PF_PDL_ENTRY();
  __shared__ float yh[128], yl[128];
  __shared__ double yd[128];
  __shared__ int wide;
  if (threadIdx.x == 0) wide = 0;
  __syncthreads();
  if (threadIdx.x < k) {
    const double v = y[threadIdx.x];
    const float h = __double2float_rn(v);
    const float l = __double2float_rn(v - (double)h);
    yd[threadIdx.x] = v;
    yh[threadIdx.x] = h;
    yl[threadIdx.x] = l;
    // the split is exact to the two-float precision only with yh and yl in
    // the normal FP32 range (or both zero)
    const float ah = fabsf(h), al = fabsf(l);
    const bool ok = isfinite(h) && (h == 0.0f || (ah >= 1.0e-30f && ah <= 1.0e30f)) &&
                    (l == 0.0f || al >= 1.17549435e-38f);
    if (!ok) atomicOr(&wide, 1);
  }
  __syncthreads();
  if (wide) {
    GRID_STRIDE(i, n) {
      double s = x[i];
      for (int j = 0; j < k; ++j) s += (double)Zf[(size_t)j * ld + i] * yd[j];
      x[i] = s;
    }
    return;
  }
  GRID_STRIDE(i, n) {
    float sh = 0.0f, sl = 0.0f;
    for (int j = 0; j < k; ++j) {
      const float z = Zf[(size_t)j * ld + i];
      const float ph = __fmul_rn(z, yh[j]);
      const float pl = __fmaf_rn(z, yl[j], __fmaf_rn(z, yh[j], -ph));  // z yl + the error of z yh
      float s, e;
      two_sum_f(sh, ph, s, e);
      const float t = __fadd_rn(sl, __fadd_rn(pl, e));
      two_sum_f(s, t, sh, sl);  // renormalise (no ordering of |s| and |t| assumed)
    }
    x[i] = x[i] + ((double)sh + (double)sl);
  }
}

void launch_multi_axpy_add_f32(long long n, int k, const float* Zf, long long ld, const double* y, double* x,
                               cudaStream_t st) {
  launch(k_multi_axpy_add_f32, grid_for(n, 256), 256, 0, st, n, k, Zf, ld, y, x);
}

void launch_dot(long long n, const double* a, const double* b, double* partial, int nblocks, double* out,
                unsigned int* counter, cudaStream_t st) {
  launch(k_multidot, nblocks, 256, 0, st, n, 1, a, 0, b, partial, 72, out, counter, 0, nullptr,
         (const double*)nullptr, (double*)nullptr, (double*)nullptr, (int*)nullptr, 0.0);
}

// explicit instantiations
template void launch_spmv<double>(const Grid&, const Wells&, const double*, const double*, const double*,
                                  const double*, const double*, double*, cudaStream_t, int);
template void launch_spmv<float>(const Grid&, const Wells&, const float*, const float*, const float*, const float*,
                                 const double*, double*, cudaStream_t, int);
template void launch_bjacobi_setup<double, double>(const Grid&, const Wells&, const double*, const double*, double*,
                                                   double*, cudaStream_t);
template void launch_bjacobi_setup<float, float>(const Grid&, const Wells&, const float*, const float*, float*, float*,
                                                 cudaStream_t);
template void launch_ilu_setup<double, double>(const Grid&, const Wells&, const double*, const double*, double*,
                                               double*, double, const IluCompact&, cudaStream_t, double, double);
template void launch_ilu_setup<float, float>(const Grid&, const Wells&, const float*, const float*, float*, float*,
                                             double, const IluCompact&, cudaStream_t, double, double);
template int launch_ilu_apply<double, double, double, double>(const Grid&, int, const double*, const double*,
                                                              const double*, const double*, double*, int,
                                                              const IluCompact&, cudaStream_t);
template int launch_ilu_apply<float, float, float, float>(const Grid&, int, const float*, const float*, const float*,
                                                          const float*, float*, int, const IluCompact&, cudaStream_t);
template int launch_ilu_apply<float, float, double, double>(const Grid&, int, const float*, const float*,
                                                            const float*, const double*, double*, int,
                                                            const IluCompact&, cudaStream_t);
template void launch_stage2_ilu<double, double>(const Grid&, const Wells&, const double*, const IluCompact&,
                                                const double*, const double*, const double*, double, double, double*,
                                                double*, const double*, int, int, cudaStream_t);
template void launch_stage2_ilu<float, float>(const Grid&, const Wells&, const float*, const IluCompact&,
                                              const float*, const float*, const float*, float, float, float*, float*,
                                              const float*, int, int, cudaStream_t);
template void launch_bjacobi_apply<double>(const Grid&, int, const double*, const double*, const double*, double*,
                                           cudaStream_t);
template void launch_bjacobi_apply<float>(const Grid&, int, const float*, const float*, const double*, double*,
                                          cudaStream_t);

}  // namespace pf
