// CPR-FP preconditioner (Alg. 2) with a structured aggregation multigrid for
// the pressure stage.  See pf_cpr.cuh for the decoupling and the hierarchy.
#include <math.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "pf_cpr.cuh"

namespace pf {

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxCoarse = 64;
constexpr long long kTwoSlotCells = 1 << 20;  // levels from this size relax two cells per thread

struct Dims {
  int nx, ny, nz;
  long long n, nxy;
};

Dims dims_of(const CprLevel& L) { return Dims{L.nx, L.ny, L.nz, L.n, (long long)L.nx * L.ny}; }

// 32-bit division: grids hold fewer than 2^31 cells (pf_create checks)
__device__ __forceinline__ void coords(const Dims& d, long long i, int& x, int& y, int& z) {
  const unsigned int ui = (unsigned int)i, nxy = (unsigned int)d.nxy, nx = (unsigned int)d.nx;
  const unsigned int zz = ui / nxy;
  const unsigned int r = ui - zz * nxy;
  const unsigned int yy = r / nx;
  z = (int)zz;
  y = (int)yy;
  x = (int)(r - yy * nx);
}

// neighbour of (x,y,z) in slot s (1..6) if inside the grid
__device__ __forceinline__ bool nbr(const Dims& d, int x, int y, int z, int s, long long& j) {
  switch (s) {
    case SL_XM: if (x == 0) return false; j = x - 1 + d.nx * (y + (long long)d.ny * z); return true;
    case SL_XP: if (x + 1 >= d.nx) return false; j = x + 1 + d.nx * (y + (long long)d.ny * z); return true;
    case SL_YM: if (y == 0) return false; j = x + d.nx * (y - 1 + (long long)d.ny * z); return true;
    case SL_YP: if (y + 1 >= d.ny) return false; j = x + d.nx * (y + 1 + (long long)d.ny * z); return true;
    case SL_ZM: if (z == 0) return false; j = x + d.nx * (y + (long long)d.ny * (z - 1)); return true;
    default: if (z + 1 >= d.nz) return false; j = x + d.nx * (y + (long long)d.ny * (z + 1)); return true;
  }
}

#define GSTRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// A_p from the P columns of the oil and water rows of J, in the hierarchy's
// precision (the FP32 form reads FP32 J: no FP64 unit time)
template <typename T>
__global__ void __launch_bounds__(256) k_extract_pressure(long long n, const T* __restrict__ J, T* __restrict__ A,
                                                          T* __restrict__ dinv, double w_o, double w_w) {
  PF_PDL_ENTRY();
  const T wo = (T)w_o, ww = (T)w_w;
  GSTRIDE(i, n) {
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      const T a = wo * J[((size_t)s * 9 + 0) * n + i] + ww * J[((size_t)s * 9 + 3) * n + i];
      A[(size_t)s * n + i] = a;
      if (s == SL_D) dinv[i] = (T)1 / a;
    }
  }
}

// Eight lanes per coarse cell, one per child (dx, dy, dz) = bits of the lane
// index within its group; groups are warp-aligned and every lane of a warp
// takes part in every round, so the shuffles see full warps.  The child sums
// use a fixed xor tree (deterministic).
// c - a b with one rounding (written out so that the per-level kernels and the
// single-block cycle round identically whatever the compiler contracts)
__device__ __forceinline__ double fnms(double a, double b, double c) { return __fma_rn(-a, b, c); }
__device__ __forceinline__ float fnms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }

__device__ __forceinline__ double grp8_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// Galerkin coarse operator with piecewise-constant aggregation
template <typename T>
__global__ void __launch_bounds__(256) k_galerkin(Dims f, Dims c, const T* __restrict__ Af, T* __restrict__ Ac,
                                                  T* __restrict__ dinv_c) {
  PF_PDL_ENTRY();
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  const long long total = 8 * c.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long t = base + threadIdx.x;
    const long long I = t >> 3;
    const int child = (int)(t & 7);
    const int dx = child & 1, dy = (child >> 1) & 1, dz = child >> 2;
    double acc[SL_COUNT];
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) acc[s] = 0.0;
    if (t < total && dx < fx && dy < fy && dz < fz) {
      int cx, cy, cz;
      coords(c, I, cx, cy, cz);
      const int x = cx * fx + dx, y = cy * fy + dy, z = cz * fz + dz;
      if (x < f.nx && y < f.ny && z < f.nz) {
        const long long i = x + f.nx * (y + (long long)f.ny * z);
        acc[SL_D] = (double)Af[i];
#pragma unroll
        for (int s = 1; s < SL_COUNT; ++s) {
          long long j;
          if (!nbr(f, x, y, z, s, j)) continue;
          const double a = (double)Af[(size_t)s * f.n + i];
          int jx, jy, jz;
          coords(f, j, jx, jy, jz);
          if (jx / fx == cx && jy / fy == cy && jz / fz == cz) acc[SL_D] += a;
          else acc[s] += a;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) acc[s] = grp8_sum(acc[s]);
    if (t < total && child == 0) {
#pragma unroll
      for (int s = 0; s < SL_COUNT; ++s) Ac[(size_t)s * c.n + I] = (T)acc[s];
      dinv_c[I] = (T)(1.0 / acc[SL_D]);
    }
  }
}

// The preconditioner's output, written by the last post-smoothing pass on the
// finest pressure level (saves a pass over the vector): mode 1 (FP64 path)
// z[3i] += x_i on every cell; mode 2 (mixed) z = zf + Pi_p x in FP64 (z may
// be null: the Krylov solver then keeps only the FP32 copy, which holds the
// same values) and its FP32 copy zf_out (may be null), wells included.
struct TopOut {
  int mode = 0;
  int nw = 0;
  double* z = nullptr;
  const float* zf = nullptr;
  float* zf_out = nullptr;
};

template <typename T>
__device__ __forceinline__ void top_write(const TopOut& t, long long i, T xi) {
  if (t.mode == 1) {
    t.z[3 * i] += (double)xi;
  } else {
    const float p = t.zf[3 * i] + (float)xi, sv = t.zf[3 * i + 1], cv = t.zf[3 * i + 2];
    if (t.z) {
      t.z[3 * i] = (double)p;
      t.z[3 * i + 1] = (double)sv;
      t.z[3 * i + 2] = (double)cv;
    }
    if (t.zf_out) { t.zf_out[3 * i] = p; t.zf_out[3 * i + 1] = sv; t.zf_out[3 * i + 2] = cv; }
  }
}

// Slots of one colour: ceil(nx / 2) per (y, z) row.
__device__ __forceinline__ long long rb_slots(const Dims& d) { return (long long)((d.nx + 1) / 2) * d.ny * d.nz; }

// Cell of colour `color` in colour slot q = (y + ny z) ceil(nx / 2) + x / 2
// (false past the row's end when nx is odd).
__device__ __forceinline__ bool slot_cell(const Dims& d, unsigned int hx, int color, long long q, int& cx, int& cy,
                                          int& cz) {
  const unsigned int uq = (unsigned int)q, row = uq / hx, m = uq - row * hx;
  cz = (int)(row / (unsigned int)d.ny);
  cy = (int)(row - (unsigned int)cz * (unsigned int)d.ny);
  cx = (int)((((unsigned int)(cy + cz + color)) & 1u) + 2u * m);
  return cx < d.nx;
}

// One Gauss-Seidel relaxation of cell i at (cx, cy, cz): x_i = (b_i - sum over
// neighbours a_ij x_j) / a_ii with the neighbours in slot order; zero_init:
// x holds no valid values yet (first half-sweep), so neighbours count as zero.
// With xc (the coarse correction of dims c) the neighbours are read as
// x_j + xc[agg(j)], i.e. the prolongation x += P xc is applied on the fly: a
// colour pass overwrites every cell of its colour, so only the other colour's
// values (the neighbours) need the correction; the next pass overwrites those.
// off(sl) gives the coefficient of slot sl (1..6), inv_diag 1 / a_ii.
template <typename T, typename Coef>
__device__ __forceinline__ T relax_cell(const Dims& d, long long i, int cx, int cy, int cz, const T* __restrict__ b,
                                        T* __restrict__ x, int zero_init, const T* __restrict__ xc, const Dims& c,
                                        int fx, int fy, int fz, Coef off, T inv_diag) {
  T s = b[i];
  if (!zero_init) {
#pragma unroll
    for (int sl = 1; sl < SL_COUNT; ++sl) {
      long long j;
      if (!nbr(d, cx, cy, cz, sl, j)) continue;
      T xj = x[j];
      if (xc) {  // the neighbour's coordinates follow from the slot (no division)
        const int jx = cx + (sl == SL_XM ? -1 : sl == SL_XP ? 1 : 0);
        const int jy = cy + (sl == SL_YM ? -1 : sl == SL_YP ? 1 : 0);
        const int jz = cz + (sl == SL_ZM ? -1 : sl == SL_ZP ? 1 : 0);
        xj += xc[jx / fx + c.nx * (jy / fy + (long long)c.ny * (jz / fz))];
      }
      s = fnms(off(sl), xj, s);
    }
  }
  const T xi = s * inv_diag;
  x[i] = xi;
  return xi;
}

// One colour of a red-black Gauss-Seidel sweep on a level in the natural
// layout (A[slot][cell], dinv[cell]).  Without TOP the threads take the
// colour's slots (every lane relaxes a cell).  With TOP (the last pass on the
// finest level, which also writes the preconditioner's output) each thread
// takes a pair of cells along x, one of each colour: it relaxes the one of
// this colour and writes the output of both (the other colour's value is
// final), so no lane of a warp idles on the other colour; threads past the
// pairs write the well rows of the mixed output.
template <typename T, bool TOP, int CPT = 1>
__global__ void __launch_bounds__(256) k_rbgs(Dims d, const T* __restrict__ A, const T* __restrict__ dinv,
                                              const T* __restrict__ b, T* __restrict__ x, int color, int zero_init,
                                              const T* __restrict__ xc, Dims c, TopOut top) {
  PF_PDL_ENTRY();
  const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
  const long long nq = rb_slots(d);
  const unsigned int hx = ((unsigned int)d.nx + 1u) >> 1;
  if (!TOP) {
    // CPT consecutive slots of a row per thread: one coordinate computation
    const unsigned int hp = (hx + CPT - 1u) / CPT;  // slot groups per row
    GSTRIDE(t, (long long)hp * d.ny * d.nz) {
      const unsigned int ut = (unsigned int)t, row = ut / hp, m0 = CPT * (ut - row * hp);
      const int cz = (int)(row / (unsigned int)d.ny), cy = (int)(row - (unsigned int)cz * (unsigned int)d.ny);
      const int par = (int)(((unsigned int)(cy + cz + color)) & 1u);
      const long long base = (long long)d.nx * row;
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        const int cx = par + 2 * (int)(m0 + e);
        if (m0 + e >= hx || cx >= d.nx) break;
        const long long i = base + cx;
        relax_cell<T>(d, i, cx, cy, cz, b, x, zero_init, xc, c, fx, fy, fz,
                      [&](int sl) { return A[(size_t)sl * d.n + i]; }, dinv[i]);
      }
    }
  } else {
    GSTRIDE(p, nq + (top.mode == 2 ? top.nw : 0)) {
      if (p >= nq) {  // well rows of the mixed output: stage-1 values
        const long long wv = 3 * d.n + (p - nq);
        const float v = top.zf[wv];
        if (top.z) top.z[wv] = (double)v;
        if (top.zf_out) top.zf_out[wv] = v;
        continue;
      }
      int cx, cy, cz;
      const bool own = slot_cell(d, hx, color, p, cx, cy, cz);
      const long long i = cx + (long long)d.nx * (cy + (long long)d.ny * cz);
      const int ox = cx ^ 1;  // the pair's cell of the other colour: final value
      if (ox < d.nx) top_write(top, i - cx + ox, x[i - cx + ox]);
      if (own)
        top_write(top, i, relax_cell<T>(d, i, cx, cy, cz, b, x, zero_init, xc, c, fx, fy, fz,
                                        [&](int sl) { return A[(size_t)sl * d.n + i]; }, dinv[i]));
    }
  }
}

// Per-colour copies of the finest level's six off-diagonal stencil slots and
// 1/diag, indexed by the colour slot q = (y + ny z) ceil(nx / 2) + x / 2: a
// colour pass then reads only its own colour's coefficients (in the natural
// layout every line also carries the other colour's).
template <typename T>
__global__ void __launch_bounds__(256) k_rb_compact(Dims d, const T* __restrict__ A, const T* __restrict__ dinv,
                                                    T* __restrict__ c0, T* __restrict__ c1) {
  PF_PDL_ENTRY();
  const long long nq = rb_slots(d);
  const unsigned int hx = ((unsigned int)d.nx + 1u) >> 1;
  GSTRIDE(i, d.n) {
    int cx, cy, cz;
    coords(d, i, cx, cy, cz);
    T* dst = ((cx + cy + cz) & 1) ? c1 : c0;
    const long long q = ((long long)cy + (long long)d.ny * cz) * hx + (cx >> 1);
#pragma unroll
    for (int sl = 1; sl < SL_COUNT; ++sl) dst[(size_t)(sl - 1) * nq + q] = A[(size_t)sl * d.n + i];
    dst[(size_t)6 * nq + q] = dinv[i];
  }
}

// k_rbgs on the finest level reading this colour's copy cp (the same
// arithmetic in the same order); the same thread mappings as k_rbgs.  In the
// TOP pass the pair's cell of this colour has the pair's index as its slot.
template <typename T, bool TOP, int CPT = 1>
__global__ void __launch_bounds__(256) k_rbgs_cp(Dims d, const T* __restrict__ cp, const T* __restrict__ b,
                                                 T* __restrict__ x, int color, int zero_init,
                                                 const T* __restrict__ xc, Dims c, TopOut top) {
  PF_PDL_ENTRY();
  const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
  const long long nq = rb_slots(d);
  const unsigned int hx = ((unsigned int)d.nx + 1u) >> 1;
  if (!TOP) {
    // CPT consecutive slots of a row per thread: one coordinate computation
    const unsigned int hp = (hx + CPT - 1u) / CPT;  // slot groups per row
    GSTRIDE(t, (long long)hp * d.ny * d.nz) {
      const unsigned int ut = (unsigned int)t, row = ut / hp, m0 = CPT * (ut - row * hp);
      const int cz = (int)(row / (unsigned int)d.ny), cy = (int)(row - (unsigned int)cz * (unsigned int)d.ny);
      const int par = (int)(((unsigned int)(cy + cz + color)) & 1u);
      const long long base = (long long)d.nx * row;
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        const int cx = par + 2 * (int)(m0 + e);
        if (m0 + e >= hx || cx >= d.nx) break;
        const long long i = base + cx, q = (long long)row * hx + m0 + e;
        relax_cell<T>(d, i, cx, cy, cz, b, x, zero_init, xc, c, fx, fy, fz,
                      [&](int sl) { return cp[(size_t)(sl - 1) * nq + q]; }, cp[(size_t)6 * nq + q]);
      }
    }
  } else {
    GSTRIDE(p, nq + (top.mode == 2 ? top.nw : 0)) {
      if (p >= nq) {  // well rows of the mixed output: stage-1 values
        const long long wv = 3 * d.n + (p - nq);
        const float v = top.zf[wv];
        if (top.z) top.z[wv] = (double)v;
        if (top.zf_out) top.zf_out[wv] = v;
        continue;
      }
      int cx, cy, cz;
      const bool own = slot_cell(d, hx, color, p, cx, cy, cz);
      const long long i = cx + (long long)d.nx * (cy + (long long)d.ny * cz);
      const int ox = cx ^ 1;  // the pair's cell of the other colour: final value
      if (ox < d.nx) top_write(top, i - cx + ox, x[i - cx + ox]);
      if (own)
        top_write(top, i, relax_cell<T>(d, i, cx, cy, cz, b, x, zero_init, xc, c, fx, fy, fz,
                                        [&](int sl) { return cp[(size_t)(sl - 1) * nq + p]; },
                                        cp[(size_t)6 * nq + p]));
    }
  }
}

// Residual b - A x of child `child` (bits dx, dy, dz) of coarse cell (cx, cy,
// cz), in FP64; 0 for a child outside the aggregate or the grid, and with
// red_only for a black child.  After a pre-smoothing whose last pass is black,
// the black residuals are zero up to rounding (that pass solved the black rows
// for the red values it read), so only the red children carry the coarse
// right-hand side.
template <typename T>
__device__ __forceinline__ double child_residual(const Dims& f, const T* __restrict__ A, const T* __restrict__ b,
                                                 const T* __restrict__ x, int cx, int cy, int cz, int fx, int fy,
                                                 int fz, int child, bool red_only) {
  const int dx = child & 1, dy = (child >> 1) & 1, dz = child >> 2;
  if (dx >= fx || dy >= fy || dz >= fz) return 0.0;
  const int X = cx * fx + dx, Y = cy * fy + dy, Z = cz * fz + dz;
  if (X >= f.nx || Y >= f.ny || Z >= f.nz) return 0.0;
  if (red_only && ((X + Y + Z) & 1)) return 0.0;
  const long long i = X + f.nx * (Y + (long long)f.ny * Z);
  T ri = fnms(A[i], x[i], b[i]);
#pragma unroll
  for (int sl = 1; sl < SL_COUNT; ++sl) {
    long long j;
    if (nbr(f, X, Y, Z, sl, j)) ri = fnms(A[(size_t)sl * f.n + i], x[j], ri);
  }
  return (double)ri;
}

// coarse right-hand side: sum over each aggregate of the fine residual b - A x
// (RED: the red children only, see child_residual; four lanes per coarse
// cell, lane q taking children q and q + 4, of which at most one is red in a
// full aggregate; otherwise eight lanes, one per child).  The lanes' values
// are summed by a fixed xor tree, which the single-block cycle reproduces.
// With xc (the coarse level's iterate) the first red pass of the coarse
// level's cycle from a zero initial guess is done here too: a red coarse cell
// gets xc = bc / a_cc (bc as stored, times the stored 1 / diagonal: the value
// that pass would compute), so the coarse cycle starts with its black pass.
template <typename T, bool RED>
__global__ void __launch_bounds__(256) k_residual_restrict(Dims f, Dims c, const T* __restrict__ A,
                                                           const T* __restrict__ b, const T* __restrict__ x,
                                                           T* __restrict__ bc, T* __restrict__ xc,
                                                           const T* __restrict__ dinv_c) {
  PF_PDL_ENTRY();
  constexpr int kLanes = RED ? 4 : 8;
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  const long long total = kLanes * c.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long t = base + threadIdx.x;
    const long long I = t / kLanes;
    const int lane = (int)(t % kLanes);
    double r = 0.0;
    if (t < total) {
      int cx, cy, cz;
      coords(c, I, cx, cy, cz);
      if (RED)
        r = child_residual<T>(f, A, b, x, cx, cy, cz, fx, fy, fz, lane, true) +
            child_residual<T>(f, A, b, x, cx, cy, cz, fx, fy, fz, lane + 4, true);
      else
        r = child_residual<T>(f, A, b, x, cx, cy, cz, fx, fy, fz, lane, false);
    }
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    if (!RED) r += __shfl_xor_sync(0xffffffffu, r, 4);
    if (t < total && lane == 0) {
      const T bI = (T)r;
      bc[I] = bI;
      if (xc) {
        int cx, cy, cz;
        coords(c, I, cx, cy, cz);
        if (((cx + cy + cz) & 1) == 0) xc[I] = bI * dinv_c[I];
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(Dims f, Dims c, const T* __restrict__ xc, T* __restrict__ x) {
  PF_PDL_ENTRY();
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  GSTRIDE(i, f.n) {
    int X, Y, Z;
    coords(f, i, X, Y, Z);
    x[i] += xc[X / fx + c.nx * (Y / fy + (long long)c.ny * (Z / fz))];
  }
}

// Dense inverse of the coarsest stencil matrix (n <= 64) by Gauss-Jordan
// elimination in place with partial pivoting (row swaps, undone as column
// swaps of the inverse at the end), in shared memory by one block of 1024
// threads: each step's n x n update is spread over the whole block, so the
// SM's FP64 lanes stay full (one thread per row would leave them nearly all
// idle, and FP64 on one SM is slow on this part).  Step k with pivot p:
// row k is divided by p, every other row i takes row i - a_ik (row k), and
// column k becomes a_kk = 1/p, a_ik = -a_ik / p.  A zero pivot sets *status
// and skips its step.  Row-major storage: M[r * kLd + c].
constexpr int kLd = kMaxCoarse + 1;
constexpr size_t kCoarseSmem = sizeof(double) * (kMaxCoarse * kLd + kMaxCoarse + 1) + sizeof(int) * (kMaxCoarse + 1);

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_factor(Dims d, const T* __restrict__ A, T* __restrict__ inv,
                                                         int* status) {
  PF_PDL_ENTRY();
  extern __shared__ double sm[];
  double* M = sm;                                              // [n][kLd]
  double* fk = sm + kMaxCoarse * kLd;                          // column k before the step, then 1 / pivot
  int* swp = reinterpret_cast<int*>(fk + kMaxCoarse + 1);      // pivot row of each step
  int* pivok = swp + kMaxCoarse;                               // this step's pivot is non-zero
  const int n = (int)d.n;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < kMaxCoarse * kLd; e += nt) M[e] = 0.0;
  if (t == 0) *status = 0;
  __syncthreads();
  if (t < n) {
    int x, y, z;
    coords(d, t, x, y, z);
    M[t * kLd + t] = (double)A[t];
    for (int s = 1; s < SL_COUNT; ++s) {
      long long j;
      if (nbr(d, x, y, z, s, j)) M[t * kLd + (int)j] = (double)A[(size_t)s * n + t];
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < 32) {  // pivot search by one warp: largest |a_rk|, r >= k (ties: the lower row)
      int p = k;
      double best = -1.0;
      for (int r = k + t; r < n; r += 32) {
        const double v = fabs(M[r * kLd + k]);
        if (v > best) { best = v; p = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (t == 0) {
        swp[k] = p;
        *pivok = best > 0.0 ? 1 : 0;
        if (!(best > 0.0)) *status = 1;
      }
    }
    __syncthreads();
    const int p = swp[k];
    if (p != k) {
      for (int c = t; c < n; c += nt) {
        const double tmp = M[k * kLd + c];
        M[k * kLd + c] = M[p * kLd + c];
        M[p * kLd + c] = tmp;
      }
    }
    __syncthreads();
    if (!*pivok) continue;  // uniform over the block
    // one FP64 division per step (by one thread: FP64 on one SM is scarce)
    if (t == 0) fk[kMaxCoarse] = 1.0 / M[k * kLd + k];
    for (int i = t; i < n; i += nt) fk[i] = M[i * kLd + k];
    __syncthreads();
    const double rp = fk[kMaxCoarse];
    for (int c = t; c < n; c += nt) M[k * kLd + c] = c == k ? rp : M[k * kLd + c] * rp;
    __syncthreads();
    for (int e = t; e < n * n; e += nt) {
      const int i = e / n, c = e - i * n;
      if (i == k) continue;
      M[i * kLd + c] = c == k ? -fk[i] * rp : fnms(fk[i], M[k * kLd + c], M[i * kLd + c]);
    }
    __syncthreads();
  }
  // (P A)^{-1} = A^{-1} P^T: undo the row swaps as column swaps, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = swp[k];
    if (p != k) {
      for (int r = t; r < n; r += nt) {
        const double tmp = M[r * kLd + k];
        M[r * kLd + k] = M[r * kLd + p];
        M[r * kLd + p] = tmp;
      }
    }
    __syncthreads();
  }
  for (int e = t; e < n * n; e += nt) {
    const int r = e / n, c = e - r * n;
    inv[e] = (T)M[r * kLd + c];
  }
}

// All levels from l0 down run inside one thread block (levels small enough
// that launch latency, not work, would dominate): the same smoother,
// restriction, prolongation and coarse inverse as the per-level kernels.
constexpr int kMaxLev = 24;
// The size up to which a level (and every coarser one) runs in the single
// block is CprData::block_cells: FP64 runs at a small fraction of the FP32
// rate per SM, so its default is lower; the launch-shape tuner may raise it.

template <typename T>
struct BlockLevels {
  int l0, nlev, pre, post, gamma;
  int pre0, post0;  // sweeps on the finest level (pre, post: on the coarser ones)
  Dims d[kMaxLev];
  T* A[kMaxLev];
  T* dinv[kMaxLev];
  T* x[kMaxLev];
  T* b[kMaxLev];
  const T* inv;
};

// The threads that run the small levels together: one block, or every block
// of a thread-block cluster (up to 16 SMs) with the cluster barrier between
// phases (its release/acquire ordering makes one block's writes to the level
// arrays visible to the others).
template <bool CL>
struct Team {
  int tid, stride;
  __device__ Team() {
    if (CL) {
      cg::cluster_group c = cg::this_cluster();
      tid = (int)(c.block_rank() * blockDim.x + threadIdx.x);
      stride = (int)(c.num_blocks() * blockDim.x);
    } else {
      tid = threadIdx.x;
      stride = blockDim.x;
    }
  }
  __device__ void sync() const {
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
  }
};

template <typename T, bool CL>
__device__ void b_rbgs(const Team<CL>& tm, const Dims& d, const T* A, const T* dinv, const T* b, T* x, int color,
                       bool zero_init) {
  // the threads take the colour's slots, as in k_rbgs
  const long long nq = rb_slots(d);
  const unsigned int hx = ((unsigned int)d.nx + 1u) >> 1;
  for (long long q = tm.tid; q < nq; q += tm.stride) {
    int cx, cy, cz;
    if (!slot_cell(d, hx, color, q, cx, cy, cz)) continue;
    const long long i = cx + (long long)d.nx * (cy + (long long)d.ny * cz);
    T s = b[i];
    if (!zero_init) {
      for (int sl = 1; sl < SL_COUNT; ++sl) {
        long long j;
        if (nbr(d, cx, cy, cz, sl, j)) s = fnms(A[(size_t)sl * d.n + i], x[j], s);
      }
    }
    x[i] = s * dinv[i];
  }
  tm.sync();
}

// The cycle below the block levels, written as a loop over an explicit level
// pointer (no device recursion, no per-thread copy of the descriptors: they
// live in shared memory).  cnt[l] counts the coarse cycles finished at level
// l in the current visit; level l runs gamma_l of them (1 at the finest
// level, L.gamma below), the first from a zero initial guess.
template <typename T, bool CL>
__global__ void __launch_bounds__(1024) k_block_cycle(BlockLevels<T> Lp, int zero_init) {
  PF_PDL_ENTRY();
  __shared__ BlockLevels<T> L;
  __shared__ int cnt[kMaxLev];
  __shared__ int zi[kMaxLev];
  const Team<CL> tm;
  if (threadIdx.x == 0) {  // every block keeps its own copy of the (identical) control state
    L = Lp;
    zi[L.l0] = zero_init;
  }
  tm.sync();
  const int last = L.nlev - 1;
  int l = L.l0;
  bool down = true;
  for (int guard = 0; guard < (1 << 20); ++guard) {
    if (down) {
      const Dims d = L.d[l];
      if (l == last) {  // coarsest: dense inverse
        const int n = (int)d.n;
        for (int r = tm.tid; r < n; r += tm.stride) {
          double sacc = 0.0;
          for (int c = 0; c < n; ++c) sacc += (double)L.inv[(size_t)r * n + c] * (double)L.b[l][c];
          L.x[l][r] = (T)sacc;
        }
        tm.sync();
        if (l == L.l0) return;
        --l;
        down = false;
        continue;
      }
      const int npre = l == 0 ? L.pre0 : L.pre;
      for (int sweep = 0; sweep < npre; ++sweep) {
        b_rbgs<T, CL>(tm, d, L.A[l], L.dinv[l], L.b[l], L.x[l], 0, zi[l] && sweep == 0);
        b_rbgs<T, CL>(tm, d, L.A[l], L.dinv[l], L.b[l], L.x[l], 1, false);
      }
      if (npre == 0 && zi[l]) {  // no pre-smoothing: the iterate is the zero initial guess
        for (long long i = tm.tid; i < d.n; i += tm.stride) L.x[l][i] = (T)0;
        tm.sync();
      }
      const Dims c = L.d[l + 1];
      const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
      const T* A = L.A[l];
      const T* x = L.x[l];
      const T* b = L.b[l];
      for (long long I = tm.tid; I < c.n; I += tm.stride) {
        int cx, cy, cz;
        coords(c, I, cx, cy, cz);
        // the children's residuals in FP64, summed in the order of the
        // per-level kernel's lanes and xor tree: with pre-smoothing (its last
        // pass black) the red children, lane q holding children q and q + 4,
        // ((v0 + v1) + (v2 + v3)); without, ((0+1)+(2+3))+((4+5)+(6+7))
        auto child_res = [&](int child, bool red) -> double {
          return child_residual<T>(d, A, b, x, cx, cy, cz, fx, fy, fz, child, red);
        };
        double v;
        if (npre > 0) {
          const double v0 = child_res(0, true) + child_res(4, true), v1 = child_res(1, true) + child_res(5, true);
          const double v2 = child_res(2, true) + child_res(6, true), v3 = child_res(3, true) + child_res(7, true);
          v = (v0 + v1) + (v2 + v3);
        } else {
          double lo = child_res(0, false) + child_res(1, false);
          lo = lo + (child_res(2, false) + child_res(3, false));
          double hi = child_res(4, false) + child_res(5, false);
          hi = hi + (child_res(6, false) + child_res(7, false));
          v = lo + hi;
        }
        L.b[l + 1][I] = (T)v;
      }
      if (threadIdx.x == 0) {
        cnt[l] = 0;
        zi[l + 1] = 1;
      }
      tm.sync();
      ++l;
      continue;
    }
    // back at level l from a finished cycle on level l + 1
    const int gamma_l = (l == 0) ? 1 : L.gamma;
    __syncthreads();
    if (threadIdx.x == 0) cnt[l] += 1;
    __syncthreads();
    if (cnt[l] < gamma_l) {  // another coarse cycle from the current coarse iterate
      if (threadIdx.x == 0) zi[l + 1] = 0;
      __syncthreads();
      // the coarse right-hand side is unchanged: re-enter level l + 1 directly
      ++l;
      down = true;
      continue;
    }
    const Dims d = L.d[l];
    const Dims c = L.d[l + 1];
    const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
    for (long long i = tm.tid; i < d.n; i += tm.stride) {
      int X, Y, Z;
      coords(d, i, X, Y, Z);
      L.x[l][i] += L.x[l + 1][X / fx + c.nx * (Y / fy + (long long)c.ny * (Z / fz))];
    }
    tm.sync();
    const int npost = l == 0 ? L.post0 : L.post;
    for (int sweep = 0; sweep < npost; ++sweep) {
      b_rbgs<T, CL>(tm, d, L.A[l], L.dinv[l], L.b[l], L.x[l], 1, false);
      b_rbgs<T, CL>(tm, d, L.A[l], L.dinv[l], L.b[l], L.x[l], 0, false);
    }
    if (l == L.l0) return;
    --l;
  }
}

template <typename T>
__global__ void k_coarse_apply(int n, const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  PF_PDL_ENTRY();
  const int r = threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int c = 0; c < n; ++c) s += (double)inv[(size_t)r * n + c] * (double)b[c];
  x[r] = (T)s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_top(long long n, const T* __restrict__ x0, double* __restrict__ y) {
  PF_PDL_ENTRY();
  GSTRIDE(i, n) y[3 * i] += (double)x0[i];
}

size_t aup(size_t v) { return (v + 255) / 256 * 256; }

// Whether the cycle on level l starts (from a zero initial guess) with a
// per-level red pass that the producer of its right-hand side can do instead:
// the level runs per-level kernels (not the coarsest direct solve, the single
// block or the cluster) and pre-smooths.
bool folds_first_red(const CprData& c, int l) {
  const CprLevel& L = c.lev[l];
  if (l == c.nlev - 1 || L.n <= c.block_cells || L.n <= c.cluster_cells) return false;
  return (l == 0 ? c.pre : c.cpre) >= 1;
}

// One cycle on level l (and below).  With top.mode set (only at l = 0), the
// last post-smoothing pass also writes the preconditioner's output; returns
// whether it did (not when the level runs in the single block or has no
// post-smoothing).
template <typename T>
// first_red_done: the producer of this level's right-hand side also did the
// first (zero initial guess) red pass (only for a level with per-level passes
// and pre-smoothing; see folds_first_red).
bool cycle(CprData& c, int l, bool zero_init, cudaStream_t st, int& k, const TopOut& top = TopOut{},
           bool first_red_done = false) {
  CprLevel& L = c.lev[l];
  const Dims d = dims_of(L);
  const int gb = grid_for(L.n, 256);
  T* x = (T*)L.x;
  const T* A = (const T*)L.A;
  const T* dinv = (const T*)L.dinv;
  const T* b = (const T*)L.b;
  if (l == c.nlev - 1) {
    launch(k_coarse_apply<T>, 1, kMaxCoarse, 0, st, (int)L.n, (const T*)c.coarse_inv, b, x);
    k += 1;
    return false;
  }
  if (L.n <= c.block_cells || L.n <= c.cluster_cells) {  // this level and all coarser ones in one block or cluster
    BlockLevels<T> B;
    B.l0 = l; B.nlev = c.nlev; B.gamma = c.cycle_gamma;
    B.pre0 = c.pre; B.post0 = c.post; B.pre = c.cpre; B.post = c.cpost;
    for (int q = 0; q < c.nlev; ++q) {
      B.d[q] = dims_of(c.lev[q]);
      B.A[q] = (T*)c.lev[q].A; B.dinv[q] = (T*)c.lev[q].dinv; B.x[q] = (T*)c.lev[q].x; B.b[q] = (T*)c.lev[q].b;
    }
    B.inv = (const T*)c.coarse_inv;
    if (L.n <= c.block_cells) {
      launch(k_block_cycle<T, false>, 1, 1024, 0, st, B, zero_init ? 1 : 0);
    } else {
      unsigned int cs = 2;  // a power of two, about one cell per thread, at most 16 blocks
      while (cs < 16 && (long long)cs * 1024 < L.n) cs *= 2;
      launch_cluster(k_block_cycle<T, true>, cs, 1024, st, B, zero_init ? 1 : 0);
    }
    k += 1;
    return false;
  }
  const int npre = l == 0 ? c.pre : c.cpre, npost = l == 0 ? c.post : c.cpost;
  const int bs = l == 0 ? c.block_rbgs0 : 256;
  const TopOut none;
  // one colour pass; on the finest level with per-colour copies the threads
  // take that colour's slots only (or every cell, for the output-writing pass)
  const bool cp = l == 0 && c.rb_cp[0] != nullptr;
  const long long nq = ((long long)(L.nx + 1) / 2) * L.ny * L.nz;
  auto pass = [&](int color, int zi, const T* xc, const Dims& dxc, const TopOut& to) {
    const bool wtop = to.mode != 0;
    // the plain passes take one colour slot per thread, or from 1M cells two
    // consecutive slots of a row (fewer coordinate computations; at smaller
    // sizes the extra threads' parallelism counts for more: measured); the
    // output-writing pass the colour slots (cell pairs), then the well rows
    const bool two = L.n >= kTwoSlotCells;
    const long long np = two ? (long long)((((L.nx + 1) / 2) + 1) / 2) * L.ny * L.nz : nq;
    const long long nt = wtop ? nq + (to.mode == 2 ? to.nw : 0) : np;
    const int grid = grid_for(nt, bs);
    if (cp) {
      const T* cc = (const T*)c.rb_cp[color];
      if (wtop) launch(k_rbgs_cp<T, true>, grid, bs, 0, st, d, cc, b, x, color, zi, xc, dxc, to);
      else if (two) launch(k_rbgs_cp<T, false, 2>, grid, bs, 0, st, d, cc, b, x, color, zi, xc, dxc, to);
      else launch(k_rbgs_cp<T, false, 1>, grid, bs, 0, st, d, cc, b, x, color, zi, xc, dxc, to);
    } else {
      if (wtop) launch(k_rbgs<T, true>, grid, bs, 0, st, d, A, dinv, b, x, color, zi, xc, dxc, to);
      else if (two) launch(k_rbgs<T, false, 2>, grid, bs, 0, st, d, A, dinv, b, x, color, zi, xc, dxc, to);
      else launch(k_rbgs<T, false, 1>, grid, bs, 0, st, d, A, dinv, b, x, color, zi, xc, dxc, to);
    }
  };
  for (int sweep = 0; sweep < npre; ++sweep) {
    if (!(sweep == 0 && zero_init && first_red_done)) {
      pass(0, (zero_init && sweep == 0) ? 1 : 0, (const T*)nullptr, Dims{}, none);
      k += 1;
    }
    pass(1, 0, (const T*)nullptr, Dims{}, none);
    k += 1;
  }
  if (npre == 0 && zero_init) cudaMemsetAsync(x, 0, (size_t)L.n * sizeof(T), st);  // the zero initial guess
  CprLevel& C = c.lev[l + 1];
  const Dims dc = dims_of(C);
  const bool fold = folds_first_red(c, l + 1);
  // after pre-smoothing (its last pass black) only the red residuals count
  if (npre > 0)
    launch(k_residual_restrict<T, true>, grid_for(4 * C.n, 256), 256, 0, st, d, dc, A, b, x, (T*)C.b,
           fold ? (T*)C.x : (T*)nullptr, (const T*)C.dinv);
  else
    launch(k_residual_restrict<T, false>, grid_for(8 * C.n, 256), 256, 0, st, d, dc, A, b, x, (T*)C.b,
           fold ? (T*)C.x : (T*)nullptr, (const T*)C.dinv);
  k += 1;
  for (int g = 0; g < (l == 0 ? 1 : c.cycle_gamma); ++g) cycle<T>(c, l + 1, g == 0, st, k, TopOut{}, g == 0 && fold);
  if (npost == 0) {
    launch(k_prolong_add<T>, gb, 256, 0, st, d, dc, (const T*)C.x, x);
    k += 1;
    return false;
  }
  for (int sweep = 0; sweep < npost; ++sweep) {
    // the first black pass applies the prolongation to the red neighbours it reads
    pass(1, 0, sweep == 0 ? (const T*)C.x : (const T*)nullptr, sweep == 0 ? dc : Dims{}, none);
    const bool last = sweep + 1 == npost && top.mode != 0;
    pass(0, 0, (const T*)nullptr, Dims{}, last ? top : none);
    k += 2;
  }
  return top.mode != 0;
}

template <typename T>
void setup_t(CprData& c, const void* J, cudaStream_t st, int& k) {
  CprLevel& L0 = c.lev[0];
  launch(k_extract_pressure<T>, grid_for(L0.n, 256), 256, 0, st, L0.n, (const T*)J, (T*)L0.A, (T*)L0.dinv, c.w_o, c.w_w);
  k += 1;
  if (c.rb_cp[0]) {
    launch(k_rb_compact<T>, grid_for(L0.n, 256), 256, 0, st, dims_of(L0), (const T*)L0.A, (const T*)L0.dinv,
           (T*)c.rb_cp[0], (T*)c.rb_cp[1]);
    k += 1;
  }
  for (int l = 0; l + 1 < c.nlev; ++l) {
    CprLevel& F = c.lev[l];
    CprLevel& C = c.lev[l + 1];
    launch(k_galerkin<T>, grid_for(8 * C.n, 256), 256, 0, st, dims_of(F), dims_of(C), (const T*)F.A, (T*)C.A,
                                                          (T*)C.dinv);
    k += 1;
  }
  CprLevel& Lc = c.lev[c.nlev - 1];
  cudaFuncSetAttribute(k_coarse_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmem);
  launch(k_coarse_factor<T>, 1, 1024, kCoarseSmem, st, dims_of(Lc), (const T*)Lc.A, (T*)c.coarse_inv,
                                                         c.coarse_status);
  k += 1;
}

// ----- FP32 CPR apply (mixed precision): every stage in FP32 -----

// stage 1 in FP32: zf = D^{-1} (float) v, cells and wells
__global__ void __launch_bounds__(256) k_stage1_f32(long long n, int nw, const float* __restrict__ Dinv,
                                                    const float* __restrict__ Dwinv, const float* __restrict__ v,
                                                    float* __restrict__ zf) {
  PF_PDL_ENTRY();
  GSTRIDE(i, n + nw) {
    if (i >= n) { zf[3 * n + (i - n)] = Dwinv[i - n] * v[3 * n + (i - n)]; continue; }
    const float r0 = v[3 * i], r1 = v[3 * i + 1], r2 = v[3 * i + 2];
    const float* D = Dinv + i;
    zf[3 * i] = D[0] * r0 + D[n] * r1 + D[2 * n] * r2;
    zf[3 * i + 1] = D[3 * n] * r0 + D[4 * n] * r1 + D[5 * n] * r2;
    zf[3 * i + 2] = D[6 * n] * r0 + D[7 * n] * r1 + D[8 * n] * r2;
  }
}

// stage 2, restricted on the fly: b0 = w_o (v - J y)_oil + w_w (v - J y)_water in
// the preconditioner's precision T (only the oil and water rows of J are read;
// a perforated cell also takes its well column B y_w)
template <typename T, typename VT>
__global__ void __launch_bounds__(256, 4) k_stage2(Grid g, Wells w, const T* __restrict__ J,
                                                const T* __restrict__ Bw, const T* __restrict__ y,
                                                const VT* __restrict__ v, T w_o, T w_w, T* __restrict__ b0,
                                                T* __restrict__ x0, const T* __restrict__ d0, int d0_slot) {
  PF_PDL_ENTRY();
  const long long n = g.n;
  GSTRIDE(i, n) {
    const unsigned int ui = (unsigned int)i, nxy = (unsigned int)g.nxy, nxu = (unsigned int)g.nx;
    const long long k = ui / nxy;
    const unsigned int rem = ui - (unsigned int)k * nxy;
    const long long j = rem / nxu;
    const long long ii = rem - (unsigned int)j * nxu;
    T t0 = 0, t1 = 0;
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
      const T* B = J + (size_t)s * 9 * n + i;
      const T x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
      t0 = fma2(B[0], B[n], x0, x1, t0);  // oil row: no polymer column
      t1 = fma3(B[3 * n], B[4 * n], B[5 * n], x0, x1, x2, t1);
    }
    T r = w_o * ((T)v[3 * i] - t0) + w_w * ((T)v[3 * i + 1] - t1);
    if (w.nw > 0) {
      const int m = w.perf_of[i];
      if (m >= 0) r -= (w_o * Bw[m] + w_w * Bw[w.npf + m]) * y[3 * n + w.pwell[m]];
    }
    b0[i] = r;
    // the multigrid's first red pass from a zero guess (as in k_stage2_ilu)
    if (x0 && ((ii + j + k) & 1) == 0) {
      const long long q = (j + (long long)g.ny * k) * ((g.nx + 1) / 2) + ii / 2;
      x0[i] = r * d0[d0_slot ? q : i];
    }
  }
}

// z = zf + Pi_p x0, written as FP64 for the Krylov basis (z may be null) and
// as an FP32 copy for the mixed-precision operator (the two hold the same float
// values)
__global__ void __launch_bounds__(256) k_out_f32(long long n, int nw, const float* __restrict__ zf,
                                                 const float* __restrict__ x0, double* __restrict__ z,
                                                 float* __restrict__ zf_out) {
  PF_PDL_ENTRY();
  GSTRIDE(i, n + nw) {
    if (i >= n) {
      const float v = zf[3 * n + (i - n)];
      if (z) z[3 * n + (i - n)] = (double)v;
      if (zf_out) zf_out[3 * n + (i - n)] = v;
      continue;
    }
    const float p = zf[3 * i] + x0[i], sv = zf[3 * i + 1], cv = zf[3 * i + 2];
    if (z) {
      z[3 * i] = (double)p;
      z[3 * i + 1] = (double)sv;
      z[3 * i + 2] = (double)cv;
    }
    if (zf_out) { zf_out[3 * i] = p; zf_out[3 * i + 1] = sv; zf_out[3 * i + 2] = cv; }
  }
}

// stage 2 in the form that matches stage 1: after the ILU(0) solve only the
// black rows need the product (k_stage2_ilu), after block-Jacobi every row
// fold: also the multigrid's first red pass from a zero guess on the finest
// level (folds_first_red(c, 0)), reading 1 / diagonal from the red per-colour
// copy when the smoother uses one
template <typename T, typename VT>
void launch_stage2(const CprData& c, const Grid& g, const Wells& w, const void* J, const void* Bw, const T* y,
                   const VT* v, int block, cudaStream_t st, bool fold = false) {
  const CprLevel& L0 = c.lev[0];
  T* b0 = (T*)L0.b;
  T* x0 = fold ? (T*)L0.x : nullptr;
  const long long nq = ((long long)(L0.nx + 1) / 2) * L0.ny * L0.nz;
  const bool slot = c.rb_cp[0] != nullptr;
  const T* d0 = slot ? (const T*)c.rb_cp[0] + 6 * nq : (const T*)L0.dinv;
  if (c.ilu)
    launch_stage2_ilu<T, VT>(g, w, (const T*)J, c.ilu_cp, (const T*)Bw, y, v, (T)c.w_o, (T)c.w_w, b0, x0, d0,
                             slot ? 1 : 0, block, st);
  else
    launch(k_stage2<T, VT>, grid_for(g.n, block), block, 0, st, g, w, (const T*)J, (const T*)Bw, y, v, (T)c.w_o,
           (T)c.w_w, b0, x0, d0, slot ? 1 : 0);
}

template <typename T>
void apply_t(CprData& c, const Grid& g, const Wells& w, const void* J, const void* Bw, const void* Dinv,
             const void* Dwinv, const double* v, double* z, cudaStream_t st, int& k) {
  // stage 1: y = D^{-1} f, or the red-black block ILU(0) solve (cells; wells by their diagonal)
  if (c.ilu) {
    k += launch_ilu_apply<T, T, double, double>(g, w.nw, (const T*)J, (const T*)Dinv, (const T*)Dwinv, v, z,
                                                c.ilu_fused, c.ilu_cp, st);
  } else {
    launch_bjacobi_apply<T>(g, w.nw, (const T*)Dinv, (const T*)Dwinv, v, z, st);
    k += 1;
  }
  // stage 2: r = f - J y restricted to the pressure equation (oil and water rows only)
  CprLevel& L0 = c.lev[0];
  const bool fold = folds_first_red(c, 0);
  launch_stage2<T, double>(c, g, w, J, Bw, (const T*)z, v, c.block_stage2, st, fold);
  k += 1;
  // stage 3: pressure multigrid cycle, then y += Pi_p x (in the cycle's last pass when it can)
  TopOut top;
  top.mode = 1;
  top.z = z;
  if (!cycle<T>(c, 0, true, st, k, top, fold)) {
    launch(k_prolong_top<T>, grid_for(g.n, 256), 256, 0, st, g.n, (const T*)L0.x, z);
    k += 1;
  }
}

}  // namespace

void cpr_time_stage2(CprData& c, const Grid& g, const Wells& w, bool mixed, const void* J, const void* Bw,
                     const double* v, double* tmp, int block, cudaStream_t st) {
  // the mixed form reads the FP32 copy of its input; any float values serve for timing
  if (mixed)
    launch_stage2<float, float>(c, g, w, J, Bw, reinterpret_cast<const float*>(tmp), reinterpret_cast<const float*>(v),
                                block, st);
  else launch_stage2<double, double>(c, g, w, J, Bw, (const double*)tmp, v, block, st);
}

void cpr_carve(CprData& c, const Grid& g, bool mixed, size_t& off, char* base) {
  const size_t ts = mixed ? sizeof(float) : sizeof(double);
  const int limit = std::min(std::max(c.coarse_limit, 1), kMaxCoarse);
  c.lev.clear();
  CprLevel L;
  L.nx = g.nx; L.ny = g.ny; L.nz = g.nz; L.n = g.n;
  c.lev.push_back(L);
  while (c.lev.back().n > limit && (int)c.lev.size() < kMaxLev) {
    const CprLevel& F = c.lev.back();
    CprLevel C;
    C.nx = F.nx > 1 ? (F.nx + 1) / 2 : 1;
    C.ny = F.ny > 1 ? (F.ny + 1) / 2 : 1;
    C.nz = F.nz > 1 ? (F.nz + 1) / 2 : 1;
    C.n = (long long)C.nx * C.ny * C.nz;
    c.lev.push_back(C);
  }
  c.nlev = (int)c.lev.size();
  auto take = [&](size_t bytes) -> void* {
    off = aup(off);
    void* p = base ? (void*)(base + off) : nullptr;
    off += bytes;
    return p;
  };
  for (auto& lv : c.lev) {
    lv.A = take((size_t)SL_COUNT * lv.n * ts);
    lv.dinv = take((size_t)lv.n * ts);
    lv.x = take((size_t)lv.n * ts);
    lv.b = take((size_t)lv.n * ts);
  }
  c.coarse_inv = take((size_t)kMaxCoarse * kMaxCoarse * ts);
  c.coarse_status = (int*)take(sizeof(int));
  const size_t nq = (size_t)((g.nx + 1) / 2) * g.ny * g.nz;
  for (int q = 0; q < 2; ++q) c.rb_cp[q] = c.rb_copy ? take(7 * nq * ts) : nullptr;
}

pf_status cpr_init(CprData& c, const Grid&, bool mixed, const pf_solver_opts& o, cudaStream_t) {
  c.block_cells = mixed ? 4096 : 512;
  c.pre = std::max(0, o.amg_pre_sweeps);
  c.post = std::max(0, o.amg_post_sweeps);
  c.cpre = o.amg_coarse_sweeps >= 0 ? o.amg_coarse_sweeps : c.pre;
  c.cpost = o.amg_coarse_sweeps >= 0 ? o.amg_coarse_sweeps : c.post;
  c.cycle_gamma = o.amg_cycle == 2 ? 2 : 1;
  if (c.lev.empty() || c.lev.back().n > kMaxCoarse) return PF_EINVAL;
  c.ready = true;
  return PF_OK;
}

void cpr_weights(CprData& c, const Phys& ph) {
  c.w_o = 1.0 / ph.rho_o;
  c.w_w = 1.0 / ph.rho_w;
}

void cpr_setup(CprData& c, const Grid&, const Phys& ph, const double*, const Wells&, bool mixed, const void* J,
               const void*, const void*, cudaStream_t st, int* launches) {
  int k = 0;
  cpr_weights(c, ph);
  if (mixed) setup_t<float>(c, J, st, k);
  else setup_t<double>(c, J, st, k);
  *launches = k;
}

void cpr_apply(CprData& c, const Grid& g, const Wells& w, bool mixed, const void* J, const void* Bw, const void* Cw,
               const void* Dw, const void* Dinv, const void* Dwinv, const double* v, const float* vf, double* z,
               double* tmp, float* zf_out, cudaStream_t st, int* launches) {
  int k = 0;
  if (mixed) {
    // the FP32 stages read vf, the FP32 copy of v (the same values they
    // would round v to)
    // every stage in FP32; tmp serves as the FP32 stage-1 vector
    float* zf = reinterpret_cast<float*>(tmp);
    CprLevel& L0 = c.lev[0];
    const int gb = grid_for(g.n + w.nw, 256);
    if (c.ilu) {
      k += launch_ilu_apply<float, float, float, float>(g, w.nw, (const float*)J, (const float*)Dinv,
                                                        (const float*)Dwinv, vf, zf, c.ilu_fused, c.ilu_cp, st);
    } else {
      launch(k_stage1_f32, gb, 256, 0, st, g.n, w.nw, (const float*)Dinv, (const float*)Dwinv, vf, zf);
      k += 1;
    }
    const bool fold = folds_first_red(c, 0);
    launch_stage2<float, float>(c, g, w, J, Bw, (const float*)zf, vf, c.block_stage2, st, fold);
    k += 1;
    TopOut top;
    top.mode = 2;
    top.nw = w.nw;
    top.z = z;
    top.zf = zf;
    top.zf_out = zf_out;
    if (!cycle<float>(c, 0, true, st, k, top, fold)) {
      launch(k_out_f32, gb, 256, 0, st, g.n, w.nw, zf, (const float*)L0.x, z, zf_out);
      k += 1;
    }
  } else {
    apply_t<double>(c, g, w, J, Bw, Dinv, Dwinv, v, z, st, k);
  }
  *launches = k;
}

}  // namespace pf
