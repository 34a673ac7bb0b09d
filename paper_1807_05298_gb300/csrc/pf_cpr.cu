// CPR-FP preconditioner (Alg. 2) with a structured aggregation multigrid for
// the pressure stage.  See pf_cpr.cuh for the decoupling and the hierarchy.
#include <math.h>

#include <algorithm>

#include "pf_cpr.cuh"

namespace pf {

namespace {

constexpr int kMaxCoarse = 64;

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

// A_p from the P columns of the oil and water rows of J
template <typename T>
__global__ void __launch_bounds__(256) k_extract_pressure(long long n, const T* __restrict__ J, T* __restrict__ A,
                                                          T* __restrict__ dinv, double w_o, double w_w) {
  GSTRIDE(i, n) {
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) {
      const double a = w_o * (double)J[((size_t)s * 9 + 0) * n + i] + w_w * (double)J[((size_t)s * 9 + 3) * n + i];
      A[(size_t)s * n + i] = (T)a;
      if (s == SL_D) dinv[i] = (T)(1.0 / a);
    }
  }
}

// Eight lanes per coarse cell, one per child (dx, dy, dz) = bits of the lane
// index within its group; groups are warp-aligned and every lane of a warp
// takes part in every round, so the shuffles see full warps.  The child sums
// use a fixed xor tree (deterministic).
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

// one colour of a red-black Gauss-Seidel sweep; zero_init: x holds no valid
// values yet (first half-sweep), so neighbours count as zero.  With xc (the
// coarse correction of dims c): the neighbours are read as x_j + xc[agg(j)],
// i.e. the prolongation x += P xc is applied on the fly.  A colour pass
// overwrites every cell of its colour, so only the other colour's values
// (the neighbours) need the correction; the next pass overwrites those.
template <typename T>
__global__ void __launch_bounds__(256) k_rbgs(Dims d, const T* __restrict__ A, const T* __restrict__ dinv,
                                              const T* __restrict__ b, T* __restrict__ x, int color, int zero_init,
                                              const T* __restrict__ xc = nullptr, Dims c = Dims{}) {
  const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
  GSTRIDE(i, d.n) {
    int cx, cy, cz;
    coords(d, i, cx, cy, cz);
    if (((cx + cy + cz) & 1) != color) continue;
    T s = b[i];
    if (!zero_init) {
#pragma unroll
      for (int sl = 1; sl < SL_COUNT; ++sl) {
        long long j;
        if (!nbr(d, cx, cy, cz, sl, j)) continue;
        T xj = x[j];
        if (xc) {
          int jx, jy, jz;
          coords(d, j, jx, jy, jz);
          xj += xc[jx / fx + c.nx * (jy / fy + (long long)c.ny * (jz / fz))];
        }
        s -= A[(size_t)sl * d.n + i] * xj;
      }
    }
    x[i] = s * dinv[i];
  }
}

// coarse right-hand side: sum over each aggregate of the fine residual b - A x
template <typename T>
__global__ void __launch_bounds__(256) k_residual_restrict(Dims f, Dims c, const T* __restrict__ A,
                                                           const T* __restrict__ b, const T* __restrict__ x,
                                                           T* __restrict__ bc) {
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  const long long total = 8 * c.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long t = base + threadIdx.x;
    const long long I = t >> 3;
    const int child = (int)(t & 7);
    const int dx = child & 1, dy = (child >> 1) & 1, dz = child >> 2;
    double r = 0.0;
    if (t < total && dx < fx && dy < fy && dz < fz) {
      int cx, cy, cz;
      coords(c, I, cx, cy, cz);
      const int X = cx * fx + dx, Y = cy * fy + dy, Z = cz * fz + dz;
      if (X < f.nx && Y < f.ny && Z < f.nz) {
        const long long i = X + f.nx * (Y + (long long)f.ny * Z);
        T ri = b[i] - A[i] * x[i];
#pragma unroll
        for (int sl = 1; sl < SL_COUNT; ++sl) {
          long long j;
          if (nbr(f, X, Y, Z, sl, j)) ri -= A[(size_t)sl * f.n + i] * x[j];
        }
        r = (double)ri;
      }
    }
    r = grp8_sum(r);
    if (t < total && child == 0) bc[I] = (T)r;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(Dims f, Dims c, const T* __restrict__ xc, T* __restrict__ x) {
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  GSTRIDE(i, f.n) {
    int X, Y, Z;
    coords(f, i, X, Y, Z);
    x[i] += xc[X / fx + c.nx * (Y / fy + (long long)c.ny * (Z / fz))];
  }
}

// Dense inverse of the coarsest stencil matrix (n <= 64): LU with partial
// pivoting in shared memory by one block, then one column of the inverse per
// thread.  Storage is column-major (M[c * ld + r]) so that the threads of a
// warp, one per row, touch consecutive words.  A zero pivot sets *status and
// leaves that column zero.
constexpr int kLd = kMaxCoarse + 1;
constexpr size_t kCoarseSmem = sizeof(double) * (2 * kMaxCoarse * kLd) + sizeof(int) * (kMaxCoarse + 1);

template <typename T>
__global__ void k_coarse_factor(Dims d, const T* __restrict__ A, T* __restrict__ inv, int* status) {
  extern __shared__ double sm[];
  double* M = sm;                       // [n][kLd] column-major: M[c * kLd + r]
  double* X = sm + kMaxCoarse * kLd;     // [n][kLd] column j of the inverse: X[j * kLd + r]
  int* perm = reinterpret_cast<int*>(X + kMaxCoarse * kLd);
  int* piv = perm + kMaxCoarse;
  const int n = (int)d.n;
  const int t = threadIdx.x;
  for (int e = t; e < kMaxCoarse * kLd; e += blockDim.x) M[e] = 0.0;
  if (t < n) perm[t] = t;
  if (t == 0) *status = 0;
  __syncthreads();
  if (t < n) {
    int x, y, z;
    coords(d, t, x, y, z);
    M[t * kLd + t] = (double)A[t];
    for (int s = 1; s < SL_COUNT; ++s) {
      long long j;
      if (nbr(d, x, y, z, s, j)) M[(int)j * kLd + t] = (double)A[(size_t)s * n + t];
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < 32) {  // pivot search by one warp
      int p = k;
      double best = -1.0;
      for (int r = k + t; r < n; r += 32) {
        const double v = fabs(M[k * kLd + r]);
        if (v > best) { best = v; p = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (t == 0) {
        *piv = p;
        if (!(best > 0.0)) *status = 1;
      }
    }
    __syncthreads();
    const int p = *piv;
    if (p != k) {
      for (int c = t; c < n; c += blockDim.x) {
        const double tmp = M[c * kLd + k]; M[c * kLd + k] = M[c * kLd + p]; M[c * kLd + p] = tmp;
      }
      if (t == 0) { const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp; }
    }
    __syncthreads();
    const double pk = M[k * kLd + k];
    if (t > k && t < n && pk != 0.0) {
      const double m = M[k * kLd + t] / pk;
      M[k * kLd + t] = m;
      for (int c = k + 1; c < n; ++c) M[c * kLd + t] -= m * M[c * kLd + k];
    }
    __syncthreads();
  }
  // column j of the inverse solves L U x = P e_j; thread j owns X[j][*]
  if (t < n) {
    double* xc = X + t * kLd;
    for (int r = 0; r < n; ++r) {
      double v = (perm[r] == t) ? 1.0 : 0.0;
      for (int c = 0; c < r; ++c) v -= M[c * kLd + r] * xc[c];
      xc[r] = v;
    }
    for (int r = n - 1; r >= 0; --r) {
      double v = xc[r];
      for (int c = r + 1; c < n; ++c) v -= M[c * kLd + r] * xc[c];
      const double dg = M[r * kLd + r];
      xc[r] = dg != 0.0 ? v / dg : 0.0;
    }
  }
  __syncthreads();
  for (int e = t; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e % n;
    inv[e] = (T)X[c * kLd + r];
  }
}

// All levels from l0 down run inside one thread block (levels small enough
// that launch latency, not work, would dominate): the same smoother,
// restriction, prolongation and coarse inverse as the per-level kernels.
constexpr int kMaxLev = 24;
// FP64 runs at a small fraction of the FP32 rate per SM, so one block may only
// take the tiny FP64 levels; FP32 levels up to 4096 cells fit one block well.
template <typename T> constexpr long long block_level_cells() { return sizeof(T) == 8 ? 256 : 4096; }

template <typename T>
struct BlockLevels {
  int l0, nlev, pre, post, gamma;
  Dims d[kMaxLev];
  T* A[kMaxLev];
  T* dinv[kMaxLev];
  T* x[kMaxLev];
  T* b[kMaxLev];
  const T* inv;
};

template <typename T>
__device__ void b_rbgs(const Dims& d, const T* A, const T* dinv, const T* b, T* x, int color, bool zero_init) {
  for (long long i = threadIdx.x; i < d.n; i += blockDim.x) {
    int cx, cy, cz;
    coords(d, i, cx, cy, cz);
    if (((cx + cy + cz) & 1) != color) continue;
    T s = b[i];
    if (!zero_init) {
      for (int sl = 1; sl < SL_COUNT; ++sl) {
        long long j;
        if (nbr(d, cx, cy, cz, sl, j)) s -= A[(size_t)sl * d.n + i] * x[j];
      }
    }
    x[i] = s * dinv[i];
  }
  __syncthreads();
}

// The cycle below the block levels, written as a loop over an explicit level
// pointer (no device recursion, no per-thread copy of the descriptors: they
// live in shared memory).  cnt[l] counts the coarse cycles finished at level
// l in the current visit; level l runs gamma_l of them (1 at the finest
// level, L.gamma below), the first from a zero initial guess.
template <typename T>
__global__ void __launch_bounds__(1024) k_block_cycle(BlockLevels<T> Lp, int zero_init) {
  __shared__ BlockLevels<T> L;
  __shared__ int cnt[kMaxLev];
  __shared__ int zi[kMaxLev];
  if (threadIdx.x == 0) {
    L = Lp;
    zi[L.l0] = zero_init;
  }
  __syncthreads();
  const int last = L.nlev - 1;
  int l = L.l0;
  bool down = true;
  for (int guard = 0; guard < (1 << 20); ++guard) {
    if (down) {
      const Dims d = L.d[l];
      if (l == last) {  // coarsest: dense inverse
        const int n = (int)d.n;
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
          double sacc = 0.0;
          for (int c = 0; c < n; ++c) sacc += (double)L.inv[(size_t)r * n + c] * (double)L.b[l][c];
          L.x[l][r] = (T)sacc;
        }
        __syncthreads();
        if (l == L.l0) return;
        --l;
        down = false;
        continue;
      }
      for (int sweep = 0; sweep < L.pre; ++sweep) {
        b_rbgs<T>(d, L.A[l], L.dinv[l], L.b[l], L.x[l], 0, zi[l] && sweep == 0);
        b_rbgs<T>(d, L.A[l], L.dinv[l], L.b[l], L.x[l], 1, false);
      }
      const Dims c = L.d[l + 1];
      const int fx = c.nx < d.nx ? 2 : 1, fy = c.ny < d.ny ? 2 : 1, fz = c.nz < d.nz ? 2 : 1;
      const T* A = L.A[l];
      const T* x = L.x[l];
      const T* b = L.b[l];
      for (long long I = threadIdx.x; I < c.n; I += blockDim.x) {
        int cx, cy, cz;
        coords(c, I, cx, cy, cz);
        T acc = 0;
        for (int dz = 0; dz < fz; ++dz)
          for (int dy = 0; dy < fy; ++dy)
            for (int dx = 0; dx < fx; ++dx) {
              const int X = cx * fx + dx, Y = cy * fy + dy, Z = cz * fz + dz;
              if (X >= d.nx || Y >= d.ny || Z >= d.nz) continue;
              const long long i = X + d.nx * (Y + (long long)d.ny * Z);
              T r = b[i] - A[i] * x[i];
              for (int sl = 1; sl < SL_COUNT; ++sl) {
                long long j;
                if (nbr(d, X, Y, Z, sl, j)) r -= A[(size_t)sl * d.n + i] * x[j];
              }
              acc += r;
            }
        L.b[l + 1][I] = acc;
      }
      if (threadIdx.x == 0) {
        cnt[l] = 0;
        zi[l + 1] = 1;
      }
      __syncthreads();
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
    for (long long i = threadIdx.x; i < d.n; i += blockDim.x) {
      int X, Y, Z;
      coords(d, i, X, Y, Z);
      L.x[l][i] += L.x[l + 1][X / fx + c.nx * (Y / fy + (long long)c.ny * (Z / fz))];
    }
    __syncthreads();
    for (int sweep = 0; sweep < L.post; ++sweep) {
      b_rbgs<T>(d, L.A[l], L.dinv[l], L.b[l], L.x[l], 1, false);
      b_rbgs<T>(d, L.A[l], L.dinv[l], L.b[l], L.x[l], 0, false);
    }
    if (l == L.l0) return;
    --l;
  }
}

template <typename T>
__global__ void k_coarse_apply(int n, const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  const int r = threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int c = 0; c < n; ++c) s += (double)inv[(size_t)r * n + c] * (double)b[c];
  x[r] = (T)s;
}

// Pi_r (f - J y): weighted oil and water rows of the residual, per cell
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_top(long long n, const double* __restrict__ f,
                                                      const double* __restrict__ Jy, double w_o, double w_w,
                                                      T* __restrict__ b0) {
  GSTRIDE(i, n) b0[i] = (T)(w_o * (f[3 * i] - Jy[3 * i]) + w_w * (f[3 * i + 1] - Jy[3 * i + 1]));
}

// y += Pi_p x0
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_top(long long n, const T* __restrict__ x0, double* __restrict__ y) {
  GSTRIDE(i, n) y[3 * i] += (double)x0[i];
}

size_t aup(size_t v) { return (v + 255) / 256 * 256; }

template <typename T>
void cycle(CprData& c, int l, bool zero_init, cudaStream_t st, int& k) {
  CprLevel& L = c.lev[l];
  const Dims d = dims_of(L);
  const int gb = grid_for(L.n, 256);
  T* x = (T*)L.x;
  const T* A = (const T*)L.A;
  const T* dinv = (const T*)L.dinv;
  const T* b = (const T*)L.b;
  if (l == c.nlev - 1) {
    k_coarse_apply<T><<<1, kMaxCoarse, 0, st>>>((int)L.n, (const T*)c.coarse_inv, b, x);
    k += 1;
    return;
  }
  if (L.n <= block_level_cells<T>()) {  // this level and all coarser ones in one block
    BlockLevels<T> B;
    B.l0 = l; B.nlev = c.nlev; B.pre = c.pre; B.post = c.post; B.gamma = c.cycle_gamma;
    for (int q = 0; q < c.nlev; ++q) {
      B.d[q] = dims_of(c.lev[q]);
      B.A[q] = (T*)c.lev[q].A; B.dinv[q] = (T*)c.lev[q].dinv; B.x[q] = (T*)c.lev[q].x; B.b[q] = (T*)c.lev[q].b;
    }
    B.inv = (const T*)c.coarse_inv;
    k_block_cycle<T><<<1, 1024, 0, st>>>(B, zero_init ? 1 : 0);
    k += 1;
    return;
  }
  const int bs = l == 0 ? c.block_rbgs0 : 256;
  const int gs = grid_for(L.n, bs);
  for (int sweep = 0; sweep < c.pre; ++sweep) {
    k_rbgs<T><<<gs, bs, 0, st>>>(d, A, dinv, b, x, 0, (zero_init && sweep == 0) ? 1 : 0);
    k_rbgs<T><<<gs, bs, 0, st>>>(d, A, dinv, b, x, 1, 0);
    k += 2;
  }
  CprLevel& C = c.lev[l + 1];
  const Dims dc = dims_of(C);
  k_residual_restrict<T><<<grid_for(8 * C.n, 256), 256, 0, st>>>(d, dc, A, b, x, (T*)C.b);
  k += 1;
  for (int g = 0; g < (l == 0 ? 1 : c.cycle_gamma); ++g) cycle<T>(c, l + 1, g == 0, st, k);
  if (c.post == 0) {
    k_prolong_add<T><<<gb, 256, 0, st>>>(d, dc, (const T*)C.x, x);
    k += 1;
  }
  for (int sweep = 0; sweep < c.post; ++sweep) {
    // the first black pass applies the prolongation to the red neighbours it reads
    if (sweep == 0) k_rbgs<T><<<gs, bs, 0, st>>>(d, A, dinv, b, x, 1, 0, (const T*)C.x, dc);
    else k_rbgs<T><<<gs, bs, 0, st>>>(d, A, dinv, b, x, 1, 0);
    k_rbgs<T><<<gs, bs, 0, st>>>(d, A, dinv, b, x, 0, 0);
    k += 2;
  }
}

template <typename T>
void setup_t(CprData& c, const void* J, cudaStream_t st, int& k) {
  CprLevel& L0 = c.lev[0];
  k_extract_pressure<T><<<grid_for(L0.n, 256), 256, 0, st>>>(L0.n, (const T*)J, (T*)L0.A, (T*)L0.dinv, c.w_o, c.w_w);
  k += 1;
  for (int l = 0; l + 1 < c.nlev; ++l) {
    CprLevel& F = c.lev[l];
    CprLevel& C = c.lev[l + 1];
    k_galerkin<T><<<grid_for(8 * C.n, 256), 256, 0, st>>>(dims_of(F), dims_of(C), (const T*)F.A, (T*)C.A,
                                                          (T*)C.dinv);
    k += 1;
  }
  CprLevel& Lc = c.lev[c.nlev - 1];
  cudaFuncSetAttribute(k_coarse_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmem);
  k_coarse_factor<T><<<1, kMaxCoarse, kCoarseSmem, st>>>(dims_of(Lc), (const T*)Lc.A, (T*)c.coarse_inv,
                                                         c.coarse_status);
  k += 1;
}

// ----- FP32 CPR apply (mixed precision): every stage in FP32 -----

// stage 1 in FP32: zf = D^{-1} (float) v, cells and wells
__global__ void __launch_bounds__(256) k_stage1_f32(long long n, int nw, const float* __restrict__ Dinv,
                                                    const float* __restrict__ Dwinv, const double* __restrict__ v,
                                                    float* __restrict__ zf) {
  GSTRIDE(i, n + nw) {
    if (i >= n) { zf[3 * n + (i - n)] = Dwinv[i - n] * (float)v[3 * n + (i - n)]; continue; }
    const float r0 = (float)v[3 * i], r1 = (float)v[3 * i + 1], r2 = (float)v[3 * i + 2];
    const float* D = Dinv + i;
    zf[3 * i] = D[0] * r0 + D[n] * r1 + D[2 * n] * r2;
    zf[3 * i + 1] = D[3 * n] * r0 + D[4 * n] * r1 + D[5 * n] * r2;
    zf[3 * i + 2] = D[6 * n] * r0 + D[7 * n] * r1 + D[8 * n] * r2;
  }
}

// stage 2 in FP32, restricted on the fly: b0 = w_o (v - J zf)_oil + w_w (v - J zf)_water
// (only the oil and water rows of J are read)
__global__ void __launch_bounds__(256, 4) k_stage2_f32(Grid g, const float* __restrict__ J, const float* __restrict__ zf,
                                                    const double* __restrict__ v, float w_o, float w_w,
                                                    float* __restrict__ b0) {
  const long long n = g.n;
  GSTRIDE(i, n) {
    const unsigned int ui = (unsigned int)i, nxy = (unsigned int)g.nxy, nxu = (unsigned int)g.nx;
    const long long k = ui / nxy;
    const unsigned int rem = ui - (unsigned int)k * nxy;
    const long long j = rem / nxu;
    const long long ii = rem - (unsigned int)j * nxu;
    float t0 = 0.f, t1 = 0.f;
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
      const float* B = J + (size_t)s * 9 * n + i;
      const float x0 = zf[3 * c], x1 = zf[3 * c + 1], x2 = zf[3 * c + 2];
      t0 += B[0] * x0 + B[n] * x1 + B[2 * n] * x2;
      t1 += B[3 * n] * x0 + B[4 * n] * x1 + B[5 * n] * x2;
    }
    b0[i] = w_o * ((float)v[3 * i] - t0) + w_w * ((float)v[3 * i + 1] - t1);
  }
}

// the well border's share of J zf in the oil and water rows of perforated cells
__global__ void k_stage2_wells_f32(Wells w, long long n, const float* __restrict__ Bw, const float* __restrict__ zf,
                                   float w_o, float w_w, float* __restrict__ b0) {
  const int wi = blockIdx.x;
  if (wi >= w.nw) return;
  const float zw = zf[3 * n + wi];
  for (int m = w.ptr[wi] + threadIdx.x; m < w.ptr[wi + 1]; m += 32) {
    const long long c = w.cell[m];
    b0[c] -= (w_o * Bw[m] + w_w * Bw[w.npf + m]) * zw;
  }
}

// z = zf + Pi_p x0, written as FP64 for the Krylov basis and as an FP32 copy
// for the mixed-precision operator (the two hold the same float values)
__global__ void __launch_bounds__(256) k_out_f32(long long n, int nw, const float* __restrict__ zf,
                                                 const float* __restrict__ x0, double* __restrict__ z,
                                                 float* __restrict__ zf_out) {
  GSTRIDE(i, n + nw) {
    if (i >= n) {
      const float v = zf[3 * n + (i - n)];
      z[3 * n + (i - n)] = (double)v;
      if (zf_out) zf_out[3 * n + (i - n)] = v;
      continue;
    }
    const float p = zf[3 * i] + x0[i], sv = zf[3 * i + 1], cv = zf[3 * i + 2];
    z[3 * i] = (double)p;
    z[3 * i + 1] = (double)sv;
    z[3 * i + 2] = (double)cv;
    if (zf_out) { zf_out[3 * i] = p; zf_out[3 * i + 1] = sv; zf_out[3 * i + 2] = cv; }
  }
}

template <typename T>
void apply_t(CprData& c, const Grid& g, const Wells& w, const void* J, const void* Bw, const void* Cw, const void* Dw,
             const void* Dinv, const void* Dwinv, const double* v, double* z, double* tmp, cudaStream_t st, int& k) {
  // stage 1: y = D^{-1} f, or the red-black block ILU(0) solve (cells; wells by their diagonal)
  if (c.ilu) {
    launch_ilu_apply<T, T, double>(g, w.nw, (const T*)J, (const T*)Dinv, (const T*)Dwinv, v, z, st);
    k += 3;
  } else {
    launch_bjacobi_apply<T>(g, w.nw, (const T*)Dinv, (const T*)Dwinv, v, z, st);
    k += 1;
  }
  // stage 2: r = f - J y, restricted to the pressure equation
  launch_spmv<T>(g, w, (const T*)J, (const T*)Bw, (const T*)Cw, (const T*)Dw, z, tmp, st);
  k += 1 + (w.nw > 0);
  CprLevel& L0 = c.lev[0];
  k_restrict_top<T><<<grid_for(g.n, 256), 256, 0, st>>>(g.n, v, tmp, c.w_o, c.w_w, (T*)L0.b);
  k += 1;
  // stage 3: pressure multigrid cycle, then y += Pi_p x
  cycle<T>(c, 0, true, st, k);
  k_prolong_top<T><<<grid_for(g.n, 256), 256, 0, st>>>(g.n, (const T*)L0.x, z);
  k += 1;
}

}  // namespace

void cpr_time_rbgs0(CprData& c, bool mixed, int block, cudaStream_t st) {
  CprLevel& L = c.lev[0];
  const Dims d = dims_of(L);
  if (mixed)
    k_rbgs<float><<<grid_for(L.n, block), block, 0, st>>>(d, (const float*)L.A, (const float*)L.dinv,
                                                          (const float*)L.b, (float*)L.x, 0, 0);
  else
    k_rbgs<double><<<grid_for(L.n, block), block, 0, st>>>(d, (const double*)L.A, (const double*)L.dinv,
                                                           (const double*)L.b, (double*)L.x, 0, 0);
}

void cpr_time_stage2(CprData& c, const Grid& g, const void* J, const double* v, double* tmp, int block,
                     cudaStream_t st) {
  k_stage2_f32<<<grid_for(g.n, block), block, 0, st>>>(g, (const float*)J, reinterpret_cast<const float*>(tmp), v,
                                                       (float)c.w_o, (float)c.w_w, (float*)c.lev[0].b);
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
}

pf_status cpr_init(CprData& c, const Grid&, bool, const pf_solver_opts& o, cudaStream_t) {
  c.pre = std::max(0, o.amg_pre_sweeps);
  c.post = std::max(0, o.amg_post_sweeps);
  c.cycle_gamma = o.amg_cycle == 2 ? 2 : 1;
  if (c.lev.empty() || c.lev.back().n > kMaxCoarse) return PF_EINVAL;
  c.ready = true;
  return PF_OK;
}

void cpr_setup(CprData& c, const Grid&, const Phys& ph, const double*, const Wells&, bool mixed, const void* J,
               const void*, const void*, cudaStream_t st, int* launches) {
  int k = 0;
  c.w_o = 1.0 / ph.rho_o;
  c.w_w = 1.0 / ph.rho_w;
  if (mixed) setup_t<float>(c, J, st, k);
  else setup_t<double>(c, J, st, k);
  *launches = k;
}

void cpr_apply(CprData& c, const Grid& g, const Wells& w, bool mixed, const void* J, const void* Bw, const void* Cw,
               const void* Dw, const void* Dinv, const void* Dwinv, const double* v, double* z, double* tmp,
               float* zf_out, cudaStream_t st, int* launches) {
  int k = 0;
  if (mixed) {
    // every stage in FP32; tmp serves as the FP32 stage-1 vector
    float* zf = reinterpret_cast<float*>(tmp);
    CprLevel& L0 = c.lev[0];
    const int gb = grid_for(g.n + w.nw, 256);
    if (c.ilu) {
      launch_ilu_apply<float, float, float>(g, w.nw, (const float*)J, (const float*)Dinv, (const float*)Dwinv, v, zf,
                                            st);
      k += 3;
    } else {
      k_stage1_f32<<<gb, 256, 0, st>>>(g.n, w.nw, (const float*)Dinv, (const float*)Dwinv, v, zf);
      k += 1;
    }
    k_stage2_f32<<<grid_for(g.n, c.block_stage2), c.block_stage2, 0, st>>>(g, (const float*)J, zf, v, (float)c.w_o,
                                                                         (float)c.w_w, (float*)L0.b);
    k += 1;
    if (w.nw > 0) {
      k_stage2_wells_f32<<<w.nw, 32, 0, st>>>(w, g.n, (const float*)Bw, zf, (float)c.w_o, (float)c.w_w,
                                              (float*)L0.b);
      k += 1;
    }
    cycle<float>(c, 0, true, st, k);
    k_out_f32<<<gb, 256, 0, st>>>(g.n, w.nw, zf, (const float*)L0.x, z, zf_out);
    k += 1;
  } else {
    apply_t<double>(c, g, w, J, Bw, Cw, Dw, Dinv, Dwinv, v, z, tmp, st, k);
  }
  *launches = k;
}

}  // namespace pf
