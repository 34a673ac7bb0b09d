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

__device__ __forceinline__ void coords(const Dims& d, long long i, int& x, int& y, int& z) {
  z = (int)(i / d.nxy);
  const long long r = i - (long long)z * d.nxy;
  y = (int)(r / d.nx);
  x = (int)(r - (long long)y * d.nx);
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

// Galerkin coarse operator with piecewise-constant aggregation
template <typename T>
__global__ void __launch_bounds__(256) k_galerkin(Dims f, Dims c, const T* __restrict__ Af, T* __restrict__ Ac,
                                                  T* __restrict__ dinv_c) {
  const int fx = c.nx < f.nx ? 2 : 1, fy = c.ny < f.ny ? 2 : 1, fz = c.nz < f.nz ? 2 : 1;
  GSTRIDE(I, c.n) {
    int cx, cy, cz;
    coords(c, I, cx, cy, cz);
    double acc[SL_COUNT];
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) acc[s] = 0.0;
    for (int dz = 0; dz < fz; ++dz)
      for (int dy = 0; dy < fy; ++dy)
        for (int dx = 0; dx < fx; ++dx) {
          const int x = cx * fx + dx, y = cy * fy + dy, z = cz * fz + dz;
          if (x >= f.nx || y >= f.ny || z >= f.nz) continue;
          const long long i = x + f.nx * (y + (long long)f.ny * z);
          acc[SL_D] += (double)Af[i];
#pragma unroll
          for (int s = 1; s < SL_COUNT; ++s) {
            const double a = (double)Af[(size_t)s * f.n + i];
            long long j;
            if (!nbr(f, x, y, z, s, j)) continue;
            int jx, jy, jz;
            coords(f, j, jx, jy, jz);
            if (jx / fx == cx && jy / fy == cy && jz / fz == cz) acc[SL_D] += a;
            else acc[s] += a;
          }
        }
#pragma unroll
    for (int s = 0; s < SL_COUNT; ++s) Ac[(size_t)s * c.n + I] = (T)acc[s];
    dinv_c[I] = (T)(1.0 / acc[SL_D]);
  }
}

// one colour of a red-black Gauss-Seidel sweep; zero_init: x holds no valid
// values yet (first half-sweep), so neighbours count as zero
template <typename T>
__global__ void __launch_bounds__(256) k_rbgs(Dims d, const T* __restrict__ A, const T* __restrict__ dinv,
                                              const T* __restrict__ b, T* __restrict__ x, int color, int zero_init) {
  GSTRIDE(i, d.n) {
    int cx, cy, cz;
    coords(d, i, cx, cy, cz);
    if (((cx + cy + cz) & 1) != color) continue;
    T s = b[i];
    if (!zero_init) {
#pragma unroll
      for (int sl = 1; sl < SL_COUNT; ++sl) {
        long long j;
        if (nbr(d, cx, cy, cz, sl, j)) s -= A[(size_t)sl * d.n + i] * x[j];
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
  GSTRIDE(I, c.n) {
    int cx, cy, cz;
    coords(c, I, cx, cy, cz);
    T acc = 0;
    for (int dz = 0; dz < fz; ++dz)
      for (int dy = 0; dy < fy; ++dy)
        for (int dx = 0; dx < fx; ++dx) {
          const int X = cx * fx + dx, Y = cy * fy + dy, Z = cz * fz + dz;
          if (X >= f.nx || Y >= f.ny || Z >= f.nz) continue;
          const long long i = X + f.nx * (Y + (long long)f.ny * Z);
          T r = b[i] - A[i] * x[i];
#pragma unroll
          for (int sl = 1; sl < SL_COUNT; ++sl) {
            long long j;
            if (nbr(f, X, Y, Z, sl, j)) r -= A[(size_t)sl * f.n + i] * x[j];
          }
          acc += r;
        }
    bc[I] = acc;
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
// thread.  A zero pivot sets *status and leaves that column zero.
template <typename T>
__global__ void k_coarse_factor(Dims d, const T* __restrict__ A, T* __restrict__ inv, int* status) {
  __shared__ double M[kMaxCoarse][kMaxCoarse];
  __shared__ int perm[kMaxCoarse];
  __shared__ int piv;
  const int n = (int)d.n;
  const int t = threadIdx.x;
  for (int e = t; e < n * n; e += blockDim.x) M[e / n][e % n] = 0.0;
  if (t < n) perm[t] = t;
  if (t == 0) *status = 0;
  __syncthreads();
  if (t < n) {
    int x, y, z;
    coords(d, t, x, y, z);
    M[t][t] = (double)A[t];
    for (int s = 1; s < SL_COUNT; ++s) {
      long long j;
      if (nbr(d, x, y, z, s, j)) M[t][j] = (double)A[(size_t)s * n + t];
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      int p = k;
      double best = fabs(M[k][k]);
      for (int r = k + 1; r < n; ++r)
        if (fabs(M[r][k]) > best) { best = fabs(M[r][k]); p = r; }
      piv = p;
      if (best == 0.0) *status = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int cidx = t; cidx < n; cidx += blockDim.x) {
        const double tmp = M[k][cidx]; M[k][cidx] = M[p][cidx]; M[p][cidx] = tmp;
      }
      if (t == 0) { const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp; }
    }
    __syncthreads();
    const double pk = M[k][k];
    if (t > k && t < n && pk != 0.0) {
      const double m = M[t][k] / pk;
      M[t][k] = m;
      for (int cidx = k + 1; cidx < n; ++cidx) M[t][cidx] -= m * M[k][cidx];
    }
    __syncthreads();
  }
  // column j of the inverse solves L U x = P e_j
  if (t < n) {
    double xcol[kMaxCoarse];
    for (int r = 0; r < n; ++r) xcol[r] = (perm[r] == t) ? 1.0 : 0.0;
    for (int r = 0; r < n; ++r)
      for (int cidx = 0; cidx < r; ++cidx) xcol[r] -= M[r][cidx] * xcol[cidx];
    for (int r = n - 1; r >= 0; --r) {
      for (int cidx = r + 1; cidx < n; ++cidx) xcol[r] -= M[r][cidx] * xcol[cidx];
      xcol[r] = M[r][r] != 0.0 ? xcol[r] / M[r][r] : 0.0;
    }
    for (int r = 0; r < n; ++r) inv[(size_t)r * n + t] = (T)xcol[r];
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
  for (int sweep = 0; sweep < c.pre; ++sweep) {
    k_rbgs<T><<<gb, 256, 0, st>>>(d, A, dinv, b, x, 0, (zero_init && sweep == 0) ? 1 : 0);
    k_rbgs<T><<<gb, 256, 0, st>>>(d, A, dinv, b, x, 1, 0);
    k += 2;
  }
  CprLevel& C = c.lev[l + 1];
  const Dims dc = dims_of(C);
  k_residual_restrict<T><<<grid_for(C.n, 256), 256, 0, st>>>(d, dc, A, b, x, (T*)C.b);
  k += 1;
  for (int g = 0; g < (l == 0 ? 1 : c.cycle_gamma); ++g) cycle<T>(c, l + 1, g == 0, st, k);
  k_prolong_add<T><<<gb, 256, 0, st>>>(d, dc, (const T*)C.x, x);
  k += 1;
  for (int sweep = 0; sweep < c.post; ++sweep) {
    k_rbgs<T><<<gb, 256, 0, st>>>(d, A, dinv, b, x, 1, 0);
    k_rbgs<T><<<gb, 256, 0, st>>>(d, A, dinv, b, x, 0, 0);
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
    k_galerkin<T><<<grid_for(C.n, 256), 256, 0, st>>>(dims_of(F), dims_of(C), (const T*)F.A, (T*)C.A, (T*)C.dinv);
    k += 1;
  }
  CprLevel& Lc = c.lev[c.nlev - 1];
  k_coarse_factor<T><<<1, kMaxCoarse, 0, st>>>(dims_of(Lc), (const T*)Lc.A, (T*)c.coarse_inv, c.coarse_status);
  k += 1;
}

template <typename T>
void apply_t(CprData& c, const Grid& g, const Wells& w, const void* J, const void* Bw, const void* Cw, const void* Dw,
             const void* Dinv, const void* Dwinv, const double* v, double* z, double* tmp, cudaStream_t st, int& k) {
  // stage 1: y = D^{-1} f (cells and wells)
  launch_bjacobi_apply<T>(g, w.nw, (const T*)Dinv, (const T*)Dwinv, v, z, st);
  // stage 2: r = f - J y, restricted to the pressure equation
  launch_spmv<T>(g, w, (const T*)J, (const T*)Bw, (const T*)Cw, (const T*)Dw, z, tmp, st);
  k += 2 + (w.nw > 0);
  CprLevel& L0 = c.lev[0];
  k_restrict_top<T><<<grid_for(g.n, 256), 256, 0, st>>>(g.n, v, tmp, c.w_o, c.w_w, (T*)L0.b);
  k += 1;
  // stage 3: pressure multigrid cycle, then y += Pi_p x
  cycle<T>(c, 0, true, st, k);
  k_prolong_top<T><<<grid_for(g.n, 256), 256, 0, st>>>(g.n, (const T*)L0.x, z);
  k += 1;
}

}  // namespace

void cpr_carve(CprData& c, const Grid& g, bool mixed, size_t& off, char* base) {
  const size_t ts = mixed ? sizeof(float) : sizeof(double);
  const int limit = std::min(std::max(c.coarse_limit, 1), kMaxCoarse);
  c.lev.clear();
  CprLevel L;
  L.nx = g.nx; L.ny = g.ny; L.nz = g.nz; L.n = g.n;
  c.lev.push_back(L);
  while (c.lev.back().n > limit && c.lev.size() < 24) {
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
               cudaStream_t st, int* launches) {
  int k = 0;
  if (mixed) apply_t<float>(c, g, w, J, Bw, Cw, Dw, Dinv, Dwinv, v, z, tmp, st, k);
  else apply_t<double>(c, g, w, J, Bw, Cw, Dw, Dinv, Dwinv, v, z, tmp, st, k);
  *launches = k;
}

}  // namespace pf
