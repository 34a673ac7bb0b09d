// Internal declarations of the polyflood CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pf_launch.cuh"
#include "polyflood.h"

namespace pf {

// Rock, fluid and polymer constants with the derived quantities the kernels
// use (passed by value as a kernel argument).
struct Phys {
  double rho_w, rho_o, c_w, c_o, p_ref, mu_w, mu_o, c_r, p_r;
  double swc, sor, nw, no, krw_max, kro_max, pc_e, pc_n;
  double ads_a, ads_b, rrf, ipv, omega, mu_p0, c_ref, g;
  int mixing;
  // derived
  double inv_den;        // 1 / (1 - swc - sor)
  double ln_mu_w, ln_mu_ratio;   // ln mu_w, ln mu_p0 - ln mu_w
  double rk_coef;        // (rrf - 1) / A_d,max, or 0 without adsorption
  double mu_p0_pow, mu_w_pow;    // mu_p0^(1-omega), mu_w^(1-omega)
  double inv_c_ref, inv_rho_w;   // 1 / c_ref, 1 / rho_w,ref
  double inv_mu_o;               // 1 / mu_o
  // optional tables on the device, structure of arrays with the segment
  // slopes: sat = S, k_rw, k_ro, P_c, then their slopes (7 x n_sat);
  // poly = C, multiplier, A_d, then their slopes (5 x n_poly)
  const double* sat = nullptr;
  const double* poly = nullptr;
  int n_sat = 0, n_poly = 0;
};

// Message returned by pf_last_error on this thread (set by host code outside pf_api.cu).
void set_last_error(const std::string& msg);

struct Grid {
  int nx, ny, nz;
  long long n, nxy;
  double dx, dy, dz, top, V;
};

// Per-cell property scratch: values (FP64) and derivatives (DT).
enum {
  PV_RHO_O = 0, PV_RHO_W, PV_PW, PV_KRW, PV_KRO, PV_RK, PV_MUWE, PV_MUPE, PV_COUNT
};
enum {
  PD_RHO_O = 0, PD_RHO_WP, PD_RHO_WS, PD_PW_S, PD_KRW, PD_KRO, PD_RK, PD_MUWE, PD_MUPE, PD_COUNT
};

// Jacobian block slots of a cell row.
enum { SL_D = 0, SL_XM, SL_XP, SL_YM, SL_YP, SL_ZM, SL_ZP, SL_COUNT };

// Device views of the well data.
struct Wells {
  int nw;
  long long npf;
  const int* ptr;          // [nw+1] perforation range of each well
  const long long* cell;   // [npf]
  const double* wi;        // [npf] Peaceman index
  const double* dzb;       // [npf] z_m - z_b
  const int* kind;         // [nw]
  const int* ctrl;         // [nw]
  const double* target;    // [nw] Pa or mass rate coefficient target (rho_t * q)
  const double* cinj;      // [nw]
  const double* W;         // [nw] BHP row scale sum(WI) rho_w / mu_w
  const double* sw;        // [nw] rate coefficient of the water sum
  const double* so;        // [nw] rate coefficient of the oil sum
  const double* scale;     // [nw] scaled-residual denominator / dt
  const double* gamma;     // [nw] lagged wellbore unit weight
  const int* perf_of;      // [N] perforation index of each cell, -1 if none
  const int* pwell;        // [npf] well of each perforation
};

// Block sizes of the per-cell kernels (autotuned or 256).  Every cell's
// arithmetic is independent of the launch shape, so results do not depend on
// these values.
struct Tuning {
  int props = 256, face = 256, gather = 256, spmv = 256, stage2 = 256, rbgs = 256;
  int block_cells = 0;  // single-block multigrid levels up to this size (0: the CPR default)
  int cluster_cells = -1;  // thread-block-cluster levels up to this size (-1: the CPR default)
  int ilu_fused = 1;    // ILU(0) solve: diagonal red sweep folded into the black sweep (1) or separate (0)
};

// One row of a 3x3 block times a 3-vector, accumulated as three fused
// multiply-adds: acc + b0 x0 + b1 x1 + b2 x2 (fma3) and acc - b0 x0 - b1 x1
// - b2 x2 (fnms3), in that order.  Written out so that an FP64 block product
// costs one FP64-pipe instruction per product, with no separate multiply and
// add around a partial sum.
__device__ __forceinline__ double fma3(double b0, double b1, double b2, double x0, double x1, double x2,
                                       double acc) {
  return __fma_rn(b2, x2, __fma_rn(b1, x1, __fma_rn(b0, x0, acc)));
}
__device__ __forceinline__ float fma3(float b0, float b1, float b2, float x0, float x1, float x2, float acc) {
  return __fmaf_rn(b2, x2, __fmaf_rn(b1, x1, __fmaf_rn(b0, x0, acc)));
}
__device__ __forceinline__ double fnms3(double b0, double b1, double b2, double x0, double x1, double x2,
                                        double acc) {
  return __fma_rn(-b2, x2, __fma_rn(-b1, x1, __fma_rn(-b0, x0, acc)));
}
__device__ __forceinline__ float fnms3(float b0, float b1, float b2, float x0, float x1, float x2, float acc) {
  return __fmaf_rn(-b2, x2, __fmaf_rn(-b1, x1, __fmaf_rn(-b0, x0, acc)));
}

// The oil row of every Jacobian block has a zero in its polymer column: the
// oil accumulation, the oil flux (k_ro, mu_o, rho_o and the oil potential) and
// the oil well rate do not depend on C (the assembly writes that entry as 0).
// Products with the oil row therefore skip the column: the same sum (adding
// 0 x to a finite value changes nothing), one FMA and one load fewer.
__device__ __forceinline__ double fma2(double b0, double b1, double x0, double x1, double acc) {
  return __fma_rn(b1, x1, __fma_rn(b0, x0, acc));
}
__device__ __forceinline__ float fma2(float b0, float b1, float x0, float x1, float acc) {
  return __fmaf_rn(b1, x1, __fmaf_rn(b0, x0, acc));
}
__device__ __forceinline__ double fnms2(double b0, double b1, double x0, double x1, double acc) {
  return __fma_rn(-b1, x1, __fma_rn(-b0, x0, acc));
}
__device__ __forceinline__ float fnms2(float b0, float b1, float x0, float x1, float acc) {
  return __fmaf_rn(-b1, x1, __fmaf_rn(-b0, x0, acc));
}

// Launch helpers ------------------------------------------------------------
// slots of one colour of the red-black ordering: ceil(nx / 2) per (j, k) row
inline long long colour_slots_host(const Grid& g) { return (long long)((g.nx + 1) / 2) * g.ny * g.nz; }

inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (int)g;
}

// Assembly (pf_assembly.cu) -------------------------------------------------
// mode 0: properties + accumulation into R and the diagonal; mode 1: old masses
// (and the values the lagged wellbore weight needs); mode 2: property values only.
template <typename DT>
void launch_cell_props(const Grid& g, const Phys& ph, const double* phi_r, const double* x,
                       double* pv, DT* pd, const double* Mold, double* R, DT* J, double* Mold_out,
                       int mode, cudaStream_t st, int block = 256);
template <typename DT>
// wL3[d * N + i]: pore-volume weight of cell i on its face towards +d
void launch_face_flux(const Grid& g, const Phys& ph, const double* wL3, const double* T3,
                      const double* x, const double* pv, const DT* pd, double dt, DT* J,
                      double* Fbuf, cudaStream_t st, int block = 256);
// Fbuf (written by launch_face_flux) holds dt F per face
template <typename DT>
void launch_gather(const Grid& g, const double* Fbuf, double* R, DT* J, cudaStream_t st, int block = 256);
template <typename DT>
void launch_wells(const Grid& g, const Phys& ph, const Wells& w, const double* x, const double* pv,
                  const DT* pd, double dt, double* R, DT* J, DT* Bw, DT* Cw, DT* Dw, cudaStream_t st);

// Packed assembly: the four assembly kernels of several simulators in one
// launch each, with every cell's arithmetic that of its own simulator's
// kernels (results bit-identical).  The members travel in the launch
// parameters; block b of a cell kernel belongs to the member m with
// cblock0[m] <= b < cblock0[m + 1] (256 threads per block), block b of the well
// kernel to the member with wblock0[m] <= b < wblock0[m + 1] (one warp per well).
constexpr int kPackMax = 24;
template <typename DT>
struct AsmMember {
  Grid g;
  Phys ph;
  Wells w;
  const double *phi_r, *x, *Mold, *wL3, *T3;
  double *pv, *R, *Fbuf;
  DT *pd, *J, *Bw, *Cw, *Dw;
  double dt;
};
template <typename DT, int CAP = kPackMax>
struct AsmPack {
  int nm;
  int cblock0[CAP + 1];
  int wblock0[CAP + 1];
  AsmMember<DT> m[CAP];
};
// launches the pack on st (cblock0/wblock0 filled by the caller, 256 threads
// per cell block); returns the kernel count.  A simulator's own assembly runs
// the same kernels on a pack of one (launch_cell_props mode 0,
// launch_face_flux, launch_gather, launch_wells), so packed and own results
// are the same compiled arithmetic.
template <typename DT>
int launch_assemble_packed(const AsmPack<DT>& pk, cudaStream_t st);
// The assembly of n simulators (one precision) in packs of up to kPackMax on
// stream st; the caller orders st after each simulator's stream and each
// simulator's stream after st.  *launches (may be null): kernels launched.
pf_status assemble_packed(pf_sim* const* sims, int n, cudaStream_t st, int* launches);
// Routes a simulator's assembly through fn(ctx, s) (null: its own launches).
void set_assembly_packer(pf_sim* s, pf_status (*fn)(void*, pf_sim*), void* ctx);
cudaStream_t sim_stream(const pf_sim* s);
void launch_well_gamma(const Grid& g, const Phys& ph, const Wells& w, const double* x,
                       const double* pv, double* gamma, cudaStream_t st);
// out[3w + {0,1,2}] = water, oil, polymer mass rate of well w (needs a mode-2 pv).
void launch_well_totals(const Grid& g, const Phys& ph, const Wells& w, const double* x, const double* pv,
                        double* out, cudaStream_t st);
// Scaled max-norm and squared 2-norm of R: out[0] = max, out[1] = sum of squares.
void launch_residual_norms(const Grid& g, const Phys& ph, const double* inv_pv, const Wells& w,
                           const double* R, double dt, double* partial, int nblocks, double* out,
                           cudaStream_t st);
// x += dx with |dS| <= ds_max and |dC| <= dc_max per cell, then S in [0, 1], C >= 0
void launch_newton_update(const Grid& g, int nw, double* x, const double* dx, double ds_max, double dc_max,
                          cudaStream_t st);

// Linear algebra (pf_linalg.cu) ---------------------------------------------
template <typename DT>
void launch_spmv(const Grid& g, const Wells& w, const DT* J, const DT* Bw, const DT* Cw,
                 const DT* Dw, const double* x, double* y, cudaStream_t st, int block = 256);
template <typename DT, typename PT>
void launch_bjacobi_setup(const Grid& g, const Wells& w, const DT* J, const DT* Dw, PT* Dinv,
                          PT* Dwinv, cudaStream_t st);
// Compact per-colour copies of the off-diagonal blocks for the ILU(0) sweeps:
// kind 0 none (the sweeps read J and the inverses by cell), 1 in the
// Jacobian's precision, 2 BF16.
struct IluCompact {
  int kind = 0;
  // [6 slots][9 entries][colour slots] per colour: c[0] the red cells' blocks,
  // c[1] the black cells' products J_bj D_j^-1 with their red neighbours'
  // inverses (formed by the set-up for the Schur update anyway), through which
  // the black sweep takes f_j of the red neighbours, so the solve is two
  // launches with no diagonal red sweep
  void* c[2] = {nullptr, nullptr};
  // the black rows' pressure combination w_o (oil row) + w_w (water row) of
  // every block, for the CPR stage 2 (null without CPR): off-diagonal blocks
  // [6 slots][3 columns][black slots] in the copy's type, the diagonal block
  // [3 columns][black slots] in the preconditioner's type
  void* p = nullptr;
  void* pd = nullptr;
  // FP64 with the copies: both colours' block inverses per colour slot, [9
  // entries][red slots] then [9 entries][black slots] (in place of the by-cell
  // array, whose lines carry both colours); null otherwise
  void* dr = nullptr;
};
// w_o, w_w: the CPR stage-2 weights (used when cp.p is set)
template <typename DT, typename PT>
void launch_ilu_setup(const Grid& g, const Wells& w, const DT* J, const DT* Dw, PT* Dinv, PT* Dwinv, double guard,
                      const IluCompact& cp, cudaStream_t st, double w_o = 0.0, double w_w = 0.0);
// f: the right-hand side, FP64 or (mixed-precision CPR) its FP32 copy
template <typename DT, typename PT, typename OT, typename VT>
int launch_ilu_apply(const Grid& g, int nw, const DT* J, const PT* Dinv, const PT* Dwinv, const VT* f, OT* y,
                     int fused, const IluCompact& cp, cudaStream_t st);  // returns the number of launches
// CPR stage 2 after the ILU(0) first stage: black rows in full, red rows their
// well column only (the red sweep solved their cell part exactly).  x0 (may be
// null): also the multigrid's first red pass from a zero guess, x0 = b0 * d0
// (d0 indexed by the red colour slot when d0_slot, else by the cell).
template <typename T, typename VT>
void launch_stage2_ilu(const Grid& g, const Wells& w, const T* J, const IluCompact& cp, const T* Bw, const T* y,
                       const VT* v, T w_o, T w_w, T* b0, T* x0, const T* d0, int d0_slot, int block,
                       cudaStream_t st);
template <typename PT>
void launch_bjacobi_apply(const Grid& g, int nw, const PT* Dinv, const PT* Dwinv, const double* r,
                          double* z, cudaStream_t st);

// Vector kernels over n FP64 entries.
void launch_copy(long long n, const double* a, double* b, cudaStream_t st);
void launch_to_f32(long long n, const double* a, float* b, cudaStream_t st);
void launch_fill(long long n, double v, double* a, cudaStream_t st);
// b = a * s[0] or a / sqrt(s[0]); with bf also bf = (float) b
void launch_scale_by_dev(long long n, const double* a, const double* s, int inv_sqrt, double* b,
                         cudaStream_t st, float* bf = nullptr);
void launch_axpy(long long n, double alpha, const double* x, double* y, cudaStream_t st);
void launch_xpay(long long n, const double* x, double beta, double* y, cudaStream_t st); // y = x + beta y
void launch_sub(long long n, const double* a, const double* b, double* c, cudaStream_t st); // c = a - b
// out[j] = sum_i V[j*ld + i] w[i], j < k (and out[k] = <w, w> with
// self_dot).  Per-block rows (stride 72) go to `partial`; the last block
// reduces them in a fixed order (deterministic) and re-arms `counter` (a
// zeroed device word shared by the reductions of one stream).  run_if (may
// be null): skip the whole kernel unless *run_if.
// vs (may be null): V_j holds the basis vector before its normalisation, the
// basis vector is vs[j] V_j, and out[j] = vs[j] <V_j, w>.
// pyth (may be null, with self_dot): pyth[0] = |w|^2 - sum_j out[j]^2, the
// squared norm of w after its projection on the orthonormal v_j, pyth[1] =
// 1 / sqrt(pyth[0]) (also into *vs_next when given), and *decide = 1 when
// pyth[0] < eta2 |w|^2.
void launch_multidot(long long n, int k, const double* V, long long ld, const double* w,
                     double* partial, int nblocks, double* out, unsigned int* counter, cudaStream_t st,
                     int self_dot = 0, const int* run_if = nullptr, const double* vs = nullptr,
                     double* pyth = nullptr, double* vs_next = nullptr, int* decide = nullptr, double eta2 = 0.0);
// w -= sum_j V[j] h[j]; out[0] = |w|^2, out[1] = 1/|w|; *decide = 1 if
// |w|^2 < eta2 norm0[0] (a second Gram-Schmidt pass is needed); with out
// null the projection alone (no norm, no reduction).
// vs as in launch_multidot; wf (may be null) gets an FP32 copy of the new w;
// vs_next (may be null) gets 1 / |w|, the normalisation of w as the next
// basis vector.
void launch_axpy_norm(long long n, int k, const double* V, long long ld, const double* h, double* w,
                      double* partial, int nblocks, double* out, unsigned int* counter, const double* norm0,
                      int* decide, const int* run_if, cudaStream_t st,
                      double eta2 = 0.5, const double* vs = nullptr, float* wf = nullptr, double* vs_next = nullptr);
void launch_spmv_f32(const Grid& g, const Wells& w, const float* J, const float* Bw, const float* Cw,
                     const float* Dw, const float* x, double* y, cudaStream_t st, int block = 256);
// x += sum_j Z[j] y[j]
void launch_multi_axpy_add(long long n, int k, const double* Z, long long ld, const double* y,
                           double* x, cudaStream_t st);
// the same with FP32 vectors Zf, summed in two-float arithmetic (about 47
// significant bits) on the FP32 pipe
void launch_multi_axpy_add_f32(long long n, int k, const float* Zf, long long ld, const double* y, double* x,
                               cudaStream_t st);
void launch_dot(long long n, const double* a, const double* b, double* partial, int nblocks,
                double* out, unsigned int* counter, cudaStream_t st);

}  // namespace pf
