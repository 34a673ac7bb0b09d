// CPR-FP preconditioner (Alg. 2): y = D_r(J)^{-1} f by block-Jacobi (one
// subdomain per GPU, so the restricted additive Schwarz step reduces to its
// local block solve); r = f - J y; y += Pi_p M_g(A_p)^{-1} Pi_r r with M_g a
// multigrid cycle on the pressure matrix.
//
// The pressure matrix A_p takes the P-columns of the oil and water rows of J
// weighted by 1/rho_o,ref and 1/rho_w,ref (a volume-balance decoupling: it
// cancels the saturation derivative of the accumulation); Pi_r applies the
// same weights to the residual and Pi_p injects the pressure correction into
// the P component of every cell (well unknowns untouched).
//
// The multigrid uses 2x2x2 (or 2x2 / 2) aggregates of the structured grid with
// piecewise-constant transfer, so each Galerkin coarse operator is again a
// 7-point stencil; red-black Gauss-Seidel smoothing; a dense inverse on the
// coarsest level (at most 64 cells).
#pragma once

#include <vector>

#include "pf_internal.cuh"

namespace pf {

struct CprLevel {
  int nx = 0, ny = 0, nz = 0;
  long long n = 0;
  void* A = nullptr;     // [7][n] stencil (slot order of SL_*), type T
  void* dinv = nullptr;  // [n] 1 / diagonal
  void* x = nullptr;     // [n]
  void* b = nullptr;     // [n]
};

struct CprData {
  bool ready = false;
  int nlev = 0;
  int pre = 1, post = 1, cycle_gamma = 1, coarse_limit = 64;
  int cpre = 1, cpost = 1;      // sweeps on the levels below the finest
  int block_rbgs0 = 256, block_stage2 = 256;  // launch shapes of the finest smoother and stage 2
  bool ilu = false;             // first stage: red-black block ILU(0) instead of block-Jacobi
  int ilu_fused = 1;            // ILU solve in two launches (1) or three (0); same results
  IluCompact ilu_cp;            // compact per-colour block copies read by the ILU sweeps
  bool rb_copy = false;         // the finest smoother reads per-colour copies (rb_cp) of its stencil
  void* rb_cp[2] = {nullptr, nullptr};  // red, black: [6 off-diagonal slots + 1/diag][colour slots]
  long long block_cells = 512;  // levels of at most this many cells run in one thread block
  long long cluster_cells = 0;  // larger levels up to this size run in one thread-block cluster (0: none)
  double w_o = 0.0, w_w = 0.0;
  std::vector<CprLevel> lev;
  void* coarse_inv = nullptr;   // [nc][nc] dense inverse of the coarsest matrix
  int* coarse_status = nullptr; // device flag: 1 if a zero pivot was met
};

// One launch of stage 2 with a given block size (used by the launch-shape
// tuner; the values computed are scratch).
void cpr_time_stage2(CprData& c, const Grid& g, const Wells& w, bool mixed, const void* J, const void* Bw,
                     const double* v, double* tmp, int block, cudaStream_t st);

// Lays out the CPR arrays in the arena (base == nullptr: sizing only).
void cpr_carve(CprData& c, const Grid& g, bool mixed, size_t& off, char* base);
pf_status cpr_init(CprData& c, const Grid& g, bool mixed, const pf_solver_opts& o, cudaStream_t st);
// the stage-2 weights w_o = 1 / rho_o,ref and w_w = 1 / rho_w,ref (the ILU(0)
// set-up needs them before cpr_setup, for the pressure rows it precomputes)
void cpr_weights(CprData& c, const Phys& ph);
void cpr_setup(CprData& c, const Grid& g, const Phys& ph, const double* phi_r, const Wells& w, bool mixed,
               const void* J, const void* Bw, const void* Dw, cudaStream_t st, int* launches);
// z = M^{-1} v.  Mixed precision runs every stage in FP32 from vf, the FP32
// copy of v (tmp then holds an FP32 vector), and also writes an FP32 copy of z
// to zf_out (may be null); the FP64 form reads v (vf unused).
void cpr_apply(CprData& c, const Grid& g, const Wells& w, bool mixed, const void* J, const void* Bw, const void* Cw,
               const void* Dw, const void* Dinv, const void* Dwinv, const double* v, const float* vf, double* z,
               double* tmp, float* zf_out, cudaStream_t st, int* launches);

}  // namespace pf
