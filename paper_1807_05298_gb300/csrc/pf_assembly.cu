// Residual and 3x3 block-Jacobian assembly of the water/oil/polymer model.
//
// Equations (arXiv 1807.05298): porosity law Sec. 2.1; phase mass
// conservation with Darcy flux and gravity Sec. 2.2; polymer conservation,
// permeability reduction R_k, equilibrium adsorption, Todd-Longstaff
// viscosities and mixing rules, inaccessible pore volume Sec. 2.3; wells
// (perforation rate, hydrostatic wellbore, BHP / rate constraints) Sec. 2.4;
// backward Euler Sec. 3.1; two-point transmissibility with harmonic geometry and
// permeability, pore-volume weighted rho and mu, upstream k_r Sec. 3.2.
//
// Kernel sequence per assembly (all deterministic, no atomics):
//   cell_props  one thread per cell: properties and their derivatives into a
//               scratch (values FP64, derivatives DT), accumulation masses into
//               R and their derivatives into the diagonal block;
//   face_flux   one thread per cell for its +x, +y, +z faces: phase potentials,
//               upstream selection, fluxes into a face buffer, and the two
//               off-diagonal blocks of the face written straight into J;
//   gather      one thread per cell: residual flux sum in the fixed order
//               -x, +x, -y, +y, -z, +z and the flux part of the diagonal block
//               as minus the sum of the column's off-diagonal blocks (a flux
//               depends only on its two cells, so dF/dx_L = J[H][L] / dt);
//   wells       one warp per well: perforation rates, their derivatives into
//               the perforated cell rows and the well border, the well row.
#include <math.h>

#include "pf_internal.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// cell properties and accumulation
// ---------------------------------------------------------------------------

// Values in FP64 (they build the residual); derivatives in the Jacobian's
// type DT (FP64, or FP32 in mixed precision, where the derivative arithmetic
// runs in FP32 from the FP64 values rounded once).
template <typename DT>
struct CellEval {
  double phi, rho_o, rho_w, Pw, krw, kro, Rk, mu_we, mu_pe, ads;
  DT dphi, drho_o, drho_wP, drho_wS, dPw_S, dkrw, dkro, dRk, dmu_we, dmu_pe, dads;
};

__device__ __forceinline__ double powi_or_pow(double b, double e) {
  if (e == 2.0) return b * b;
  if (e == 1.0) return b;
  return pow(b, e);
}
__device__ __forceinline__ float powi_or_pow(float b, float e) {
  if (e == 2.0f) return b * b;
  if (e == 1.0f) return b;
  return powf(b, e);
}

// Segment of a strictly increasing abscissa table: k with x[k] <= u < x[k+1],
// -1 below the first knot, K - 1 from the last knot on (binary search).
__device__ __forceinline__ int table_segment(const double* __restrict__ x, int K, double u) {
  if (u < __ldg(x)) return -1;
  if (u >= __ldg(x + K - 1)) return K - 1;
  int lo = 0, hi = K - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(x + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Value and derivative of column col (1-based) of a structure-of-arrays
// table with `cols` value columns: the segment's line inside the table, the
// end value with derivative 0 outside it.
__device__ __forceinline__ void table_eval(const double* __restrict__ T, int K, int cols, int col, int k, double u,
                                           double& v, double& d) {
  const double* y = T + (size_t)col * K;
  if (k < 0) { v = __ldg(y); d = 0.0; return; }
  if (k >= K - 1) { v = __ldg(y + K - 1); d = 0.0; return; }
  const double sl = __ldg(T + (size_t)(cols + col) * K + k);
  v = (u - __ldg(T + k)) * sl + __ldg(y + k);
  d = sl;
}

template <typename DT>
__device__ __forceinline__ void eval_cell(const Phys& ph, double phi_r, double P, double S, double C,
                                          CellEval<DT>& c) {
  c.phi = phi_r + ph.c_r * (P - ph.p_r);
  c.dphi = (DT)ph.c_r;
  c.rho_o = ph.rho_o * (1.0 + ph.c_o * (P - ph.p_ref));
  c.drho_o = (DT)ph.rho_o * (DT)ph.c_o;
  double pc = 0.0;
  DT dpc = 0;
  if (ph.n_sat > 0) {  // tabulated k_rw, k_ro, P_c of S_w
    const int k = table_segment(ph.sat, ph.n_sat, S);
    double d1, d2, d3;
    table_eval(ph.sat, ph.n_sat, 3, 1, k, S, c.krw, d1);
    table_eval(ph.sat, ph.n_sat, 3, 2, k, S, c.kro, d2);
    table_eval(ph.sat, ph.n_sat, 3, 3, k, S, pc, d3);
    c.dkrw = (DT)d1;
    c.dkro = (DT)d2;
    dpc = (DT)d3;
  } else {
    // normalised saturation, clipped; derivative of the interior formula on [0, 1]
    double sn = (S - ph.swc) * ph.inv_den, dsn = ph.inv_den;
    if (sn < 0.0) { sn = 0.0; dsn = 0.0; }
    if (sn > 1.0) { sn = 1.0; dsn = 0.0; }
    const double so = 1.0 - sn;
    c.krw = ph.krw_max * powi_or_pow(sn, ph.nw);
    c.dkrw = (sn == 0.0 && ph.nw > 1.0)
                 ? (DT)0
                 : (DT)ph.krw_max * (DT)ph.nw * powi_or_pow((DT)sn, (DT)(ph.nw - 1.0)) * (DT)dsn;
    c.kro = ph.kro_max * powi_or_pow(so, ph.no);
    c.dkro = (so == 0.0 && ph.no > 1.0)
                 ? (DT)0
                 : -(DT)ph.kro_max * (DT)ph.no * powi_or_pow((DT)so, (DT)(ph.no - 1.0)) * (DT)dsn;
    if (ph.pc_e != 0.0) {
      pc = ph.pc_e * powi_or_pow(so, ph.pc_n);
      dpc = (so == 0.0 && ph.pc_n > 1.0)
                ? (DT)0
                : -(DT)ph.pc_e * (DT)ph.pc_n * powi_or_pow((DT)so, (DT)(ph.pc_n - 1.0)) * (DT)dsn;
    }
  }
  c.Pw = P - pc;
  c.dPw_S = -dpc;
  c.rho_w = ph.rho_w * (1.0 + ph.c_w * (c.Pw - ph.p_ref));
  c.drho_wP = (DT)ph.rho_w * (DT)ph.c_w;
  c.drho_wS = (DT)ph.rho_w * (DT)ph.c_w * c.dPw_S;
  const double beta = C * ph.inv_c_ref;
  double mu_m;
  DT dmu_m;
  if (ph.n_poly > 0) {  // tabulated A_d(C) and water viscosity multiplier
    const int k = table_segment(ph.poly, ph.n_poly, C);
    double mult, dmult, dads;
    table_eval(ph.poly, ph.n_poly, 2, 1, k, C, mult, dmult);
    table_eval(ph.poly, ph.n_poly, 2, 2, k, C, c.ads, dads);
    c.dads = (DT)dads;
    mu_m = mult * ph.mu_w;
    dmu_m = (DT)dmult * (DT)ph.mu_w;
  } else {
    // Langmuir adsorption (one reciprocal: FP64 division is costly on this part)
    const double rden = 1.0 / (1.0 + ph.ads_b * C);
    c.ads = ph.ads_a * C * rden;
    c.dads = (DT)ph.ads_a * (DT)rden * (DT)rden;
  }
  // permeability reduction
  c.Rk = 1.0 + ph.rk_coef * c.ads;
  c.dRk = (DT)ph.rk_coef * c.dads;
  // mixing rule (the table already gave mu_m)
  if (ph.n_poly > 0) {
    // mu_m, dmu_m from the viscosity multiplier above
  } else if (ph.mixing == PF_MIX_NONLINEAR) {
    mu_m = exp(ph.ln_mu_w + beta * ph.ln_mu_ratio);
    dmu_m = (DT)mu_m * (DT)ph.ln_mu_ratio * (DT)ph.inv_c_ref;
  } else {
    mu_m = ph.mu_w + beta * (ph.mu_p0 - ph.mu_w);
    dmu_m = (DT)(ph.mu_p0 - ph.mu_w) * (DT)ph.inv_c_ref;
  }
  // Todd-Longstaff effective viscosities
  double alpha = beta;
  DT dalpha = (DT)ph.inv_c_ref;
  if (alpha < 0.0) { alpha = 0.0; dalpha = 0; }
  if (alpha > 1.0) { alpha = 1.0; dalpha = 0; }
  // 1/mu_w,e = alpha/mu_p,e + (1-alpha)/mu_w,partial, with one reciprocal per
  // viscosity.  With omega = 1 both are mu_m, so 1/mu_w,e = 1/mu_m: the
  // effective viscosities are the mixture's, exactly (no reciprocal at all)
  if (ph.omega == 1.0) {
    c.mu_we = mu_m;
    c.dmu_we = dmu_m;
    c.mu_pe = mu_m;
    c.dmu_pe = dmu_m;
    return;
  }
  double mu_pe, mu_wp, rpe, rwp;
  DT dmu_pe, dmu_wp;
  {
    const double mo = pow(mu_m, ph.omega);
    const DT dmo = (DT)ph.omega * (DT)mo / (DT)mu_m * dmu_m;
    mu_pe = mo * ph.mu_p0_pow; dmu_pe = dmo * (DT)ph.mu_p0_pow;
    mu_wp = mo * ph.mu_w_pow; dmu_wp = dmo * (DT)ph.mu_w_pow;
    rpe = 1.0 / mu_pe;
    rwp = 1.0 / mu_wp;
  }
  const double inv = alpha * rpe + (1.0 - alpha) * rwp;
  const DT a = (DT)alpha, p = (DT)rpe, w = (DT)rwp;
  const DT dinv = dalpha * p - a * dmu_pe * p * p - dalpha * w - ((DT)1 - a) * dmu_wp * w * w;
  c.mu_we = 1.0 / inv;
  c.dmu_we = -dinv * (DT)c.mu_we * (DT)c.mu_we;
  c.mu_pe = mu_pe;
  c.dmu_pe = dmu_pe;
}

// One cell of the property kernel (mode as in launch_cell_props).
template <typename DT>
__device__ __forceinline__ void cell_props_at(const Grid& g, const Phys& ph, const double* __restrict__ phi_r,
                                              const double* __restrict__ x, double* __restrict__ pv,
                                              DT* __restrict__ pd, const double* __restrict__ Mold,
                                              double* __restrict__ R, DT* __restrict__ J,
                                              double* __restrict__ Mold_out, int mode, long long i) {
  const long long n = g.n;
  {
    const double P = x[3 * i], S = x[3 * i + 1], C = x[3 * i + 2];
    CellEval<DT> c;
    eval_cell<DT>(ph, phi_r[i], P, S, C, c);
    const double V = g.V;
    // accumulation masses (oil, water, polymer)
    const double Mo = V * c.phi * c.rho_o * (1.0 - S);
    const double Mw = V * c.phi * c.rho_w * S;
    const double k1 = V * (1.0 - ph.ipv) * ph.inv_rho_w;
    const double Mp = k1 * c.phi * S * c.rho_w * C + V * (1.0 - c.phi) * c.ads;
    if (mode == 2) {  // values only, for well totals
      pv[PV_RHO_O * n + i] = c.rho_o;
      pv[PV_RHO_W * n + i] = c.rho_w;
      pv[PV_PW * n + i] = c.Pw;
      pv[PV_KRW * n + i] = c.krw;
      pv[PV_KRO * n + i] = c.kro;
      pv[PV_RK * n + i] = c.Rk;
      pv[PV_MUWE * n + i] = c.mu_we;
      pv[PV_MUPE * n + i] = c.mu_pe;
      return;
    }
    if (mode == 1) {
      Mold_out[3 * i] = Mo;
      Mold_out[3 * i + 1] = Mw;
      Mold_out[3 * i + 2] = Mp;
      pv[PV_RHO_O * n + i] = c.rho_o;
      pv[PV_RHO_W * n + i] = c.rho_w;
      pv[PV_KRW * n + i] = c.krw;
      pv[PV_KRO * n + i] = c.kro;
      pv[PV_RK * n + i] = c.Rk;
      pv[PV_MUWE * n + i] = c.mu_we;
      return;
    }
    pv[PV_RHO_O * n + i] = c.rho_o;
    pv[PV_RHO_W * n + i] = c.rho_w;
    pv[PV_PW * n + i] = c.Pw;
    pv[PV_KRW * n + i] = c.krw;
    pv[PV_KRO * n + i] = c.kro;
    pv[PV_RK * n + i] = c.Rk;
    pv[PV_MUWE * n + i] = c.mu_we;
    pv[PV_MUPE * n + i] = c.mu_pe;
    pd[PD_RHO_O * n + i] = c.drho_o;
    pd[PD_RHO_WP * n + i] = c.drho_wP;
    pd[PD_RHO_WS * n + i] = c.drho_wS;
    pd[PD_PW_S * n + i] = c.dPw_S;
    pd[PD_KRW * n + i] = c.dkrw;
    pd[PD_KRO * n + i] = c.dkro;
    pd[PD_RK * n + i] = c.dRk;
    pd[PD_MUWE * n + i] = c.dmu_we;
    pd[PD_MUPE * n + i] = c.dmu_pe;
    R[3 * i] = Mo - Mold[3 * i];
    R[3 * i + 1] = Mw - Mold[3 * i + 1];
    R[3 * i + 2] = Mp - Mold[3 * i + 2];
    // d(M)/d(P, S, C): rows oil, water, polymer
    DT* Jd = J + (size_t)SL_D * 9 * n;
    // in DT: the FP64 values rounded once, then the derivative arithmetic
    const DT Vd = (DT)V, k1d = (DT)k1, Sd = (DT)S, Cd = (DT)C, phid = (DT)c.phi;
    const DT rho_od = (DT)c.rho_o, rho_wd = (DT)c.rho_w, adsd = (DT)c.ads;
    const DT dMoP = Vd * (c.dphi * rho_od + phid * c.drho_o) * ((DT)1 - Sd);
    const DT dMoS = -Vd * phid * rho_od;
    const DT dMwP = Vd * (c.dphi * rho_wd + phid * c.drho_wP) * Sd;
    const DT dMwS = Vd * phid * (c.drho_wS * Sd + rho_wd);
    const DT dMpP = k1d * Sd * Cd * (c.dphi * rho_wd + phid * c.drho_wP) - Vd * c.dphi * adsd;
    const DT dMpS = k1d * Cd * phid * (rho_wd + Sd * c.drho_wS);
    const DT dMpC = k1d * phid * Sd * rho_wd + Vd * ((DT)1 - phid) * c.dads;
    Jd[0 * n + i] = dMoP;
    Jd[1 * n + i] = dMoS;
    Jd[2 * n + i] = (DT)0;
    Jd[3 * n + i] = dMwP;
    Jd[4 * n + i] = dMwS;
    Jd[5 * n + i] = (DT)0;
    Jd[6 * n + i] = dMpP;
    Jd[7 * n + i] = dMpS;
    Jd[8 * n + i] = dMpC;
  }
}

// modes 1 and 2 (the old masses at the start of a step, the property values
// for the well totals); mode 0 runs in the assembly kernel k_cell_props
template <typename DT>
__global__ void __launch_bounds__(256) k_cell_values(Grid g, Phys ph, const double* __restrict__ phi_r,
                                                     const double* __restrict__ x, double* __restrict__ pv,
                                                     DT* __restrict__ pd, const double* __restrict__ Mold,
                                                     double* __restrict__ R, DT* __restrict__ J,
                                                     double* __restrict__ Mold_out, int mode) {
  PF_PDL_ENTRY();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n;
       i += (long long)gridDim.x * blockDim.x)
    cell_props_at<DT>(g, ph, phi_r, x, pv, pd, Mold, R, J, Mold_out, mode, i);
}

// ---------------------------------------------------------------------------
// face fluxes with upstream weighting
// ---------------------------------------------------------------------------

struct SideV {
  double P, C, rho_o, rho_w, Pw, krw, kro, Rk, mu_we, mu_pe;
};
template <typename DT>
struct SideD {
  DT drho_o, drho_wP, drho_wS, dPw_S, dkrw, dkro, dRk, dmu_we, dmu_pe;
};

template <typename DT>
__device__ __forceinline__ void load_side(long long i, long long n, const double* __restrict__ x,
                                          const double* __restrict__ pv, const DT* __restrict__ pd,
                                          SideV& v, SideD<DT>& d) {
  v.P = x[3 * i];
  v.C = x[3 * i + 2];
  v.rho_o = pv[PV_RHO_O * n + i];
  v.rho_w = pv[PV_RHO_W * n + i];
  v.Pw = pv[PV_PW * n + i];
  v.krw = pv[PV_KRW * n + i];
  v.kro = pv[PV_KRO * n + i];
  v.Rk = pv[PV_RK * n + i];
  v.mu_we = pv[PV_MUWE * n + i];
  v.mu_pe = pv[PV_MUPE * n + i];
  d.drho_o = pd[PD_RHO_O * n + i];
  d.drho_wP = pd[PD_RHO_WP * n + i];
  d.drho_wS = pd[PD_RHO_WS * n + i];
  d.dPw_S = pd[PD_PW_S * n + i];
  d.dkrw = pd[PD_KRW * n + i];
  d.dkro = pd[PD_KRO * n + i];
  d.dRk = pd[PD_RK * n + i];
  d.dmu_we = pd[PD_MUWE * n + i];
  d.dmu_pe = pd[PD_MUPE * n + i];
}

// Mass fluxes F (oil, water, polymer) from H into L across one face and their
// derivatives dL = dF/d(P_L, S_L, C_L), dH = dF/d(P_H, S_H, C_H), row-major
// 3x3 (rows oil, water, polymer).  gdz = g (Z_H - Z_L).  Every output is
// linear in the transmissibility T, so a caller that passes T dt gets the
// time-step integrals dt F and dt dF directly.
template <typename DT>
__device__ __forceinline__ void face_flux(const Phys& ph, double T, double gdz, double wL,
                                          const SideV& a, const SideD<DT>& da, const SideV& b,
                                          const SideD<DT>& db, double F[3], DT dL[9], DT dH[9]) {
  const double wH = 1.0 - wL;
  // oil phase
  const double rho_o = wL * a.rho_o + wH * b.rho_o;
  const double dPo = (b.P - a.P) - rho_o * gdz;
  const bool upHo = dPo >= 0.0;
  const double kro = upHo ? b.kro : a.kro;
  const DT dkro = upHo ? db.dkro : da.dkro;
  const double To = T * ph.inv_mu_o;
  F[0] = To * kro * rho_o * dPo;
  {
    // d(rho dPhi)/dP_L = wL rho'_L (dPhi - g dz rho) - rho, and the H side with
    // +rho: the averaged density enters dPhi once more through g dz
    const DT Tk = (DT)(To * kro);
    const DT qo = (DT)dPo - (DT)gdz * (DT)rho_o;
    dL[0] = Tk * ((DT)wL * da.drho_o * qo - (DT)rho_o);
    dH[0] = Tk * ((DT)wH * db.drho_o * qo + (DT)rho_o);
    const DT dS = (DT)To * dkro * (DT)(rho_o * dPo);
    dL[1] = upHo ? (DT)0 : dS;
    dH[1] = upHo ? dS : (DT)0;
    dL[2] = (DT)0;
    dH[2] = (DT)0;
  }
  // water phase (and polymer carried by it)
  const double rho_w = wL * a.rho_w + wH * b.rho_w;
  const double dPw = (b.Pw - a.Pw) - rho_w * gdz;
  const bool upHw = dPw >= 0.0;
  const double krw = upHw ? b.krw : a.krw;
  const double Rk = upHw ? b.Rk : a.Rk;
  const double Cu = upHw ? b.C : a.C;
  const DT dkrw = upHw ? db.dkrw : da.dkrw;
  const DT dRk = upHw ? db.dRk : da.dRk;
  const double mu_we = wL * a.mu_we + wH * b.mu_we;
  const double mu_pe = wL * a.mu_pe + wH * b.mu_pe;
  const double A = rho_w * dPw;
  // two FP64 divisions per face; with omega = 1 (mu_p,e = mu_w,e = mu_m in
  // every cell, so on every face) one, and the polymer flux and its
  // derivatives are the water ones times c / rho_w,ref; 1/mu and 1/R_k follow
  // by multiplication
  const bool tl1 = ph.omega == 1.0;  // the same for every thread
  const double irw = 1.0 / (Rk * mu_we), irp = tl1 ? irw : 1.0 / (Rk * mu_pe);
  const double inv_mu_we = Rk * irw, inv_mu_pe = Rk * irp, inv_Rk = mu_we * irw;
  const double mw = krw * irw;
  const double mp = krw * irp;
  const double cf = Cu * ph.inv_rho_w;
  F[1] = T * mw * A;
  F[2] = tl1 ? F[1] * cf : T * mp * A * cf;
  // dA/d(P_L, S_L, P_H, S_H), A = rho_w dPhi_w, with qw = dPhi_w - g dz rho_w
  // as for the oil phase
  const DT qw = (DT)dPw - (DT)gdz * (DT)rho_w;
  const DT dA_PL = (DT)wL * da.drho_wP * qw - (DT)rho_w;
  const DT dA_SL = (DT)wL * da.drho_wS * qw - (DT)rho_w * da.dPw_S;
  const DT dA_PH = (DT)wH * db.drho_wP * qw + (DT)rho_w;
  const DT dA_SH = (DT)wH * db.drho_wS * qw + (DT)rho_w * db.dPw_S;
  const DT Tmw = (DT)(T * mw), Tmp = (DT)(T * mp * cf);
  // pressure and saturation columns through A
  dL[3] = Tmw * dA_PL;
  dH[3] = Tmw * dA_PH;
  dL[4] = Tmw * dA_SL;
  dH[4] = Tmw * dA_SH;
  dL[6] = Tmp * dA_PL;
  dH[6] = Tmp * dA_PH;
  dL[7] = Tmp * dA_SL;
  dH[7] = Tmp * dA_SH;
  // concentration columns through the averaged viscosities
  const DT TA = (DT)(T * A);
  const DT cw = -TA * (DT)(mw * inv_mu_we);
  dL[5] = cw * (DT)wL * da.dmu_we;
  dH[5] = cw * (DT)wH * db.dmu_we;
  // upstream cell: k_rw (saturation), R_k and the carried concentration
  const DT dFw_S = TA * dkrw * (DT)irw;
  const DT dFw_C = -TA * (DT)(mw * inv_Rk) * dRk;
  DT dFp_S, dFp_C;
  if (tl1) {
    const DT cfd = (DT)cf;
    dL[8] = dL[5] * cfd;
    dH[8] = dH[5] * cfd;
    dFp_S = dFw_S * cfd;
    dFp_C = cfd * dFw_C + TA * (DT)(mw * ph.inv_rho_w);
  } else {
    const DT cp = -TA * (DT)(mp * cf * inv_mu_pe);
    dL[8] = cp * (DT)wL * da.dmu_pe;
    dH[8] = cp * (DT)wH * db.dmu_pe;
    dFp_S = TA * (DT)cf * dkrw * (DT)irp;
    dFp_C = TA * ((DT)(mp * cf * inv_Rk) * (-dRk) + (DT)(mp * ph.inv_rho_w));
  }
  if (upHw) {
    dH[4] += dFw_S; dH[7] += dFp_S; dH[5] += dFw_C; dH[8] += dFp_C;
  } else {
    dL[4] += dFw_S; dL[7] += dFp_S; dL[5] += dFw_C; dL[8] += dFp_C;
  }
}

// The three faces of cell i towards +x, +y, +z (one thread per cell).
template <typename DT>
__device__ __forceinline__ void face_flux_at(const Grid& g, const Phys& ph, const double* __restrict__ wL3,
                                             const double* __restrict__ T3, const double* __restrict__ x,
                                             const double* __restrict__ pv, const DT* __restrict__ pd, double dt,
                                             DT* __restrict__ J, double* __restrict__ Fbuf, long long i) {
  const long long n = g.n;
  {
    const unsigned int ui = (unsigned int)i, nxy = (unsigned int)g.nxy, nxu = (unsigned int)g.nx;
    const long long k = ui / nxy;  // 32-bit division: fewer than 2^31 cells
    const unsigned int rem = ui - (unsigned int)k * nxy;
    const long long j = rem / nxu;
    const long long ii = rem - (unsigned int)j * nxu;
    SideV a; SideD<DT> da;
    load_side<DT>(i, n, x, pv, pd, a, da);
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      bool has;
      long long s;
      double gdz = 0.0;
      if (d == 0) { has = ii + 1 < g.nx; s = 1; }
      else if (d == 1) { has = j + 1 < g.ny; s = g.nx; }
      else { has = k + 1 < g.nz; s = g.nxy; gdz = ph.g * g.dz; }
      double* Fd = Fbuf + (size_t)d * 3 * n;
      if (!has) {
        Fd[i] = 0.0; Fd[n + i] = 0.0; Fd[2 * n + i] = 0.0;
        continue;
      }
      const long long h = i + s;
      SideV b; SideD<DT> db;
      load_side<DT>(h, n, x, pv, pd, b, db);
      const double wL = wL3[(size_t)d * n + i];
      double F[3]; DT dL[9], dH[9];
      // with T dt: F and its derivatives come out as dt F and dt dF (one
      // multiply per face instead of one per Jacobian entry and flux)
      face_flux<DT>(ph, T3[(size_t)d * n + i] * dt, gdz, wL, a, da, b, db, F, dL, dH);
      Fd[i] = F[0]; Fd[n + i] = F[1]; Fd[2 * n + i] = F[2];
      // row L, column H: -dt dF/dx_H  (slot +d of row i)
      DT* Jp = J + (size_t)(SL_XP + 2 * d) * 9 * n;
      // row H, column L: +dt dF/dx_L  (slot -d of row h)
      DT* Jm = J + (size_t)(SL_XM + 2 * d) * 9 * n;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        Jp[(size_t)e * n + i] = -dH[e];
        Jm[(size_t)e * n + h] = dL[e];
      }
    }
    // slots that leave the grid on the minus side are zero
    if (ii == 0) { DT* Jm = J + (size_t)SL_XM * 9 * n; for (int e = 0; e < 9; ++e) Jm[(size_t)e * n + i] = (DT)0; }
    if (j == 0) { DT* Jm = J + (size_t)SL_YM * 9 * n; for (int e = 0; e < 9; ++e) Jm[(size_t)e * n + i] = (DT)0; }
    if (k == 0) { DT* Jm = J + (size_t)SL_ZM * 9 * n; for (int e = 0; e < 9; ++e) Jm[(size_t)e * n + i] = (DT)0; }
    if (ii + 1 == g.nx) { DT* Jp = J + (size_t)SL_XP * 9 * n; for (int e = 0; e < 9; ++e) Jp[(size_t)e * n + i] = (DT)0; }
    if (j + 1 == g.ny) { DT* Jp = J + (size_t)SL_YP * 9 * n; for (int e = 0; e < 9; ++e) Jp[(size_t)e * n + i] = (DT)0; }
    if (k + 1 == g.nz) { DT* Jp = J + (size_t)SL_ZP * 9 * n; for (int e = 0; e < 9; ++e) Jp[(size_t)e * n + i] = (DT)0; }
  }
}


// ---------------------------------------------------------------------------
// gather: residual flux sums and the flux part of the diagonal block
// ---------------------------------------------------------------------------

// Row i of the gather.
template <typename DT>
__device__ __forceinline__ void gather_at(const Grid& g, const double* __restrict__ Fbuf, double* __restrict__ R,
                                          DT* __restrict__ J, long long i) {
  const long long n = g.n;
  {
    const unsigned int ui = (unsigned int)i, nxy = (unsigned int)g.nxy, nxu = (unsigned int)g.nx;
    const long long k = ui / nxy;  // 32-bit division: fewer than 2^31 cells
    const unsigned int rem = ui - (unsigned int)k * nxy;
    const long long j = rem / nxu;
    const long long ii = rem - (unsigned int)j * nxu;
    double fs[3] = {0.0, 0.0, 0.0};
    DT dsum[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) dsum[e] = (DT)0;
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      const long long s = d == 0 ? 1 : (d == 1 ? g.nx : g.nxy);
      const bool has_m = d == 0 ? ii > 0 : (d == 1 ? j > 0 : k > 0);
      const bool has_p = d == 0 ? ii + 1 < g.nx : (d == 1 ? j + 1 < g.ny : k + 1 < g.nz);
      const double* Fd = Fbuf + (size_t)d * 3 * n;
      if (has_m) {  // face (i - s, i): i is H; R_H += dt F; diag += +dt dF/dx_H = -J[i-s][+d]
        const long long l = i - s;
        fs[0] -= Fd[l]; fs[1] -= Fd[n + l]; fs[2] -= Fd[2 * n + l];
        const DT* Jp = J + (size_t)(SL_XP + 2 * d) * 9 * n;
#pragma unroll
        for (int e = 0; e < 9; ++e)
          if (e != 2) dsum[e] += Jp[(size_t)e * n + l];  // (oil, C) is structurally zero
      }
      if (has_p) {  // face (i, i + s): i is L; R_L -= dt F; diag += -dt dF/dx_L = -J[i+s][-d]
        const long long h = i + s;
        fs[0] += Fd[i]; fs[1] += Fd[n + i]; fs[2] += Fd[2 * n + i];
        const DT* Jm = J + (size_t)(SL_XM + 2 * d) * 9 * n;
#pragma unroll
        for (int e = 0; e < 9; ++e)
          if (e != 2) dsum[e] += Jm[(size_t)e * n + h];
      }
    }
    R[3 * i] -= fs[0];  // Fbuf holds dt F
    R[3 * i + 1] -= fs[1];
    R[3 * i + 2] -= fs[2];
    DT* Jd = J + (size_t)SL_D * 9 * n;
#pragma unroll
    for (int e = 0; e < 9; ++e) Jd[(size_t)e * n + i] -= dsum[e];
  }
}



// ---------------------------------------------------------------------------
// wells: one warp per well
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Well wi, one warp (lane 0..31).
template <typename DT>
__device__ __forceinline__ void wells_at(const Grid& g, const Phys& ph, const Wells& w, const double* __restrict__ x,
                                         const double* __restrict__ pv, const DT* __restrict__ pd, double dt,
                                         double* __restrict__ R, DT* __restrict__ J, DT* __restrict__ Bw,
                                         DT* __restrict__ Cw, DT* __restrict__ Dw, int wi, int lane) {
  const long long n = g.n;
  const long long npf = w.npf;
  const double Pb = x[3 * n + wi];
  const double gam = w.gamma[wi];
  const int kind = w.kind[wi];
  const int ctrl = w.ctrl[wi];
  const double sw = w.sw[wi], so = w.so[wi];
  const double cinj = w.cinj[wi];
  double sum_q = 0.0, sum_dPb = 0.0;
  DT* Jd = J + (size_t)SL_D * 9 * n;
  for (int m = w.ptr[wi] + lane; m < w.ptr[wi + 1]; m += 32) {
    const long long c = w.cell[m];
    const double WI = w.wi[m];
    const double P = x[3 * c], C = x[3 * c + 2];
    const double rho_o = pv[PV_RHO_O * n + c], rho_w = pv[PV_RHO_W * n + c];
    const double Pw = pv[PV_PW * n + c];
    const double krw = pv[PV_KRW * n + c], kro = pv[PV_KRO * n + c];
    const double Rk = pv[PV_RK * n + c], mu_we = pv[PV_MUWE * n + c];
    const double drho_o = pd[PD_RHO_O * n + c], drho_wP = pd[PD_RHO_WP * n + c];
    const double drho_wS = pd[PD_RHO_WS * n + c], dPw_S = pd[PD_PW_S * n + c];
    const double dkrw = pd[PD_KRW * n + c], dkro = pd[PD_KRO * n + c];
    const double dRk = pd[PD_RK * n + c], dmu_we = pd[PD_MUWE * n + c];
    const double Pbm = Pb + gam * w.dzb[m];
    // water mobility and derivatives (S, C)
    const double lw = krw / (Rk * mu_we);
    const double dlw_S = dkrw / (Rk * mu_we);
    const double dlw_C = -lw * (dRk / Rk + dmu_we / mu_we);
    const double lo = kro / ph.mu_o;
    const double dlo_S = dkro / ph.mu_o;
    const double dw = Pbm - Pw;  // water drawdown
    double qw, qo, qp;
    double dqw[4], dqo[4], dqp[4];  // d/d(P, S, C, Pb)
    if (kind == PF_WELL_INJECTOR) {
      const double lt = lw + lo, dlt_S = dlw_S + dlo_S, dlt_C = dlw_C;
      qw = WI * lt * rho_w * dw;
      dqw[0] = WI * lt * (drho_wP * dw - rho_w);
      dqw[1] = WI * (dlt_S * rho_w * dw + lt * drho_wS * dw - lt * rho_w * dPw_S);
      dqw[2] = WI * dlt_C * rho_w * dw;
      dqw[3] = WI * lt * rho_w;
      qo = 0.0;
      dqo[0] = dqo[1] = dqo[2] = dqo[3] = 0.0;
      const double cf = cinj * ph.inv_rho_w;
      qp = qw * cf;
      for (int t = 0; t < 4; ++t) dqp[t] = dqw[t] * cf;
    } else {
      qw = WI * lw * rho_w * dw;
      dqw[0] = WI * lw * (drho_wP * dw - rho_w);
      dqw[1] = WI * (dlw_S * rho_w * dw + lw * drho_wS * dw - lw * rho_w * dPw_S);
      dqw[2] = WI * dlw_C * rho_w * dw;
      dqw[3] = WI * lw * rho_w;
      const double dox = Pbm - P;
      qo = WI * lo * rho_o * dox;
      dqo[0] = WI * lo * (drho_o * dox - rho_o);
      dqo[1] = WI * dlo_S * rho_o * dox;
      dqo[2] = 0.0;
      dqo[3] = WI * lo * rho_o;
      const double cf = C * ph.inv_rho_w;
      qp = qw * cf;
      dqp[0] = dqw[0] * cf;
      dqp[1] = dqw[1] * cf;
      dqp[2] = dqw[2] * cf + qw * ph.inv_rho_w;
      dqp[3] = dqw[3] * cf;
    }
    // cell rows (a cell holds at most one perforation: no race)
    R[3 * c] -= dt * qo;
    R[3 * c + 1] -= dt * qw;
    R[3 * c + 2] -= dt * qp;
    for (int b = 0; b < 3; ++b) {
      Jd[(size_t)(0 + b) * n + c] -= (DT)(dt * dqo[b]);
      Jd[(size_t)(3 + b) * n + c] -= (DT)(dt * dqw[b]);
      Jd[(size_t)(6 + b) * n + c] -= (DT)(dt * dqp[b]);
    }
    Bw[0 * npf + m] = (DT)(-dt * dqo[3]);
    Bw[1 * npf + m] = (DT)(-dt * dqw[3]);
    Bw[2 * npf + m] = (DT)(-dt * dqp[3]);
    if (ctrl == PF_CTRL_BHP) {
      Cw[0 * npf + m] = (DT)0; Cw[1 * npf + m] = (DT)0; Cw[2 * npf + m] = (DT)0;
    } else {
      for (int b = 0; b < 3; ++b) Cw[(size_t)b * npf + m] = (DT)(dt * (sw * dqw[b] + so * dqo[b]));
      sum_q += sw * qw + so * qo;
      sum_dPb += sw * dqw[3] + so * dqo[3];
    }
  }
  sum_q = warp_sum(sum_q);
  sum_dPb = warp_sum(sum_dPb);
  if (lane == 0) {
    if (ctrl == PF_CTRL_BHP) {
      R[3 * n + wi] = dt * w.W[wi] * (Pb - w.target[wi]);
      Dw[wi] = (DT)(dt * w.W[wi]);
    } else {
      R[3 * n + wi] = dt * (sum_q - w.target[wi]);
      Dw[wi] = (DT)(dt * sum_dPb);
    }
  }
}



// Lagged wellbore unit weight (frozen over a step): rho_w(P_b) g for an
// injector, the mobility-weighted mixture density over the perforations
// times g for a producer.  Needs pv from a mode-1 cell_props pass.
__global__ void k_well_gamma(Grid g, Phys ph, Wells w, const double* __restrict__ x,
                             const double* __restrict__ pv, double* __restrict__ gamma) {
  PF_PDL_ENTRY();
  const int wi = blockIdx.x;
  if (wi >= w.nw) return;
  const int lane = threadIdx.x;
  const long long n = g.n;
  if (w.kind[wi] == PF_WELL_INJECTOR) {
    if (lane == 0) gamma[wi] = ph.g * ph.rho_w * (1.0 + ph.c_w * (x[3 * n + wi] - ph.p_ref));
    return;
  }
  double num = 0.0, den = 0.0;
  for (int m = w.ptr[wi] + lane; m < w.ptr[wi + 1]; m += 32) {
    const long long c = w.cell[m];
    const double lw = pv[PV_KRW * n + c] / (pv[PV_RK * n + c] * pv[PV_MUWE * n + c]);
    const double lo = pv[PV_KRO * n + c] / ph.mu_o;
    num += lw * pv[PV_RHO_W * n + c] + lo * pv[PV_RHO_O * n + c];
    den += lw + lo;
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if (lane == 0) {
    if (den > 0.0) gamma[wi] = ph.g * num / den;
    else gamma[wi] = ph.g * pv[PV_RHO_O * n + w.cell[w.ptr[wi]]];
  }
}

// Summed water, oil and polymer mass rates of each well at the current state
// (the perforation rates of Sec. 2.4 with the lagged gamma); needs pv from a
// mode-2 pass.
__global__ void k_well_totals(Grid g, Phys ph, Wells w, const double* __restrict__ x,
                              const double* __restrict__ pv, double* __restrict__ out) {
  PF_PDL_ENTRY();
  const int wi = blockIdx.x;
  if (wi >= w.nw) return;
  const int lane = threadIdx.x;
  const long long n = g.n;
  const double Pb = x[3 * n + wi];
  double sw = 0.0, so = 0.0, sp = 0.0;
  for (int m = w.ptr[wi] + lane; m < w.ptr[wi + 1]; m += 32) {
    const long long c = w.cell[m];
    const double Pbm = Pb + w.gamma[wi] * w.dzb[m];
    const double lw = pv[PV_KRW * n + c] / (pv[PV_RK * n + c] * pv[PV_MUWE * n + c]);
    const double lo = pv[PV_KRO * n + c] / ph.mu_o;
    const double rho_w = pv[PV_RHO_W * n + c], rho_o = pv[PV_RHO_O * n + c];
    const double dw = Pbm - pv[PV_PW * n + c];
    if (w.kind[wi] == PF_WELL_INJECTOR) {
      const double qw = w.wi[m] * (lw + lo) * rho_w * dw;
      sw += qw;
      sp += qw * w.cinj[wi] * ph.inv_rho_w;
    } else {
      const double qw = w.wi[m] * lw * rho_w * dw;
      sw += qw;
      so += w.wi[m] * lo * rho_o * (Pbm - x[3 * c]);
      sp += qw * x[3 * c + 2] * ph.inv_rho_w;
    }
  }
  sw = warp_sum(sw);
  so = warp_sum(so);
  sp = warp_sum(sp);
  if (lane == 0) {
    out[3 * wi] = sw;
    out[3 * wi + 1] = so;
    out[3 * wi + 2] = sp;
  }
}

void launch_well_totals(const Grid& g, const Phys& ph, const Wells& w, const double* x, const double* pv,
                        double* out, cudaStream_t st) {
  if (w.nw == 0) return;
  launch(k_well_totals, w.nw, 32, 0, st, g, ph, w, x, pv, out);
}

void launch_well_gamma(const Grid& g, const Phys& ph, const Wells& w, const double* x, const double* pv,
                       double* gamma, cudaStream_t st) {
  if (w.nw == 0) return;
  launch(k_well_gamma, w.nw, 32, 0, st, g, ph, w, x, pv, gamma);
}

// ---------------------------------------------------------------------------
// residual norms
// ---------------------------------------------------------------------------

// max that propagates NaN (fmax would drop it and hide a broken iterate)
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(256) k_res_norm_partial(Grid g, Phys ph, const double* __restrict__ inv_pv,
                                                          const double* __restrict__ R, double* __restrict__ partial) {
  PF_PDL_ENTRY();
  const long long n = g.n;
  double mx = 0.0, ss = 0.0;
  const double io = 1.0 / ph.rho_o, iw = ph.inv_rho_w, ic = ph.inv_c_ref;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ip = inv_pv[i];  // 1 / (V phi_r)
    const double r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
    mx = nanmax(mx, fabs(r0) * ip * io);
    mx = nanmax(mx, fabs(r1) * ip * iw);
    mx = nanmax(mx, fabs(r2) * ip * ic);
    ss += r0 * r0 + r1 * r1 + r2 * r2;
  }
  __shared__ double smx[8], sss[8];
  mx = warp_max(mx);
  ss = warp_sum(ss);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { smx[wid] = mx; sss[wid] = ss; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) { a = nanmax(a, smx[t]); b += sss[t]; }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_res_norm_final(int nblocks, Wells w, long long n, const double* __restrict__ R, double dt,
                                 const double* __restrict__ partial, double* __restrict__ out) {
  PF_PDL_ENTRY();
  // one warp: fixed-order reduction of the block partials, then the well rows
  const int lane = threadIdx.x;
  double mx = 0.0, ss = 0.0;
  for (int b = lane; b < nblocks; b += 32) { mx = nanmax(mx, partial[2 * b]); ss += partial[2 * b + 1]; }
  for (int wi = lane; wi < w.nw; wi += 32) {
    const double r = R[3 * n + wi];
    mx = nanmax(mx, fabs(r) / (dt * w.scale[wi]));
    ss += r * r;
  }
  mx = warp_max(mx);
  ss = warp_sum(ss);
  if (lane == 0) { out[0] = mx; out[1] = ss; }
}

void launch_residual_norms(const Grid& g, const Phys& ph, const double* inv_pv, const Wells& w, const double* R,
                           double dt, double* partial, int nblocks, double* out, cudaStream_t st) {
  launch(k_res_norm_partial, nblocks, 256, 0, st, g, ph, inv_pv, R, partial);
  launch(k_res_norm_final, 1, 32, 0, st, nblocks, w, g.n, R, dt, partial, out);
}

// ---------------------------------------------------------------------------
// Newton update with the saturation chop and the bounds on S and C
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_newton_update(long long n, int nw, double* __restrict__ x,
                                                       const double* __restrict__ dx, double ds_max, double dc_max) {
  PF_PDL_ENTRY();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n + nw;
       i += (long long)gridDim.x * blockDim.x) {
    if (i >= n) { x[3 * n + (i - n)] += dx[3 * n + (i - n)]; continue; }
    x[3 * i] += dx[3 * i];
    const double ds = fmin(fmax(dx[3 * i + 1], -ds_max), ds_max);
    x[3 * i + 1] = fmin(fmax(x[3 * i + 1] + ds, 0.0), 1.0);
    const double dc = fmin(fmax(dx[3 * i + 2], -dc_max), dc_max);
    x[3 * i + 2] = fmax(x[3 * i + 2] + dc, 0.0);
  }
}

void launch_newton_update(const Grid& g, int nw, double* x, const double* dx, double ds_max, double dc_max,
                          cudaStream_t st) {
  launch(k_newton_update, grid_for(g.n + nw, 256), 256, 0, st, g.n, nw, x, dx, ds_max, dc_max);
}

// explicit instantiations
// ---------------------------------------------------------------------------
// assembly kernels over a pack of simulators (one or up to kPackMax)
// ---------------------------------------------------------------------------

// The member that block b belongs to (b0 ascending, b0[0] = 0).
__device__ __forceinline__ int pack_member(const int* b0, int nm, int b) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b0[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the pack travels in the launch parameters (at most 32,764 bytes)
static_assert(sizeof(AsmPack<double>) <= 32000 && sizeof(AsmPack<float>) <= 32000, "pack size");

template <typename DT>
struct PackWords {
  static constexpr int n = (int)(sizeof(AsmMember<DT>) / sizeof(unsigned long long));
  static_assert(sizeof(AsmMember<DT>) % sizeof(unsigned long long) == 0, "descriptor size");
};

// Copies member m's descriptor from the launch parameters into shared memory
// (every thread of a block serves the same member), so that the per-cell
// arithmetic reads it the same way in every pack size.
template <typename DT, int CAP>
__device__ __forceinline__ const AsmMember<DT>& pack_load(const AsmPack<DT, CAP>& pk, int m,
                                                          unsigned long long* sm) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&pk.m[m]);
  for (int w = threadIdx.x; w < PackWords<DT>::n; w += blockDim.x) sm[w] = src[w];
  __syncthreads();
  return *reinterpret_cast<const AsmMember<DT>*>(sm);
}

// cell index of this thread within its member (blockDim.x threads per block)
template <typename DT, int CAP>
__device__ __forceinline__ long long pack_cell(const AsmPack<DT, CAP>& pk, int m) {
  return (long long)(blockIdx.x - pk.cblock0[m]) * blockDim.x + threadIdx.x;
}

template <typename DT, int CAP>
__global__ void __launch_bounds__(256) k_cell_props(const __grid_constant__ AsmPack<DT, CAP> pk) {
  PF_PDL_ENTRY();
  __shared__ unsigned long long sm[PackWords<DT>::n];
  const int m = CAP == 1 ? 0 : pack_member(pk.cblock0, pk.nm, blockIdx.x);
  const AsmMember<DT>& a = pack_load(pk, m, sm);
  const long long i = pack_cell(pk, m);
  if (i < a.g.n) cell_props_at<DT>(a.g, a.ph, a.phi_r, a.x, a.pv, a.pd, a.Mold, a.R, a.J, nullptr, 0, i);
}

template <typename DT, int CAP>
__global__ void __launch_bounds__(256) k_face_flux(const __grid_constant__ AsmPack<DT, CAP> pk) {
  PF_PDL_ENTRY();
  __shared__ unsigned long long sm[PackWords<DT>::n];
  const int m = CAP == 1 ? 0 : pack_member(pk.cblock0, pk.nm, blockIdx.x);
  const AsmMember<DT>& a = pack_load(pk, m, sm);
  const long long i = pack_cell(pk, m);
  if (i < a.g.n) face_flux_at<DT>(a.g, a.ph, a.wL3, a.T3, a.x, a.pv, a.pd, a.dt, a.J, a.Fbuf, i);
}

template <typename DT, int CAP>
__global__ void __launch_bounds__(256) k_gather(const __grid_constant__ AsmPack<DT, CAP> pk) {
  PF_PDL_ENTRY();
  __shared__ unsigned long long sm[PackWords<DT>::n];
  const int m = CAP == 1 ? 0 : pack_member(pk.cblock0, pk.nm, blockIdx.x);
  const AsmMember<DT>& a = pack_load(pk, m, sm);
  const long long i = pack_cell(pk, m);
  if (i < a.g.n) gather_at<DT>(a.g, a.Fbuf, a.R, a.J, i);
}

// one warp per well
template <typename DT, int CAP>
__global__ void k_wells(const __grid_constant__ AsmPack<DT, CAP> pk) {
  PF_PDL_ENTRY();
  __shared__ unsigned long long sm[PackWords<DT>::n];
  const int m = CAP == 1 ? 0 : pack_member(pk.wblock0, pk.nm, blockIdx.x);
  const AsmMember<DT>& a = pack_load(pk, m, sm);
  wells_at<DT>(a.g, a.ph, a.w, a.x, a.pv, a.pd, a.dt, a.R, a.J, a.Bw, a.Cw, a.Dw, (int)(blockIdx.x - pk.wblock0[m]),
               (int)threadIdx.x);
}

template <typename DT>
int launch_assemble_packed(const AsmPack<DT>& pk, cudaStream_t st) {
  const int cb = pk.cblock0[pk.nm], wb = pk.wblock0[pk.nm];
  if (cb == 0) return 0;
  launch(k_cell_props<DT, kPackMax>, cb, 256, 0, st, pk);
  launch(k_face_flux<DT, kPackMax>, cb, 256, 0, st, pk);
  launch(k_gather<DT, kPackMax>, cb, 256, 0, st, pk);
  if (wb > 0) launch(k_wells<DT, kPackMax>, wb, 32, 0, st, pk);
  return 3 + (wb > 0);
}

// A pack of one simulator for its own launches (fields a kernel does not read
// stay null).
template <typename DT>
AsmPack<DT, 1> pack_of_one(const Grid& g, const Phys& ph) {
  AsmPack<DT, 1> pk{};
  pk.nm = 1;
  pk.cblock0[0] = 0;
  pk.wblock0[0] = 0;
  pk.m[0].g = g;
  pk.m[0].ph = ph;
  return pk;
}

template <typename DT>
void launch_cell_props(const Grid& g, const Phys& ph, const double* phi_r, const double* x, double* pv,
                       DT* pd, const double* Mold, double* R, DT* J, double* Mold_out, int mode,
                       cudaStream_t st, int block) {
  if (mode != 0) {
    launch(k_cell_values<DT>, grid_for(g.n, block), block, 0, st, g, ph, phi_r, x, pv, pd, Mold, R, J, Mold_out,
           mode);
    return;
  }
  AsmPack<DT, 1> pk = pack_of_one<DT>(g, ph);
  AsmMember<DT>& a = pk.m[0];
  a.phi_r = phi_r; a.x = x; a.pv = pv; a.pd = pd; a.Mold = Mold; a.R = R; a.J = J;
  launch(k_cell_props<DT, 1>, grid_for(g.n, block), block, 0, st, pk);
}

template <typename DT>
void launch_face_flux(const Grid& g, const Phys& ph, const double* wL3, const double* T3, const double* x,
                      const double* pv, const DT* pd, double dt, DT* J, double* Fbuf, cudaStream_t st, int block) {
  AsmPack<DT, 1> pk = pack_of_one<DT>(g, ph);
  AsmMember<DT>& a = pk.m[0];
  a.wL3 = wL3; a.T3 = T3; a.x = x; a.pv = const_cast<double*>(pv); a.pd = const_cast<DT*>(pd); a.dt = dt;
  a.J = J; a.Fbuf = Fbuf;
  launch(k_face_flux<DT, 1>, grid_for(g.n, block), block, 0, st, pk);
}

template <typename DT>
void launch_gather(const Grid& g, const double* Fbuf, double* R, DT* J, cudaStream_t st, int block) {
  AsmPack<DT, 1> pk = pack_of_one<DT>(g, Phys{});
  AsmMember<DT>& a = pk.m[0];
  a.Fbuf = const_cast<double*>(Fbuf); a.R = R; a.J = J;
  launch(k_gather<DT, 1>, grid_for(g.n, block), block, 0, st, pk);
}

template <typename DT>
void launch_wells(const Grid& g, const Phys& ph, const Wells& w, const double* x, const double* pv, const DT* pd,
                  double dt, double* R, DT* J, DT* Bw, DT* Cw, DT* Dw, cudaStream_t st) {
  if (w.nw == 0) return;
  AsmPack<DT, 1> pk = pack_of_one<DT>(g, ph);
  AsmMember<DT>& a = pk.m[0];
  a.w = w; a.x = x; a.pv = const_cast<double*>(pv); a.pd = const_cast<DT*>(pd); a.dt = dt; a.R = R; a.J = J;
  a.Bw = Bw; a.Cw = Cw; a.Dw = Dw;
  pk.wblock0[1] = w.nw;
  launch(k_wells<DT, 1>, w.nw, 32, 0, st, pk);
}

template void launch_cell_props<double>(const Grid&, const Phys&, const double*, const double*, double*, double*,
                                        const double*, double*, double*, double*, int, cudaStream_t, int);
template void launch_cell_props<float>(const Grid&, const Phys&, const double*, const double*, double*, float*,
                                       const double*, double*, float*, double*, int, cudaStream_t, int);
template void launch_face_flux<double>(const Grid&, const Phys&, const double*, const double*, const double*,
                                       const double*, const double*, double, double*, double*, cudaStream_t, int);
template void launch_face_flux<float>(const Grid&, const Phys&, const double*, const double*, const double*,
                                      const double*, const float*, double, float*, double*, cudaStream_t, int);
template void launch_gather<double>(const Grid&, const double*, double*, double*, cudaStream_t, int);
template void launch_gather<float>(const Grid&, const double*, double*, float*, cudaStream_t, int);
template void launch_wells<double>(const Grid&, const Phys&, const Wells&, const double*, const double*,
                                   const double*, double, double*, double*, double*, double*, double*, cudaStream_t);
template void launch_wells<float>(const Grid&, const Phys&, const Wells&, const double*, const double*,
                                  const float*, double, double*, float*, float*, float*, float*, cudaStream_t);

template int launch_assemble_packed<double>(const AsmPack<double>&, cudaStream_t);
template int launch_assemble_packed<float>(const AsmPack<float>&, cudaStream_t);

}  // namespace pf
