// Capillary-gravity equilibrium initial state (Sec. 4.1.3 of the paper: the
// datum-phase pressure is marched through the reservoir with the density
// recomputed along the way, the other phase's pressure from the contact, and
// the saturations balance the capillary pressure).  Host code: this runs
// once, before pf_create, on the caller's host arrays.
//
// Each column is marched cell to cell with the discrete relation of the
// assembly's vertical faces, P_D - P_U = (w_U rho(P_U) + w_D rho(P_D)) g dz
// (reference-pore-volume face weights), solved in closed form for the linear
// density law, so the discrete phase potential difference of every vertical
// face is zero.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pf_internal.cuh"

namespace {

pf_status init_fail(const std::string& m) {
  pf::set_last_error(m);
  return PF_EINVAL;
}

struct PhaseLaw {
  double rho_ref, c, p_ref, g;
  double rho(double P) const { return rho_ref * (1.0 + c * (P - p_ref)); }
  // dP/dz = g rho(P) from (z0, p0) to z1: for c != 0,
  // P = p0 + (p0 - p_ref + 1/c) (exp(g rho_ref c (z1 - z0)) - 1)
  double along(double p0, double z0, double z1) const {
    if (c == 0.0) return p0 + g * rho_ref * (z1 - z0);
    return p0 + (p0 - p_ref + 1.0 / c) * expm1(g * rho_ref * c * (z1 - z0));
  }
  // lower cell from the upper: P_D (1 - g dz w_D rho_ref c) = P_U + g dz (w_U rho(P_U) + w_D rho_ref (1 - c p_ref))
  double down(double pu, double wu, double wd, double dz) const {
    const double a = g * dz;
    return (pu + a * (wu * rho(pu) + wd * rho_ref * (1.0 - c * p_ref))) / (1.0 - a * wd * rho_ref * c);
  }
  // upper cell from the lower: P_U (1 + g dz w_U rho_ref c) = P_D - g dz (w_U rho_ref (1 - c p_ref) + w_D rho(P_D))
  double up(double pd, double wu, double wd, double dz) const {
    const double a = g * dz;
    return (pd - a * (wu * rho_ref * (1.0 - c * p_ref) + wd * rho(pd))) / (1.0 + a * wu * rho_ref * c);
  }
};

// Capillary pressure of the model at S (Corey curve or table).
double pc_at(const pf_model_desc& m, double S) {
  if (m.n_sat > 0) {
    const double* t = m.sat_table;
    const int K = m.n_sat;
    if (S < t[0]) return t[3];
    if (S >= t[4 * (K - 1)]) return t[4 * (K - 1) + 3];
    int k = 0;
    while (k + 1 < K - 1 && t[4 * (k + 1)] <= S) ++k;
    const double sl = (t[4 * (k + 1) + 3] - t[4 * k + 3]) / (t[4 * (k + 1)] - t[4 * k]);
    return (S - t[4 * k]) * sl + t[4 * k + 3];
  }
  const pf_physics& p = m.phys;
  if (p.pc_e == 0.0) return 0.0;
  double sn = (S - p.swc) / (1.0 - p.swc - p.sor);
  sn = std::min(std::max(sn, 0.0), 1.0);
  return p.pc_e * pow(1.0 - sn, p.pc_n);
}

// Largest S in [0, 1] with P_c(S) >= dP; the irreducible saturation (first
// knot, or swc) when none qualifies.  P_c does not increase with S.
double saturation_for(const pf_model_desc& m, double dP) {
  if (pc_at(m, 1.0) >= dP) return 1.0;
  if (m.n_sat > 0) {
    const double* t = m.sat_table;
    const int K = m.n_sat;
    int j = -1;  // last knot with P_c >= dP
    for (int k = K - 1; k >= 0; --k)
      if (t[4 * k + 3] >= dP) { j = k; break; }
    if (j < 0) return t[0];
    // P_c(x_j) >= dP > P_c(x_{j+1}) (j < K - 1 since P_c(1) < dP)
    const double x0 = t[4 * j], x1 = t[4 * (j + 1)], y0 = t[4 * j + 3], y1 = t[4 * (j + 1) + 3];
    return x0 + (y0 - dP) / (y0 - y1) * (x1 - x0);
  }
  const pf_physics& p = m.phys;
  if (p.pc_e == 0.0 || dP > p.pc_e) return p.swc;  // dP > 0 here
  // pc_e (1 - Sn)^n >= dP  <=>  Sn <= 1 - (dP / pc_e)^(1/n)
  const double sn = 1.0 - pow(dP / p.pc_e, 1.0 / p.pc_n);
  return p.swc + sn * (1.0 - p.swc - p.sor);
}

}  // namespace

extern "C" {

pf_status pf_equilibrium_init(const pf_model_desc* m, double datum_depth, double datum_p, double contact_depth,
                              double* p0, double* s0) {
  if (!m || !p0 || !s0) return init_fail("NULL argument");
  if (m->nx < 1 || m->ny < 1 || m->nz < 1) return init_fail("grid dimensions must be >= 1");
  if (!(m->dz > 0.0) || !std::isfinite(m->top) || !m->phi) return init_fail("invalid grid or porosity");
  if (!std::isfinite(datum_depth) || !std::isfinite(datum_p) || !std::isfinite(contact_depth))
    return init_fail("datum and contact must be finite");
  const pf_physics& p = m->phys;
  if (!(p.rho_o > 0.0) || !(p.rho_w > 0.0) || !std::isfinite(p.c_o) || !std::isfinite(p.c_w) || !std::isfinite(p.g))
    return init_fail("invalid fluid constants");
  if (m->n_sat < 0 || m->n_sat > PF_MAX_KNOTS || (m->n_sat > 0 && !m->sat_table))
    return init_fail("invalid saturation table size");
  for (int k = 1; k < m->n_sat; ++k) {
    const double* r = m->sat_table + 4 * k;
    if (!(r[0] > r[-4]) || !(r[3] <= r[-1])) return init_fail("saturation table: S must increase, P_c must not");
  }
  if (m->n_sat == 0 && p.pc_e < 0.0) return init_fail("negative capillary entry pressure");
  if (m->n_sat == 0 && p.pc_e > 0.0 && !(p.pc_n > 0.0)) return init_fail("invalid capillary exponent");
  const long long nxy = (long long)m->nx * m->ny, n = nxy * m->nz;
  for (long long i = 0; i < n; ++i)
    if (!(m->phi[i] > 0.0)) return init_fail("porosity must be positive");
  const PhaseLaw oil{p.rho_o, p.c_o, p.p_ref, p.g}, wat{p.rho_w, p.c_w, p.p_ref, p.g};
  const int nz = m->nz;
  const double dz = m->dz;
  auto layer_of = [&](double depth) {
    const double f = floor((depth - m->top) / dz);
    return (int)std::min(std::max(f, 0.0), (double)(nz - 1));
  };
  auto zc = [&](int k) { return m->top + (k + 0.5) * dz; };
  const int kd = layer_of(datum_depth), kc = layer_of(contact_depth);
  std::vector<double> po(nz), pw(nz);
  auto march = [&](const PhaseLaw& law, long long col, int k0, double pk0, std::vector<double>& out) {
    out[k0] = pk0;
    for (int k = k0; k + 1 < nz; ++k) {
      const double fu = m->phi[col + k * nxy], fd = m->phi[col + (k + 1) * nxy];
      const double wu = fu / (fu + fd);
      out[k + 1] = law.down(out[k], wu, 1.0 - wu, dz);
    }
    for (int k = k0; k > 0; --k) {
      const double fu = m->phi[col + (k - 1) * nxy], fd = m->phi[col + k * nxy];
      const double wu = fu / (fu + fd);
      out[k - 1] = law.up(out[k], wu, 1.0 - wu, dz);
    }
  };
  for (long long col = 0; col < nxy; ++col) {
    march(oil, col, kd, oil.along(datum_p, datum_depth, zc(kd)), po);
    const double p_contact = oil.along(po[kc], zc(kc), contact_depth);  // P_w = P_o at the contact
    march(wat, col, kc, wat.along(p_contact, contact_depth, zc(kc)), pw);
    for (int k = 0; k < nz; ++k) {
      const long long i = col + k * nxy;
      const double dP = po[k] - pw[k];
      const double S = saturation_for(*m, dP);
      const double pc = pc_at(*m, S);
      s0[i] = S;
      p0[i] = pc > dP ? pw[k] + pc : po[k];  // below the contact: water pressure on its gradient
    }
  }
  return PF_OK;
}

}  // extern "C"
