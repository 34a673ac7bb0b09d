"""FP64 CPU oracle of the fully implicit water/oil/polymer model.

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.

Everything is written from the paper's equations (arXiv 1807.05298):

  rock        phi(P) = phi_r + c_r (P - P_r)                       (Sec. 2.1)
  closure     S_w + S_o = 1, P_c = P_o - P_w                       (Sec. 2.2)
  Darcy       phase mass flux  k k_r rho / mu  grad(P - gamma Z)   (Sec. 2.2)
  oil, water  d/dt(phi S rho) = div(...) + q                       (Sec. 2.2)
  polymer     d/dt(phi S_w rho_w C + (1 - phi) A_d) = div(...) + q_w C  (Sec. 2.3)
  R_k         1 + (RRF - 1) A_d / A_d,max                          (Sec. 2.3)
  viscosity   Todd-Longstaff mu_p,e, mu_w,partial, mu_w,e; linear or
              nonlinear mixing rule in beta = C / C_ref             (Sec. 2.3)
  wells       Peaceman index with its equivalent radius and
              permeability; perforation rate; hydrostatic wellbore;
              BHP and rate constraints                              (Sec. 2.4)
  time        backward Euler                                       (Sec. 3.1)
  space       two-point transmissibility, harmonic k and geometry,
              pore-volume weighted rho and mu, upstream k_r          (Sec. 3.2)
  Newton      Algorithm 1 with forcing term of Sec. 3.3, third choice

Where the paper is silent the following readings are taken (the CUDA path
takes the same ones):
  * rho_a(P_a) = rho_a,ref (1 + c_a (P_a - P_ref)); formation volume factor 1.
  * C is kg of polymer per m^3 of water at reference conditions, so polymer
    mass per unit water volume is rho_w C / rho_w,ref; A_d is kg per m^3 of
    rock; the polymer well source is q_w C / rho_w,ref.
  * inaccessible pore volume: polymer sees the fraction (1 - IPV) of the
    water-filled pore space in the accumulation term; the flux is unchanged.
  * Todd-Longstaff alpha = clip(C / C_ref, 0, 1).
  * face averages of rho and mu weight the two cells by their reference pore
    volumes V phi_r; k_r, R_k and the polymer concentration of a face come
    from the upstream cell of the water (or oil) potential; for the face
    (L, H) with H the higher natural index, H is upstream iff
    Phi_H - Phi_L >= 0, where Phi_H - Phi_L = (P_H - P_L) - rho_bar g (Z_H - Z_L)
    and Z is depth (positive downward).
  * Langmuir adsorption A_d = a C / (1 + b C), A_d,max = a / b.
  * Corey k_rw = krw_max Sn^nw, k_ro = kro_max (1 - Sn)^no,
    Sn = (S - Swc) / (1 - Swc - Sor), clipped to [0, 1] (derivative of the
    interior formula on the closed interval, 0 outside);
    P_c = pc_e (1 - Sn)^pc_n.
  * injector perforations use the cell's total mobility and rho_w; producer
    perforations use phase mobilities; water phase flow is driven by P_w.
  * gamma_well is evaluated at the start of the step and frozen: rho_w(P_b) g
    for an injector, the mobility-weighted perforation mixture density times
    g for a producer.
  * residuals are masses [kg]; a BHP well row is dt * W (P_b - target) with
    W = sum(WI) rho_w,ref / mu_w; a rate row is dt (sum of signed phase mass
    rates - rho_ref * target).
  * Newton update: S change per cell chopped to +-ds_max and C change to
    +-0.5 C_ref, then S clipped to [0, 1] and C to >= 0.
"""

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dual as D
from .dual import Dual

NPHASE = 3  # rows per cell: oil, water, polymer; columns P_o, S_w, C


# ---------------------------------------------------------------------------
# set-up: geometry, transmissibility and well index
# ---------------------------------------------------------------------------

def faces(nx, ny, nz):
    """Interior faces per direction as (L, H) natural-index arrays, H = L + stride."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    out = {}
    out["x"] = (idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel())
    out["y"] = (idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel())
    out["z"] = (idx[:-1, :, :].ravel(), idx[1:, :, :].ravel())
    return out


def transmissibility(sc):
    """Geometric transmissibility per face: area over the harmonic sum of the
    two half-cell resistances, A / (dd/(2 k_L) + dd/(2 k_H))  (Sec. 3.2)."""
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    dx, dy, dz = sc["dx"], sc["dy"], sc["dz"]
    f = faces(nx, ny, nz)
    geo = {"x": (dy * dz, dx, sc["kx"]), "y": (dx * dz, dy, sc["ky"]), "z": (dx * dy, dz, sc["kz"])}
    T = {}
    for d, (L, H) in f.items():
        area, dd, k = geo[d]
        T[d] = area / (dd / (2.0 * k[L]) + dd / (2.0 * k[H]))
    return f, T


def cell_depth(sc):
    nz = sc["nz"]
    zc = sc["top"] + (np.arange(nz) + 0.5) * sc["dz"]
    return np.repeat(zc, sc["nx"] * sc["ny"])


def peaceman_wi(kx, ky, kz, dx, dy, dz, direction, rw, skin, gf=0.249, f=1.0, fh=1.0):
    """Peaceman well index (Sec. 2.4) with its equivalent radius r_e and
    permeability k_a.

    The printed form is for a well along x (perpendicular directions y, z);
    a well along y or z uses the same expression with the two directions
    perpendicular to it."""
    if direction == "x":
        k1, k2, h1, h2, h = ky, kz, dy, dz, dx
    elif direction == "y":
        k1, k2, h1, h2, h = kx, kz, dx, dz, dy
    else:
        k1, k2, h1, h2, h = kx, ky, dx, dy, dz
    # r_e and k_a of Sec. 2.4 with (y, z) -> (1, 2)
    re = (2.0 * gf / math.sqrt(math.pi)) * math.sqrt(math.sqrt(k2 / k1) * h1 ** 2 + math.sqrt(k1 / k2) * h2 ** 2) \
        / ((k2 / k1) ** 0.25 + (k1 / k2) ** 0.25)
    ka = math.sqrt(k1 * k2)
    return 2.0 * math.pi * f * h * fh * ka / (math.log(re / rw) + skin)


class Setup:
    """Static per-scenario data derived from the scenario dict."""

    def __init__(self, sc):
        self.sc = sc
        self.ph = sc["physics"]
        self.nx, self.ny, self.nz = sc["nx"], sc["ny"], sc["nz"]
        self.n = self.nx * self.ny * self.nz
        self.V = sc["dx"] * sc["dy"] * sc["dz"]
        self.phi_r = sc["phi"]
        self.Z = cell_depth(sc)
        self.faces, self.T = transmissibility(sc)
        self.wells = []
        for w in sc["wells"]:
            cells = np.asarray(w["cells"], dtype=np.int64)
            wi = np.array([peaceman_wi(sc["kx"][c], sc["ky"][c], sc["kz"][c], sc["dx"], sc["dy"], sc["dz"],
                                       d, w["rw"], w["skin"], w["gf"], w["f"], w["fh"])
                           for c, d in zip(cells, w["dirs"])])
            self.wells.append(dict(kind=w["kind"], cells=cells, WI=wi, z=self.Z[cells],
                                   zb=self.Z[cells[0]],
                                   W=float(wi.sum()) * self.ph["rho_w"] / self.ph["mu_w"]))
        self.nw = len(self.wells)
        self.nunk = NPHASE * self.n + self.nw


# ---------------------------------------------------------------------------
# cell properties (Sec. 2.1 - 2.3), generic in float arrays or Dual
# ---------------------------------------------------------------------------

def _clip01_dual(x):
    x = D.where(x.v < 0.0, 0.0, x)
    return D.where(x.v > 1.0, 1.0, x)


def table_lookup(xs, ys, u):
    """Piecewise-linear interpolation of the knots (xs, ys) at the Dual u:
    on [x_k, x_{k+1}) the segment's line (so the derivative at a knot is the
    right-hand slope); below x_0 and from x_{K-1} on, the end value with
    derivative 0."""
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    K = len(xs)
    k = np.searchsorted(xs, u.v, side="right") - 1          # x_k <= u < x_{k+1}
    inside = (k >= 0) & (k < K - 1)
    kk = np.clip(k, 0, max(K - 2, 0))
    if K > 1:
        slope = (ys[kk + 1] - ys[kk]) / (xs[kk + 1] - xs[kk])
        line = (u - xs[kk]) * slope + ys[kk]
    else:
        line = Dual.const(np.full_like(u.v, ys[0]), u.k)
    end = Dual.const(np.where(k < 0, ys[0], ys[K - 1]), u.k)
    return D.where(inside, line, end)


def cell_properties(ph, phi_r, P, S, C):
    """All per-cell quantities as Duals in the cell's own (P, S, C)."""
    phi = phi_r + ph["c_r"] * (P - ph["p_r"])                       # porosity law
    rho_o = ph["rho_o"] * (1.0 + ph["c_o"] * (P - ph["p_ref"]))
    sat = ph.get("sat_table")
    if sat is not None:                      # tabulated k_rw, k_ro, P_c (Sec. 2.2)
        sat = np.asarray(sat, dtype=np.float64)
        krw = table_lookup(sat[:, 0], sat[:, 1], S)
        kro = table_lookup(sat[:, 0], sat[:, 2], S)
        pc = table_lookup(sat[:, 0], sat[:, 3], S)
    else:
        sn = _clip01_dual((S - ph["swc"]) / (1.0 - ph["swc"] - ph["sor"]))
        krw = ph["krw_max"] * (sn ** ph["nw"])
        kro = ph["kro_max"] * ((1.0 - sn) ** ph["no"])
        if ph["pc_e"] != 0.0:
            pc = ph["pc_e"] * ((1.0 - sn) ** ph["pc_n"])
        else:
            pc = Dual.const(np.zeros_like(P.v), P.k)
    Pw = P - pc                                                      # P_c = P_o - P_w
    rho_w = ph["rho_w"] * (1.0 + ph["c_w"] * (Pw - ph["p_ref"]))
    poly = ph.get("poly_table")
    if poly is not None:                     # tabulated A_d(C) and viscosity multiplier (Sec. 2.3)
        poly = np.asarray(poly, dtype=np.float64)
        ads = table_lookup(poly[:, 0], poly[:, 2], C)
        ads_max = float(poly[:, 2].max())
    else:
        ads = ph["ads_a"] * C / (1.0 + ph["ads_b"] * C)              # Langmuir A_d(C)
        ads_max = ph["ads_a"] / ph["ads_b"]
    if ads_max > 0.0:                                                # permeability reduction
        Rk = 1.0 + (ph["rrf"] - 1.0) * ads / ads_max
    else:                                                            # no adsorption: R_k = 1
        Rk = Dual.const(np.ones_like(P.v), P.k)
    beta = C / ph["c_ref"]
    if poly is not None:                     # mu_m = mu_w x multiplier(C)
        mu_m = table_lookup(poly[:, 0], poly[:, 1], C) * ph["mu_w"]
    elif ph["mixing"] == 0:                  # nonlinear rule mu_p0^beta mu_w^(1-beta)
        mu_m = D.exp(beta * math.log(ph["mu_p0"]) + (1.0 - beta) * math.log(ph["mu_w"]))
    else:                                                            # linear rule
        mu_m = beta * ph["mu_p0"] + (1.0 - beta) * ph["mu_w"]
    om = ph["omega"]
    mu_pe = (mu_m ** om) * (ph["mu_p0"] ** (1.0 - om))                # Todd-Longstaff
    mu_wp = (mu_m ** om) * (ph["mu_w"] ** (1.0 - om))
    alpha = _clip01_dual(C / ph["c_ref"])
    mu_we = 1.0 / (alpha / mu_pe + (1.0 - alpha) / mu_wp)
    return dict(phi=phi, rho_o=rho_o, rho_w=rho_w, krw=krw, kro=kro, Pw=Pw, ads=ads, Rk=Rk,
                mu_pe=mu_pe, mu_we=mu_we, S=S, C=C, P=P)


def accumulation(st, ph, pr):
    """Component masses per cell [kg]: oil, water, polymer (Sec. 2.2, 2.3)."""
    V = st.V
    Mo = V * pr["phi"] * pr["rho_o"] * (1.0 - pr["S"])
    Mw = V * pr["phi"] * pr["rho_w"] * pr["S"]
    Mp = V * (1.0 - ph["ipv"]) * pr["phi"] * pr["S"] * pr["rho_w"] * pr["C"] / ph["rho_w"] \
        + V * (1.0 - pr["phi"]) * pr["ads"]
    return Mo, Mw, Mp


def _cell_duals(st, x):
    P = Dual.variable(x[0::3][: st.n], 3, 0)
    S = Dual.variable(x[1::3][: st.n], 3, 1)
    C = Dual.variable(x[2::3][: st.n], 3, 2)
    return P, S, C


def unpack(st, x):
    n = st.n
    xc = x[: 3 * n]
    return xc[0::3], xc[1::3], xc[2::3], x[3 * n:]


# ---------------------------------------------------------------------------
# capillary-gravity equilibrium initialisation (Sec. 4.1.3)
# ---------------------------------------------------------------------------

def _phase_density(ph, a, P):
    key, c = ("rho_o", "c_o") if a == "o" else ("rho_w", "c_w")
    return ph[key] * (1.0 + ph[c] * (P - ph["p_ref"]))


def _march_continuous(ph, a, p0, z0, z1, steps=4000):
    """dP/dz = g rho_a(P) from (z0, p0) to z1 by many small RK4 steps (the
    paper marches the hydrostatic pressure in small steps, recomputing the
    density at each one)."""
    if z1 == z0:
        return p0
    h = (z1 - z0) / steps
    g = ph["g"]
    f = lambda P: g * _phase_density(ph, a, P)
    P = p0
    for _ in range(steps):
        k1 = f(P)
        k2 = f(P + 0.5 * h * k1)
        k3 = f(P + 0.5 * h * k2)
        k4 = f(P + h * k3)
        P = P + h * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0
    return P


def _face_balance_step(ph, a, P_known, known_is_upper, wU, wD, dz):
    """Pressure of the neighbouring cell that makes the discrete potential
    difference of phase a across a vertical face vanish:
    P_D - P_U = (wU rho(P_U) + wD rho(P_D)) g dz, U the upper (lower index)
    cell, D the lower; solved for the unknown side by scalar Newton."""
    g = ph["g"]
    P = P_known
    for _ in range(50):
        if known_is_upper:
            F = P - P_known - (wU * _phase_density(ph, a, P_known) + wD * _phase_density(ph, a, P)) * g * dz
            dF = 1.0 - wD * g * dz * (_phase_density(ph, a, P + 1.0) - _phase_density(ph, a, P))
        else:
            F = P_known - P - (wU * _phase_density(ph, a, P) + wD * _phase_density(ph, a, P_known)) * g * dz
            dF = -1.0 - wU * g * dz * (_phase_density(ph, a, P + 1.0) - _phase_density(ph, a, P))
        step = F / dF
        P -= step
        if abs(step) <= 1e-13 * abs(P):
            break
    return P


def _capillary_pressure(ph, S):
    """P_c = P_o - P_w of the model at the saturations S (array)."""
    S = np.atleast_1d(np.asarray(S, dtype=np.float64))
    z = np.zeros_like(S)
    pr = cell_properties(ph, z, Dual.variable(z, 3, 0), Dual.variable(S, 3, 1), Dual.variable(z, 3, 2))
    return -pr["Pw"].v


def _saturation_for(ph, dP):
    """Per entry of dP: the largest S in [0, 1] with P_c(S) >= dP (P_c is
    non-increasing in S), by bisection; the irreducible saturation where no S
    qualifies."""
    dP = np.asarray(dP, dtype=np.float64)
    sat = ph.get("sat_table")
    s_irr = float(np.asarray(sat)[0, 0]) if sat is not None else ph["swc"]
    ones = np.ones_like(dP)
    at_one = _capillary_pressure(ph, ones) >= dP
    none = _capillary_pressure(ph, 0.0 * ones) < dP
    lo, hi = np.zeros_like(dP), ones.copy()          # P_c(lo) >= dP > P_c(hi) where bracketed
    for _ in range(1100):
        mid = 0.5 * (lo + hi)
        moving = (mid != lo) & (mid != hi)
        if not moving.any():
            break
        up = _capillary_pressure(ph, mid) >= dP
        lo = np.where(moving & up, mid, lo)
        hi = np.where(moving & ~up, mid, hi)
    return np.where(at_one, 1.0, np.where(none, s_irr, lo))


def equilibrium_state(sc, datum_depth, datum_p, contact_depth):
    """Capillary-gravity equilibrium (Sec. 4.1.3): oil pressure from the
    datum, water pressure from the oil-water contact (free water level, where
    P_o = P_w), each column marched cell to cell so that the discrete phase
    potential difference of every vertical face is zero with the face density
    of the discretisation (pore-volume weighted); saturations then balance
    the capillary pressure, S = max{S : P_c(S) >= P_o - P_w}.  Below the
    contact (no S balances it) the oil pressure of a cell is set to
    P_w + P_c(S) so that its water pressure stays on the water gradient.
    The datum-to-cell and contact-to-cell legs are continuous marches.
    Returns (P_o, S_w) per cell."""
    ph = sc["physics"]
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    top, dz = sc["top"], sc["dz"]
    zc = top + (np.arange(nz) + 0.5) * dz
    phi = np.asarray(sc["phi"], dtype=np.float64).reshape(nz, ny * nx)
    kd = int(min(max(math.floor((datum_depth - top) / dz), 0), nz - 1))
    kc = int(min(max(math.floor((contact_depth - top) / dz), 0), nz - 1))
    P_o = np.empty((nz, ny * nx))
    P_w = np.empty((nz, ny * nx))
    for col in range(ny * nx):
        def march(a, k0, p_k0, out):
            out[k0] = p_k0
            for k in range(k0, nz - 1):                  # downwards
                wU = phi[k, col] / (phi[k, col] + phi[k + 1, col])
                out[k + 1] = _face_balance_step(ph, a, out[k], True, wU, 1.0 - wU, dz)
            for k in range(k0, 0, -1):                   # upwards
                wU = phi[k - 1, col] / (phi[k - 1, col] + phi[k, col])
                out[k - 1] = _face_balance_step(ph, a, out[k], False, wU, 1.0 - wU, dz)
        march("o", kd, _march_continuous(ph, "o", datum_p, datum_depth, zc[kd]), P_o[:, col])
        p_contact = _march_continuous(ph, "o", P_o[kc, col], zc[kc], contact_depth)
        march("w", kc, _march_continuous(ph, "w", p_contact, contact_depth, zc[kc]), P_w[:, col])
    P = P_o.ravel().copy()
    Pw = P_w.ravel()
    S = _saturation_for(ph, P - Pw)
    pc = _capillary_pressure(ph, S)
    below = pc > P - Pw                                 # below the contact
    P[below] = Pw[below] + pc[below]
    return P, S


# ---------------------------------------------------------------------------
# face fluxes (Sec. 3.2)
# ---------------------------------------------------------------------------

def face_fluxes(st, pr, L, H, T, dZ):
    """Mass fluxes from H into L for oil, water, polymer as Duals in
    (x_L, x_H) (6 derivative columns)."""
    ph = st.ph
    g = ph["g"]
    w_L = st.phi_r[L] / (st.phi_r[L] + st.phi_r[H])
    w_H = 1.0 - w_L

    def lift(q):
        a = q.take(L).embed(6, 0)
        b = q.take(H).embed(6, 3)
        return a, b

    def avg(q):
        a, b = lift(q)
        return a * w_L + b * w_H

    def upstream(q, up_H):
        a, b = lift(q)
        return D.where(up_H, b, a)

    rho_o = avg(pr["rho_o"])
    rho_w = avg(pr["rho_w"])
    mu_we = avg(pr["mu_we"])
    mu_pe = avg(pr["mu_pe"])
    PL, PH = lift(pr["P"])
    PwL, PwH = lift(pr["Pw"])
    dPhi_o = (PH - PL) - rho_o * (g * dZ)
    dPhi_w = (PwH - PwL) - rho_w * (g * dZ)
    up_o = dPhi_o.v >= 0.0
    up_w = dPhi_w.v >= 0.0
    kro = upstream(pr["kro"], up_o)
    krw = upstream(pr["krw"], up_w)
    Rk = upstream(pr["Rk"], up_w)
    Cu = upstream(pr["C"], up_w)
    Fo = T * (kro / ph["mu_o"]) * rho_o * dPhi_o
    Fw = T * (krw / (Rk * mu_we)) * rho_w * dPhi_w
    Fp = T * (krw / (Rk * mu_pe)) * rho_w * dPhi_w * Cu / ph["rho_w"]
    return Fo, Fw, Fp


# ---------------------------------------------------------------------------
# wells (Sec. 2.4)
# ---------------------------------------------------------------------------

def well_gamma(st, x, controls):
    """Wellbore fluid unit weight per well at the state x (frozen over a step)."""
    ph = st.ph
    P, S, C, Pb = unpack(st, x)
    pr = cell_properties(ph, st.phi_r, *_cell_duals(st, x))
    out = np.zeros(st.nw)
    for w, (wl, ctl) in enumerate(zip(st.wells, controls)):
        if wl["kind"] == "inj":
            out[w] = ph["g"] * ph["rho_w"] * (1.0 + ph["c_w"] * (Pb[w] - ph["p_ref"]))
        else:
            c = wl["cells"]
            lw = pr["krw"].v[c] / (pr["Rk"].v[c] * pr["mu_we"].v[c])
            lo = pr["kro"].v[c] / ph["mu_o"]
            lt = float(np.sum(lw + lo))
            if lt > 0.0:
                out[w] = ph["g"] * float(np.sum(lw * pr["rho_w"].v[c] + lo * pr["rho_o"].v[c])) / lt
            else:
                out[w] = ph["g"] * float(pr["rho_o"].v[c[0]])
    return out


RATE_COEF = {  # control, kind -> (s_w, s_o, reference density key)
    ("wrate", "inj"): (1.0, 0.0, "rho_w"),
    ("wrate", "prod"): (-1.0, 0.0, "rho_w"),
    ("orate", "prod"): (0.0, -1.0, "rho_o"),
    ("lrate", "prod"): (-1.0, None, "rho_w"),   # s_o = -rho_w,ref / rho_o,ref
}


def rate_coefficients(ph, ctrl, kind):
    s_w, s_o, key = RATE_COEF[(ctrl, kind)]
    if s_o is None:
        s_o = -ph["rho_w"] / ph["rho_o"]
    return s_w, s_o, ph[key]


def perforation_rates(st, pr, w, Pb_w, gamma_w, c_inj):
    """Phase mass rates (water, oil, polymer) into the perforated cells of
    well w: the perforation rate of Sec. 2.4 with the hydrostatic wellbore
    pressure of the same section; Duals in (x_cell, P_b): 4 columns."""
    ph = st.ph
    wl = st.wells[w]
    c = wl["cells"]
    m = len(c)

    def cellq(q):
        return q.take(c).embed(4, 0)

    Pb = Dual(np.full(m, Pb_w), np.tile(np.array([0.0, 0.0, 0.0, 1.0]), (m, 1)))
    Pbm = Pb + gamma_w * (wl["z"] - wl["zb"])
    krw, kro, Rk, mu_we = cellq(pr["krw"]), cellq(pr["kro"]), cellq(pr["Rk"]), cellq(pr["mu_we"])
    rho_w, rho_o, P, Pw, C = cellq(pr["rho_w"]), cellq(pr["rho_o"]), cellq(pr["P"]), cellq(pr["Pw"]), cellq(pr["C"])
    lam_w = krw / (Rk * mu_we)
    lam_o = kro / ph["mu_o"]
    WI = wl["WI"]
    if wl["kind"] == "inj":
        qw = WI * (lam_w + lam_o) * rho_w * (Pbm - Pw)
        qo = Dual.const(np.zeros(m), 4)
        qp = qw * (c_inj / ph["rho_w"])
    else:
        qw = WI * lam_w * rho_w * (Pbm - Pw)
        qo = WI * lam_o * rho_o * (Pbm - P)
        qp = qw * C / ph["rho_w"]
    return qw, qo, qp


# ---------------------------------------------------------------------------
# residual and Jacobian
# ---------------------------------------------------------------------------

def assemble(st, x, M_old, dt, controls, gamma, with_jacobian=True):
    """Residual R (length 3N + W) and sparse Jacobian dR/dx at the state x.

    Cell rows: R = M(x) - M^n - dt (sum of face inflows + well sources)
    (backward Euler, Sec. 3.1).  Well rows: the active constraint."""
    n, ph = st.n, st.ph
    P, S, C = _cell_duals(st, x)
    pr = cell_properties(ph, st.phi_r, P, S, C)
    Mo, Mw, Mp = accumulation(st, ph, pr)
    R = np.zeros(st.nunk)
    R[0:3 * n:3] = Mo.v - M_old[0]
    R[1:3 * n:3] = Mw.v - M_old[1]
    R[2:3 * n:3] = Mp.v - M_old[2]
    rows, cols, vals = [], [], []
    cell = np.arange(n)

    def add_block(rblk, cblk, blk):
        # blk: (m, 3, 3) derivative blocks d R[3 rblk + a] / d x[3 cblk + b]
        a = np.arange(3)
        rows.append((3 * rblk[:, None, None] + a[None, :, None]).repeat(3, axis=2).ravel())
        cols.append((3 * cblk[:, None, None] + a[None, None, :]).repeat(3, axis=1).ravel())
        vals.append(blk.ravel())

    if with_jacobian:
        add_block(cell, cell, np.stack([Mo.d, Mw.d, Mp.d], axis=1))

    for d, (L, H) in st.faces.items():
        if L.size == 0:
            continue
        dZ = st.Z[H] - st.Z[L]
        Fo, Fw, Fp = face_fluxes(st, pr, L, H, st.T[d], dZ)
        F = np.stack([Fo.v, Fw.v, Fp.v], axis=1)      # (f, 3) H -> L
        np.add.at(R, 3 * L[:, None] + np.arange(3), -dt * F)
        np.add.at(R, 3 * H[:, None] + np.arange(3), dt * F)
        if with_jacobian:
            dF = np.stack([Fo.d, Fw.d, Fp.d], axis=1)  # (f, 3, 6)
            dL, dH = dF[:, :, :3], dF[:, :, 3:]
            add_block(L, L, -dt * dL)
            add_block(L, H, -dt * dH)
            add_block(H, L, dt * dL)
            add_block(H, H, dt * dH)

    Pb = x[3 * n:]
    for w, wl in enumerate(st.wells):
        ctl = controls[w]
        qw, qo, qp = perforation_rates(st, pr, w, Pb[w], gamma[w], ctl["c_inj"])
        c = wl["cells"]
        q = np.stack([qo.v, qw.v, qp.v], axis=1)       # rows ordered oil, water, polymer
        np.add.at(R, 3 * c[:, None] + np.arange(3), -dt * q)
        wrow = 3 * n + w
        if ctl["ctrl"] == "bhp":
            R[wrow] = dt * wl["W"] * (Pb[w] - ctl["target"])
        else:
            s_w, s_o, rho_t = rate_coefficients(ph, ctl["ctrl"], wl["kind"])
            R[wrow] = dt * (s_w * qw.v.sum() + s_o * qo.v.sum() - rho_t * ctl["target"])
        if with_jacobian:
            dq = np.stack([qo.d, qw.d, qp.d], axis=1)   # (m, 3, 4)
            add_block(c, c, -dt * dq[:, :, :3])
            for r in range(3):                         # d R_cell / d P_b
                rows.append(3 * c + r)
                cols.append(np.full(len(c), wrow))
                vals.append(-dt * dq[:, r, 3])
            if ctl["ctrl"] == "bhp":
                rows.append(np.array([wrow])); cols.append(np.array([wrow]))
                vals.append(np.array([dt * wl["W"]]))
            else:
                dsum = s_w * qw.d + s_o * qo.d             # (m, 4)
                for b in range(3):
                    rows.append(np.full(len(c), wrow)); cols.append(3 * c + b)
                    vals.append(dt * dsum[:, b])
                rows.append(np.array([wrow])); cols.append(np.array([wrow]))
                vals.append(np.array([dt * dsum[:, 3].sum()]))
    if not with_jacobian:
        return R, None
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(st.nunk, st.nunk)).tocsr()
    J.sum_duplicates()
    return R, J


def masses(st, x):
    P, S, C = _cell_duals(st, x)
    pr = cell_properties(st.ph, st.phi_r, P, S, C)
    Mo, Mw, Mp = accumulation(st, st.ph, pr)
    return np.stack([Mo.v, Mw.v, Mp.v])


def scaled_residual(st, R, dt, controls):
    """Max-norm of the residual in dimensionless units: cell rows over
    V phi_r rho_ref (polymer over V phi_r C_ref), rate rows over
    dt rho_ref |target|, BHP rows over dt W * 1 bar."""
    n, ph = st.n, st.ph
    pv = st.V * st.phi_r
    s = np.abs(R[0:3 * n:3]) / (pv * ph["rho_o"])
    s = np.maximum(s, np.abs(R[1:3 * n:3]) / (pv * ph["rho_w"]))
    s = np.maximum(s, np.abs(R[2:3 * n:3]) / (pv * ph["c_ref"]))
    out = float(s.max()) if n else 0.0
    for w, wl in enumerate(st.wells):
        ctl = controls[w]
        if ctl["ctrl"] == "bhp":
            sc = dt * wl["W"] * 1.0e5
        else:
            _, _, rho_t = rate_coefficients(ph, ctl["ctrl"], wl["kind"])
            sc = dt * rho_t * max(abs(ctl["target"]), 1e-30)
        out = max(out, abs(R[3 * n + w]) / sc)
    return out


# ---------------------------------------------------------------------------
# Newton (Algorithm 1) and the forcing term of Sec. 3.3
# ---------------------------------------------------------------------------

GOLDEN = (math.sqrt(5.0) + 1.0) / 2.0


def forcing_term(norm_b, norm_b_prev, gamma=0.5, beta=GOLDEN, lo=0.01, hi=0.1):
    """Third choice of the Sec. 3.3 forcing term, restricted to [0.01, 0.1]; the first
    iteration (no previous norm) takes the upper bound."""
    if norm_b_prev is None or norm_b_prev <= 0.0:
        return hi
    eta = gamma * (norm_b / norm_b_prev) ** beta
    return min(max(eta, lo), hi)


def forcing_term_difference(b, r_prev, norm_b_prev, lo=0.01, hi=0.1):
    """First choice of the Sec. 3.3 forcing term: |b^l - r^{l-1}| / |b^{l-1}|, where b^l is
    the current right-hand side (-R) and r^{l-1} = b^{l-1} - J^{l-1} dx^{l-1}
    the residual the previous Newton iteration's linear solve left; the
    numerator measures how far the linear model of the previous iteration
    missed the new residual.  Restricted to [0.01, 0.1]; the first iteration
    (no previous solve) takes the upper bound."""
    if r_prev is None or norm_b_prev is None or norm_b_prev <= 0.0:
        return hi
    eta = float(np.linalg.norm(np.asarray(b) - np.asarray(r_prev))) / norm_b_prev
    return min(max(eta, lo), hi)


def forcing_term_norms(norm_b, norm_r_prev, norm_b_prev, lo=0.01, hi=0.1):
    """Second choice of the Sec. 3.3 forcing term: (|b^l| - |r^{l-1}|) / |b^{l-1}|, taken
    as printed (no absolute value: a negative value is restricted to the
    lower bound).  Restricted to [0.01, 0.1]; first iteration: upper bound."""
    if norm_r_prev is None or norm_b_prev is None or norm_b_prev <= 0.0:
        return hi
    eta = (norm_b - norm_r_prev) / norm_b_prev
    return min(max(eta, lo), hi)


def update(st, x, dx, ds_max, dc_frac=0.5):
    """x + dx with the saturation change chopped to +-ds_max and the
    concentration change to +-dc_frac * C_ref per cell, then S clipped to
    [0, 1] and C to >= 0 (these limits shape the path, not the root)."""
    n = st.n
    y = x.copy()
    y[0:3 * n:3] += dx[0:3 * n:3]
    ds = np.clip(dx[1:3 * n:3], -ds_max, ds_max)
    y[1:3 * n:3] = np.clip(x[1:3 * n:3] + ds, 0.0, 1.0)
    dc_max = dc_frac * st.ph["c_ref"]
    dc = np.clip(dx[2:3 * n:3], -dc_max, dc_max)
    y[2:3 * n:3] = np.maximum(x[2:3 * n:3] + dc, 0.0)
    y[3 * n:] += dx[3 * n:]
    return y


def solve_linear(J, b):
    """Direct sparse solve of J x = b (the plain definition of the Newton
    correction); a library LU serves as the step."""
    return spla.spsolve(J.tocsc(), b)


def initial_state(st):
    sc = st.sc
    x = np.empty(st.nunk)
    x[0:3 * st.n:3] = sc["P0"]
    x[1:3 * st.n:3] = sc["S0"]
    x[2:3 * st.n:3] = sc["C0"]
    x[3 * st.n:] = [w["Pb0"] for w in sc["wells"]]
    return x


def limit_crossings(st, x, controls, switched):
    """In-iteration limit check: a rate well with a BHP limit whose current
    P_b crosses it (above for an injector, below for a producer) is moved onto
    BHP = limit for the rest of the step.  Returns True if anything switched."""
    changed = False
    for w, c in enumerate(controls):
        if c["ctrl"] == "bhp" or not c.get("limit") or switched[w]:
            continue
        pb = x[3 * st.n + w]
        kind = st.wells[w]["kind"]
        if (kind == "inj" and pb > c["limit"]) or (kind == "prod" and pb < c["limit"]):
            switched[w] = True
            changed = True
    return changed


def newton_step(st, x_old, dt, controls, tol=1e-10, max_iter=25, ds_max=0.2, record=None, switched=None,
                div=1e6):
    """One backward-Euler step by Newton's method (Algorithm 1) under the user
    controls; rate wells flagged in ``switched`` (updated in place by the
    in-iteration limit check) run on their BHP limit.  The step fails at the
    iteration cap, on a non-finite residual, or once the scaled residual
    exceeds ``div`` times its first value (runaway iterates; 0 disables).

    Returns (x_new, converged, iterations)."""
    if switched is None:
        switched = [False] * st.nw
    eff = effective_controls(st, controls, switched)
    M_old = masses(st, x_old)
    gamma = well_gamma(st, x_old, eff)
    x = x_old.copy()
    for it in range(max_iter + 1):
        R, J = assemble(st, x, M_old, dt, eff, gamma)
        res = scaled_residual(st, R, dt, eff)
        if record is not None:
            record.append(res)
        if res <= tol:
            return x, True, it
        if it == 0:
            res0 = res
        elif div > 0.0 and res > div * res0:
            break
        if it == max_iter or not np.all(np.isfinite(R)):
            break
        dx = solve_linear(J, -R)
        x = update(st, x, dx, ds_max)
        if limit_crossings(st, x, controls, switched):
            eff = effective_controls(st, controls, switched)
    return x_old, False, max_iter


def controls_with_defaults(controls):
    return [dict(c) for c in controls]


def well_totals(st, x, controls, gamma):
    """Per well: summed water and oil mass rates into the reservoir (positive
    for injection) at the state x (the perforation rate of Sec. 2.4), and the
    reference BHP."""
    pr = cell_properties(st.ph, st.phi_r, *_cell_duals(st, x))
    out = []
    for w in range(st.nw):
        qw, qo, _ = perforation_rates(st, pr, w, x[3 * st.n + w], gamma[w], controls[w]["c_inj"])
        out.append((float(qw.v.sum()), float(qo.v.sum()), float(x[3 * st.n + w])))
    return out


def controlled_rate(ph, kind, ctrl, qw, qo):
    """The volume rate a rate constraint refers to (Sec. 2.4), positive."""
    if kind == "inj":
        return qw / ph["rho_w"]
    if ctrl == "wrate":
        return -qw / ph["rho_w"]
    if ctrl == "orate":
        return -qo / ph["rho_o"]
    return -(qw / ph["rho_w"] + qo / ph["rho_o"])


def effective_controls(st, controls, switched):
    """Rate wells switched onto their BHP limit run under BHP = limit."""
    out = []
    for w, c in enumerate(controls):
        if switched[w]:
            out.append(dict(c, ctrl="bhp", target=c["limit"]))
        else:
            out.append(dict(c))
    return out


def update_switches(st, controls, switched, totals):
    """Limit check after a converged step.  A rate well whose BHP crosses its
    limit (above it for an injector, below it for a producer) moves to BHP
    control at the limit; a switched well whose rate at the limit exceeds its
    target returns to rate control.  Returns True if anything changed."""
    changed = False
    for w, c in enumerate(controls):
        if c["ctrl"] == "bhp" or not c.get("limit"):
            continue
        kind = st.wells[w]["kind"]
        qw, qo, pb = totals[w]
        if not switched[w]:
            if (kind == "inj" and pb > c["limit"]) or (kind == "prod" and pb < c["limit"]):
                switched[w] = True
                changed = True
        else:
            if controlled_rate(st.ph, kind, c["ctrl"], qw, qo) > c["target"]:
                switched[w] = False
                changed = True
    return changed


def run(sc, n_steps=None, tol=1e-10, max_iter=25, ds_max=0.2, max_cuts=6, max_switch_solves=2,
        callback=None):
    """Time loop over the scenario schedule with fixed steps; on a Newton
    failure the step is cut in half and retried (Sec. 3, step 4(a)); controls
    stay fixed within a step (step 4(b)) except that a rate well crossing its
    BHP limit during the iterations moves onto the limit (``limit_crossings``);
    after convergence ``update_switches`` may switch it back, with up to
    ``max_switch_solves`` re-solves.  After an accepted sub-step the step
    doubles again, never beyond the schedule's step, so the loop keeps trying
    to lengthen the step (step 4(c)-(d))."""
    st = Setup(sc)
    x = initial_state(st)
    t = 0.0
    history = []
    done = 0
    switched = [False] * st.nw
    prev = None
    for period in sc["schedule"]:
        ctl = controls_with_defaults(period["controls"])
        if prev is not None:   # a well keeps its switched state while its constraint is unchanged
            for w in range(st.nw):
                if any(ctl[w].get(k) != prev[w].get(k) for k in ("ctrl", "target", "limit")):
                    switched[w] = False
        prev = ctl
        for _ in range(period["n_steps"]):
            if n_steps is not None and done >= n_steps:
                return st, x, history
            dt_left = period["dt"]
            dt = dt_left
            cuts = 0
            newton_total = 0
            accepted = []
            while dt_left > 0.0:
                dt = min(dt, dt_left)
                for attempt in range(max_switch_solves + 1):
                    xn, ok, its = newton_step(st, x, dt, ctl, tol=tol, max_iter=max_iter, ds_max=ds_max,
                                              switched=switched)
                    newton_total += its
                    if not ok or attempt == max_switch_solves:
                        break
                    eff = effective_controls(st, ctl, switched)
                    gam = well_gamma(st, x, eff)
                    if not update_switches(st, ctl, switched, well_totals(st, xn, eff, gam)):
                        break
                if ok:
                    x = xn
                    t += dt
                    dt_left -= dt
                    accepted.append(dt)
                    # after a cut the step grows again, doubling up to the
                    # schedule's step (Sec. 3 step 4(c)-(d))
                    dt = min(2.0 * dt, period["dt"])
                else:
                    cuts += 1
                    if cuts > max_cuts:
                        raise RuntimeError("time step cut limit reached")
                    dt = 0.5 * dt
            done += 1
            history.append(dict(t=t, x=x.copy(), newton=newton_total, cuts=cuts, switched=list(switched),
                                substeps=accepted))
            if callback is not None:
                callback(st, x, history[-1])
    return st, x, history
