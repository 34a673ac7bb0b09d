"""Pins of the FP64 oracle against closed forms, invariants and independent
computations (no GPU).  Each test names the paper passage it pins.

A plausible slip in the oracle -- a dropped term, a wrong sign or index, a
transposed operand -- is meant to fail at least one of these.
"""

import math

import numpy as np
import pytest

from oracle import model as M
from oracle.linalg import lu_solve_dense
from scenarios import generate as G

DAY, BAR, MD, CP = G.DAY, G.BAR, G.MD, G.CP


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def one_d(n, L=1000.0, area=100.0, phi=0.2, perm_md=100.0, physics=None, q_day=20.0,
          c_inj=0.0, s0=None, c0=0.0, dt_days=1.0, n_steps=10, bhp=200.0 * BAR, perm=None):
    side = math.sqrt(area)
    dx = L / n
    k = np.full(n, perm_md * MD) if perm is None else perm
    wells = [dict(kind="inj", cells=[0]), dict(kind="prod", cells=[n - 1])]
    ctl = [dict(ctrl="wrate", target=q_day / DAY, limit=None, c_inj=c_inj),
           dict(ctrl="bhp", target=bhp, limit=None, c_inj=0.0)]
    sched = [dict(n_steps=n_steps, dt=dt_days * DAY, controls=ctl)]
    return G.make_scenario(n, 1, 1, dx, side, side, 1000.0, k, k, k, np.full(n, phi), physics,
                           wells, sched, p_top=200.0 * BAR, s0=s0, c0=c0)


def incompressible(**over):
    base = dict(c_w=0.0, c_o=0.0, c_r=0.0, g=0.0, pc_e=0.0)
    base.update(over)
    return G.default_physics(**base)


def field(st, x, comp):
    return x[comp:3 * st.n:3]


# ---------------------------------------------------------------------------
# Buckley-Leverett waterflood (Sec. 2.2 flow equations, Sec. 3.2 upstream k_r)
# ---------------------------------------------------------------------------

def _fractional_flow(ph):
    def f(S):
        sn = np.clip((S - ph["swc"]) / (1.0 - ph["swc"] - ph["sor"]), 0.0, 1.0)
        lw = sn ** ph["nw"] / ph["mu_w"]
        lo = (1.0 - sn) ** ph["no"] / ph["mu_o"]
        return lw / (lw + lo)

    def df(S, h=1e-7):
        return (f(S + h) - f(S - h)) / (2.0 * h)

    return f, df


def welge_profile(ph, x, t, u, phi):
    """Self-similar Buckley-Leverett saturation with the Welge tangent front."""
    f, df = _fractional_flow(ph)
    si, smax = ph["swc"], 1.0 - ph["sor"]
    lo, hi = si + 1e-6, smax - 1e-9
    g = lambda s: df(s) * (s - si) - f(s)
    for _ in range(200):                      # g > 0 below the tangent point
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    sf = 0.5 * (lo + hi)
    xf = u * t * df(sf) / phi
    out = np.full_like(x, si)
    for i, xi in enumerate(x):
        if xi < xf:
            a, b = sf, smax                       # df decreasing on [sf, smax]
            for _ in range(100):
                mid = 0.5 * (a + b)
                if u * t * df(mid) / phi > xi:
                    a = mid
                else:
                    b = mid
            out[i] = 0.5 * (a + b)
    return out, sf, xf


@pytest.mark.slow
def test_buckley_leverett_front_and_refinement():
    ph = incompressible(mu_w=1.0 * CP, mu_o=2.0 * CP, ads_a=0.0, rrf=1.0, ipv=0.0, mu_p0=1.0 * CP)
    t_end = 150.0
    errs, fronts = [], []
    for n, dt in [(50, 2.0), (200, 0.5)]:
        sc = one_d(n, physics=ph, dt_days=dt, n_steps=int(round(t_end / dt)))
        st, x, hist = M.run(sc)
        S = field(st, x, 1)
        dx = 1000.0 / n
        xc = (np.arange(n) + 0.5) * dx
        u = 20.0 / DAY / 100.0
        Sex, sf, xf = welge_profile(ph, xc, t_end * DAY, u, 0.2)
        errs.append(np.sum(np.abs(S - Sex)) * dx / 1000.0)
        mid = 0.5 * (sf + ph["swc"])
        i = int(np.nonzero(S < mid)[0][0])
        x_mid = xc[i - 1] + (S[i - 1] - mid) / (S[i - 1] - S[i]) * dx
        fronts.append((x_mid, xf, dx))
    assert errs[1] < 0.7 * errs[0], errs
    for x_mid, xf, dx in fronts:
        assert abs(x_mid - xf) < max(3.0 * dx, 0.03 * xf), (x_mid, xf, dx)


# ---------------------------------------------------------------------------
# polymer shock speed (Sec. 2.3 polymer equation, adsorption, IPV)
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("ads_a", [0.0, 0.05])
def test_polymer_front_rankine_hugoniot(ads_a):
    ph = incompressible(swc=0.0, sor=0.0, ads_a=ads_a, ads_b=10.0, ipv=0.1, rrf=1.5,
                        mu_w=1.0 * CP, mu_p0=4.0 * CP, c_ref=2.0)
    n, t_end, dt = 200, 150.0, 0.5
    sc = one_d(n, physics=ph, q_day=20.0, c_inj=1.0, s0=1.0, c0=0.0, dt_days=dt,
               n_steps=int(round(t_end / dt)))
    st, x, hist = M.run(sc)
    C = field(st, x, 2)
    phi, u, cin = 0.2, 20.0 / DAY / 100.0, 1.0
    ads = ads_a * cin / (1.0 + 10.0 * cin)
    vs = u * cin / (phi * (1.0 - 0.1) * cin + (1.0 - phi) * ads)
    xs = vs * t_end * DAY
    dx = 1000.0 / n
    xc = (np.arange(n) + 0.5) * dx
    i = int(np.nonzero(C < 0.5 * cin)[0][0])
    x_half = xc[i - 1] + (C[i - 1] - 0.5 * cin) / (C[i - 1] - C[i]) * dx
    assert abs(x_half - xs) < 3.0 * dx, (x_half, xs)
    assert np.allclose(field(st, x, 1), 1.0)


# ---------------------------------------------------------------------------
# Darcy series resistance (Darcy's law Sec. 2.2, harmonic averaging Sec. 3.2,
# R_k and mixing rule Sec. 2.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mixing,omega", [(0, 1.0), (1, 1.0)])
def test_darcy_pressure_drop_series(mixing, omega):
    c_ref, mu_w, mu_p0, rrf = 2.0, 1.0 * CP, 9.0 * CP, 2.2
    ph = incompressible(swc=0.0, sor=0.0, ads_a=0.3, ads_b=1.0, ipv=0.1, rrf=rrf, mu_w=mu_w,
                        mu_p0=mu_p0, c_ref=c_ref, mixing=mixing, omega=omega)
    n = 12
    rng = np.random.default_rng(5)
    perm = np.exp(rng.normal(math.log(100.0), 0.8, n)) * MD
    C = 1.0                                    # beta = 1/2 and b C = 1
    sc = one_d(n, physics=ph, q_day=30.0, c_inj=C, s0=1.0, c0=C, n_steps=1, perm=perm)
    st, x, _ = M.run(sc)
    P = field(st, x, 0)
    mu = math.sqrt(mu_p0 * mu_w) if mixing == 0 else 0.5 * (mu_p0 + mu_w)
    Rk = 1.0 + (rrf - 1.0) * 0.5               # A_d / A_d,max = bC / (1 + bC) = 1/2
    q, A, dx = 30.0 / DAY, 100.0, 1000.0 / n
    for i in range(n - 1):
        expect = q * mu * Rk * (dx / (2.0 * perm[i]) + dx / (2.0 * perm[i + 1])) / A
        assert P[i] - P[i + 1] == pytest.approx(expect, rel=1e-7)


# ---------------------------------------------------------------------------
# gravity: hydrostatic rest and segregation (Sec. 2.2 gravity term)
# ---------------------------------------------------------------------------

def test_static_wellbore_in_a_water_column_does_not_flow():
    """Sec. 2.4, the perforation rate and the hydrostatic wellbore: a producer
    perforated through a water-filled column at rest, held at the static wellbore pressure of its
    top perforation, draws nothing from any perforation: the wellbore gradient
    gamma of a producer is the mobility-weighted mixture density (here water)
    times g, and the perforation pressures shift by gamma (z_m - z_b).  The same
    state with an oil-density gradient would flow (checked as the control)."""
    ph = G.default_physics(c_w=0.0, c_o=0.0, c_r=0.0, pc_e=0.0)
    nx, ny, nz, dz, top = 3, 3, 6, 4.0, 1500.0
    n = nx * ny * nz
    k = np.full(n, 200.0 * MD)
    col = [1 + nx * (1 + ny * kk) for kk in range(nz)]
    sc = G.make_scenario(nx, ny, nz, 20.0, 20.0, dz, top, k, k, 0.1 * k, np.full(n, 0.2), ph,
                         [dict(kind="prod", cells=col)], [dict(n_steps=1, dt=DAY, controls=[])], s0=1.0)
    st = M.Setup(sc)
    z = top + (np.arange(nz) + 0.5) * dz
    p_top = 180.0 * BAR
    P = np.repeat(p_top + ph["rho_w"] * ph["g"] * (z - z[0]), nx * ny)   # water hydrostatics
    x = np.zeros(st.nunk)
    x[0:3 * n:3], x[1:3 * n:3], x[2:3 * n:3] = P, 1.0, 0.0
    x[3 * n] = P[col[0]]
    ctl = [dict(ctrl="bhp", target=P[col[0]], limit=None, c_inj=0.0)]
    gam = M.well_gamma(st, x, ctl)
    assert gam[0] == pytest.approx(ph["g"] * ph["rho_w"], rel=1e-14)
    R, _ = M.assemble(st, x, M.masses(st, x), DAY, ctl, gam, with_jacobian=False)
    assert M.scaled_residual(st, R, DAY, ctl) < 1e-12
    R_oil, _ = M.assemble(st, x, M.masses(st, x), DAY, ctl, np.array([ph["g"] * ph["rho_o"]]),
                          with_jacobian=False)
    assert M.scaled_residual(st, R_oil, DAY, ctl) > 1e-6


def test_rate_controls_deliver_their_reference_volumes():
    """Sec. 2.4 rate constraints with B = 1: after a converged step, a water-
    rate injector puts in its target water volume at reference conditions,
    and producers on liquid-rate and oil-rate control take out their target
    liquid (water + oil) and oil volumes, each phase's mass rate divided by its
    own reference density."""
    ph = G.default_physics()
    nx, ny, nz = 7, 6, 2
    n = nx * ny * nz
    k = np.full(n, 150.0 * MD)
    col = lambda i, j: [i + nx * (j + ny * kk) for kk in range(nz)]
    wells = [dict(kind="inj", cells=col(0, 0)), dict(kind="prod", cells=col(nx - 1, ny - 1)),
             dict(kind="prod", cells=col(nx - 1, 0))]
    ctl = [dict(ctrl="wrate", target=60.0 / DAY, limit=None, c_inj=0.5),
           dict(ctrl="lrate", target=25.0 / DAY, limit=None, c_inj=0.0),
           dict(ctrl="orate", target=15.0 / DAY, limit=None, c_inj=0.0)]
    sc = G.make_scenario(nx, ny, nz, 20.0, 20.0, 4.0, 1500.0, k, k, 0.1 * k, np.full(n, 0.2), ph, wells,
                         [dict(n_steps=1, dt=DAY, controls=ctl)], s0=0.45)
    st = M.Setup(sc)
    x0 = M.initial_state(st)
    x1, ok, _ = M.newton_step(st, x0, 2.0 * DAY, ctl, tol=1e-12)
    assert ok
    (qw0, qo0, _), (qw1, qo1, _), (qw2, qo2, _) = M.well_totals(st, x1, ctl, M.well_gamma(st, x0, ctl))
    rw, ro = ph["rho_w"], ph["rho_o"]
    assert qw0 / rw == pytest.approx(60.0 / DAY, rel=1e-9) and qo0 == 0.0
    assert -(qw1 / rw + qo1 / ro) == pytest.approx(25.0 / DAY, rel=1e-9)
    assert -qo2 / ro == pytest.approx(15.0 / DAY, rel=1e-9)
    assert qw1 < 0.0 and qo1 < 0.0 and qw2 <= 0.0          # both phases flow out of the producers


def test_rock_compressibility_closed_tank():
    """Sec. 2.1 porosity law phi(P) = phi_r + c_r (P - P_r), pinned by a
    closed tank: one 10 m cube full of water (S_w = 1, so k_ro = 0 and only
    water moves), incompressible fluids, c_r = 1e-4 / bar, and a producer that
    takes q = 0.5 m^3/day of water.  The water mass V phi(P) rho_w can only fall
    by rho_w q dt, so with the additive law V c_r (P1 - P0) = -q dt:
        P1 = P0 - q dt / (V c_r) = 250 bar - 0.5 / (1000 * 1e-9 / Pa) = 245 bar
    after one day, and 240 bar after a second one.  The multiplicative form
    phi_r (1 + c_r (P - P_r)) would give 225 bar (a drop divided by phi_r =
    0.2), and a flipped sign would raise the pressure.  P0 = 250 bar differs
    from P_r = 200 bar, so a law anchored at P instead of P_r fails as well."""
    ph = G.default_physics(c_w=0.0, c_o=0.0, c_r=1.0e-4 / BAR, p_r=200.0 * BAR, pc_e=0.0)
    k = np.full(1, 100.0 * MD)
    wells = [dict(kind="prod", cells=[0])]
    ctl = [dict(ctrl="wrate", target=0.5 / DAY, limit=None, c_inj=0.0)]
    sc = G.make_scenario(1, 1, 1, 10.0, 10.0, 10.0, 1000.0, k, k, k, np.full(1, 0.2), ph, wells,
                         [dict(n_steps=2, dt=DAY, controls=ctl)], p_top=250.0 * BAR, s0=1.0, c0=0.0)
    st = M.Setup(sc)
    x0 = M.initial_state(st)
    assert x0[0] == 250.0 * BAR and x0[1] == 1.0
    x1, ok, _ = M.newton_step(st, x0, DAY, ctl, tol=1e-11)
    assert ok
    assert x1[0] == pytest.approx(245.0 * BAR, rel=1e-9)
    assert x1[1] == pytest.approx(1.0, abs=1e-12) and abs(x1[2]) < 1e-15
    x2, ok, _ = M.newton_step(st, x1, DAY, ctl, tol=1e-11)
    assert ok
    assert x2[0] == pytest.approx(240.0 * BAR, rel=1e-9)


def test_hydrostatic_rest_is_a_root():
    ph = G.default_physics(c_w=0.0, c_o=0.0, c_r=0.0)
    nx, ny, nz = 3, 2, 6
    n = nx * ny * nz
    k = np.exp(np.random.default_rng(1).normal(math.log(50.0), 1.0, n)) * MD
    phi = np.repeat(np.linspace(0.1, 0.3, nz), nx * ny)
    sc = G.make_scenario(nx, ny, nz, 10.0, 10.0, 3.0, 1500.0, k, k, k, phi, ph, [], [
        dict(n_steps=2, dt=10 * DAY, controls=[])])
    st = M.Setup(sc)
    x = M.initial_state(st)
    R, _ = M.assemble(st, x, M.masses(st, x), 10 * DAY, [], np.zeros(0), with_jacobian=False)
    assert M.scaled_residual(st, R, 10 * DAY, []) < 1e-12
    st, x2, hist = M.run(sc)
    assert np.allclose(x2, x, rtol=1e-12, atol=1e-9)
    assert hist[0]["newton"] == 0


def test_water_sinks_below_oil():
    ph = G.default_physics()
    nx, ny, nz = 1, 1, 4
    k = np.full(4, 500.0 * MD)
    sc = G.make_scenario(nx, ny, nz, 10.0, 10.0, 2.0, 1500.0, k, k, k, np.full(4, 0.25), ph, [],
                         [dict(n_steps=1, dt=1 * DAY, controls=[])])
    sc["S0"] = np.array([0.8, 0.8, 0.2, 0.2])
    st, x, _ = M.run(sc)
    S = field(st, x, 1)
    assert S[0] < 0.8 and S[1] < 0.8 and S[3] > 0.2
    # total water is conserved without wells (masses change only through compression)
    assert abs(S.sum() - 2.0) < 1e-3


# ---------------------------------------------------------------------------
# conservation, symmetry and special cases
# ---------------------------------------------------------------------------

def _random_state(st, rng):
    x = M.initial_state(st)
    n = st.n
    x[0:3 * n:3] += rng.normal(0.0, 2.0 * BAR, n)
    x[1:3 * n:3] = rng.uniform(0.25, 0.75, n)
    x[2:3 * n:3] = rng.uniform(0.1, 1.5, n)
    return x


def test_interior_fluxes_cancel_mass_balance():
    sc = G.scenario_c1(nx=5, ny=4, nz=3)
    st = M.Setup(sc)
    rng = np.random.default_rng(7)
    x_old = _random_state(st, rng)
    x = _random_state(st, rng)
    ctl = sc["schedule"][0]["controls"]
    gam = M.well_gamma(st, x_old, ctl)
    dt = 2.0 * DAY
    M_old = M.masses(st, x_old)
    R, _ = M.assemble(st, x, M_old, dt, ctl, gam, with_jacobian=False)
    Mnew = M.masses(st, x)
    pr = M.cell_properties(st.ph, st.phi_r, *M._cell_duals(st, x))
    src = np.zeros(3)
    for w in range(st.nw):
        qw, qo, qp = M.perforation_rates(st, pr, w, x[3 * st.n + w], gam[w], ctl[w]["c_inj"])
        src += [qo.v.sum(), qw.v.sum(), qp.v.sum()]
    for a in range(3):
        lhs = R[a:3 * st.n:3].sum()
        rhs = Mnew[a].sum() - M_old[a].sum() - dt * src[a]
        scale = Mnew[a].sum()
        assert abs(lhs - rhs) <= 1e-12 * scale


def test_five_spot_symmetry():
    ph = G.default_physics()
    nx = ny = 7
    n = nx * ny
    k = np.full(n, 100.0 * MD)
    corners = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]
    wells = [dict(kind="inj", cells=[i + nx * j]) for (i, j) in corners]
    wells.append(dict(kind="prod", cells=[nx // 2 + nx * (ny // 2)]))
    ctl = [dict(ctrl="wrate", target=50.0 / DAY, limit=None, c_inj=1.0)] * 4 + \
          [dict(ctrl="bhp", target=150.0 * BAR, limit=None, c_inj=0.0)]
    sc = G.make_scenario(nx, ny, 1, 20.0, 20.0, 5.0, 2000.0, k, k, k, np.full(n, 0.2), ph, wells,
                         [dict(n_steps=4, dt=5 * DAY, controls=ctl)])
    st, x, _ = M.run(sc)
    for comp in range(3):
        f = field(st, x, comp).reshape(ny, nx)
        scale = np.abs(f).max()
        assert np.abs(f - f.T).max() <= 1e-8 * scale
        assert np.abs(f - f[:, ::-1]).max() <= 1e-8 * scale
        assert np.abs(f - f[::-1, :]).max() <= 1e-8 * scale


def test_passive_tracer_special_case():
    base = dict(rrf=1.0, ads_a=0.0, ipv=0.0, mu_p0=G.default_physics()["mu_w"])
    runs = []
    for c in (0.0, 0.7):
        sc = G.scenario_c1(nx=5, ny=5, nz=2, n_steps=4)
        sc["physics"] = G.default_physics(**base)
        sc["C0"][:] = c
        sc["schedule"][0]["controls"] = [dict(cc, c_inj=c) if cc["ctrl"] != "bhp" else dict(cc)
                                         for cc in sc["schedule"][0]["controls"]]
        st, x, _ = M.run(sc)
        runs.append((st, x))
    (st, x0), (_, x1) = runs
    assert np.allclose(field(st, x1, 2), 0.7, rtol=1e-9)
    for comp in (0, 1):
        assert np.allclose(field(st, x1, comp), field(st, x0, comp), rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------------------
# Jacobian: exact (dual numbers) versus central finite differences
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mixing,omega,pc", [(0, 0.6, 0.3 * BAR), (1, 1.0, 0.0)])
def test_jacobian_matches_finite_differences(mixing, omega, pc):
    sc = G.scenario_c1(nx=4, ny=3, nz=2)
    sc["physics"] = G.default_physics(mixing=mixing, omega=omega, pc_e=pc)
    ctl = [dict(ctrl="wrate", target=100.0 / DAY, limit=None, c_inj=1.2),
           dict(ctrl="lrate", target=80.0 / DAY, limit=None, c_inj=0.0)]
    st = M.Setup(sc)
    rng = np.random.default_rng(3)
    x_old = _random_state(st, rng)
    x = _random_state(st, rng)
    x[3 * st.n:] += [10.0 * BAR, -10.0 * BAR]
    gam = M.well_gamma(st, x_old, ctl)
    dt = 3.0 * DAY
    M_old = M.masses(st, x_old)
    R, J = M.assemble(st, x, M_old, dt, ctl, gam)
    J = J.toarray()
    for j in range(st.nunk):
        h = 1e-7 * abs(x[j]) if (j >= 3 * st.n or j % 3 == 0) else 1e-7
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        Rp, _ = M.assemble(st, xp, M_old, dt, ctl, gam, with_jacobian=False)
        Rm, _ = M.assemble(st, xm, M_old, dt, ctl, gam, with_jacobian=False)
        col = (Rp - Rm) / (2.0 * h)
        scale = max(np.abs(J[:, j]).max(), 1e-300)
        assert np.abs(col - J[:, j]).max() <= 2e-6 * scale, j


# ---------------------------------------------------------------------------
# linear solve, forcing term, well index
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["corey", "capillary_linear_omega", "tables"])
def test_oil_rows_do_not_depend_on_polymer(variant):
    """Sec. 2.2-2.4: the oil accumulation (phi rho_o S_o), the oil flux
    (k k_ro(S) rho_o / mu_o times the oil potential) and the oil perforation
    rate (WI lambda_o rho_o (P_bm - P)) hold no polymer concentration, so every
    oil row of the Jacobian has an exact zero in every polymer column (the
    block products of the CUDA path skip that entry).  Checked on the oracle's
    dual-number Jacobian at a random state with injector and producers, for
    Corey curves, capillary pressure with the linear mixing rule and omega < 1,
    and tabulated curves."""
    if variant == "corey":
        ph = G.default_physics()
    elif variant == "capillary_linear_omega":
        ph = G.default_physics(pc_e=0.4 * BAR, mixing=1, omega=0.6, rrf=2.0)
    else:
        ph = G.default_physics(omega=0.7, sat_table=np.array([[0.1, 0.0, 1.0, 0.9 * BAR], [0.4, 0.1, 0.4, 0.3 * BAR],
                                                             [0.85, 0.8, 0.0, 0.01 * BAR]]),
                               poly_table=np.array([[0.0, 1.0, 0.0], [1.0, 3.5, 0.05], [2.5, 6.0, 0.065]]))
    nx, ny, nz = 5, 4, 3
    n = nx * ny * nz
    rng = np.random.default_rng(11)
    k = np.exp(rng.normal(math.log(100.0), 0.7, n)) * MD
    col = lambda i, j: [i + nx * (j + ny * kk) for kk in range(nz)]
    wells = [dict(kind="inj", cells=col(0, 0)), dict(kind="prod", cells=col(nx - 1, ny - 1)),
             dict(kind="prod", cells=col(nx - 1, 0))]
    ctl = [dict(ctrl="wrate", target=40.0 / DAY, limit=None, c_inj=1.0),
           dict(ctrl="bhp", target=150.0 * BAR, limit=None, c_inj=0.0),
           dict(ctrl="lrate", target=10.0 / DAY, limit=None, c_inj=0.0)]
    sc = G.make_scenario(nx, ny, nz, 20.0, 20.0, 4.0, 1500.0, k, k, 0.1 * k, np.full(n, 0.2), ph, wells,
                         [dict(n_steps=1, dt=DAY, controls=ctl)], s0=0.45, c0=0.3)
    st = M.Setup(sc)
    x_old = M.initial_state(st)
    x = x_old.copy()
    x[0:3 * n:3] += rng.normal(0.0, 2.0 * BAR, n)
    x[1:3 * n:3] = rng.uniform(0.22, 0.78, n)
    x[2:3 * n:3] = rng.uniform(0.05, 1.6, n)
    _, J = M.assemble(st, x, M.masses(st, x_old), DAY, ctl, M.well_gamma(st, x_old, ctl))
    J = J.tocsr()
    oil_C = J[0:3 * n:3, :][:, 2:3 * n:3]
    assert oil_C.count_nonzero() == 0
    # the other rows do carry polymer columns (the check is not vacuous)
    assert J[1:3 * n:3, :][:, 2:3 * n:3].count_nonzero() > n
    assert J[0:3 * n:3, :][:, 1:3 * n:3].count_nonzero() > n


def test_sparse_solve_matches_own_dense_lu():
    sc = G.scenario_c1(nx=4, ny=4, nz=2)
    st = M.Setup(sc)
    x = _random_state(st, np.random.default_rng(11))
    ctl = sc["schedule"][0]["controls"]
    gam = M.well_gamma(st, x, ctl)
    R, J = M.assemble(st, x, M.masses(st, x) * 0.999, DAY, ctl, gam)
    d1 = M.solve_linear(J, -R)
    d2 = lu_solve_dense(J.toarray(), -R)
    assert np.allclose(d1, d2, rtol=1e-9, atol=0.0) or \
        np.abs(d1 - d2).max() <= 1e-9 * np.abs(d2).max()
    assert np.linalg.norm(J @ d2 + R) <= 1e-10 * np.linalg.norm(R)


def test_forcing_term_third_choice():
    beta = (math.sqrt(5.0) + 1.0) / 2.0
    assert M.forcing_term(1.0, None) == 0.1
    assert M.forcing_term(1.0, 1.0) == 0.1                  # 0.5 clipped to 0.1
    assert M.forcing_term(0.1, 1.0) == pytest.approx(0.5 * 0.1 ** beta)
    assert M.forcing_term(1e-4, 1.0) == 0.01
    assert 0.5 * 0.1 ** beta == pytest.approx(0.0120486, rel=1e-5)


def test_forcing_term_first_and_second_choices():
    """Forcing term of Sec. 3.3, first and second choices.  For a linear F the previous
    linear model is exact, so b^l = r^{l-1} whatever the step: both
    numerators vanish and eta takes the lower bound.  For F(x) = x*x - c the
    model misses by exactly s*s (closed form).  The second choice never
    exceeds the first (triangle inequality) and, after an exact solve, is the
    ratio of the right-hand side norms."""
    inf = float("inf")
    rng = np.random.default_rng(7)
    A = rng.standard_normal((6, 6)) + 6.0 * np.eye(6)
    c = rng.standard_normal(6)
    x = rng.standard_normal(6)
    s = 0.3 * rng.standard_normal(6)                      # any step, not the Newton one
    b0, b1 = -(A @ x - c), -(A @ (x + s) - c)
    r0 = b0 - A @ s
    assert M.forcing_term_difference(b1, r0, np.linalg.norm(b0)) == 0.01
    assert M.forcing_term_norms(np.linalg.norm(b1), np.linalg.norm(r0), np.linalg.norm(b0)) == 0.01
    assert M.forcing_term_difference(b1, None, None) == 0.1
    assert M.forcing_term_norms(1.0, None, None) == 0.1
    # F(x) = x*x - c, J = diag(2x)
    xq = np.array([1.0, 2.0, 3.0])
    cq = np.array([0.5, 3.0, 8.0])
    sq = np.array([-0.2, -0.2, -0.15])
    F = lambda v: v * v - cq
    b0, b1 = -F(xq), -F(xq + sq)
    r0 = b0 - 2.0 * xq * sq
    eta1 = M.forcing_term_difference(b1, r0, np.linalg.norm(b0))
    assert eta1 == pytest.approx(math.sqrt(0.04 ** 2 + 0.04 ** 2 + 0.0225 ** 2) / 1.5, rel=1e-12)
    assert 0.01 < eta1 < 0.1
    for _ in range(20):
        b0, b1, r0 = rng.standard_normal((3, 5))
        e1 = M.forcing_term_difference(b1, r0, np.linalg.norm(b0), lo=-inf, hi=inf)
        e2 = M.forcing_term_norms(np.linalg.norm(b1), np.linalg.norm(r0), np.linalg.norm(b0), lo=-inf, hi=inf)
        assert e2 <= e1 + 1e-12
        assert M.forcing_term_norms(np.linalg.norm(b1), 0.0, np.linalg.norm(b0), lo=-inf, hi=inf) == \
            pytest.approx(np.linalg.norm(b1) / np.linalg.norm(b0))


def test_peaceman_equivalent_radius():
    h, rw = 20.0, 0.1
    k = 100.0 * MD
    wi = M.peaceman_wi(k, k, k, h, h, 4.0, "z", rw, 0.0)
    re = rw * math.exp(2.0 * math.pi * 4.0 * k / wi)
    assert re / h == pytest.approx(0.198, rel=5e-3)          # Peaceman's square-cell value
    kx, ky, hx, hy = 300.0 * MD, 30.0 * MD, 20.0, 10.0
    wi = M.peaceman_wi(kx, ky, k, hx, hy, 4.0, "z", rw, 0.5)
    re = rw * math.exp(2.0 * math.pi * 4.0 * math.sqrt(kx * ky) / wi - 0.5)
    expect = 0.28 * math.sqrt(math.sqrt(ky / kx) * hx ** 2 + math.sqrt(kx / ky) * hy ** 2) / \
        ((ky / kx) ** 0.25 + (kx / ky) ** 0.25)
    assert re == pytest.approx(expect, rel=5e-3)             # Peaceman's anisotropic form
    # a well along x sees (y, z): same value as a z-well with the axes rotated
    a = M.peaceman_wi(k, 2 * k, 3 * k, 7.0, 11.0, 13.0, "x", rw, 0.0)
    b = M.peaceman_wi(2 * k, 3 * k, k, 11.0, 13.0, 7.0, "z", rw, 0.0)
    assert a == pytest.approx(b, rel=1e-14)


def test_viscosity_special_cases():
    from oracle.dual import Dual
    ph = G.default_physics(mu_w=0.5 * CP, mu_p0=8.0 * CP, c_ref=2.0)

    def props(C, **over):
        p = dict(ph, **over)
        n = len(C)
        P = Dual.variable(np.full(n, 200 * BAR), 3, 0)
        S = Dual.variable(np.full(n, 0.5), 3, 1)
        Cd = Dual.variable(np.asarray(C, float), 3, 2)
        return M.cell_properties(p, np.full(n, 0.2), P, S, Cd)

    pr = props([0.0, 2.0, 1.0], omega=1.0)
    assert pr["mu_we"].v[0] == pytest.approx(0.5 * CP)       # beta = 0: pure water
    assert pr["mu_we"].v[1] == pytest.approx(8.0 * CP)       # beta = 1: mu_p0
    assert pr["mu_we"].v[2] == pytest.approx(2.0 * CP)       # geometric mean at beta = 1/2
    pr = props([1.0], omega=1.0, mixing=1)
    assert pr["mu_we"].v[0] == pytest.approx(4.25 * CP)      # linear rule at beta = 1/2
    pr = props([1.0, 0.0, 3.0], omega=0.0)                    # fully segregated
    assert pr["mu_pe"].v[0] == pytest.approx(8.0 * CP)
    assert pr["mu_we"].v[1] == pytest.approx(0.5 * CP)        # alpha = 0 -> water
    assert pr["mu_we"].v[2] == pytest.approx(8.0 * CP)        # alpha = 1 -> polymer
    # alpha = 1/2, omega = 0: harmonic mean of mu_w and mu_p0
    assert pr["mu_we"].v[0] == pytest.approx(1.0 / (0.5 / (8.0 * CP) + 0.5 / (0.5 * CP)))


# ---------------------------------------------------------------------------
# well constraints with a BHP limit (Sec. 2.4, Sec. 4.1.2)
# ---------------------------------------------------------------------------

def limited_injector_scenario(rate_day, limit_bar, n_steps=4):
    ph = G.default_physics()
    nx, ny, nz = 6, 6, 2
    n = nx * ny * nz
    k = np.full(n, 20.0 * MD)
    wells = [dict(kind="inj", cells=[0, nx * ny]), dict(kind="prod", cells=[n - 1 - nx * ny, n - 1])]
    ctl = [dict(ctrl="wrate", target=rate_day / DAY, limit=limit_bar * BAR, c_inj=1.0),
           dict(ctrl="bhp", target=150.0 * BAR, limit=None, c_inj=0.0)]
    return G.make_scenario(nx, ny, nz, 20.0, 20.0, 5.0, 2000.0, k, k, k, np.full(n, 0.2), ph, wells,
                           [dict(n_steps=n_steps, dt=2.0 * DAY, controls=ctl)])


def test_bhp_limit_switches_rate_injector():
    sc = limited_injector_scenario(2000.0, 260.0)
    st, x, hist = M.run(sc)
    assert hist[-1]["switched"][0]
    assert x[3 * st.n] == pytest.approx(260.0 * BAR, rel=1e-12)
    gam = M.well_gamma(st, hist[-2]["x"], M.effective_controls(st, sc["schedule"][0]["controls"],
                                                                 hist[-1]["switched"]))
    qw, qo, pb = M.well_totals(st, x, sc["schedule"][0]["controls"], gam)[0]
    assert 0.0 < qw / st.ph["rho_w"] < 2000.0 / DAY


def test_rate_injector_below_limit_stays_on_rate():
    sc = limited_injector_scenario(20.0, 400.0)
    st, x, hist = M.run(sc)
    assert not any(h["switched"][0] for h in hist)
    assert x[3 * st.n] < 400.0 * BAR


def test_time_step_cut_then_grow():
    """Sec. 3 step 4: a failed Newton solve halves the step, and the loop
    then tries to lengthen it again (doubling, capped by the period's step and
    by what is left of it); the accepted sub-steps cover the step exactly."""
    sc = G.scenario_c1(n_steps=2, dt_days=30.0)
    _, _, hist = M.run(sc, max_iter=6)
    dt = sc["schedule"][0]["dt"]
    first = hist[0]
    assert first["cuts"] >= 1
    sub = first["substeps"]
    assert abs(sum(sub) - dt) <= 1e-9 * dt
    grew = False
    left = dt
    for a, b in zip(sub, sub[1:]):
        left -= a
        assert b <= min(2.0 * a, left) * (1 + 1e-12)
        grew |= b > a * (1 + 1e-12)
    assert grew
    assert hist[1]["cuts"] == 0 and hist[1]["substeps"] == [dt]


# ---------------------------------------------------------------------------
# tabulated properties (Sec. 2.2 k_r and P_c of saturation; Sec. 2.3 "specified
# in the form of a table" for adsorption, and the water viscosity multiplier)
# ---------------------------------------------------------------------------

def _props(ph, P, S, C):
    n = len(P)
    return M.cell_properties(ph, np.full(n, 0.2), M.Dual.variable(np.asarray(P, float), 3, 0),
                             M.Dual.variable(np.asarray(S, float), 3, 1), M.Dual.variable(np.asarray(C, float), 3, 2))


def test_tables_reproduce_linear_closed_forms():
    """Two-knot tables are straight lines, so they must give exactly the
    linear Corey curves (n = 1), the linear mixing rule and a linear isotherm,
    values and derivatives, including the flat ends outside the knots."""
    swc, sor, pce, c_ref, mu_w, mu_p0, rrf, K = 0.15, 0.25, 0.7 * BAR, 2.0, 0.5 * CP, 6.0 * CP, 1.8, 0.03
    corey = G.default_physics(swc=swc, sor=sor, nw=1.0, no=1.0, krw_max=0.6, kro_max=0.9, pc_e=pce, pc_n=1.0,
                              mixing=1, c_ref=c_ref, mu_w=mu_w, mu_p0=mu_p0, rrf=rrf)
    sat = np.array([[swc, 0.0, 0.9, pce], [1.0 - sor, 0.6, 0.0, 0.0]])
    cmax = 40.0
    poly = np.array([[0.0, 1.0, 0.0], [cmax, 1.0 + cmax / c_ref * (mu_p0 / mu_w - 1.0), K * cmax]])
    tab = dict(corey, sat_table=sat, poly_table=poly)
    rng = np.random.default_rng(11)
    S = rng.uniform(0.0, 1.0, 64)
    C = rng.uniform(0.0, 0.99 * cmax, 64)
    P = rng.uniform(150.0, 250.0, 64) * BAR
    a, b = _props(corey, P, S, C), _props(tab, P, S, C)
    for key in ("krw", "kro", "Pw", "mu_we", "mu_pe", "rho_w"):
        assert np.allclose(a[key].v, b[key].v, rtol=1e-13, atol=0.0), key
        assert np.allclose(a[key].d, b[key].d, rtol=1e-11, atol=1e-300), key
    assert np.allclose(b["ads"].v, K * C, rtol=1e-13)
    assert np.allclose(b["ads"].d[:, 2], K, rtol=1e-13)
    assert np.allclose(b["Rk"].v, 1.0 + (rrf - 1.0) * C / cmax, rtol=1e-13)


def test_table_knots_take_the_right_slope_and_flat_ends():
    ph = G.default_physics(sat_table=np.array([[0.2, 0.0, 1.0, 3.0e4], [0.5, 0.1, 0.3, 1.0e4],
                                               [0.8, 0.7, 0.0, 0.0]]))
    S = np.array([0.5, 0.2, 0.8, 0.1, 0.95, 0.35])
    p = _props(ph, np.full(6, 200.0 * BAR), S, np.zeros(6))
    krw_slope = np.array([2.0, 1.0 / 3.0, 0.0, 0.0, 0.0, 1.0 / 3.0])
    assert np.allclose(p["krw"].d[:, 1], krw_slope, rtol=1e-12, atol=0.0)
    assert np.allclose(p["krw"].v, [0.1, 0.0, 0.7, 0.0, 0.7, 0.05], rtol=1e-12, atol=1e-15)
    assert np.allclose(p["Pw"].v, 200.0 * BAR - np.array([1.0e4, 3.0e4, 0.0, 3.0e4, 0.0, 2.0e4]), rtol=1e-15)


def test_polymer_front_with_tabulated_linear_isotherm():
    """Sec. 2.3 table form of A_d(C): a linear isotherm A_d = K C retards the
    polymer front to u / (phi (1 - IPV) + (1 - phi) K) (mass balance of the
    front)."""
    K, cmax = 0.02, 20.0
    poly = np.array([[0.0, 1.0, 0.0], [cmax, 5.0, K * cmax]])
    ph = incompressible(swc=0.0, sor=0.0, ipv=0.1, rrf=1.5, mu_w=1.0 * CP, poly_table=poly)
    n, t_end, dt = 200, 150.0, 0.5
    sc = one_d(n, physics=ph, q_day=20.0, c_inj=1.0, s0=1.0, c0=0.0, dt_days=dt, n_steps=int(round(t_end / dt)))
    st, x, hist = M.run(sc)
    C = field(st, x, 2)
    phi, u = 0.2, 20.0 / DAY / 100.0
    vs = u / (phi * (1.0 - 0.1) + (1.0 - phi) * K)
    xs = vs * t_end * DAY
    dx = 1000.0 / n
    xc = (np.arange(n) + 0.5) * dx
    i = int(np.nonzero(C < 0.5)[0][0])
    x_half = xc[i - 1] + (C[i - 1] - 0.5) / (C[i - 1] - C[i]) * dx
    assert abs(x_half - xs) < 3.0 * dx, (x_half, xs)


# ---------------------------------------------------------------------------
# capillary-gravity equilibrium initialisation (Sec. 4.1.3)
# ---------------------------------------------------------------------------

def _layered_no_wells(ph, nz=30, dz=1.0, nx=3, ny=2):
    n = nx * ny * nz
    phi = np.repeat(np.linspace(0.12, 0.3, nz), nx * ny)
    k = np.repeat(np.exp(np.linspace(math.log(20.0), math.log(500.0), nz)), nx * ny) * MD
    sched = [dict(n_steps=1, dt=DAY, controls=[])]
    return G.make_scenario(nx, ny, nz, 20.0, 20.0, dz, 2000.0, k, k, 0.1 * k, phi, ph, [], sched)


@pytest.mark.parametrize("kind", ["corey", "table"])
def test_equilibrium_state_is_a_discrete_rest_state(kind):
    """With no wells the equilibrated state is a root of the discrete
    equations for any step: every face flux cancels (both phases), across
    the oil zone, the capillary transition zone and the water zone."""
    if kind == "corey":
        ph = G.default_physics(pc_e=0.8 * BAR, pc_n=2.0)
    else:
        ph = G.default_physics(sat_table=np.array([[0.2, 0.0, 1.0, 1.2 * BAR], [0.45, 0.08, 0.45, 0.35 * BAR],
                                                   [0.8, 0.6, 0.0, 0.0], [1.0, 1.0, 0.0, 0.0]]))
    sc = _layered_no_wells(ph)
    P, S = M.equilibrium_state(sc, 2005.0, 200.0 * BAR, 2022.0)
    trans = (S > 0.2 + 1e-6) & (S < 0.8 - 1e-6)
    assert trans.sum() >= 6 * 5 and (S == 1.0).sum() >= 6 * 5
    sc["P0"], sc["S0"] = P, S
    st = M.Setup(sc)
    x = M.initial_state(st)
    for dt in (DAY, 100.0 * DAY):
        R, _ = M.assemble(st, x, M.masses(st, x), dt, [], [], with_jacobian=False)
        assert M.scaled_residual(st, R, dt, []) < 1e-11


def test_equilibrium_incompressible_closed_form():
    """Incompressible phases: hydrostatic lines from the datum (oil) and from
    the contact (water); in the transition zone P_c(S) = (rho_w - rho_o) g
    (z_c - z), the capillary rise of the textbook, inverted in closed form
    for the Corey curve."""
    pce, pcn, swc, sor = 0.8 * BAR, 2.0, 0.2, 0.2
    ph = G.default_physics(c_w=0.0, c_o=0.0, pc_e=pce, pc_n=pcn, swc=swc, sor=sor)
    sc = _layered_no_wells(ph, nz=40, dz=0.5)
    zd, pd, zc_ = 2003.3, 190.0 * BAR, 2014.2
    P, S = M.equilibrium_state(sc, zd, pd, zc_)
    z = M.cell_depth(sc)
    g, ro, rw = ph["g"], ph["rho_o"], ph["rho_w"]
    Po = pd + ro * g * (z - zd)
    Pw = pd + ro * g * (zc_ - zd) + rw * g * (z - zc_)
    dP = Po - Pw
    sn = 1.0 - np.clip(dP / pce, 0.0, 1.0) ** (1.0 / pcn)
    S_expect = np.where(dP <= 0.0, 1.0, swc + sn * (1.0 - swc - sor))
    # the datum and contact legs are marched in thousands of small steps, whose
    # rounding (~1e-5 Pa) moves S by ~1e-10 on the steep part of the curve
    assert np.allclose(S, S_expect, rtol=0.0, atol=1e-9)
    expectP = np.where(dP < 0.0, Pw, Po)
    assert np.allclose(P, expectP, rtol=1e-12, atol=0.0)


def test_equilibrium_continuous_leg_is_the_exponential_profile():
    """dP/dz = g rho_ref (1 + c (P - P_ref)) has the closed-form solution
    P = P_ref - 1/c + (P_0 - P_ref + 1/c) exp(g rho_ref c (z - z_0))."""
    ph = G.default_physics(c_o=5e-4 / BAR)
    c, r, g, pref = ph["c_o"], ph["rho_o"], ph["g"], ph["p_ref"]
    p0, z0, z1 = 180.0 * BAR, 1000.0, 1350.0
    exact = pref - 1.0 / c + (p0 - pref + 1.0 / c) * math.exp(g * r * c * (z1 - z0))
    assert M._march_continuous(ph, "o", p0, z0, z1) == pytest.approx(exact, rel=1e-13)


def test_newton_gives_up_on_runaway_iterates():
    """A 300-day first step on the 10x10x3 case runs away (the scaled
    residual grows by orders of magnitude); with the divergence test the
    step fails as soon as the residual passes 1e6 times its first value,
    without it only at the iteration cap; the time loop then cuts."""
    sc = G.scenario_c1(n_steps=1, dt_days=300.0)
    st = M.Setup(sc)
    x0 = M.initial_state(st)
    ctl = M.controls_with_defaults(sc["schedule"][0]["controls"])
    rec_off, rec_on = [], []
    _, ok_off, _ = M.newton_step(st, x0, 300.0 * DAY, ctl, record=rec_off, switched=[False] * st.nw, div=0.0)
    _, ok_on, _ = M.newton_step(st, x0, 300.0 * DAY, ctl, record=rec_on, switched=[False] * st.nw, div=1e6)
    assert not ok_off and not ok_on
    assert len(rec_off) == 26 and len(rec_on) < len(rec_off)
    assert rec_on[-1] > 1e6 * rec_on[0] and max(rec_on[:-1]) <= 1e6 * rec_on[0]
    assert rec_on == rec_off[:len(rec_on)]
    _, _, hist = M.run(sc)
    assert hist[0]["cuts"] >= 1 and abs(sum(hist[0]["substeps"]) - 300.0 * DAY) <= 1e-6 * DAY


@pytest.mark.parametrize("mixing", [0, 1])
def test_todd_longstaff_limits(mixing):
    """Sec. 2.3, the Todd-Longstaff limits of the effective viscosities, for
    either mixing rule: full mixing (omega = 1) gives both phases the
    mixture's viscosity, mu_p,e = mu_w,e = mu_m (so the GPU path may use mu_m
    directly); no mixing (omega = 0) leaves the polymer solution at mu_p0 and
    gives the water its own viscosity blended by the harmonic rule
    1/mu_w,e = a/mu_p0 + (1 - a)/mu_w, a = C/C_ref clipped to [0, 1].  The
    mixture viscosity is taken from the mixing rule written out here: mu_w at
    C = 0 and mu_p0 at C = C_ref for both rules, the geometric or arithmetic
    blend in between."""
    mu_w, mu_p0, c_ref = 0.6 * CP, 7.0 * CP, 1.5
    C = np.array([0.0, 0.3, 0.75, 1.2, 1.5, 1.9])
    b = C / c_ref                      # the rules extrapolate above C_ref
    mu_m = mu_w ** (1.0 - b) * mu_p0 ** b if mixing == 0 else b * mu_p0 + (1.0 - b) * mu_w
    n = len(C)
    P, S = np.full(n, 200.0 * BAR), np.full(n, 0.5)
    ph1 = G.default_physics(mixing=mixing, omega=1.0, mu_w=mu_w, mu_p0=mu_p0, c_ref=c_ref)
    pr = _props(ph1, P, S, C)
    assert np.allclose(pr["mu_pe"].v, mu_m, rtol=1e-14, atol=0.0)
    assert np.allclose(pr["mu_we"].v, mu_m, rtol=1e-14, atol=0.0)
    # and their C-derivatives agree (the Jacobian's concentration column)
    assert np.allclose(pr["mu_we"].d[2], pr["mu_pe"].d[2], rtol=1e-12, atol=0.0)
    ph0 = G.default_physics(mixing=mixing, omega=0.0, mu_w=mu_w, mu_p0=mu_p0, c_ref=c_ref)
    pr = _props(ph0, P, S, C)
    a = np.clip(C / c_ref, 0.0, 1.0)
    assert np.allclose(pr["mu_pe"].v, mu_p0, rtol=1e-14, atol=0.0)
    assert np.allclose(pr["mu_we"].v, 1.0 / (a / mu_p0 + (1.0 - a) / mu_w), rtol=1e-14, atol=0.0)
