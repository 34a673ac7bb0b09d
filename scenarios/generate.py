"""Seeded synthetic scenarios shaped after the paper's workloads.

A scenario is a plain dict of numpy arrays and numbers (SI units throughout:
Pa, m, m^2, s, kg, Pa*s).  Keys:

  nx, ny, nz, dx, dy, dz, top        Cartesian grid; cell (i,j,k) has the
                                     natural index i + nx*(j + ny*k); k grows
                                     downward; ``top`` is the depth of the top
                                     face of layer 0.
  kx, ky, kz, phi                    per-cell absolute permeability [m^2] and
                                     reference porosity.
  P0, S0, C0                         initial oil pressure [Pa], water
                                     saturation, polymer concentration [kg/m^3].
  physics                            dict of scalar constants (see
                                     ``default_physics``).
  wells                              list of dicts: kind ('inj'|'prod'), cells
                                     (int64 natural indices, top first), dirs
                                     (per perforation 'x'|'y'|'z'), rw, skin,
                                     gf, f, fh, Pb0.
  schedule                           list of periods: {'n_steps', 'dt',
                                     'controls': [per-well {ctrl, target,
                                     limit, c_inj}]}.  ctrl is 'bhp' (target
                                     in Pa), 'wrate', 'orate' or 'lrate'
                                     (target a positive volume rate at
                                     reference conditions, m^3/s).

Nothing in this module evaluates a property law, a transmissibility, a well
index or a residual: those belong to the two implementations that read it.
"""

import math

import numpy as np

DAY = 86400.0
BAR = 1.0e5
MD = 9.869233e-16
CP = 1.0e-3
PSI = 6894.757293168
FT = 0.3048
G = 9.80665

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z):
    """SplitMix64 output function applied to uint64 array ``z`` (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_base(seed, stream):
    with np.errstate(over="ignore"):
        s = splitmix64(np.uint64(seed) * _GOLDEN + np.uint64(stream))
    return s


def uniform01(seed, stream, n):
    """n uniforms in (0, 1]: counter k of (seed, stream) -> top 53 bits."""
    base = _stream_base(seed, stream)
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64(base + k * _GOLDEN)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed, stream, n):
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


def default_physics(**over):
    """Constants used by the synthetic scenarios.

    Fluid values follow the paper's Table 1 (densities 1025.18 / 832.96 kg/m^3,
    compressibilities 3.03e-6 and 1e-5 per bar, water viscosity 0.5 cp) and
    Table 2 (oil viscosity 2 cp).  Constants the paper leaves open (rock
    compressibility, Corey end points, Langmuir constants, mixing parameters)
    take documented defaults.
    """
    p = dict(
        rho_w=1025.18, rho_o=832.96,
        c_w=3.03e-6 / BAR, c_o=1.0e-5 / BAR, p_ref=200.0 * BAR,
        mu_w=0.5 * CP, mu_o=2.0 * CP,
        c_r=2.0e-6 / BAR, p_r=200.0 * BAR,
        swc=0.2, sor=0.2, nw=2.0, no=2.0, krw_max=1.0, kro_max=1.0,
        pc_e=0.0, pc_n=2.0,
        ads_a=0.5, ads_b=10.0,          # Langmuir A_d = a C / (1 + b C)  [kg/m^3 rock]
        rrf=1.5, ipv=0.1,
        omega=1.0, mu_p0=5.0 * CP, c_ref=2.0, mixing=0,   # 0 nonlinear, 1 linear rule
        g=G,
        sat_table=None,     # optional (K, 4) knots: S_w, k_rw, k_ro, P_c [Pa]
        poly_table=None,    # optional (K, 3) knots: C, water viscosity multiplier, A_d [kg/m^3 rock]
    )
    p.update(over)
    return p


def _hydrostatic_guess(nz, dz, top, p_top, rho):
    """Linear pressure profile with a constant density: an input guess only."""
    zc = top + (np.arange(nz) + 0.5) * dz
    return p_top + rho * G * (zc - zc[0])


def make_scenario(nx, ny, nz, dx, dy, dz, top, kx, ky, kz, phi, physics, wells,
                  schedule, p_top=200.0 * BAR, s0=None, c0=0.0, name="custom"):
    n = nx * ny * nz
    pk = _hydrostatic_guess(nz, dz, top, p_top, physics["rho_o"])
    P0 = np.repeat(pk, nx * ny).astype(np.float64)
    S0 = np.full(n, physics["swc"] if s0 is None else s0, dtype=np.float64)
    C0 = np.full(n, c0, dtype=np.float64)
    for w in wells:
        w.setdefault("rw", 0.1)
        w.setdefault("skin", 0.0)
        w.setdefault("gf", 0.249)
        w.setdefault("f", 1.0)
        w.setdefault("fh", 1.0)
        w["cells"] = np.asarray(w["cells"], dtype=np.int64)
        w.setdefault("dirs", ["z"] * len(w["cells"]))
        if "Pb0" not in w:
            w["Pb0"] = float(P0[w["cells"][0]] + (5.0 * BAR if w["kind"] == "inj" else -5.0 * BAR))
    return dict(name=name, nx=nx, ny=ny, nz=nz, dx=float(dx), dy=float(dy), dz=float(dz),
                top=float(top), kx=np.ascontiguousarray(kx, np.float64),
                ky=np.ascontiguousarray(ky, np.float64), kz=np.ascontiguousarray(kz, np.float64),
                phi=np.ascontiguousarray(phi, np.float64), P0=P0, S0=S0, C0=C0,
                physics=physics, wells=wells, schedule=schedule)


def _column(nx, ny, nz, i, j, k0=0, k1=None):
    k1 = nz if k1 is None else k1
    return [i + nx * (j + ny * k) for k in range(k0, k1)]


def _ctrl(ctrl, target, limit=None, c_inj=0.0):
    return dict(ctrl=ctrl, target=float(target), limit=None if limit is None else float(limit),
                c_inj=float(c_inj))


def scenario_c1(seed=1, nx=10, ny=10, nz=3, n_steps=30, dt_days=1.0):
    """10x10x3 of 20 m cubes, lognormal perm (arithmetic mean 100 mD, sigma 1),
    porosity 0.2, injector (0,0) at 200 m^3/d water with 1 kg/m^3 polymer and a
    400 bar cap, producer (nx-1, ny-1) at 150 bar; daily steps."""
    n = nx * ny * nz
    sigma = 1.0
    logk = math.log(100.0) - 0.5 * sigma * sigma + sigma * normal(seed, 0, n)
    k = np.exp(logk) * MD
    phys = default_physics(rrf=1.5, ipv=0.1)
    wells = [dict(kind="inj", cells=_column(nx, ny, nz, 0, 0)),
             dict(kind="prod", cells=_column(nx, ny, nz, nx - 1, ny - 1))]
    controls = [_ctrl("wrate", 200.0 / DAY, limit=400.0 * BAR, c_inj=1.0),
                _ctrl("bhp", 150.0 * BAR)]
    sched = [dict(n_steps=n_steps, dt=dt_days * DAY, controls=controls)]
    return make_scenario(nx, ny, nz, 20.0, 20.0, 20.0, 2000.0, k, k, k, np.full(n, 0.2),
                         phys, wells, sched, name=f"c1_{nx}x{ny}x{nz}")


def _layered_lognormal(seed, nx, ny, nz, sigma, mean_md):
    n = nx * ny * nz
    lay = normal(seed, 1, nz)
    eps = normal(seed, 2, n)
    Lk = np.repeat(lay, nx * ny)
    logk = math.log(mean_md) - 0.5 * sigma * sigma + sigma * (math.sqrt(0.8) * Lk + math.sqrt(0.2) * eps)
    return np.exp(logk) * MD


def _five_spot_wells(nx, ny, nz):
    corners = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]
    wells = [dict(kind="inj", cells=_column(nx, ny, nz, i, j)) for (i, j) in corners]
    wells.append(dict(kind="prod", cells=_column(nx, ny, nz, nx // 2, ny // 2)))
    return wells


def scenario_c2(seed=2, nx=100, ny=100, nz=10, n_steps=100, dt_days=10.0, slug_steps=30,
                c_slug=1.0, rrf=1.5):
    """Layered lognormal perm (sigma 1.5, kv/kh 0.1), 20x20x4 m cells, 5-spot
    (4 corner injectors, centre producer), 1 PV per 1000 d split equally,
    polymer slug at ``c_slug`` kg/m^3 for ``slug_steps`` steps then water."""
    n = nx * ny * nz
    dx, dy, dz = 20.0, 20.0, 4.0
    kh = _layered_lognormal(seed, nx, ny, nz, 1.5, 100.0)
    phi = np.full(n, 0.2)
    pv = float(phi.sum()) * dx * dy * dz
    q_inj = pv / (1000.0 * DAY) / 4.0
    phys = default_physics(rrf=rrf)
    wells = _five_spot_wells(nx, ny, nz)
    inj = lambda c: _ctrl("wrate", q_inj, limit=400.0 * BAR, c_inj=c)
    ctrl_slug = [inj(c_slug)] * 4 + [_ctrl("bhp", 150.0 * BAR)]
    ctrl_chase = [inj(0.0)] * 4 + [_ctrl("bhp", 150.0 * BAR)]
    sched = [dict(n_steps=min(slug_steps, n_steps), dt=dt_days * DAY, controls=ctrl_slug)]
    if n_steps > slug_steps:
        sched.append(dict(n_steps=n_steps - slug_steps, dt=dt_days * DAY, controls=ctrl_chase))
    return make_scenario(nx, ny, nz, dx, dy, dz, 2000.0, kh, kh, 0.1 * kh, phi, phys, wells,
                         sched, name=f"c2_{nx}x{ny}x{nz}")


def scenario_c3(seed=3, nx=600, ny=450, nz=100, n_steps=3, dt_days=10.0, n_inj=(5, 8),
                n_prod=(8, 10), channels=6, q_inj_m3_day=2000.0):
    """Channelised reservoir: background log k ~ N(ln 20 mD, 0.5); per layer
    ``channels`` sinusoidal channels with log k ~ N(ln 1000 mD, 0.3), porosity
    0.25 in channels and 0.15 outside, kv/kh 0.1; injectors (water at
    ``q_inj_m3_day`` each with 1 kg/m^3 polymer, 400 bar cap) and producers
    (150 bar) on offset lattices, fully perforated; 20x20x2 m cells."""
    n = nx * ny * nz
    dx, dy, dz = 20.0, 20.0, 2.0
    back = np.exp(math.log(20.0) + 0.5 * normal(seed, 1, n))
    chan = np.exp(math.log(1000.0) + 0.3 * normal(seed, 2, n))
    par = uniform01(seed, 3, nz * channels * 4).reshape(nz, channels, 4)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    inchan = np.zeros((nz, ny, nx), dtype=bool)
    for k in range(nz):
        for c in range(channels):
            amp = 20.0 + 40.0 * par[k, c, 0]
            lam = 150.0 + 250.0 * par[k, c, 1]
            width = 6.0 + 9.0 * par[k, c, 2]
            ph = 2.0 * math.pi * par[k, c, 3]
            y0 = (c + 0.5) * ny / channels
            yc = y0 + amp * np.sin(2.0 * math.pi * x / lam + ph)
            inchan[k] |= np.abs(y - yc) < 0.5 * width
    m = inchan.reshape(-1)
    kh = np.where(m, chan, back) * MD
    phi = np.where(m, 0.25, 0.15)
    wells = []
    for (ni, nj) in [n_inj]:
        for a in range(ni):
            for b in range(nj):
                i = int((a + 0.5) * nx / ni)
                j = int((b + 0.5) * ny / nj)
                wells.append(dict(kind="inj", cells=_column(nx, ny, nz, min(i, nx - 1), min(j, ny - 1))))
    for a in range(n_prod[0]):
        for b in range(n_prod[1]):
            i = int((a + 0.25) * nx / n_prod[0])
            j = int((b + 0.25) * ny / n_prod[1])
            wells.append(dict(kind="prod", cells=_column(nx, ny, nz, min(i, nx - 1), min(j, ny - 1))))
    ninj = n_inj[0] * n_inj[1]
    q_inj = q_inj_m3_day / DAY
    phys = default_physics()
    controls = [_ctrl("wrate", q_inj, limit=400.0 * BAR, c_inj=1.0)] * ninj + \
               [_ctrl("bhp", 150.0 * BAR)] * (len(wells) - ninj)
    sched = [dict(n_steps=n_steps, dt=dt_days * DAY, controls=controls)]
    return make_scenario(nx, ny, nz, dx, dy, dz, 2000.0, kh, kh, 0.1 * kh, phi, phys, wells,
                         sched, name=f"c3_{nx}x{ny}x{nz}")


def scenario_size(seed, n_cells, nz=10):
    """(nx, ny, nz) for a member of an uneven ensemble of about ``n_cells``."""
    side = max(2, int(round(math.sqrt(n_cells / nz))))
    return side, side, nz


def scenario_member(index, base_seed=100, n_lo=2.0e4, n_hi=4.0e5, n_steps=20, nz=10):
    """Ensemble member ``index``: cell count log-uniform in [n_lo, n_hi],
    slug concentration U(0.5, 2) kg/m^3, RRF U(1.2, 2.0), otherwise the
    100x100x10 recipe."""
    seed = base_seed + index
    u = uniform01(seed, 7, 3)
    n_cells = math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u[0])
    nx, ny, nz = scenario_size(seed, n_cells, nz)
    return scenario_c2(seed=seed, nx=nx, ny=ny, nz=nz, n_steps=n_steps,
                       slug_steps=max(1, n_steps // 3), c_slug=0.5 + 1.5 * u[1],
                       rrf=1.2 + 0.8 * u[2])


def scenario_1d_table1(n_steps=60, dt_days=30.0, block=100.0):
    """The paper's 1-D case (Table 1): 15 blocks, porosity 0.5, 100 mD, initial
    water saturation 0.4 and polymer 0.1 kg/m^3, 1000 m^3/d injector in block 1
    and producer in block 15; water 300 d, polymer 6 kg/m^3 for 500 d, then
    water to 1800 d.  The block cross-section is not printed; ``block`` sets
    all three cell sizes."""
    nx, ny, nz = 15, 1, 1
    k = np.full(nx, 100.0 * MD)
    phys = default_physics(rho_w=1025.18, rho_o=832.96, c_w=3.03e-6 / BAR, c_o=1.0e-5 / BAR,
                           mu_w=0.5 * CP, mu_o=0.5 * CP, ipv=0.15, rrf=2.67, swc=0.2, sor=0.2)
    wells = [dict(kind="inj", cells=[0]), dict(kind="prod", cells=[nx - 1])]
    q = 1000.0 / DAY
    water = [_ctrl("wrate", q, limit=1000.0 * BAR, c_inj=0.0), _ctrl("lrate", q)]
    poly = [_ctrl("wrate", q, limit=1000.0 * BAR, c_inj=6.0), _ctrl("lrate", q)]
    dt = dt_days * DAY
    n1 = int(round(300.0 / dt_days)); n2 = int(round(500.0 / dt_days))
    n3 = max(0, int(round(1800.0 / dt_days)) - n1 - n2)
    sched = [dict(n_steps=n1, dt=dt, controls=water), dict(n_steps=n2, dt=dt, controls=poly),
             dict(n_steps=n3, dt=dt, controls=water)]
    total = n1 + n2 + n3
    if n_steps < total:
        left = n_steps
        out = []
        for p in sched:
            take = min(left, p["n_steps"])
            if take > 0:
                out.append(dict(p, n_steps=take))
            left -= take
        sched = out
    return make_scenario(nx, ny, nz, block, block, block, 1000.0, k, k, k, np.full(nx, 0.5),
                         phys, wells, sched, s0=0.4, c0=0.1, name="table1_1d")


def scenario_2d_table2(n_steps=34, dt_days=50.0):
    """The paper's 2-D case (Table 2): 10x10 blocks of 75 ft, porosity 0.2,
    50 mD, initially oil saturated; injector at one corner at 200 STB/d with
    50 lbm/STB polymer for 200 d under a 2e5 psia cap, producer at the other
    corner at 3999 psia; 1700 d."""
    nx, ny, nz = 10, 10, 1
    n = nx * ny
    k = np.full(n, 50.0 * MD)
    lbm_ft3 = 0.45359237 / FT ** 3
    stb = 0.158987294928
    phys = default_physics(rho_w=64.0 * lbm_ft3, rho_o=52.0 * lbm_ft3, c_w=3.03e-6 / PSI,
                           c_o=1.0e-5 / PSI, p_ref=4000.0 * PSI, p_r=4000.0 * PSI,
                           mu_w=0.5 * CP, mu_o=2.0 * CP, swc=0.0, sor=0.0,
                           c_ref=50.0 * 0.45359237 / stb)
    wells = [dict(kind="inj", cells=[0]), dict(kind="prod", cells=[n - 1])]
    q = 200.0 * stb / DAY
    c_inj = 50.0 * 0.45359237 / stb
    poly = [_ctrl("wrate", q, limit=2.0e5 * PSI, c_inj=c_inj), _ctrl("bhp", 3999.0 * PSI)]
    water = [_ctrl("wrate", q, limit=2.0e5 * PSI, c_inj=0.0), _ctrl("bhp", 3999.0 * PSI)]
    dt = dt_days * DAY
    n1 = int(round(200.0 / dt_days))
    sched = [dict(n_steps=min(n1, n_steps), dt=dt, controls=poly)]
    if n_steps > n1:
        sched.append(dict(n_steps=n_steps - n1, dt=dt, controls=water))
    return make_scenario(nx, ny, nz, 75.0 * FT, 75.0 * FT, 75.0 * FT, 6000.0 * FT, k, k, k,
                         np.full(n, 0.2), phys, wells, sched, p_top=4000.0 * PSI, s0=0.0,
                         name="table2_2d")


TABLE4 = [  # layer: porosity, kx, ky, kz [mD]  (paper, Table 4)
    (0.17393, 326.4, 980.6, 163.4),
    (0.1694, 445.3, 1335.8, 222.6),
    (0.25714, 148.9, 446.6, 74.4),
    (0.17344, 118.8, 356.4, 59.4),
    (0.1187, 71.2, 213.6, 35.6),
]


def scenario_layered_table4(nx=95, ny=192, refine_z=1, n_steps=5, dt_days=10.0, dx=None, dy=None,
                            dz=None):
    """Layered reservoir of the paper's Table 4 (5 layers; ``refine_z`` splits
    each), initial 4000 psi at 6150 ft, four vertical corner injectors and a
    horizontal producer along x through the centre of the middle layer.
    Cell sizes are not printed; defaults give a 95x192x5 grid of 20x20x4 m."""
    nz = 5 * refine_z
    dx = 20.0 if dx is None else dx
    dy = 20.0 if dy is None else dy
    dz = 4.0 / refine_z if dz is None else dz
    n = nx * ny * nz
    kx = np.empty(n); ky = np.empty(n); kz = np.empty(n); phi = np.empty(n)
    for k in range(nz):
        por, a, b, c = TABLE4[k // refine_z]
        sl = slice(k * nx * ny, (k + 1) * nx * ny)
        phi[sl] = por; kx[sl] = a * MD; ky[sl] = b * MD; kz[sl] = c * MD
    wells = [dict(kind="inj", cells=_column(nx, ny, nz, i, j))
             for (i, j) in [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]]
    kmid = nz // 2
    i0, i1 = nx // 4, 3 * nx // 4
    wells.append(dict(kind="prod", cells=[i + nx * (ny // 2 + ny * kmid) for i in range(i0, i1)],
                      dirs=["x"] * (i1 - i0)))
    pv = float(phi.sum()) * dx * dy * dz
    q = pv / (3000.0 * DAY) / 4.0
    phys = default_physics(p_ref=4000.0 * PSI, p_r=4000.0 * PSI)
    controls = [_ctrl("wrate", q, limit=8000.0 * PSI, c_inj=1.0)] * 4 + [_ctrl("bhp", 3000.0 * PSI)]
    sched = [dict(n_steps=n_steps, dt=dt_days * DAY, controls=controls)]
    return make_scenario(nx, ny, nz, dx, dy, dz, 6150.0 * FT, kx, ky, kz, phi, phys, wells, sched,
                         p_top=4000.0 * PSI, name=f"table4_{nx}x{ny}x{nz}")
