"""pf_equilibrium_init (host code of the library, no GPU) against the
oracle's equilibrium (Sec. 4.1.3): same oil pressures and saturations on
layered and laterally heterogeneous grids, Corey and tabulated capillary
pressure; invalid tables are refused."""

import numpy as np
import pytest

from oracle import model as M
from scenarios import generate as G

BAR, MD, DAY = G.BAR, G.MD, G.DAY


@pytest.fixture(scope="module")
def B():
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding
    binding.lib()
    return binding


SAT = np.array([[0.2, 0.0, 1.0, 1.2 * BAR], [0.45, 0.08, 0.45, 0.35 * BAR], [0.8, 0.6, 0.0, 0.0],
                [1.0, 1.0, 0.0, 0.0]])


def column_model(ph, layered=True, nx=4, ny=3, nz=24, dz=0.75, seed=3):
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    if layered:
        phi = np.repeat(rng.uniform(0.1, 0.3, nz), nx * ny)
    else:
        phi = rng.uniform(0.1, 0.3, n)
    k = np.exp(rng.normal(np.log(100.0), 1.0, n)) * MD
    sched = [dict(n_steps=1, dt=DAY, controls=[])]
    return G.make_scenario(nx, ny, nz, 15.0, 15.0, dz, 1800.0, k, k, 0.1 * k, phi, ph, [], sched)


@pytest.mark.parametrize("kind,layered", [("corey", True), ("corey", False), ("table", True),
                                          ("incompressible", True)])
def test_equilibrium_matches_oracle(B, kind, layered):
    if kind == "corey":
        ph = G.default_physics(pc_e=0.6 * BAR, pc_n=1.7)
    elif kind == "table":
        ph = G.default_physics(sat_table=SAT)
    else:
        ph = G.default_physics(c_w=0.0, c_o=0.0, pc_e=0.3 * BAR, pc_n=2.0)
    sc = column_model(ph, layered=layered)
    args = (1803.1, 185.0 * BAR, 1811.6)
    P_o, S_o = M.equilibrium_state(sc, *args)
    P_g, S_g = B.equilibrium_init(sc, *args)
    assert np.allclose(P_g, P_o, rtol=1e-12, atol=0.0)
    assert np.allclose(S_g, S_o, rtol=0.0, atol=1e-9)
    assert ((S_g > 0.21) & (S_g < 0.79)).any() and (S_g == 1.0).any()


def test_equilibrium_refuses_increasing_capillary_pressure(B):
    bad = SAT.copy()
    bad[2, 3] = 2.0 * BAR
    sc = column_model(G.default_physics(sat_table=bad))
    with pytest.raises(B.PfError) as e:
        B.equilibrium_init(sc, 1803.0, 185.0 * BAR, 1811.0)
    assert e.value.status == B.PF_EINVAL


def test_model_tables_are_validated(B):
    bad = SAT.copy()
    bad[2, 0] = 0.3                       # abscissae must increase
    sc = column_model(G.default_physics(sat_table=bad))
    with pytest.raises(B.PfError) as e:
        B.footprint(sc)
    assert e.value.status == B.PF_EINVAL
    poly = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.1]])   # multiplier must be positive
    sc = column_model(G.default_physics(poly_table=poly))
    with pytest.raises(B.PfError):
        B.footprint(sc)
    ok = column_model(G.default_physics(sat_table=SAT, poly_table=np.array([[0.0, 1.0, 0.0], [2.0, 4.0, 0.05]])))
    assert B.footprint(ok) > 0
