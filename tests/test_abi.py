"""The C-ABI library loads, exports every symbol include/polyflood.h
declares, and rejects invalid models before touching the GPU (no GPU needed)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding
    binding.lib()
    return binding


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "polyflood.h")).read()
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(B):
    syms = declared_symbols()
    assert len(syms) >= 18
    for name in syms:
        assert hasattr(B.lib(), name), name
    L = C.CDLL(B.LIB_PATH)
    for name in syms:
        getattr(L, name)


def test_version_and_defaults(B):
    assert b"sm_103a" in B.lib().pf_version()
    o = B.default_opts()
    assert o.gmres_restart == 30 and o.newton_tol == 1e-10 and o.ds_max == 0.2
    assert o.precision == B.PF_PREC_FP64
    assert o.ilu_store == -1 and o.krylov_lookahead == 1


def _model(**over):
    from scenarios import scenario_c1
    sc = scenario_c1(nx=3, ny=3, nz=2)
    sc.update(over)
    return sc


@pytest.mark.parametrize("mutate,needle", [
    (lambda sc: sc["kx"].__setitem__(0, -1.0), "permeability"),
    (lambda sc: sc["phi"].__setitem__(1, 0.0), "porosity"),
    (lambda sc: sc["P0"].__setitem__(2, np.nan), "finite"),
    (lambda sc: sc["wells"][1].__setitem__("cells", np.array([0], dtype=np.int64)), "more than one perforation"),
    (lambda sc: sc["wells"][0].__setitem__("cells", np.array([99], dtype=np.int64)), "outside"),
])
def test_invalid_models_rejected_without_gpu(B, mutate, needle):
    sc = _model()
    mutate(sc)
    with pytest.raises(B.PfError) as e:
        B.Simulator(sc)
    assert e.value.status == B.PF_EINVAL
    assert needle in str(e.value)


def test_invalid_options_rejected(B):
    with pytest.raises(B.PfError) as e:
        B.Simulator(_model(), gmres_restart=100)
    assert e.value.status == B.PF_EINVAL
    with pytest.raises(B.PfError) as e:
        B.Simulator(_model(), krylov_lookahead=2)
    assert e.value.status == B.PF_EINVAL and "krylov_lookahead" in str(e.value)


def test_tuning_calls_reject_null_arguments_without_gpu(B):
    """pf_get_tuning, pf_set_tuning and pf_autotune refuse a NULL simulator
    (and pf_get_tuning a NULL output) with PF_EINVAL before any CUDA call."""
    import ctypes as C
    L = B.lib()
    t = B.pf_tuning()
    assert L.pf_get_tuning(None, C.byref(t)) == B.PF_EINVAL
    assert L.pf_set_tuning(None, C.byref(t)) == B.PF_EINVAL
    assert L.pf_autotune(None, C.byref(t)) == B.PF_EINVAL
    assert L.pf_get_tuning(None, None) == B.PF_EINVAL
