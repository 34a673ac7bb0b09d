"""pf_footprint, the device bytes a simulator will take (the serving loop
admits requests by it), computed on the host without a GPU: it grows with the
grid, mixed precision takes less than FP64, and the per-colour copies
(ilu_store) add exactly their documented arrays."""

import pytest

from scenarios import generate as G


@pytest.fixture(scope="module")
def B():
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding
    binding.lib()
    return binding


def colour_slots(sc):
    return ((sc["nx"] + 1) // 2) * sc["ny"] * sc["nz"]


def test_footprint_grows_with_the_grid_and_shrinks_with_precision(B):
    grids = [G.scenario_c1(nx=20 * m, ny=20, nz=5) for m in (1, 2, 3)]
    f64 = [B.footprint(sc, precond=B.PF_PC_CPR, ilu_store=0) for sc in grids]
    mix = [B.footprint(sc, precond=B.PF_PC_CPR, precision=B.PF_PREC_MIXED, ilu_store=0) for sc in grids]
    # per-cell arrays on top of a fixed part: equal steps for equal steps in cells (to the
    # 256-byte alignment of each array and the multigrid's rounding of odd dimensions)
    for f in (f64, mix):
        assert f[0] < f[1] < f[2]
        assert abs((f[2] - f[1]) - (f[1] - f[0])) <= 0.02 * (f[1] - f[0])
    assert all(m < d for m, d in zip(mix, f64))


# per colour slot: both colours' 6 off-diagonal blocks of 9 in the copy's type, and the finest
# stencil's 6 slots + 1/diag of each colour in the preconditioner's type; the black rows'
# stage-2 combination (18 values) moves from the preconditioner's type (without copies) to the
# copy's.  In FP64 the block inverses move from by cell (9 per cell) to per colour slot (9 per
# slot and colour).
@pytest.mark.parametrize("precision,store,bytes_per_slot,bytes_per_cell", [
    (0, 1, 2 * 54 * 8 + 2 * 7 * 8 + 2 * 9 * 8, -9 * 8),   # FP64
    (1, 1, 2 * 54 * 4 + 2 * 7 * 4, 0),                    # mixed, FP32 block copies
    (1, 2, 2 * 54 * 2 + 2 * 7 * 4 + 18 * (2 - 4), 0),     # mixed, BF16 block copies
])
def test_per_colour_copies_add_their_arrays(B, precision, store, bytes_per_slot, bytes_per_cell):
    sc = G.scenario_c1(nx=31, ny=17, nz=6)
    base = B.footprint(sc, precond=B.PF_PC_CPR, precision=precision, ilu_store=0)
    with_copies = B.footprint(sc, precond=B.PF_PC_CPR, precision=precision, ilu_store=store)
    extra = with_copies - base
    expect = bytes_per_slot * colour_slots(sc) + bytes_per_cell * sc["nx"] * sc["ny"] * sc["nz"]
    assert abs(extra - expect) <= 5 * 256   # each array starts on a 256-byte boundary
