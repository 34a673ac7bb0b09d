"""bench.py's host-side arithmetic: the algorithmic byte counts that the
roofline fractions divide by, and the whole-job throughput of replicas."""

import sys

import pytest


@pytest.fixture(scope="module")
def bench():
    sys.argv = ["bench.py"]
    import bench as b
    return b


def test_block_and_face_counts_of_the_benchmark_grids(bench):
    # faces = (nx-1) ny nz + nx (ny-1) nz + nx ny (nz-1); blocks = N + 2F
    assert bench.spmv_algorithmic({"nx": 100, "ny": 100, "nz": 10}, 0) == (676000, 100000, 288000)
    assert bench.spmv_algorithmic({"nx": 600, "ny": 450, "nz": 100}, 0) == (188250000, 27000000, 80625000)
    assert bench.spmv_algorithmic({"nx": 10, "ny": 10, "nz": 3}, 0) == (1780, 300, 740)
    assert bench.spmv_algorithmic({"nx": 1, "ny": 1, "nz": 1}, 0) == (1, 1, 0)


def test_algorithmic_bytes_of_the_benchmark_grids(bench):
    blocks, ncell, _ = bench.spmv_algorithmic({"nx": 100, "ny": 100, "nz": 10}, 50)
    # FP64: 676,000 blocks x 8 values x 8 B (the oil row's polymer column is
    # structurally zero) + 300,000 unknowns x (8 B read + 8 B written)
    # + 50 perforations x 3 x 2 x 8 B (B and C border) + 5 wells x 8 B (D)
    assert bench.spmv_bytes(blocks, ncell, 50, 5, 8, 8) == 43_264_000 + 4_800_000 + 2_400 + 40
    # mixed: FP32 blocks and FP32 vector copy, FP64 result
    assert bench.spmv_bytes(blocks, ncell, 50, 5, 4, 4) == 21_632_000 + 3_600_000 + 1_200 + 20
    # 16 flops per block (8 multiply-adds) + 12 per perforation + 2 per well
    assert bench.spmv_flops(blocks, 50, 5) == 10_816_000 + 600 + 10
    # assembly: 632 B per cell in FP64, 380 B in mixed precision
    assert bench.assembly_bytes(ncell, 8) == 63_200_000
    assert bench.assembly_bytes(27_000_000, 4) == 10_260_000_000


def test_replicas_add_up(bench):
    assert bench.replica_throughput(1, 100_000, 20, 0.04) == pytest.approx(50e6)
    assert bench.replica_throughput(4, 100_000, 20, 0.04) == pytest.approx(200e6)  # weak scaling: whole job
