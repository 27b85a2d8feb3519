"""The benchmark's roofline accounting, on the CPU.

The algorithmic bytes per launch that `bench.py` divides by a kernel's time are counted from the
matrix pattern.  On a natural-order box with the 7-point stencil the block counts have closed
forms: (nx-1) ny nz + nx (ny-1) nz + nx ny (nz-1) lower blocks, as many upper blocks, one diagonal
block per cell.  These tests check the pattern-derived counts against that geometry and the
per-launch byte counts against what each kernel must move once.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import bench  # noqa: E402


def _box(nx, ny, nz):
    return synth.make_box(nx, ny, nz, 3.125, seed=3).system()


@pytest.mark.parametrize("dims", [(5, 4, 3), (7, 1, 1), (2, 3, 4)])
@pytest.mark.parametrize("mixed", [False, True])
def test_algorithmic_bytes_follow_the_box_geometry(dims, mixed):
    nx, ny, nz = dims
    s = _box(nx, ny, nz)
    n, b = s["n"], s["b"]
    assert n == nx * ny * nz
    lower = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert int(s["row_ptr"][-1]) == n + 2 * lower            # the pattern is the 7-point stencil
    f = 4 if mixed else 8                                    # preconditioner value and vector size
    nb, chunks = n * b, (n + 31) // 32
    blk = lambda w: w * b * b + 4                            # a block's values and its column
    got = bench.algorithmic_bytes(s, mixed)
    # outer SpMV (FP64 in both forms): every block once, the chunk offsets, z read, w written
    assert got["spmv"] == (n + 2 * lower) * blk(8) + (chunks + 1) * 8 + 2 * nb * 8
    # forward sweep: the L blocks, the positions, r read and y written
    assert got["ilu_fwd"] == lower * blk(f) + n * 4 + 2 * nb * f
    # backward sweep: the U blocks (as many as L on the stencil), the inverted pivots, two
    # position tables, y read, the intermediate written, z written in FP64, dp and dT read
    assert got["ilu_bwd"] == lower * blk(f) + n * f * b * b + n * 8 + 2 * nb * f + nb * 8 + 2 * n * f
    # stage-1 residual: the p and T columns of every block, offsets, v read (FP64), b1 written,
    # dp and dT read
    assert got["stage1_resid"] == (n + 2 * lower) * (f * 2 * b + 4) + (chunks + 1) * 8 + nb * 8 + nb * f + 2 * n * f


def test_vcycle_bytes_of_a_level_pair():
    # a level of n rows and nnz entries with an n x nc interpolation of nnzP entries: the four
    # kernels of its V-cycle step read the matrix (values + columns + row pointers) and the vectors
    info = [{"n": 1000, "nnz": 6800, "nnzP": 2400}, {"n": 300}]
    for f in (8, 4):
        got = bench.vcycle_bytes(info, f)
        mat = 6800 * (4 + f) + 4 * 1001
        assert got["down"] == mat + 4 * f * 1000              # D^-1, b read; t, r written
        assert got["post"] == mat + 4 * f * 1000              # D^-1, b, t read; x written
        assert got["restrict"] == 2400 * (4 + f) + 4 * 301 + f * 1000 + f * 300
        assert got["prolong"] == 2400 * (4 + f) + 4 * 1001 + f * 300 + 2 * f * 1000


def test_roofline_line_arithmetic():
    # 20 launches over 2 steps, 0.5 ms in all: 25 us per launch; 100 MB per launch -> 4000 GB/s
    line = bench.roofline_line("k", 100e6, 0.5, 20, 2, 8000.0, "measured", traffic=120e6)
    assert line["avg_launch_us"] == pytest.approx(25.0)
    assert line["achieved"] == pytest.approx(4000.0)
    assert line["frac"] == pytest.approx(0.5)
    assert line["launches_per_step"] == 10 and line["ms_per_step"] == pytest.approx(0.25)
    assert line["traffic"] == 120e6 and line["bound"] == "hbm"
