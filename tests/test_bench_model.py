"""The byte and flop models behind the reported rooflines, at the 1M-lattice sizes
(n = 1,000,000, m = 1,998,000, k = 3, grid cap 1023: N_int = 341, G = 1023, P = 2048),
checked against the per-unit figures written out by hand. CPU only."""
import pytest

import bench

N, M, G, P, NINT = 1_000_000, 1_998_000, 1023, 2048, 341
NH = P // 2 + 1
NBOX = NINT * NINT


@pytest.mark.parametrize("stage, expected", [
    # bin: 8 B position in, 8 B (key, slot) out; scan: count in, offset out; scatter:
    # (key, slot), position and permutation in, sorted position and permutation out
    ("sort", 48 * N + 8 * NBOX),
    # sorted positions in, box offsets in, three FP32 planes out
    ("spread", 8 * N + 4 * NBOX + 12 * G * G),
    # three FP32 planes in, three half spectra (complex64) out
    ("rows_fwd", 12 * G * G + 24 * G * NH),
    # per column: three sequences of G complex in and out, three real spectra of P
    ("cols", NH * 3 * (8 * G + 4 * P + 8 * G)),
    # three half spectra in, one float4 per grid node out
    ("rows_inv", 24 * G * NH + 16 * G * G),
    # sorted position, permutation, attraction in; the float4 grid; positions out twice
    ("gather_update", 36 * N + 16 * G * G),
    # positions, row pointers, column ids, neighbour positions in; attraction out
    ("attract", 16 * N + 4 * (N + 1) + 12 * 2 * M),
])
def test_stage_bytes(stage, expected):
    assert bench.stage_bytes(stage, N, M, G, P, NBOX) == expected


def test_column_stage_bytes_value():
    # the figure the dominant-kernel roofline divides by its launch time
    assert bench.stage_bytes("cols", N, M, G, P, NBOX) == 75_522_000


def test_lattice_grid_sizes():
    # N_int = ceil(L) capped at floor(1023 / 3) = 341 for L ~ 1000; G = 3 N_int; P the
    # next power of two of 2 G - 1
    assert 1023 // 3 == NINT and 3 * NINT == G
    assert P == 1 << (2 * G - 1 - 1).bit_length()


def test_workload_generators_sizes():
    e, xy = bench.make_workload("er_64k_exact")
    assert xy.shape == (65536, 2) and e.shape == (4 * 65536, 2)
    e, xy = bench.make_workload("er_2000_exact")
    assert xy.shape == (2000, 2) and e.shape == (8000, 2)


def test_iteration_model_bytes_lattice():
    # node bytes 28 n + 24 m and the single-pass grid model at G = 1023, P = 2048:
    # 76.0 MB + 151.1 MB
    node = 28 * N + 24 * M
    grid = 2 * 3 * 4 * G * G + 2 * 3 * P * NH * 8 + 3 * P * NH * 4
    assert bench.iteration_model_bytes(N, M, G, P) == node + grid == 227_020_696
    r = bench.iteration_roofline(N, M, G, P, 0.2270206960, 6753.1)
    assert r["achieved"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(1000.0 / 6753.1)
    assert bench.iteration_roofline(N, M, 0, 0, 1.0, 6753.1) is None
