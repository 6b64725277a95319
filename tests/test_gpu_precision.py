"""Precision mode TFDP_PREC_BF16X3: the column stage of the grid interaction (Sec. 3.4,
second step) as BF16 split-precision tensor-core products with FP32 accumulation.

The force field is compared with the FP64 oracle's ibFFT (the same reference the FP32
mode is held to) on the workloads of config 3, and with the FP32 mode itself. Each
measured error is written to $TFDP_PARITY_LOG. The tolerance MIXED_TOL is the error the
split products leave: each operand keeps about 16 bits (hi + lo), the dropped lo x lo
term and the split residues are about 2^-16 of each product, and four stages compound
them, so the grid outputs carry a few 1e-6 of relative error, which the gather can
amplify where the interpolated field nearly cancels.
"""
import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4
FORCE_TOL = 1e-5


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_03964_gb300 import tfdp as t
    return t


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def record(name, value):
    import json
    import os
    path = os.environ.get("TFDP_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, "value": value}) + "\n")
    return value


def _forces(tfdp, n, e, xy, precision, **kw):
    p = tfdp.params_default(grid_max=1023, precision=precision, **kw)
    with tfdp.Graph(n, e, xy, p) as g:
        fr, fa = g.eval_forces()
        st = g.stats()
        grid = g.debug_fetch(tfdp.DEBUG_GRID_OUTPUT)
    assert st["fft_P"] == 2048 and st["device_flags"] == 0
    return fr, fa, st, grid


def _oracle(xy, st, gamma=2.0):
    grid = oracle.grid_policy(xy, 3, 50, 1023)
    assert grid["G"] == st["grid_G"]
    return oracle.rep_fft(xy.astype(np.float64), gamma, 3, grid=grid, P=st["fft_P"], xy_f32=xy)


def test_bf16x3_small_graph_against_oracle_and_fp32(tfdp):
    rng = synth.rng_for(71)
    n = 3001
    e = synth.erdos_renyi(n, 9000, rng)
    xy = synth.uniform_positions(n, 40.0, rng)
    fr, fa, st, grid = _forces(tfdp, n, e, xy, tfdp.PREC_BF16X3)
    fr32, fa32, _, grid32 = _forces(tfdp, n, e, xy, tfdp.PREC_FP32)
    G = st["grid_G"]
    gerr = record("bf16x3_small_grid_vs_fp32", rel_l2(grid[:G, :G, :3], grid32[:G, :G, :3].astype(np.float64)))
    err = record("bf16x3_small_frep", rel_l2(fr, _oracle(xy, st)))
    record("bf16x3_small_frep_vs_fp32", rel_l2(fr, fr32.astype(np.float64)))
    assert np.array_equal(fa, fa32)  # the attraction does not touch the grid
    assert gerr <= MIXED_TOL
    assert err <= MIXED_TOL


def test_bf16x3_lattice_1m_full_size(tfdp):
    """Config 3 (i) in the mixed mode: all 1M nodes against the oracle's ibFFT."""
    e, xy = synth.lattice_1m()
    n = xy.shape[0]
    fr, _, st, _ = _forces(tfdp, n, e, xy, tfdp.PREC_BF16X3)
    assert record("bf16x3_lattice1m_frep", rel_l2(fr, _oracle(xy, st))) <= MIXED_TOL


def test_bf16x3_sbm_100k(tfdp):
    """The SBM of config 2 at the mixed mode's FFT size (grid up to 1023, P = 2048)."""
    e, xy = synth.sbm_100k()
    n = xy.shape[0]
    fr, _, st, _ = _forces(tfdp, n, e, xy, tfdp.PREC_BF16X3)
    assert record("bf16x3_sbm100k_frep", rel_l2(fr, _oracle(xy, st))) <= MIXED_TOL


def test_bf16x3_spectrum_rebuilt_on_gamma_and_mode_changes(tfdp):
    rng = synth.rng_for(72)
    n = 5000
    e = synth.erdos_renyi(n, 15000, rng)
    xy = synth.uniform_positions(n, 50.0, rng)
    p = tfdp.params_default(grid_max=1023, precision=tfdp.PREC_BF16X3)
    with tfdp.Graph(n, e, xy, p) as g:
        g.eval_forces()
        g.set_params(gamma=3.0)  # new spectrum
        fr3, _ = g.eval_forces()
        st = g.stats()
        g.set_params(gamma=3.0, precision=tfdp.PREC_FP32)  # the FP32 spectrum is rebuilt too
        fr3_32, _ = g.eval_forces()
        g.set_params(gamma=3.0, precision=tfdp.PREC_BF16X3)
        fr3b, _ = g.eval_forces()
    ref = _oracle(xy, st, gamma=3.0)
    assert record("bf16x3_gamma3_frep", rel_l2(fr3, ref)) <= MIXED_TOL
    assert rel_l2(fr3_32, ref) <= FORCE_TOL
    assert np.array_equal(fr3, fr3b)  # the same mode gives the same bits


def test_bf16x3_layout_is_reproducible(tfdp):
    rng = synth.rng_for(73)
    n = 20_000
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = synth.uniform_positions(n, 70.0, rng)
    p = tfdp.params_default(grid_max=1023, precision=tfdp.PREC_BF16X3, total_iters=50)
    out = []
    for _ in range(2):
        with tfdp.Graph(n, e, xy, p) as g:
            g.iterate(10)
            out.append(g.get_positions())
            assert g.stats()["device_flags"] == 0
    assert np.array_equal(out[0], out[1])
    ref = oracle.iterate(xy.astype(np.float64), e, 10, mode="fft", grid_max=1023, P=2048, T=50)
    record("bf16x3_sbm20k_10it_pos", rel_l2(out[0], ref))
    assert rel_l2(out[0], ref) <= 1e-3
