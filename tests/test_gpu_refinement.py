"""Local refinement (Sec. 5 "Local Refinement"): per-node weights through the C ABI
against the FP64 oracle. Reading: the pair repulsion is scaled by r_i r_j and the edge
attraction by a_i a_j; all weights 1 is the plain method."""
import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
POS_TOL = 1e-4


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_03964_gb300 import tfdp as t
    return t


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def record(name, value):
    """Append a measured parity error to $TFDP_PARITY_LOG (JSON lines), if set."""
    import json
    import os
    path = os.environ.get("TFDP_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, "value": value}) + "\n")
    return value


def _graph(n, seed, span):
    rng = np.random.default_rng(seed)
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = rng.uniform(-span, span, size=(n, 2)).astype(np.float32)
    wr = rng.uniform(0.25, 6.0, n).astype(np.float32)
    wa = rng.uniform(0.25, 6.0, n).astype(np.float32)
    return e, xy, wr, wa


def test_exact_path_weighted_forces(tfdp):
    n = 777
    e, xy, wr, wa = _graph(n - 7, 51, 10.0)
    xy = np.vstack([xy, np.random.default_rng(52).uniform(-10, 10, (7, 2)).astype(np.float32)])
    wr = np.concatenate([wr, np.full(7, 3.0, np.float32)])
    wa = np.concatenate([wa, np.full(7, 0.5, np.float32)])
    with tfdp.Graph(n, e, xy, tfdp.params_default(rep_mode=tfdp.REP_EXACT)) as g:
        g.set_node_weights(wr, wa)
        fr, fa = g.eval_forces()
    x64 = xy.astype(np.float64)
    assert record("weights_exact_frep", rel_l2(fr, oracle.rep_exact(x64, 2.0, w=wr))) <= FORCE_TOL
    assert record("weights_exact_fatt", rel_l2(fa, oracle.attraction(e, x64, 0.1, 8.0, w=wa))) <= FORCE_TOL


def test_fft_path_weighted_forces(tfdp):
    n = 20000
    e, xy, wr, wa = _graph(n, 53, 70.0)
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=255)) as g:
        g.set_node_weights(wr, wa)
        fr, fa = g.eval_forces()
        st = g.stats()
    grid = oracle.grid_policy(xy, 3, 50, 255, oracle.GRID_SNAP_H)
    ref = oracle.rep_fft(xy.astype(np.float64), 2.0, 3, grid=grid, P=st["fft_P"], xy_f32=xy, w=wr)
    assert record("weights_fft_frep", rel_l2(fr, ref)) <= FORCE_TOL
    assert record("weights_fft_fatt",
                  rel_l2(fa, oracle.attraction(e, xy.astype(np.float64), 0.1, 8.0, w=wa))) <= FORCE_TOL


def _fisheye(n, seed, span):
    """Focal nodes pull their neighbours in (attraction weight 8) while the other nodes
    repel more strongly (repulsion weight 2)."""
    rng = np.random.default_rng(seed)
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = rng.uniform(-span, span, size=(n, 2)).astype(np.float32)
    focal = rng.choice(n, 12, replace=False)
    wa = np.ones(n, np.float32)
    wa[focal] = 8.0
    wr = np.full(n, 2.0, np.float32)
    wr[focal] = 1.0
    return e, xy, wr, wa


def test_fisheye_layout_exact_path(tfdp):
    """30 iterations with exact repulsion, whose force is continuous in the positions, so
    the FP32 and FP64 trajectories stay close."""
    n = 2000
    e, xy, wr, wa = _fisheye(n, 54, 50.0)
    with tfdp.Graph(n, e, xy, tfdp.params_default(rep_mode=tfdp.REP_EXACT, total_iters=100)) as g:
        g.set_node_weights(wr, wa)
        g.iterate(30)
        out = g.get_positions()
        assert g.stats()["device_flags"] == 0
    ref = oracle.iterate(xy.astype(np.float64), e, 30, mode="exact", T=100, wrep=wr, watt=wa)
    assert record("fisheye_exact_30it_pos", rel_l2(out, ref)) <= POS_TOL


def test_fisheye_layout_fft_path(tfdp):
    """3 iterations of the ibFFT path. Longer FFT trajectories drift apart where the FP32
    and FP64 positions put a node in different boxes (the per-box interpolation is
    discontinuous at box borders), which stronger forces make more frequent; the force
    field itself is compared at full tolerance above."""
    n = 20000
    e, xy, wr, wa = _fisheye(n, 57, 70.0)
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=255, total_iters=300)) as g:
        g.set_node_weights(wr, wa)
        g.iterate(3)
        out = g.get_positions()
        assert g.stats()["device_flags"] == 0
    ref = oracle.iterate(xy.astype(np.float64), e, 3, mode="fft", k=3, grid_max=255,
                         policy=oracle.GRID_SNAP_H, P=512, T=300, wrep=wr, watt=wa)
    assert record("fisheye_fft_3it_pos", rel_l2(out, ref)) <= POS_TOL


@pytest.mark.parametrize("rep", ["exact", "fft"])
def test_unit_weights_and_reset_are_the_plain_method(tfdp, rep):
    n = 3001
    e, xy, wr, wa = _graph(n - 1, 55, 30.0)
    xy = np.vstack([xy, [[0.5, -0.25]]]).astype(np.float32)
    p = tfdp.params_default(grid_max=255, rep_mode=tfdp.REP_EXACT if rep == "exact" else tfdp.REP_FFT)
    with tfdp.Graph(n, e, xy, p) as g:
        plain = g.eval_forces()
        g.set_node_weights(np.ones(n, np.float32), np.ones(n, np.float32))
        unit = g.eval_forces()
        g.set_node_weights(np.append(wr, 1.0), np.append(wa, 1.0))
        weighted = g.eval_forces()
        g.set_node_weights(None, None)
        reset = g.eval_forces()
    for a, b in zip(plain, unit):
        assert np.array_equal(a, b)
    for a, b in zip(plain, reset):
        assert np.array_equal(a, b)
    assert not np.array_equal(plain[0], weighted[0])


def test_weight_out_of_range_changes_nothing(tfdp):
    n = 500
    e, xy, wr, wa = _graph(n, 56, 10.0)
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=255)) as g:
        before = g.eval_forces()
        bad = np.ones(n, np.float32)
        bad[7] = tfdp.WEIGHT_MAX * 2
        for args in ((bad, None), (None, -bad), (np.full(n, np.nan, np.float32), None)):
            with pytest.raises(tfdp.TfdpError) as ei:
                g.set_node_weights(*args)
            assert ei.value.status == 3
        after = g.eval_forces()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
