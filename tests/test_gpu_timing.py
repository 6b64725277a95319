"""Stage timing through the C ABI: only the stages in the mask are timed, stages the
mode does not run read zero, and timing changes no bit of the computed layout."""
import numpy as np
import pytest

from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_03964_gb300 import tfdp as t
    return t


FFT_STAGES = ["sort", "spread", "spectrum", "rows_fwd", "cols", "rows_inv", "gather_update", "attract"]


def _graph(tfdp, rep=None):
    rng = np.random.default_rng(41)
    n = 20000
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = rng.uniform(-70, 70, size=(n, 2)).astype(np.float32)
    p = tfdp.params_default(grid_max=255, total_iters=300,
                            rep_mode=tfdp.REP_FFT if rep is None else rep)
    return tfdp.Graph(n, e, xy, p)


def test_mask_times_only_selected_stages(tfdp):
    with _graph(tfdp) as g:
        g.set_stage_timing_mask(["cols", "attract"])
        g.iterate(1)
        t = g.stage_times()
        assert t["cols"] > 0 and t["attract"] > 0
        assert all(v == 0.0 for k, v in t.items() if k not in ("cols", "attract"))
        g.set_stage_timing(True)
        g.iterate(1)
        t = g.stage_times()
        assert all(t[k] > 0 for k in FFT_STAGES)
        assert t["exact"] == 0.0 and t["edge_update"] == 0.0
        g.set_stage_timing(False)
        g.iterate(1)
        with pytest.raises(tfdp.TfdpError):
            g.stage_times()


def test_exact_mode_stages(tfdp):
    with _graph(tfdp, rep=tfdp.REP_EXACT) as g:
        g.set_stage_timing(True)
        g.iterate(1)
        t = g.stage_times()
        assert t["exact"] > 0 and t["edge_update"] > 0
        assert all(t[k] == 0.0 for k in FFT_STAGES)


def test_timing_changes_no_bit_of_the_layout(tfdp):
    outs = []
    for mask in ([], ["gather_update"], list(tfdp.STAGES)):
        with _graph(tfdp) as g:
            g.set_stage_timing_mask(mask)
            g.iterate(7)
            outs.append(g.get_positions())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
