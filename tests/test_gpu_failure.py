"""Failure detection on the GPU without a GPU fault.

Two failures are made on purpose, both through the tfdp_debug_inject test hook:

* a bounded device-side wait that runs out: the first tile of the box-count scan
  withholds its status word and the look-back waits give up after a few thousand polls.
  The kernel records the timeout in the device flags and returns; the next synchronising
  call must return TFDP_ERR_TIMEOUT, and the graph must compute correct forces again
  once the hook is off (the visit order restarts from the caller order);
* an FFT-buffer allocation refused on the host, as if the device were full: the call
  that asked for a larger grid returns TFDP_ERR_OUT_OF_MEMORY, the next iteration retries
  the allocation (refused again: nothing launches, nothing moves), and once it succeeds
  the forces match the oracle at the new grid.
"""
import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
TIMEOUT, OUT_OF_MEMORY = 6, 4


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_03964_gb300 import tfdp as t
    return t


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_fft(xy32, P, k=3, grid_max=1023):
    grid = oracle.grid_policy(xy32, k, 50, grid_max)
    return oracle.rep_fft(xy32.astype(np.float64), 2.0, k, grid=grid, P=P, xy_f32=xy32)


def test_scan_wait_that_runs_out_is_reported_as_timeout(tfdp):
    rng = synth.rng_for(61)
    n = 40_000  # side 200: N_int = 200, 40,000 boxes, 20 scan tiles
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = synth.uniform_positions(n, 100.0, rng)
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=1023, total_iters=50)) as g:
        g.iterate(2)
        g.synchronize()
        assert g.stats()["device_flags"] == 0
        g.debug_inject(tfdp.INJECT_SCAN_STALL, 2000)
        g.iterate(1)
        with pytest.raises(tfdp.TfdpError) as ei:
            g.synchronize()
        assert ei.value.status == TIMEOUT
        assert g.stats()["device_flags"] & tfdp.FLAG_WAIT_TIMEOUT
        assert np.all(np.isfinite(g.get_positions()))  # reported once, then cleared
        g.debug_inject(tfdp.INJECT_SCAN_STALL, 0)
        g.set_positions(xy)
        g.set_iteration(0)
        fr, _ = g.eval_forces()
        P = g.stats()["fft_P"]
        g.iterate(1)
        g.synchronize()
    assert rel_l2(fr, _oracle_fft(xy, P)) <= FORCE_TOL


def test_refused_fft_allocation_is_retried_and_never_launches_without_buffers(tfdp):
    rng = synth.rng_for(63)
    n = 5_000
    e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
    xy = synth.uniform_positions(n, 60.0, rng)
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=255, total_iters=50)) as g:
        g.iterate(2)
        before = g.get_positions()
        it = g.stats()["iteration"]
        g.debug_inject(tfdp.INJECT_FFT_ALLOC, 2)
        with pytest.raises(tfdp.TfdpError) as ei:
            g.set_params(grid_max=511)
        assert ei.value.status == OUT_OF_MEMORY
        with pytest.raises(tfdp.TfdpError) as ei:
            g.iterate(1)
        assert ei.value.status == OUT_OF_MEMORY
        # nothing ran: same positions, same iteration counter
        assert np.array_equal(g.get_positions(), before)
        assert g.stats()["iteration"] == it
        # the third attempt is allowed: buffers for the larger grid, correct forces
        g.set_positions(xy)
        fr, _ = g.eval_forces()
        st = g.stats()
        assert st["fft_P"] == 1024
        g.iterate(3)
        g.synchronize()
        assert st["device_flags"] == 0
    assert rel_l2(fr, _oracle_fft(xy, 1024, grid_max=511)) <= FORCE_TOL
