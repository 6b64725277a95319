"""Batches: every graph of a batch must give the forces and the
short layout of its solo run (and, through it, of the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
POS_TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _mixed_graphs(count, seed, nmin=300, nmax=6000):
    """Log-uniform sizes; SBM (10 blocks, mean degree 8), BA (m0 = 2) and lattices in turn."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        kind = q % 3
        if kind == 0:
            n = max(10, n // 10 * 10)
            e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
        elif kind == 1:
            e = synth.barabasi_albert(n, 2, rng)
        else:
            side = max(2, int(np.sqrt(n)))
            n = side * side
            e = synth.lattice(side, side)
        xy = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng)
        out.append((n, e, xy))
    return out


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_03964_gb300 import tfdp as t
    return t


@pytest.mark.parametrize("phases", [True, False])
@pytest.mark.parametrize("grid_max", [255, 100])
def test_batch_forces_equal_solo(tfdp, grid_max, phases):
    """Both launch shapes (one launch per phase, one cooperative persistent launch) give
    every graph its solo run's forces."""
    graphs = _mixed_graphs(9, 31 + grid_max)
    params = [tfdp.params_default(grid_max=grid_max, gamma=2.0 + 0.5 * (q % 3)) for q in range(len(graphs))]
    with tfdp.Batch(graphs, params) as b:
        assert b.grid_blocks() > 0 and b.phase_parts() == 1
        b.set_phase_launches(phases)
        assert b.phase_parts() == (1 if phases else 0)
        for q, (n, e, xy) in enumerate(graphs):
            fr_b, fa_b = b.eval_forces(q)
            with tfdp.Graph(n, e, xy, params[q]) as g:
                fr_s, fa_s = g.eval_forces()
                st = g.stats()
            assert _rel(fr_b, fr_s) <= FORCE_TOL, (q, _rel(fr_b, fr_s))
            assert _rel(fa_b, fa_s) <= FORCE_TOL
            if q < 3:
                grid = oracle.grid_policy(xy, 3, 50, grid_max)
                ref = oracle.rep_fft(xy.astype(np.float64), params[q].gamma, 3, grid=grid, xy_f32=xy)
                assert _rel(fr_b, ref) <= FORCE_TOL
            assert b.stats(q)["grid_G"] == st["grid_G"]


@pytest.mark.parametrize("phases", [True, False])
def test_batch_layout_equals_solo(tfdp, phases):
    graphs = _mixed_graphs(6, 77, nmin=500, nmax=3000)
    params = [tfdp.params_default(grid_max=255, total_iters=50) for _ in graphs]
    T = 8
    with tfdp.Batch(graphs, params) as b:
        b.set_phase_launches(phases)
        b.iterate(3)
        b.iterate(T - 3)  # two launches (two captured graphs) in a row
        for q, (n, e, xy) in enumerate(graphs):
            out_b = b.get_positions(q)
            assert b.stats(q)["iteration"] == T and b.stats(q)["device_flags"] == 0
            with tfdp.Graph(n, e, xy, params[q]) as g:
                g.iterate(T)
                out_s = g.get_positions()
            assert _rel(out_b, out_s) <= POS_TOL, (q, _rel(out_b, out_s))


def test_batch_launch_shapes_bitwise_equal(tfdp):
    """One launch per phase and one cooperative launch run the same phase bodies, and every
    sum on the path is order-independent (the spread in exact fixed point), so a layout is
    bit for bit the same under both shapes, with a k = 1 part and a k = 3 part."""
    graphs = _mixed_graphs(6, 55, nmin=400, nmax=4000)
    params = [tfdp.params_default(k_interp=(1 if q % 2 else 3), grid_max=255, total_iters=40)
              for q in range(len(graphs))]
    outs = []
    for phases in (True, False):
        with tfdp.Batch(graphs, params) as b:
            assert b.num_parts() == 2
            b.set_phase_launches(phases)
            b.iterate(7)
            outs.append([b.get_positions(q) for q in range(len(graphs))])
    for q in range(len(graphs)):
        assert np.array_equal(outs[0][q], outs[1][q]), q


def test_batch_parts_of_mixed_k_and_fft_size_equal_solo(tfdp):
    """Graphs with different k and grid caps run as several parts (one set of launches
    per (k, FFT size)); each graph still gives its solo run's forces and layout, and the
    oracle's ibFFT at its own grid."""
    graphs = _mixed_graphs(8, 91, nmin=400, nmax=5000)
    settings = [(1, 63), (2, 127), (3, 255), (1, 255), (3, 127), (2, 63), (1, 127), (3, 255)]
    params = [tfdp.params_default(k_interp=k, grid_max=gm, total_iters=40) for k, gm in settings]
    with tfdp.Batch(graphs, params) as b:
        assert b.num_parts() == len(set((k, max(7, int(np.ceil(np.log2(2 * (gm // k) * k - 1)))))
                                        for k, gm in settings))
        for q, (n, e, xy) in enumerate(graphs):
            fr_b, _ = b.eval_forces(q)
            with tfdp.Graph(n, e, xy, params[q]) as g:
                fr_s, _ = g.eval_forces()
                st = g.stats()
            assert _rel(fr_b, fr_s) <= FORCE_TOL, (q, _rel(fr_b, fr_s))
            assert b.stats(q)["fft_P"] == st["fft_P"] and b.stats(q)["grid_G"] == st["grid_G"]
            k, gm = settings[q]
            grid = oracle.grid_policy(xy, k, 50, gm)
            ref = oracle.rep_fft(xy.astype(np.float64), 2.0, k, grid=grid, xy_f32=xy)
            assert _rel(fr_b, ref) <= FORCE_TOL, (q, _rel(fr_b, ref))
        b.iterate(6)
        for q, (n, e, xy) in enumerate(graphs):
            with tfdp.Graph(n, e, xy, params[q]) as g:
                g.iterate(6)
                assert _rel(b.get_positions(q), g.get_positions()) <= POS_TOL


def test_batch_plan_meets_its_error_bound(tfdp):
    """The grid autotuner's choice per graph: an FFT no larger than the reference's, and a
    repulsion error against the exact sum within the requested ratio of the reference
    parameters' error (checked here on every graph, also the ones it did not measure)."""
    graphs = _mixed_graphs(12, 93, nmin=800, nmax=20000)
    base = tfdp.params_default(grid_max=255)
    ratio, floor = 1.5, 0.02
    params, err = tfdp.batch_plan(graphs, base, max_error_ratio=ratio, min_error_bound=floor, probes=2)
    assert len(params) == len(graphs) and np.all(np.isfinite(err))
    sizes = []
    for q, (n, e, xy) in enumerate(graphs):
        p = params[q]
        assert p.gamma == base.gamma and p.rep_mode == tfdp.REP_FFT and 1 <= p.k_interp <= 3
        with tfdp.Graph(n, e, xy, p) as g:
            fr, _ = g.eval_forces()
            sizes.append(g.stats()["fft_P"])
        with tfdp.Graph(n, e, xy, base) as g:
            fr_ref, _ = g.eval_forces()
            assert sizes[-1] <= g.stats()["fft_P"]
        rows = np.random.default_rng(q).choice(n, min(n, 1000), replace=False)
        ex = oracle.rep_exact(xy.astype(np.float64), 2.0, rows=rows)
        e_ref, e_got = _rel(fr_ref[rows], ex), _rel(fr[rows], ex)
        # graphs the tuner did not measure share their size group's choice: allow a margin
        assert e_got <= 1.25 * max(ratio * e_ref, floor) + 1e-4, (q, n, e_got, e_ref)
    with tfdp.Batch(graphs, params) as b:
        b.iterate(2)
        b.synchronize()
        # the launch-shape autotuner keeps either shape; the layout goes on from where it is
        b.autotune(2)
        assert 0 <= b.phase_parts() <= b.num_parts()
        b.iterate(2)
        b.synchronize()
        assert all(b.stats(q)["iteration"] == 4 and b.stats(q)["device_flags"] == 0 for q in range(len(graphs)))


def test_batch_rejects_dynamic_k_and_bad_graph(tfdp):
    g1 = (10, [[0, 1]], np.zeros((10, 2), np.float32))
    bad = (10, [[0, 0]], np.zeros((10, 2), np.float32))
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.Batch([g1, bad])
    assert ei.value.status == 2
    # one fixed k per batch: the dynamic schedule is for single graphs
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.Batch([g1, g1], [tfdp.params_default(k_interp=tfdp.K_DYNAMIC)] * 2)
    assert ei.value.status == 3
