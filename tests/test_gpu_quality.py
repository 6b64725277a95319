"""Layout quality of the ibFFT path against the exact path (Sec. 4.2: the relative
SE / NP1 / NP2 / CL / MA of ibFFT layouts stay within a few percent of the exact ones,
mean near zero). Three synthetic graph classes, 300-iteration layouts from the same
start; metrics from `paper_2303_03964_gb300.quality` on the host."""
import numpy as np
import pytest

from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")

METRICS = ("SE", "NP1", "NP2", "CL", "MA")


@pytest.fixture(scope="module")
def relative():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_03964_gb300 import quality as q
    from paper_2303_03964_gb300 import tfdp
    rng = synth.rng_for(6)
    graphs = []
    e, _ = synth.sbm(2000, 10, 8.0, 0.9, rng)
    graphs.append((2000, e))
    graphs.append((1600, synth.lattice(40, 40)))
    graphs.append((2000, synth.barabasi_albert(2000, 2, rng)))
    rel = []
    for n, e in graphs:
        xy0 = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng)
        m = {}
        for rep in (tfdp.REP_EXACT, tfdp.REP_FFT):
            with tfdp.Graph(n, e, xy0, tfdp.params_default(rep_mode=rep, total_iters=300, grid_max=255)) as g:
                g.iterate(300)
                m[rep] = q.evaluate(g.get_positions(), e)
        rel.append({k: q.relative(m[tfdp.REP_FFT][k], m[tfdp.REP_EXACT][k]) for k in METRICS})
    return rel


def test_each_graph_within_six_percent(relative):
    # A single layout is one trajectory of a chaotic iteration: two exact layouts of the
    # same graph from two random starts differ by a few percent as well (the bench
    # quality line reports that spread), so the per-graph bound sits above the paper's
    # 4 % band, which is a statement about the mean.
    for r in relative:
        for k in METRICS:
            assert abs(r[k]) <= 0.06, (k, r)


def test_mean_over_graphs_within_paper_band(relative):
    # Sec. 4.2: relative values within [-4 %, +4 %], mean near zero
    for k in METRICS:
        assert abs(np.mean([r[k] for r in relative])) <= 0.04, k
