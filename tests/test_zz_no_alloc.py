"""The no-allocation exact repulsion (tfdp_exact_repulsion_noalloc), called through the
C ABI, must give the graph API's exact forces.

It exists for callers that cannot allocate device memory: code under a framework whose
caching allocator owns the device pool, and latency-critical loops where cudaMalloc /
cudaFree could synchronise the device. Its scratch is one fixed array inside the library
shared by all calls, so this test makes two calls in a row (the second one finds the
first one's partial sums in the array) and checks both.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_noalloc_exact_repulsion_matches_graph_api_twice():
    import torch
    from paper_2303_03964_gb300 import tfdp

    assert torch.cuda.is_available()
    rng = np.random.default_rng(77)
    cases = []
    for n, half in ((3001, 15.0), (1203, 9.0)):  # second call: smaller n, same scratch
        e = synth.erdos_renyi(n, 2 * n, rng)
        xy = rng.uniform(-half, half, size=(n, 2)).astype(np.float32)
        cases.append((n, e, xy))
    for n, e, xy in cases:
        p = tfdp.params_default(rep_mode=tfdp.REP_EXACT)
        with tfdp.Graph(n, e, xy, p) as g:
            ref, _ = g.eval_forces()
        xy_d = torch.from_numpy(xy).cuda()
        out = torch.full_like(xy_d, float("nan"))
        tfdp.exact_repulsion_noalloc(xy_d, out, gamma=2.0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= FORCE_TOL
        assert _rel(got, oracle.rep_exact(xy.astype(np.float64), 2.0)) <= FORCE_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2303_03964_gb300 import tfdp

    n = tfdp.NOALLOC_MAX_N + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    out = torch.empty_like(xy)
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.exact_repulsion_noalloc(xy, out)
    assert ei.value.status == 3
