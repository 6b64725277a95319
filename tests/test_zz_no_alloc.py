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


@pytest.mark.parametrize("gamma", [1.5, 2.0, 3.2, 4.0, 8.0])
@pytest.mark.parametrize("n", [11, 777])
def test_noalloc_every_gamma_branch_against_oracle(gamma, n):
    # gamma 2, 4, 8 take the squaring branch; 1.5 and 3.2 the general exp2/log2 one.
    # n = 11 leaves most of the 16 source chunks empty.
    import torch
    from paper_2303_03964_gb300 import tfdp

    rng = np.random.default_rng(1000 + n)
    xy = rng.uniform(-0.4 * np.sqrt(n), 0.4 * np.sqrt(n), size=(n, 2)).astype(np.float32)
    xy_d = torch.from_numpy(xy).cuda()
    out = torch.full_like(xy_d, float("nan"))
    tfdp.exact_repulsion_noalloc(xy_d, out, gamma=gamma)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert _rel(got, oracle.rep_exact(xy.astype(np.float64), gamma)) <= FORCE_TOL


def test_noalloc_rejects_tensors_the_kernels_cannot_read():
    import torch
    from paper_2303_03964_gb300 import tfdp

    xy = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        tfdp.exact_repulsion_noalloc(xy.double(), torch.empty_like(xy).double())
    with pytest.raises(ValueError):
        tfdp.exact_repulsion_noalloc(xy, torch.empty((32, 2), dtype=torch.float32, device="cuda"))
    # an odd float offset is not 8-byte aligned: the library refuses it before launching
    flat = torch.zeros(2 * 64 + 1, dtype=torch.float32, device="cuda")
    st = tfdp.lib.tfdp_exact_repulsion_noalloc(tfdp._p(flat.data_ptr() + 4), 64, 2.0,
                                               tfdp._p(xy.data_ptr()), None)
    assert st == 1
    # host memory is refused too
    host = np.zeros((64, 2), np.float32)
    st = tfdp.lib.tfdp_exact_repulsion_noalloc(host.ctypes.data_as(tfdp._p), 64, 2.0,
                                               tfdp._p(xy.data_ptr()), None)
    assert st == 1


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2303_03964_gb300 import tfdp

    n = tfdp.NOALLOC_MAX_N + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    out = torch.empty_like(xy)
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.exact_repulsion_noalloc(xy, out)
    assert ei.value.status == 3
