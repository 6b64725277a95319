"""Serving with continuous batching: each job's result is the same alone and in the mix,
admission respects the memory budget, and the iteration is bitwise reproducible."""
import time

import numpy as np
import pytest

from paper_2303_03964_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tfdp():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_03964_gb300 import tfdp as t
    return t


def _jobs(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(2000), np.log(20000)))) // 10 * 10
        if q % 2 == 0:
            e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
        else:
            e = synth.barabasi_albert(n, 2, rng)
        xy = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng)
        updates = []
        for _ in range(2):  # parameters drawn in the paper's ranges, alpha (1 + beta) < 1
            while True:
                a, b = rng.uniform(0.01, 0.5), rng.uniform(8.0, 50.0)
                if a * (1 + b) < 1:
                    break
            updates.append((a, b, float(rng.choice([2.0, 3.0, 4.0]))))
        out.append((n, e, xy, updates))
    return out


def _wait(server, want, timeout=120.0):
    got = {}
    t_end = time.time() + timeout
    while len(got) < want and time.time() < t_end:
        for d in server.poll(64, wait_ms=50):
            got[d["request_id"]] = d
    assert len(got) == want, "requests did not complete"
    return got


def _run(tfdp, jobs, budget, max_active, init_iters=30, upd_iters=10):
    """Submit all jobs at once, then their updates one by one as each request completes."""
    res = {}
    with tfdp.Server(budget, max_active=max_active, chunk_iters=7) as s:
        ids = []
        for (n, e, xy, ups) in jobs:
            job, _ = s.submit(n, e, xy, tfdp.params_default(grid_max=255, total_iters=init_iters), init_iters)
            ids.append(job)
        pending = {job: list(ups) for job, (_, _, _, ups) in zip(ids, jobs)}
        done_jobs = set()
        t_end = time.time() + 180
        while len(done_jobs) < len(ids) and time.time() < t_end:
            for d in s.poll(64, wait_ms=50):
                assert d["status"] == 0
                job = d["job_id"]
                if pending[job]:
                    a, b, g = pending[job].pop(0)
                    s.update(job, tfdp.params_default(alpha=a, beta=b, gamma=g, grid_max=255), upd_iters)
                else:  # last request done: read the layout, free the slot and memory
                    done_jobs.add(job)
                    res[job - ids[0]] = s.positions(job)
                    s.release(job)
        assert len(done_jobs) == len(ids)
        st = s.stats()
    return res, st


def test_iteration_is_bitwise_reproducible(tfdp):
    rng = np.random.default_rng(5)
    e, _ = synth.sbm(8000, 10, 8.0, 0.9, rng)
    xy = synth.uniform_positions(8000, 45.0, rng)
    outs = []
    for _ in range(2):
        with tfdp.Graph(8000, e, xy, tfdp.params_default(grid_max=255)) as g:
            g.iterate(25)
            outs.append(g.get_positions())
    assert np.array_equal(outs[0], outs[1])


def test_results_same_alone_and_in_the_mix(tfdp):
    jobs = _jobs(4, 11)
    big = 64 << 30
    mixed, st = _run(tfdp, jobs, big, max_active=4)
    assert st["peak_active"] >= 2  # jobs really shared the device
    for q in range(len(jobs)):
        alone, _ = _run(tfdp, [jobs[q]], big, max_active=1)
        assert np.array_equal(alone[0], mixed[q]), q
    # and a plain graph driven through the same request sequence
    n, e, xy, ups = jobs[0]
    with tfdp.Graph(n, e, xy, tfdp.params_default(grid_max=255, total_iters=30)) as g:
        g.iterate(30)
        for (a, b, gm) in ups:
            g.set_params(tfdp.params_default(alpha=a, beta=b, gamma=gm, grid_max=255, total_iters=10))
            g.set_iteration(0)
            g.iterate(10)
        assert np.array_equal(g.get_positions(), mixed[0])


def test_admission_by_memory_footprint(tfdp):
    jobs = _jobs(3, 12)
    fp = max(tfdp.graph_footprint(n, e.shape[0], tfdp.params_default(grid_max=255)) for (n, e, _, _) in jobs)
    res, st = _run(tfdp, jobs, int(1.5 * fp), max_active=8)  # room for one job at a time
    assert st["peak_active"] == 1 and len(res) == 3
    with tfdp.Server(fp // 2, max_active=2) as s:
        n, e, xy, _ = jobs[0]
        with pytest.raises(tfdp.TfdpError) as ei:
            s.submit(n, e, xy, tfdp.params_default(grid_max=255), 10)
        assert ei.value.status == 4
