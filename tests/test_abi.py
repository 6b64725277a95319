"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/tfdp.h declares, and its host-side validation behaves as documented.
No call here launches a kernel."""
import os
import re

import numpy as np
import pytest

from paper_2303_03964_gb300 import tfdp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tfdp_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert len(names) >= 15
    out = os.popen("nm -D --defined-only %s" % tfdp.LIB_PATH).read()
    exported = set(re.findall(r" T (tfdp_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(tfdp.lib, n)


def test_params_default_values_are_the_papers():
    p = tfdp.params_default()
    assert (p.alpha, p.beta, p.gamma) == (0.1, 8.0, 2.0)
    assert p.k_interp == 3 and p.n_int_min == 50
    assert tfdp.params_check(p) is True  # alpha (1 + beta) = 0.9 < 1


@pytest.mark.parametrize("field,value,status", [
    ("gamma", 1.0, 3), ("gamma", 0.5, 3), ("alpha", -0.1, 3), ("beta", -1.0, 3),
    ("k_interp", -1, 3), ("k_interp", 4, 3), ("grid_max", 2, 3), ("total_iters", 0, 3),
    ("step_min", 0.0, 3), ("grid_policy", 7, 1), ("rep_mode", 5, 1), ("grid_max", 1 << 20, 3),
])
def test_params_range_rejected(field, value, status):
    p = tfdp.params_default(**{field: value})
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.params_check(p)
    assert ei.value.status == status


def test_dynamic_k_accepted_and_sized_for_every_k():
    # Sec. 3.4 "Choices of k": k_interp = 0 runs k = 1, 2, 3 in turn with one N_int for
    # every k (capped at floor(grid_max / 3)), so the buffers hold the k = 3 grid and
    # (grid_max / 3)^2 boxes: as much as a fixed k = 3, less than a fixed k = 1 whose
    # N_int may reach grid_max
    p = tfdp.params_default(k_interp=tfdp.K_DYNAMIC, grid_max=1023)
    assert tfdp.params_check(p) is True
    dyn = tfdp.graph_footprint(100_000, 200_000, p)
    k1 = tfdp.graph_footprint(100_000, 200_000, tfdp.params_default(k_interp=1, grid_max=1023))
    k3 = tfdp.graph_footprint(100_000, 200_000, tfdp.params_default(k_interp=3, grid_max=1023))
    assert k3 <= dyn < k1
    # the dynamic schedule needs room for k = 3 boxes: grid_max >= 3
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.params_check(tfdp.params_default(k_interp=tfdp.K_DYNAMIC, grid_max=2))
    assert ei.value.status == 3


def test_soft_weight_condition_is_flagged_not_rejected():
    # Sec. 3.3 shows alpha = 0.5 with beta = 8, which breaks alpha (1 + beta) < 1
    assert tfdp.params_check(tfdp.params_default(alpha=0.5)) is False


@pytest.mark.parametrize("edges", [
    [[0, 1], [1, 1]],          # self-loop
    [[0, 1], [1, 0]],          # duplicate in the other order
    [[0, 1], [0, 1]],          # duplicate
    [[0, 3]],                  # out of range
    [[-1, 2]],                 # negative id
])
def test_bad_graph_rejected_before_any_device_work(edges):
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.Graph(3, edges, np.zeros((3, 2), np.float32))
    assert ei.value.status == 2


def test_status_strings():
    for code, name in tfdp.STATUS.items():
        assert tfdp.lib.tfdp_status_str(code).decode() == name


@pytest.mark.parametrize("xy,frep", [(0x1001, 0x2000), (0x1000, 0x2004), (0x1002, 0x2006)])
def test_noalloc_rejects_misaligned_pointers_before_any_launch(xy, frep):
    # the kernels read and write float2 pairs: a pointer that is not 8-byte aligned is
    # refused on the host, before any CUDA call (these addresses are never dereferenced)
    st = tfdp.lib.tfdp_exact_repulsion_noalloc(tfdp._p(xy), 10, 2.0, tfdp._p(frep), None)
    assert st == 1


def test_noalloc_rejects_null_and_size_before_any_launch():
    assert tfdp.lib.tfdp_exact_repulsion_noalloc(None, 10, 2.0, tfdp._p(0x2000), None) == 1
    assert tfdp.lib.tfdp_exact_repulsion_noalloc(tfdp._p(0x1000), -1, 2.0, tfdp._p(0x2000), None) == 1
    big = tfdp.NOALLOC_MAX_N + 1
    assert tfdp.lib.tfdp_exact_repulsion_noalloc(tfdp._p(0x1000), big, 2.0, tfdp._p(0x2000), None) == 3
    assert tfdp.lib.tfdp_exact_repulsion_noalloc(tfdp._p(0x1000), 10, 1.0, tfdp._p(0x2000), None) == 3


def test_bf16x3_precision_mode_accepted_only_at_its_fft_size():
    # the tensor-core column stage is built for P = 2048 (grid_max 513 .. 1024)
    assert tfdp.params_check(tfdp.params_default(precision=tfdp.PREC_BF16X3, grid_max=1023)) is True
    for gm in (255, 511, 2047):
        with pytest.raises(tfdp.TfdpError) as ei:
            tfdp.params_check(tfdp.params_default(precision=tfdp.PREC_BF16X3, grid_max=gm))
        assert ei.value.status == 3
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.params_check(tfdp.params_default(precision=7))
    assert ei.value.status == 1
    # the exact path has no grid convolution: the mode is accepted and changes nothing
    assert tfdp.params_check(tfdp.params_default(precision=tfdp.PREC_BF16X3, rep_mode=tfdp.REP_EXACT,
                                                 grid_max=255)) is True


@pytest.mark.parametrize("grid_max,n_exact,n_fft", [(255, 9000, 10000), (1023, 13000, 14000)])
def test_auto_mode_resolves_by_graph_size(grid_max, n_exact, n_fft):
    # AUTO takes the exact sum while its estimated iteration (9 us + n^2 / 3e12 s) is no
    # longer than the FFT path's (40 us at P <= 512, + 15 us per doubling of P); the
    # footprint is sized for the resolved mode
    auto = tfdp.params_default(rep_mode=tfdp.REP_AUTO, grid_max=grid_max)
    assert tfdp.params_check(auto) is True
    for n, want in ((n_exact, tfdp.REP_EXACT), (n_fft, tfdp.REP_FFT)):
        other = tfdp.REP_FFT if want == tfdp.REP_EXACT else tfdp.REP_EXACT
        fp = tfdp.graph_footprint(n, 4 * n, auto)
        assert fp == tfdp.graph_footprint(n, 4 * n, tfdp.params_default(rep_mode=want, grid_max=grid_max))
        assert fp != tfdp.graph_footprint(n, 4 * n, tfdp.params_default(rep_mode=other, grid_max=grid_max))


def test_auto_mode_is_checked_as_fft():
    # AUTO may resolve to the FFT path, so its FFT-only limits apply
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.params_check(tfdp.params_default(rep_mode=tfdp.REP_AUTO, precision=tfdp.PREC_BF16X3, grid_max=255))
    assert ei.value.status == 3
    assert tfdp.params_check(tfdp.params_default(rep_mode=tfdp.REP_AUTO, precision=tfdp.PREC_BF16X3,
                                                 grid_max=1023)) is True
    with pytest.raises(tfdp.TfdpError) as ei:
        tfdp.params_check(tfdp.params_default(rep_mode=3))
    assert ei.value.status == 1
