"""Layout-quality metrics (Sec. 4, "Metrics") against layouts whose values follow from
the definitions by hand. CPU only."""
import math

import numpy as np
import pytest

from paper_2303_03964_gb300 import quality as q
from paper_2303_03964_gb300 import synth

pytest.importorskip("scipy")


def _grid(nx, ny):
    return np.stack(np.meshgrid(np.arange(nx), np.arange(ny)), -1).reshape(-1, 2).astype(float)


def test_unit_square_cycle():
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    e = np.array([[0, 1], [1, 2], [2, 3], [3, 0]])
    # four sides: d = 1, |x| = 1; two diagonals: d = 2, |x| = sqrt 2. With a = |x| / d the
    # optimal scale is s = sum a / sum a^2 = (4 + sqrt 2) / 5 and SE = mean (s a - 1)^2.
    s = (4 + math.sqrt(2)) / 5
    se = (4 * (s - 1) ** 2 + 2 * (s * math.sqrt(2) / 2 - 1) ** 2) / 6
    assert q.stress_error(xy, e) == pytest.approx(se, rel=1e-12)
    assert q.neighbourhood_preservation(xy, e, 1) == 1.0
    assert q.crosslessness(xy, e) == 1.0
    # every corner has two edges at 90 degrees: theta = pi, theta_min = pi/2
    assert q.minimum_angle(xy, e) == pytest.approx(0.5)


def test_path_on_a_line_is_perfect():
    e = np.array([[i, i + 1] for i in range(9)])
    xy = np.stack([np.arange(10.0) * 2.5, np.zeros(10)], 1)  # any scale
    assert q.stress_error(xy, e) == pytest.approx(0.0, abs=1e-24)
    assert q.neighbourhood_preservation(xy, e, 1) == 1.0


def test_lattice_on_its_grid():
    nx, ny = 6, 5
    e = synth.lattice(nx, ny)
    xy = _grid(nx, ny)
    # 1-ring: the axis neighbours at distance 1; 2-ring: those, the diagonals (sqrt 2) and
    # the second axis neighbours (2) -- exactly the nearest layout points in both cases
    assert q.neighbourhood_preservation(xy, e, 1) == 1.0
    assert q.neighbourhood_preservation(xy, e, 2) == 1.0
    assert q.crosslessness(xy, e) == 1.0
    # interior (degree 4): perfect; border (degree 3): |120 - 90| / 120; corner: 0.5
    interior, corners = (nx - 2) * (ny - 2), 4
    border = nx * ny - interior - corners
    assert q.minimum_angle(xy, e) == pytest.approx(1 - (border * 0.25 + corners * 0.5) / (nx * ny))


def test_crossing_counts():
    # two crossing edges that share no node: c = c_max = 1
    xy = np.array([[0, 0], [1, 1], [0, 1], [1, 0]], float)
    assert q.crosslessness(xy, np.array([[0, 1], [2, 3]])) == 0.0
    # a triangle: every pair of edges shares a node, c_max = 0
    assert q.crosslessness(np.array([[0, 0], [1, 0], [0, 1]], float), np.array([[0, 1], [1, 2], [2, 0]])) == 1.0
    # K4 drawn as a square with both diagonals: 1 crossing; of its 15 edge pairs, 12 share
    # a node (4 nodes of degree 3 give 3 pairs each), so c_max = 3
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    k4 = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [0, 2], [1, 3]])
    assert q.crosslessness(xy, k4) == pytest.approx(1 - math.sqrt(1 / 3))


def test_np_detects_a_scrambled_layout():
    e = synth.lattice(10, 10)
    xy = _grid(10, 10)
    rng = np.random.default_rng(0)
    assert q.neighbourhood_preservation(rng.permutation(xy), e, 1) < 0.2


def test_stress_sampled_sources_match_full_on_all_sources():
    rng = np.random.default_rng(1)
    e = synth.erdos_renyi(60, 150, rng)
    xy = rng.normal(size=(60, 2))
    full = q.stress_error(xy, e)
    # every ordered pair from all sources counts each unordered pair twice, same ratios
    assert q.stress_error(xy, e, sources=np.arange(60)) == pytest.approx(full, rel=1e-12)


def test_relative_value():
    assert q.relative(0.9, 1.0) == pytest.approx(-0.1)
