"""Pins for the FP64 CPU oracle: each test checks the oracle against something other
than itself -- closed forms, values the paper prints, invariants, a library routine,
or brute force on tiny inputs. CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2303_03964_gb300 import synth


@pytest.fixture(scope="module")
def paper(golden_dir):
    with open(os.path.join(golden_dir, "paper_values.json")) as f:
        return json.load(f)


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    e = synth.erdos_renyi(n, m, rng)
    xy = rng.uniform(-2.0, 2.0, size=(n, 2))
    return e, xy


def _equilibrium_distance(alpha, beta, gamma):
    """Two connected nodes balance where (1+d^2)^-gamma = alpha (1 + beta/(1+d^2)),
    i.e. alpha u^gamma + alpha beta u^(gamma-1) - 1 = 0 with u = 1 + d^2 (u > 1)."""
    lo, hi = 1.0, 1.0
    while alpha * hi ** gamma + alpha * beta * hi ** (gamma - 1) - 1.0 < 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if alpha * mid ** gamma + alpha * beta * mid ** (gamma - 1) - 1.0 < 0:
            lo = mid
        else:
            hi = mid
    return math.sqrt(0.5 * (lo + hi) - 1.0)


# ---------------------------------------------------------------- t-force (Sec. 3.2)

def test_tforce_shape_matches_paper(paper):
    spec = paper["tforce_shape"]
    d = np.linspace(0.0, 3.0, 30001)
    for phi in spec["phis"]:
        f = np.array([oracle.tforce(x, phi) for x in d])
        j = int(np.argmax(f))
        assert f[j] < spec["max_below"]
        assert spec["argmax_in"][0] <= d[j] <= spec["argmax_in"][1]
        # calculus: f'(d) = 0 at d = 1/sqrt(2 phi - 1)
        dmax = 1.0 / math.sqrt(2 * phi - 1)
        assert abs(d[j] - dmax) < 2e-4
        fmax = dmax / (1 + dmax * dmax) ** phi
        assert abs(f[j] - fmax) < 1e-8
    # gamma = 2: f_max = (1/sqrt 3) (3/4)^2
    assert abs(oracle.tforce(1 / math.sqrt(3), 2.0) - 0.3247595264191645) < 1e-15


def test_tforce_requirements_R2_R3():
    for phi in (1.0, 2.0, 4.0):
        # R3: f(d) ~ d as d -> 0
        assert abs(oracle.tforce(1e-6, phi) / 1e-6 - 1.0) < 1e-9
        # R2: f(d) ~ d^-(2 phi - 1) as d -> inf
        d = 1e4
        assert abs(oracle.tforce(d, phi) * d ** (2 * phi - 1) - 1.0) < 1e-6


# ------------------------------------------------------- exact forces (Sec. 3.3)

def test_exact_two_nodes_direction_and_magnitude():
    for gamma in (2.0, 3.5):
        xy = np.array([[0.3, -0.2], [1.1, 0.4]])
        f = oracle.rep_exact(xy, gamma)
        dvec = xy[0] - xy[1]
        d = np.linalg.norm(dvec)
        # node 0 is pushed away from node 1 with the t-force magnitude
        np.testing.assert_allclose(f[0], oracle.tforce(d, gamma) * dvec / d, rtol=1e-14)
        np.testing.assert_allclose(f[1], -f[0], rtol=1e-14)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("gamma", [2.0, 3.3])
def test_exact_rows_are_the_rows_of_the_full_sum(weighted, gamma):
    """The row-sampled exact sum (used against the GPU at full size) must give, for every
    listed target, the row of the full sum of Eq. (repfK): shuffled, repeated, first and
    last rows, with and without local-refinement weights (reading R13)."""
    rng = np.random.default_rng(41)
    n = 301
    xy = rng.uniform(-6.0, 6.0, size=(n, 2))
    w = rng.uniform(0.25, 4.0, size=n) if weighted else None
    full = oracle.rep_exact(xy, gamma, w=w)
    rows = np.concatenate([rng.permutation(n)[:120], [0, n - 1, 7, 7, 7, 0]])
    got = oracle.rep_exact(xy, gamma, rows=rows, w=w)
    assert got.shape == (rows.shape[0], 2)
    assert np.array_equal(got, full[rows])
    # two nodes: the closed form of the t-force on the listed row alone
    two = np.array([[0.3, -0.2], [1.1, 0.4]])
    f1 = oracle.rep_exact(two, gamma, rows=[1])[0]
    dvec = two[1] - two[0]
    d = np.linalg.norm(dvec)
    np.testing.assert_allclose(f1, oracle.tforce(d, gamma) * dvec / d, rtol=1e-14)


@pytest.mark.parametrize("gamma", [2.0, 2.7, 4.0])
def test_forces_are_minus_energy_gradient(gamma):
    """Central finite differences of an energy written independently of the forces."""
    e, xy = _random_graph(7, 9, 11)
    alpha, beta = 0.1, 8.0
    D = oracle.rep_exact(xy, gamma) + oracle.attraction(e, xy, alpha, beta)
    h = 1e-5
    g = np.zeros_like(xy)
    for i in range(xy.shape[0]):
        for c in range(2):
            xp = xy.copy(); xp[i, c] += h
            xm = xy.copy(); xm[i, c] -= h
            g[i, c] = (oracle.energy(xp, e, alpha, beta, gamma)
                       - oracle.energy(xm, e, alpha, beta, gamma)) / (2 * h)
    np.testing.assert_allclose(D, -g, rtol=1e-7, atol=1e-9)


def test_pairwise_antisymmetry_net_force_zero():
    e, xy = _random_graph(200, 600, 3)
    fr = oracle.rep_exact(xy, 2.0)
    fa = oracle.attraction(e, xy, 0.1, 8.0)
    assert np.abs(fr.sum(0)).max() < 1e-12 * np.abs(fr).sum()
    assert np.abs(fa.sum(0)).max() < 1e-12 * np.abs(fa).sum()


def test_translation_rotation_permutation():
    e, xy = _random_graph(60, 150, 5)
    fr = oracle.rep_exact(xy, 2.0)
    fa = oracle.attraction(e, xy, 0.1, 8.0)
    # translation invariance
    c = np.array([37.25, -11.5])
    np.testing.assert_allclose(oracle.rep_exact(xy + c, 2.0), fr, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(oracle.attraction(e, xy + c, 0.1, 8.0), fa, rtol=1e-10,
                               atol=1e-12)
    # rotation equivariance (a swapped or mis-signed coordinate fails this)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    np.testing.assert_allclose(oracle.rep_exact(xy @ R.T, 2.0), fr @ R.T, rtol=1e-10,
                               atol=1e-12)
    np.testing.assert_allclose(oracle.attraction(e, xy @ R.T, 0.1, 8.0), fa @ R.T,
                               rtol=1e-10, atol=1e-12)
    # node permutation equivariance
    p = np.random.default_rng(1).permutation(60)
    inv = np.argsort(p)
    e2 = inv[e]
    np.testing.assert_allclose(oracle.rep_exact(xy[p], 2.0), fr[p], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle.attraction(e2, xy[p], 0.1, 8.0), fa[p], rtol=1e-12,
                               atol=1e-14)


def test_kernel_bounded_at_zero_distance():
    # coincident nodes: K = 1 but the pair force is 0 (f(0) = 0, R3)
    xy = np.array([[1.0, 1.0], [1.0, 1.0], [2.0, 1.0]])
    f = oracle.rep_exact(xy, 2.0)
    np.testing.assert_allclose(f[0], f[1])
    np.testing.assert_allclose(f[0], [-0.25, 0.0])  # only the third node acts: 1/(1+1)^2
    # |K (x_i - x_j)| never exceeds the t-force maximum
    rng = np.random.default_rng(2)
    for _ in range(20):
        xy = rng.normal(size=(2, 2)) * rng.uniform(0.01, 3)
        assert np.linalg.norm(oracle.rep_exact(xy, 2.0)[0]) <= 0.3247595264191645 + 1e-15


def test_limit_ratio_alpha_one_plus_beta(paper):
    """Eq. (limitweight): for two connected nodes, |F^a|/|F^r| -> alpha (1 + beta) as d -> 0."""
    alpha, beta = paper["defaults"]["alpha"], paper["defaults"]["beta"]
    xy = np.array([[0.0, 0.0], [1e-5, 0.0]])
    e = np.array([[0, 1]])
    ratio = (np.linalg.norm(oracle.attraction(e, xy, alpha, beta)[0])
             / np.linalg.norm(oracle.rep_exact(xy, 2.0)[0]))
    assert abs(ratio - alpha * (1 + beta)) < 1e-8
    assert alpha * (1 + beta) < paper["weight_condition"]["bound"]


@pytest.mark.parametrize("gamma", [2.0, 4.0, 8.0])
def test_two_connected_nodes_converge_to_closed_form(paper, gamma):
    alpha, beta = paper["defaults"]["alpha"], paper["defaults"]["beta"]
    dstar = _equilibrium_distance(alpha, beta, gamma)
    if gamma == 2.0:
        # quadratic alpha u^2 + alpha beta u - 1 = 0
        u = (-alpha * beta + math.sqrt((alpha * beta) ** 2 + 4 * alpha)) / (2 * alpha)
        assert abs(dstar - math.sqrt(u - 1)) < 1e-12
        assert abs(dstar - 0.3146737) < 1e-7
    xy = oracle.iterate(np.array([[0.0, 0.0], [1.3, 0.4]]), np.array([[0, 1]]), 300,
                        alpha=alpha, beta=beta, gamma=gamma, mode="exact", T=300)
    assert abs(np.linalg.norm(xy[0] - xy[1]) - dstar) < 1e-9


def test_connected_triangle_converges_to_equilateral(paper):
    alpha, beta, gamma = 0.1, 8.0, 2.0
    dstar = _equilibrium_distance(alpha, beta, gamma)
    xy0 = np.array([[0.0, 0.0], [1.0, 0.0], [0.3, 0.8]])
    e = np.array([[0, 1], [1, 2], [0, 2]])
    xy = oracle.iterate(xy0, e, 300, alpha=alpha, beta=beta, gamma=gamma, mode="exact", T=300)
    for a, b in e:
        assert abs(np.linalg.norm(xy[a] - xy[b]) - dstar) < 1e-7


# -------------------------------------------------- update schedule (reading)

def test_step_schedule_and_cap():
    T, s0, smin = 300, 1.0, 0.01
    s = np.array([oracle.step_size(t, T, s0, smin) for t in range(T)])
    assert s[0] == s0 and abs(s[-1] - smin) < 1e-15
    r = s[1:] / s[:-1]
    assert np.allclose(r, r[0], rtol=1e-12)
    xy = np.zeros((3, 2))
    D = np.array([[3.0, 4.0], [0.03, 0.04], [0.0, 0.0]])
    out = oracle.update(xy, D, 0.5)
    np.testing.assert_allclose(out, [[0.3, 0.4], [0.03, 0.04], [0.0, 0.0]], rtol=1e-15)


# ------------------------------------------- interpolation and FFT (Sec. 3.4)

@pytest.mark.parametrize("k", [1, 2, 3])
def test_lagrange_basis_properties(k):
    nodes = (np.arange(k) + 0.5) / k
    for u in np.linspace(-0.1, 1.1, 25):
        w = oracle.lagrange(k, u)
        for p in range(k):  # reproduces every polynomial of degree < k
            assert abs(np.dot(w, nodes ** p) - u ** p) < 1e-13
    for l in range(k):
        np.testing.assert_allclose(oracle.lagrange(k, nodes[l]), np.eye(k)[l], atol=1e-15)


def test_own_fft_matches_library():
    rng = np.random.default_rng(4)
    for N in (1, 2, 4, 8, 64, 1024):
        z = rng.normal(size=N) + 1j * rng.normal(size=N)
        np.testing.assert_allclose(oracle.fft(z), np.fft.fft(z), rtol=1e-12, atol=1e-11)
        np.testing.assert_allclose(oracle.fft(z, inverse=True), np.fft.ifft(z) * N,
                                   rtol=1e-12, atol=1e-11)
    z = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
    np.testing.assert_allclose(oracle.fft(z), np.fft.fft2(z), rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("G", [1, 2, 5, 8])
def test_fft_grid_interaction_equals_direct_sum(G):
    rng = np.random.default_rng(G)
    ch = rng.normal(size=(3, G, G))
    for gamma in (2.0, 3.3):
        d = oracle.conv_grid(ch, 0.37, gamma, direct=True)
        for P in (None, 64):
            f = oracle.conv_grid(ch, 0.37, gamma, P=P)
            np.testing.assert_allclose(f, d, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_ibfft_exact_when_nodes_sit_on_grid_nodes(k):
    """One-hot interpolation: the ibFFT sum reduces to the exact sum of Eq. (repfK)."""
    lo, h, n_int = -3.0, 0.75, 8
    G = n_int * k
    rng = np.random.default_rng(7)
    q = rng.choice(G * G, size=45, replace=False)
    qy, qx = q // G, q % G
    xy = np.stack([lo + (qx + 0.5) * h / k, lo + (qy + 0.5) * h / k], axis=1)
    for gamma in (2.0, 2.5):
        approx = oracle.rep_fft(xy, gamma, k, grid={"lo": lo, "h": h, "n_int": n_int})
        exact = oracle.rep_exact(xy, gamma)
        np.testing.assert_allclose(approx, exact, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_ibfft_net_force_zero_and_translation(k):
    rng = np.random.default_rng(8)
    # positions on a 2^-10 lattice: exact in FP32, so shifts by 16 stay exact
    xy = np.round(rng.uniform(-20, 20, size=(500, 2)) * 1024) / 1024
    f = oracle.rep_fft(xy, 2.0, k)
    assert np.abs(f.sum(0)).max() < 1e-11 * np.abs(f).sum()
    f2 = oracle.rep_fft(xy + 16.0, 2.0, k)
    np.testing.assert_allclose(f2, f, rtol=1e-9, atol=1e-11)


def test_ibfft_converges_to_exact_as_boxes_shrink():
    rng = np.random.default_rng(9)
    xy = rng.uniform(-4, 4, size=(300, 2))
    exact = oracle.rep_exact(xy, 2.0)
    errs = {}
    for k in (1, 3):
        for n_int in (8, 16, 32):
            lo = xy.min() - 1e-9
            L = xy.max() - lo + 1e-9
            f = oracle.rep_fft(xy, 2.0, k, grid={"lo": lo, "h": L / n_int, "n_int": n_int})
            errs[k, n_int] = np.linalg.norm(f - exact) / np.linalg.norm(exact)
    for k in (1, 3):
        assert errs[k, 8] > errs[k, 16] > errs[k, 32]
    # degree-(k-1) interpolation: error falls about like h^k
    assert errs[3, 16] / errs[3, 32] > 4.0
    assert errs[3, 32] < errs[1, 32]
    assert errs[3, 32] < 1e-3


# ------------------------------------------------------ grid policy (Sec. 3.4)

def _pts(lo, hi):
    return np.array([[lo, lo], [hi, hi]], dtype=np.float32)


def test_grid_rule_n_int(paper):
    nmin = paper["interpolation"]["n_int_min"]
    g = oracle.grid_policy(_pts(0, 30), 3, nmin, policy=oracle.GRID_PAPER)
    assert g["n_int"] == 50 and abs(g["h"] - 30 / 50) < 1e-15
    g = oracle.grid_policy(_pts(-60.0, 60.25), 3, nmin, policy=oracle.GRID_PAPER)
    assert g["n_int"] == 121 and abs(g["h"] - 120.25 / 121) < 1e-15
    g = oracle.grid_policy(_pts(-500, 500), 3, nmin, grid_max=1023, policy=oracle.GRID_PAPER)
    assert g["n_int"] == 341 and g["G"] == 1023
    g = oracle.grid_policy(_pts(-50, 50), 3, nmin, grid_max=255, policy=oracle.GRID_PAPER)
    assert g["n_int"] == 85 and g["G"] == 255


def test_grid_snap_h_policy():
    rng = np.random.default_rng(10)
    for _ in range(200):
        L = float(np.float32(rng.uniform(0.5, 3000)))
        g = oracle.grid_policy(_pts(0.0, L), 3, 50, grid_max=1023, policy=oracle.GRID_SNAP_H)
        h, n_int = g["h"], g["n_int"]
        m, e = math.frexp(h)  # h = m 2^e, m in [0.5, 1): 16 m 2 must be an integer in 16..31
        j = m * 32
        assert j == int(j) and 16 <= j <= 31
        assert n_int * h >= g["L"]
        prev = (j - 1) / 32 * 2 ** e if j > 16 else 31 / 32 * 2 ** (e - 1)
        assert n_int * prev < g["L"]
        if 50 <= L <= 341:
            assert h == 1.0


def test_box_decision_clamps():
    assert oracle.box_f32(10.0, 0.0, 1.0, 10) == 9  # x_max goes to the last box
    assert oracle.box_f32(0.0, 0.0, 1.0, 10) == 0
    assert oracle.box_f32(3.9999, 0.0, 1.0, 10) == 3


@pytest.mark.parametrize("k", [1, 2, 3])
def test_ibfft_equals_explicit_interpolated_kernel_matrix(k):
    """Brute force on a tiny input: build the interpolated kernel
    Kt_ij = sum_{p,q} w_ip K(y_p - y_q) w_jq explicitly (no grid arrays, no FFT) and
    form sum_j Kt_ij (x_i - x_j); the oracle's spread / FFT / gather route must agree."""
    rng = np.random.default_rng(20 + k)
    n, n_int, lo, h = 25, 4, -1.0, 0.5
    xy = rng.uniform(lo, lo + n_int * h, size=(n, 2))
    gamma = 2.0
    G = n_int * k
    nodes = lo + (np.arange(G) + 0.5) * h / k  # grid node coordinates along one axis
    W = np.zeros((n, G * G))
    for i in range(n):
        a = [min(int(np.floor((xy[i, c] - lo) / h)), n_int - 1) for c in range(2)]
        wx = np.zeros(G)
        wy = np.zeros(G)
        for c, w in ((0, wx), (1, wy)):
            u = (xy[i, c] - lo) / h - a[c]
            for l in range(k):  # Lagrange basis written out from its definition
                v = 1.0
                for q in range(k):
                    if q != l:
                        v *= (u - (q + 0.5) / k) / ((l + 0.5) / k - (q + 0.5) / k)
                w[a[c] * k + l] = v
        W[i] = np.outer(wy, wx).reshape(-1)
    gy, gx = np.meshgrid(nodes, nodes, indexing="ij")
    P = np.stack([gx.reshape(-1), gy.reshape(-1)], axis=1)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    Kt = W @ (1.0 + d2) ** (-gamma) @ W.T
    brute = (Kt.sum(1)[:, None] * xy) - Kt @ xy
    got = oracle.rep_fft(xy, gamma, k, grid={"lo": lo, "h": h, "n_int": n_int})
    np.testing.assert_allclose(got, brute, rtol=1e-10, atol=1e-12)


def test_dynamic_k_schedule_counts(paper):
    """Sec. 3.4 "Choices of k": k = 1 for 90 % of the iterations, 2 for 5 %, 3 for the
    rest; Sec. 4.2 prints the count of single-point iterations of a 300-iteration run."""
    d, it = paper["dynamic_k"], paper["dynamic_k_iterations"]
    T = it["T"]
    ks = [oracle.k_of_iter(0, t, T) for t in range(T)]
    assert ks.count(1) == it["k1_iterations"]
    counts = [ks.count(k) for k in d["k"]]
    assert counts == [round(f * T) for f in d["fractions"]]
    assert ks == sorted(ks)                      # 1s, then 2s, then 3s
    assert oracle.k_of_iter(0, T + 5, T) == 3    # past the schedule: the last k
    assert all(oracle.k_of_iter(k, t, T) == k for k in (1, 2, 3) for t in (0, T - 1))


def test_dynamic_k_iteration_is_the_fixed_k_segments():
    """A dynamic-k run equals fixed-k runs chained at the schedule's boundaries (T = 20:
    k = 1 for t < 18, k = 2 at t = 18, k = 3 at t = 19). The paper's N_int rule does not
    depend on k (Sec. 3.4 "Choices of k"), so under the dynamic strategy N_int has one
    cap, floor(grid_max / 3), and the fixed-k segment of order k runs with a cap of
    k * floor(grid_max / 3) on G (reading R9b)."""
    e, xy = _random_graph(60, 150, 7)
    xy = xy * 6.0
    kw = dict(mode="fft", n_int_min=4, T=20, alpha=0.1, beta=8.0, gamma=2.0)
    gm = 30
    L = float(np.float32(xy).max() - np.float32(xy).min())
    assert L > gm // 3  # the common cap binds, so the rule is visible
    dyn = oracle.iterate(xy, e, 20, k=0, grid_max=gm, **kw)
    x = oracle.iterate(xy, e, 18, k=1, t0=0, grid_max=1 * (gm // 3), **kw)
    x = oracle.iterate(x, e, 1, k=2, t0=18, grid_max=2 * (gm // 3), **kw)
    x = oracle.iterate(x, e, 1, k=3, t0=19, grid_max=3 * (gm // 3), **kw)
    assert np.array_equal(dyn, x)
    # and differs from a fixed-k run, so the switch is not a no-op
    assert not np.array_equal(dyn, oracle.iterate(xy, e, 20, k=3, grid_max=gm, **kw))
    # a cap of floor(grid_max / k) per k (the k = 1 grid as wide as the k = 3 grid) is
    # another run
    y = oracle.iterate(xy, e, 18, k=1, t0=0, grid_max=gm, **kw)
    y = oracle.iterate(y, e, 1, k=2, t0=18, grid_max=gm, **kw)
    y = oracle.iterate(y, e, 1, k=3, t0=19, grid_max=gm, **kw)
    assert not np.array_equal(dyn, y)
    # one N_int for every k: the k = 1 grid is a third of the k = 3 grid per axis
    g1 = oracle.grid_policy(np.float32(xy), 1, 4, 1 * (gm // 3))
    g3 = oracle.grid_policy(np.float32(xy), 3, 4, 3 * (gm // 3))
    assert g1["n_int"] == g3["n_int"] == gm // 3 and g3["G"] == 3 * g1["G"]


# ------------------------------------------------------------------ local refinement
# Sec. 5 "Local Refinement" gives no formula; the reading is per-node weights with the
# pair repulsion scaled by r_i r_j and the edge attraction by a_i a_j.

def _weights(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 3.0, n)


def test_unit_weights_are_the_plain_method():
    e, xy = _random_graph(40, 90, 31)
    one = np.ones(40)
    assert np.array_equal(oracle.rep_exact(xy, 2.0, w=one), oracle.rep_exact(xy, 2.0))
    assert np.array_equal(oracle.attraction(e, xy, 0.1, 8.0, w=one), oracle.attraction(e, xy, 0.1, 8.0))
    assert np.array_equal(oracle.rep_fft(xy, 2.0, 3, w=one, n_int_min=4), oracle.rep_fft(xy, 2.0, 3, n_int_min=4))


def test_weighted_forces_are_minus_grad_of_weighted_energy():
    e, xy = _random_graph(12, 25, 32)
    wr, wa = _weights(12, 33)
    D = oracle.rep_exact(xy, 3.0, w=wr) + oracle.attraction(e, xy, 0.2, 5.0, w=wa)
    g = np.zeros_like(xy)
    eps = 1e-6
    for i in range(12):
        for c in range(2):
            p, q = xy.copy(), xy.copy()
            p[i, c] += eps
            q[i, c] -= eps
            g[i, c] = (oracle.energy(p, e, 0.2, 5.0, 3.0, wr=wr, wa=wa)
                       - oracle.energy(q, e, 0.2, 5.0, 3.0, wr=wr, wa=wa)) / (2 * eps)
    assert np.linalg.norm(D + g) <= 1e-7 * np.linalg.norm(D)


def test_weighted_forces_are_antisymmetric():
    e, xy = _random_graph(50, 120, 34)
    wr, wa = _weights(50, 35)
    fr = oracle.rep_exact(xy, 2.0, w=wr)
    fa = oracle.attraction(e, xy, 0.1, 8.0, w=wa)
    assert np.abs(fr.sum(0)).max() <= 1e-12 * np.abs(fr).sum()
    assert np.abs(fa.sum(0)).max() <= 1e-12 * np.abs(fa).sum()


@pytest.mark.parametrize("path", ["exact", "fft"])
def test_repulsion_weight_two_is_a_duplicated_node(path):
    """A source of weight 2 acts on every other node like two unit nodes at one point;
    on itself, the force is twice the unit-weight force (both sides linear in r)."""
    rng = np.random.default_rng(36)
    n = 30
    xy = rng.uniform(-6, 6, size=(n, 2))
    w = np.ones(n)
    w[0] = 2.0
    dup = np.vstack([xy, xy[:1]])
    if path == "exact":
        fw = oracle.rep_exact(xy, 2.0, w=w)
        fd = oracle.rep_exact(dup, 2.0)
        f1 = oracle.rep_exact(xy, 2.0)
    else:
        kw = dict(k=3, n_int_min=5)
        fw = oracle.rep_fft(xy, 2.0, w=w, **kw)
        fd = oracle.rep_fft(dup, 2.0, **kw)
        f1 = oracle.rep_fft(xy, 2.0, **kw)
    assert np.allclose(fw[1:], fd[1:n], rtol=0, atol=1e-12 * np.abs(fd).max())
    # node 0 with r_0 = 2: 2 x (sum over unit sources) -- its duplicate adds no force
    assert np.allclose(fw[0], 2.0 * f1[0], rtol=1e-12, atol=1e-14)


def test_weighted_two_node_equilibrium():
    """Two connected nodes balance where r1 r2 (1+d^2)^-gamma = alpha a1 a2 (1 + beta/(1+d^2)),
    i.e. the unweighted equilibrium with alpha' = alpha a1 a2 / (r1 r2)."""
    wr, wa = np.array([1.5, 2.0]), np.array([0.8, 1.25])
    alpha = 0.1 * wa.prod() / wr.prod()
    d_star = _equilibrium_distance(alpha, 8.0, 2.0)
    xy = np.array([[0.0, 0.0], [2.0, 0.5]])
    e = np.array([[0, 1]], np.int32)
    x = oracle.iterate(xy, e, 3000, alpha=0.1, beta=8.0, gamma=2.0, mode="exact", T=3000,
                       s0=0.05, smin=1e-4, wrep=wr, watt=wa)
    assert abs(np.linalg.norm(x[0] - x[1]) - d_star) < 1e-6
