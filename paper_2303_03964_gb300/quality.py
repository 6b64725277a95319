"""Layout-quality metrics of Sec. 4 ("Metrics"), host-side NumPy/SciPy.

These evaluate finished layouts; they are not part of the force computation. The
definitions follow the paper:

* normalized stress error (SE): 2/(n(n-1)) sum_{i<j} (s |x_i - x_j| - d_ij)^2 / d_ij^2 over
  the pairs with a finite graph distance d_ij, with the scale s that minimises it;
* neighbourhood preservation (NP_r): the mean over nodes of the Jaccard index between the
  r-ring graph neighbourhood of i and its k_i nearest layout neighbours, k_i the size of
  that neighbourhood (NP1, NP2 for r = 1, 2);
* crosslessness (CL): 1 - sqrt(c / c_max) with c the number of edge crossings and
  c_max = m(m-1)/2 - sum_i deg(i)(deg(i)-1)/2 (pairs of edges that share no node), 1 when
  c_max = 0;
* minimum angle (MA): 1 - mean_i |theta(i) - theta_min(i)| / theta(i), theta(i) = 2 pi / deg(i),
  over nodes of degree >= 2 (a node of degree 1 has no angle);
* relative value of a metric between a source and a target layout:
  (M(source) - M(target)) / M(target).
"""
import numpy as np


def _csr(n, edges):
    import scipy.sparse as sp
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    data = np.ones(2 * e.shape[0], dtype=np.int8)
    rows = np.concatenate([e[:, 0], e[:, 1]])
    cols = np.concatenate([e[:, 1], e[:, 0]])
    return sp.csr_matrix((data, (rows, cols)), shape=(n, n))


def graph_distances(n, edges, sources=None):
    """Unweighted shortest-path distances (BFS) from `sources` (all nodes by default) to
    all nodes; inf where unreachable. Shape (len(sources), n)."""
    from scipy.sparse.csgraph import shortest_path
    A = _csr(n, edges)
    idx = np.arange(n) if sources is None else np.asarray(sources)
    return shortest_path(A, method="D", unweighted=True, directed=False, indices=idx)


def stress_error(xy, edges, sources=None):
    """Normalized stress error with the optimal uniform scale. `sources` restricts the
    pairs to (source, any other node) (a sample for larger graphs); the sum then runs over
    those pairs with the same normalisation per pair."""
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.shape[0]
    idx = np.arange(n) if sources is None else np.asarray(sources)
    D = graph_distances(n, edges, idx)
    X = np.linalg.norm(xy[idx][:, None, :] - xy[None, :, :], axis=2)
    mask = np.isfinite(D) & (D > 0)
    if sources is None:
        mask &= np.arange(n)[None, :] > np.arange(n)[:, None]  # i < j once
    a = X[mask] / D[mask]  # scaled distance over graph distance, per pair
    if a.size == 0:
        return 0.0
    s = a.sum() / np.dot(a, a)  # minimises sum (s a - 1)^2
    return float(np.sum((s * a - 1.0) ** 2) / a.size)


def ring_neighbours(n, edges, r):
    """r-ring graph neighbourhoods: list of arrays of the nodes within r hops (excluding i)."""
    A = _csr(n, edges)
    reach = A.copy().astype(bool)
    frontier = A.astype(bool)
    for _ in range(1, r):
        frontier = (frontier @ A).astype(bool)
        reach = (reach + frontier).astype(bool)
    reach = reach.tolil()
    out = []
    for i in range(n):
        nb = np.asarray(reach.rows[i], dtype=np.int64)
        out.append(nb[nb != i])
    return out


def neighbourhood_preservation(xy, edges, r=1):
    """NP_r: mean Jaccard index of the r-ring neighbourhood and the k_i nearest layout
    neighbours (k_i = its size); nodes without neighbours are left out."""
    from scipy.spatial import cKDTree
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.shape[0]
    rings = ring_neighbours(n, edges, r)
    tree = cKDTree(xy)
    kmax = max((len(x) for x in rings), default=0)
    if kmax == 0:
        return 0.0
    _, nn = tree.query(xy, k=min(n, kmax + 1))
    nn = np.atleast_2d(nn)
    vals = []
    for i in range(n):
        k = len(rings[i])
        if k == 0:
            continue
        cand = nn[i][nn[i] != i][:k]
        inter = np.intersect1d(rings[i], cand).size
        vals.append(inter / (2 * k - inter))
    return float(np.mean(vals))


def _segments_cross(p1, p2, q1, q2):
    """Proper crossings of segments p1p2 and q1q2 (arrays of shape (..., 2))."""
    def orient(a, b, c):
        return np.sign((b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1])
                       - (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0]))
    o1, o2 = orient(p1, p2, q1), orient(p1, p2, q2)
    o3, o4 = orient(q1, q2, p1), orient(q1, q2, p2)
    return (o1 * o2 < 0) & (o3 * o4 < 0)


def crosslessness(xy, edges):
    """CL = 1 - sqrt(c / c_max); O(m^2), for small graphs."""
    xy = np.asarray(xy, dtype=np.float64)
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    m = e.shape[0]
    deg = np.bincount(e.reshape(-1), minlength=xy.shape[0])
    c_max = m * (m - 1) / 2 - np.sum(deg * (deg - 1)) / 2
    if c_max <= 0:
        return 1.0
    c = 0
    for a in range(m - 1):
        b = np.arange(a + 1, m)
        share = (e[b, 0] == e[a, 0]) | (e[b, 0] == e[a, 1]) | (e[b, 1] == e[a, 0]) | (e[b, 1] == e[a, 1])
        b = b[~share]
        if b.size:
            c += int(np.sum(_segments_cross(xy[e[a, 0]], xy[e[a, 1]], xy[e[b, 0]], xy[e[b, 1]])))
    return float(1.0 - np.sqrt(c / c_max))


def minimum_angle(xy, edges):
    """MA = 1 - mean |theta - theta_min| / theta over nodes of degree >= 2."""
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.shape[0]
    rings = ring_neighbours(n, edges, 1)
    vals = []
    for i in range(n):
        nb = rings[i]
        if nb.size < 2:
            continue
        d = xy[nb] - xy[i]
        ang = np.sort(np.arctan2(d[:, 1], d[:, 0]))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi]))
        theta = 2 * np.pi / nb.size
        vals.append(abs(theta - gaps.min()) / theta)
    return float(1.0 - np.mean(vals)) if vals else 1.0


def relative(source, target):
    """Relative value (M(source) - M(target)) / M(target) of Sec. 4."""
    return (source - target) / target


def evaluate(xy, edges, se_sources=None, with_cl=True):
    """All four metrics of one layout (SE on sampled sources if given)."""
    out = {"SE": stress_error(xy, edges, se_sources),
           "NP1": neighbourhood_preservation(xy, edges, 1),
           "NP2": neighbourhood_preservation(xy, edges, 2),
           "MA": minimum_angle(xy, edges)}
    if with_cl:
        out["CL"] = crosslessness(xy, edges)
    return out
