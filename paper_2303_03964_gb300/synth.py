"""Seeded synthetic graphs and initial layouts.

These stand in for the paper's 50 real graphs and com-LiveJournal (Sec. 4, "Datasets"),
none of which is available: Erdos-Renyi graphs, stochastic block models (clustered
graphs, like the paper's graph-tool cluster graphs), 2D lattices (mesh-like graphs) and
Barabasi-Albert graphs (scale-free, like the social networks), with uniform random
initial positions.

This module holds none of the method's arithmetic. It is the only code that both the
oracle-side tests and the GPU library's callers share.
All graphs are undirected, without self-loops or duplicate edges, returned as an
(m, 2) int32 array of node pairs (i, j).
"""
import numpy as np

SEED_BASE = 2303039640


def rng_for(config: int) -> np.random.Generator:
    """PCG64 generator with the seed of a numbered workload (SEED_BASE + config)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config)))


def _canon_unique(pairs: np.ndarray) -> np.ndarray:
    a = np.minimum(pairs[:, 0], pairs[:, 1])
    b = np.maximum(pairs[:, 0], pairs[:, 1])
    keep = a != b
    a, b = a[keep], b[keep]
    key = np.unique(a.astype(np.int64) << 32 | b.astype(np.int64))
    return np.stack([(key >> 32), (key & 0xFFFFFFFF)], axis=1)


def _top_up(n_target: int, draw, rng, first_key_order=True) -> np.ndarray:
    """Draw batches of candidate pairs until n_target distinct edges exist."""
    have = np.zeros((0, 2), dtype=np.int64)
    need = n_target
    while need > 0:
        cand = draw(int(need * 1.1) + 16)
        have = _canon_unique(np.concatenate([have, cand]))
        need = n_target - have.shape[0]
    # keep a uniformly random subset of exactly n_target edges, in random order
    sel = rng.permutation(have.shape[0])[:n_target]
    return have[sel]


def erdos_renyi(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """m distinct uniform random pairs i != j."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")

    def draw(c):
        return rng.integers(0, n, size=(c, 2))

    return _top_up(m, draw, rng).astype(np.int32)


def sbm(n: int, blocks: int, mean_degree: float, intra_frac: float,
        rng: np.random.Generator):
    """Stochastic block model with equal blocks (node b*size .. (b+1)*size-1 in block b).

    m = round(n * mean_degree / 2) edges, a fraction intra_frac of them inside blocks,
    each inside-block edge in a uniformly chosen block, each across-block edge between
    two different uniformly chosen blocks. Returns (edges, block_of_node).
    """
    size = n // blocks
    if size * blocks != n:
        raise ValueError("n must be a multiple of blocks")
    m = int(round(n * mean_degree / 2))
    m_in = int(round(intra_frac * m))
    m_out = m - m_in

    def draw_in(c):
        b = rng.integers(0, blocks, size=c)
        return b[:, None] * size + rng.integers(0, size, size=(c, 2))

    def draw_out(c):
        b1 = rng.integers(0, blocks, size=c)
        b2 = (b1 + rng.integers(1, blocks, size=c)) % blocks
        return np.stack([b1 * size + rng.integers(0, size, size=c),
                         b2 * size + rng.integers(0, size, size=c)], axis=1)

    e_in = _top_up(m_in, draw_in, rng)
    e_out = _top_up(m_out, draw_out, rng) if m_out > 0 else np.zeros((0, 2), np.int64)
    edges = np.concatenate([e_in, e_out])
    edges = edges[rng.permutation(edges.shape[0])]
    return edges.astype(np.int32), np.arange(n) // size


def barabasi_albert(n: int, m0: int, rng: np.random.Generator) -> np.ndarray:
    """Preferential attachment: a clique on m0 + 1 nodes, then each new node links to
    m0 distinct earlier nodes drawn with probability proportional to their degree."""
    if n <= m0:
        raise ValueError("n must exceed m0")
    clique = [(i, j) for i in range(m0 + 1) for j in range(i + 1, m0 + 1)]
    m_total = len(clique) + m0 * (n - m0 - 1)
    edges = np.empty((m_total, 2), dtype=np.int32)
    edges[: len(clique)] = np.asarray(clique, dtype=np.int32).reshape(-1, 2)
    # endpoint list: node v appears deg(v) times; uniform draws from it are
    # degree-proportional draws.
    ends = np.empty(2 * m_total, dtype=np.int64)
    ne = 2 * len(clique)
    ends[:ne] = edges[: len(clique)].reshape(-1)
    pos = len(clique)
    u = rng.random(size=(n, 4 * m0))
    for v in range(m0 + 1, n):
        chosen = []
        row = u[v]
        r = 0
        while len(chosen) < m0:
            if r < row.shape[0]:
                x = row[r]
                r += 1
            else:
                x = rng.random()
            t = int(ends[int(x * ne)])
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            edges[pos, 0] = v
            edges[pos, 1] = t
            pos += 1
            ends[ne] = v
            ends[ne + 1] = t
            ne += 2
    return edges


def lattice(side_x: int, side_y: int) -> np.ndarray:
    """4-neighbour grid graph; node (x, y) has id y * side_x + x."""
    ids = np.arange(side_x * side_y, dtype=np.int64).reshape(side_y, side_x)
    h = np.stack([ids[:, :-1].reshape(-1), ids[:, 1:].reshape(-1)], axis=1)
    v = np.stack([ids[:-1, :].reshape(-1), ids[1:, :].reshape(-1)], axis=1)
    return np.concatenate([h, v]).astype(np.int32)


def uniform_positions(n: int, half_width: float, rng: np.random.Generator,
                      dtype=np.float32) -> np.ndarray:
    """Initial layout: n points uniform in [-half_width, half_width]^2, shape (n, 2)."""
    return rng.uniform(-half_width, half_width, size=(n, 2)).astype(dtype)


# --------------------------------------------------------------------------
# Named workloads (sizes and structure of the paper's graphs, Sec. 4).
# --------------------------------------------------------------------------

def er_2000(rng=None):
    """ER n=2000, m=8000, positions U[-50, 50]^2 in FP64 (exact-repulsion workload)."""
    rng = rng or rng_for(1)
    e = erdos_renyi(2000, 8000, rng)
    xy = uniform_positions(2000, 50.0, rng, dtype=np.float64)
    return e, xy


def sbm_100k(rng=None, n=100_000, blocks=20):
    """SBM n=100k in 20 blocks, mean degree 10, 90% of edges inside blocks, U[-50, 50]^2."""
    rng = rng or rng_for(2)
    e, _ = sbm(n, blocks, 10.0, 0.9, rng)
    xy = uniform_positions(n, 50.0, rng)
    return e, xy


def lattice_1m(rng=None, side=1000):
    """side x side lattice with positions U[-side/2, side/2]^2 (unit density)."""
    rng = rng or rng_for(3)
    e = lattice(side, side)
    xy = uniform_positions(side * side, side / 2.0, rng)
    return e, xy


def ba_2m(rng=None, n=2_000_000, m0=3):
    """BA n=2M, m0=3 with positions U[-sqrt(n)/2, sqrt(n)/2]^2 (unit density)."""
    rng = rng or rng_for(3)
    e = barabasi_albert(n, m0, rng)
    xy = uniform_positions(n, np.sqrt(n) / 2.0, rng)
    return e, xy


def batch_mixed(count=512, nmin=1000, nmax=50000, rng=None):
    """`count` graphs with n log-uniform in [nmin, nmax]; in turn an SBM (10 blocks, mean
    degree 8, 90% inside blocks), a Barabasi-Albert graph (m0 = 2) and a lattice
    (side floor(sqrt n)); positions uniform with unit density. Returns a list of
    (n, edges, xy)."""
    rng = rng or rng_for(4)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        kind = q % 3
        if kind == 0:
            n = max(10, n // 10 * 10)
            e, _ = sbm(n, 10, 8.0, 0.9, rng)
        elif kind == 1:
            e = barabasi_albert(n, 2, rng)
        else:
            side = max(2, int(np.sqrt(n)))
            n = side * side
            e = lattice(side, side)
        xy = uniform_positions(n, np.sqrt(n) / 2.0, rng)
        out.append((n, e, xy))
    return out
