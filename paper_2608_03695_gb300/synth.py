"""Seeded synthetic temporal graphs (inputs only).

This module produces the snapshot sequences that both the CUDA path and the
CPU oracle consume.  It holds none of the clustering method's arithmetic: no
modularity, no gains, no coupling, no supra-graph.  Every generator is driven
by numpy's PCG64 stream seeded with an explicit integer, so a (recipe, seed)
pair always yields the same graphs on any machine.

A snapshot is returned as a plain symmetric CSR over ``n`` nodes:
``(indptr int64[n+1], indices int32[nnz], weights int32[nnz])`` with sorted
column indices, no self-loops, no duplicate entries and weights >= 1.

The recipes stand in for the paper's datasets (Table 1 lists temporal graphs
from a few hundred to 1.3M nodes and 4 to 7,375 snapshots, plus SBM graphs
whose nodes/edges/snapshots are doubled in the scaling study of Sec. 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Snapshot",
    "csr_from_edges",
    "planted_partition_temporal",
    "dcsbm_powerlaw_temporal",
    "random_temporal",
    "cliques_temporal",
    "contact_temporal",
    "config_graph",
    "RECIPES",
]


@dataclass
class Snapshot:
    indptr: np.ndarray  # int64[n+1]
    indices: np.ndarray  # int32[nnz]
    weights: np.ndarray  # int32[nnz]

    @property
    def n(self) -> int:
        return len(self.indptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray) -> Snapshot:
    """Symmetric CSR from an undirected edge list with u != v and no repeats."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.int32)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    # (src, dst) pairs are distinct, so one sort of src*n + dst orders them
    order = np.argsort(src * max(n, 1) + dst)
    src, dst, ww = src[order], dst[order], ww[order]
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return Snapshot(indptr, dst.astype(np.int32), ww.astype(np.int32))


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    x = np.sort(x, kind="stable")
    if len(x) == 0:
        return x
    keep = np.empty(len(x), dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def _in_sorted(x: np.ndarray, sorted_ref: np.ndarray) -> np.ndarray:
    if len(sorted_ref) == 0:
        return np.zeros(len(x), dtype=bool)
    pos = np.searchsorted(sorted_ref, x)
    pos = np.minimum(pos, len(sorted_ref) - 1)
    return sorted_ref[pos] == x


def _edge_keys(u: np.ndarray, v: np.ndarray, n: int) -> np.ndarray:
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    return a * n + b


def _keys_to_edges(keys: np.ndarray, n: int):
    return keys // n, keys % n


def _tri_decode(k: np.ndarray):
    """Linear index into the strict upper triangle -> (i, j), i < j."""
    k = k.astype(np.int64)
    j = ((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # fix float rounding at the boundaries
    j = np.where(j * (j - 1) // 2 > k, j - 1, j)
    j = np.where((j + 1) * j // 2 <= k, j + 1, j)
    i = k - j * (j - 1) // 2
    return i, j


def _distinct_ints(rng, possible: int, m: int) -> np.ndarray:
    """m distinct integers drawn uniformly from [0, possible).  Small
    populations use numpy's sampler without replacement; large sparse ones
    draw with replacement, drop repeats and draw again for the shortfall (the
    same distribution: every m-subset is equally likely), then keep a random
    m of them."""
    if possible <= (1 << 22) or m * 4 > possible:
        return rng.choice(possible, size=m, replace=False)
    out = np.zeros(0, np.int64)
    while len(out) < m:
        need = m - len(out)
        x = rng.integers(0, possible, size=need + need // 50 + 16, dtype=np.int64)
        out = _sorted_unique(np.concatenate([out, x]))
    if len(out) > m:
        out = out[rng.permutation(len(out))[:m]]
    return out


def _sample_block_pairs(rng, members_a, members_b, p, same):
    """Distinct node pairs between two blocks, each present with prob. p."""
    na, nb = len(members_a), len(members_b)
    possible = na * (na - 1) // 2 if same else na * nb
    if possible <= 0 or p <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    m = int(rng.binomial(possible, min(p, 1.0)))
    if m == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    idx = _distinct_ints(rng, possible, m)
    if same:
        i, j = _tri_decode(idx)
        return members_a[i], members_a[j]
    return members_a[idx // nb], members_b[idx % nb]


def _sbm_edges(rng, block_of: np.ndarray, n_blocks: int, p_in: float, p_out: float):
    members = [np.flatnonzero(block_of == b).astype(np.int64) for b in range(n_blocks)]
    us, vs = [], []
    for a in range(n_blocks):
        for b in range(a, n_blocks):
            u, v = _sample_block_pairs(rng, members[a], members[b], p_in if a == b else p_out, a == b)
            us.append(u)
            vs.append(v)
    return np.concatenate(us), np.concatenate(vs)


def planted_partition_temporal(
    n: int,
    T: int,
    n_blocks: int = 4,
    p_in: float = 0.05,
    p_out: float = 0.005,
    switch_frac: float = 0.10,
    churn: float | None = None,
    w_max: int = 1,
    seed: int = 1,
):
    """Temporal planted partition (stochastic block model) snapshots.

    Node i starts in block floor(n_blocks*i/n).  Between consecutive snapshots a
    fraction ``switch_frac`` of the nodes (uniform, without replacement) moves to
    a uniformly chosen other block.  With ``churn=None`` every snapshot's edges
    are sampled afresh from the current blocks; with ``churn=f`` a fraction f of
    the previous snapshot's edges is deleted uniformly and the same number is
    drawn from the model, the surviving edges keeping their weights.
    Weights are uniform on {1..w_max}.  Returns (snapshots, blocks[T][n]).
    """
    rng = np.random.default_rng(seed)
    block_of = (np.arange(n, dtype=np.int64) * n_blocks) // max(n, 1)
    snaps, blocks = [], []
    prev_keys = prev_w = None
    for t in range(T):
        if t > 0 and switch_frac > 0 and n > 0:
            k = int(round(switch_frac * n))
            movers = rng.choice(n, size=k, replace=False)
            shift = rng.integers(1, n_blocks, size=k)
            block_of = block_of.copy()
            block_of[movers] = (block_of[movers] + shift) % n_blocks
        if churn is None or prev_keys is None:
            u, v = _sbm_edges(rng, block_of, n_blocks, p_in, p_out)
            keys = _sorted_unique(_edge_keys(u, v, n))
            w = rng.integers(1, w_max + 1, size=len(keys)).astype(np.int32)
        else:
            keys, w = _churn(rng, prev_keys, prev_w, churn, n, w_max,
                             lambda m: _sbm_edges(rng, block_of, n_blocks, p_in, p_out), m_target=len(prev_keys))
        prev_keys, prev_w = keys, w
        a, b = _keys_to_edges(keys, n)
        snaps.append(csr_from_edges(n, a, b, w))
        blocks.append(block_of.copy())
    return snaps, blocks


def _churn(rng, keys, w, frac, n, w_max, sampler, m_target):
    """Delete a fraction of edges uniformly; refill from the model to m_target."""
    m = len(keys)
    n_del = int(round(frac * m))
    keep = np.ones(m, dtype=bool)
    if n_del > 0:
        keep[rng.choice(m, size=n_del, replace=False)] = False
    keys, w = keys[keep], w[keep]  # still sorted
    need = m_target - len(keys)
    new_keys = np.zeros(0, np.int64)
    tries = 0
    while need > 0 and tries < 50:
        u, v = sampler(int(need * 1.25) + 16)
        cand = _sorted_unique(_edge_keys(u, v, n))
        cand = cand[~_in_sorted(cand, keys)]
        cand = cand[~_in_sorted(cand, new_keys)]
        if len(cand) > need:
            cand = np.sort(rng.permutation(cand)[:need])
        new_keys = np.sort(np.concatenate([new_keys, cand]))
        need -= len(cand)
        tries += 1
    new_w = rng.integers(1, w_max + 1, size=len(new_keys)).astype(np.int32)
    keys = np.concatenate([keys, new_keys])
    w = np.concatenate([w, new_w])
    order = np.argsort(keys, kind="stable")
    return keys[order], w[order]


def _powerlaw_sample(rng, size, exponent, lo, hi):
    """Continuous power law p(x) ~ x^-exponent on [lo, hi] by inversion."""
    a = 1.0 - exponent
    u = rng.random(size)
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def _powerlaw_mean(exponent, lo, hi):
    a1, a2 = 2.0 - exponent, 1.0 - exponent
    return (a2 / a1) * (hi ** a1 - lo ** a1) / (hi ** a2 - lo ** a2)


def _community_sizes(rng, n, exponent, smin, smax):
    sizes = []
    total = 0
    while total < n:
        s = int(_powerlaw_sample(rng, 1, exponent, smin, smax + 1)[0])
        s = min(max(s, smin), smax)
        if total + s > n:
            s = n - total
        sizes.append(s)
        total += s
    return np.array(sizes, dtype=np.int64)


def _chung_lu_pairs(rng, nodes, weights, m):
    """m endpoint pairs drawn with probability proportional to weight."""
    if m <= 0 or len(nodes) < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    cdf = np.cumsum(weights, dtype=np.float64)
    cdf /= cdf[-1]
    a = np.searchsorted(cdf, rng.random(m), side="right")
    b = np.searchsorted(cdf, rng.random(m), side="right")
    a = np.minimum(a, len(nodes) - 1)
    b = np.minimum(b, len(nodes) - 1)
    return nodes[a], nodes[b]


def dcsbm_powerlaw_temporal(
    n: int,
    T: int,
    deg_exp: float = 2.5,
    mean_deg: float = 20.0,
    size_exp: float = 1.5,
    size_min: int = 20,
    size_max: int = 5000,
    mixing: float = 0.3,
    churn: float = 0.05,
    w_max: int = 8,
    seed: int = 2,
):
    """Degree-corrected SBM with power-law degrees and community sizes.

    Community sizes follow a power law (exponent ``size_exp`` on
    [size_min, size_max]) until they cover n nodes; expected degrees follow a
    power law (exponent ``deg_exp``) with mean ``mean_deg`` and cutoff
    sqrt(n*mean_deg).  A fraction ``mixing`` of each node's expected stubs
    leaves its community.  Edges are drawn Chung-Lu style inside each
    community and between communities (pairs landing inside one community in
    the between-draw are rejected).  Each later snapshot deletes ``churn`` of
    the previous edges uniformly and refills from the same model; surviving
    edges keep their weight (uniform on {1..w_max}).
    Returns (snapshots, community_of[n]).
    """
    rng = np.random.default_rng(seed)
    sizes = _community_sizes(rng, n, size_exp, size_min, size_max)
    comm = np.repeat(np.arange(len(sizes), dtype=np.int64), sizes)
    comm = comm[rng.permutation(n)]
    hi = math.sqrt(n * mean_deg)
    # pick lo so that the truncated power law has the requested mean
    lo_a, lo_b = 1e-3, mean_deg
    for _ in range(200):
        mid = 0.5 * (lo_a + lo_b)
        if _powerlaw_mean(deg_exp, mid, hi) < mean_deg:
            lo_a = mid
        else:
            lo_b = mid
    theta = _powerlaw_sample(rng, n, deg_exp, 0.5 * (lo_a + lo_b), hi)
    m_total = int(round(theta.sum() / 2.0))
    order = np.argsort(comm, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(np.bincount(comm, minlength=len(sizes)))])
    w_in = (1.0 - mixing) * theta
    w_out = mixing * theta
    all_nodes = np.arange(n, dtype=np.int64)

    def sample(m_req):
        # split the request between intra and inter edges by the stub mass
        m_in = int(round(m_req * (1.0 - mixing)))
        us, vs = [], []
        mass = np.array([w_in[order[bounds[c]:bounds[c + 1]]].sum() for c in range(len(sizes))])
        counts = rng.multinomial(m_in, mass / mass.sum()) if m_in > 0 else np.zeros(len(sizes), np.int64)
        for c in np.flatnonzero(counts):
            nodes = order[bounds[c]:bounds[c + 1]]
            a, b = _chung_lu_pairs(rng, nodes, w_in[nodes], int(counts[c]))
            us.append(a)
            vs.append(b)
        a, b = _chung_lu_pairs(rng, all_nodes, w_out, m_req - m_in)
        keep = comm[a] != comm[b]
        us.append(a[keep])
        vs.append(b[keep])
        u = np.concatenate(us)
        v = np.concatenate(vs)
        ok = u != v
        return u[ok], v[ok]

    snaps = []
    keys = w = None
    for t in range(T):
        if keys is None:
            keys, w = _churn(rng, np.zeros(0, np.int64), np.zeros(0, np.int32), 0.0, n, w_max, sample, m_total)
        else:
            keys, w = _churn(rng, keys, w, churn, n, w_max, sample, len(keys))
        a, b = _keys_to_edges(keys, n)
        snaps.append(csr_from_edges(n, a, b, w))
    return snaps, comm


def random_temporal(n: int, T: int, p: float, w_max: int = 3, seed: int = 0, p_empty: float = 0.0):
    """Independent G(n,p) snapshots (tiny test graphs); a snapshot is left
    without edges with probability p_empty."""
    rng = np.random.default_rng(seed)
    snaps = []
    for _ in range(T):
        if n >= 2 and rng.random() >= p_empty:
            iu, ju = np.triu_indices(n, 1)
            keep = rng.random(len(iu)) < p
            u, v = iu[keep], ju[keep]
        else:
            u = v = np.zeros(0, np.int64)
        w = rng.integers(1, w_max + 1, size=len(u))
        snaps.append(csr_from_edges(n, u, v, w))
    return snaps


def cliques_temporal(clique_sizes, T: int, w: int = 1):
    """Disjoint cliques, the same in every snapshot."""
    us, vs = [], []
    off = 0
    for s in clique_sizes:
        iu, ju = np.triu_indices(s, 1)
        us.append(iu + off)
        vs.append(ju + off)
        off += s
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    snap = csr_from_edges(off, u, v, np.full(len(u), w, np.int32))
    return [Snapshot(snap.indptr.copy(), snap.indices.copy(), snap.weights.copy()) for _ in range(T)]


def contact_temporal(n: int, T: int, n_groups: int, static_edges: int, contacts: int, within_frac: float,
                     seed: int = 0):
    """Face-to-face contact sequences, the shape of a school contact dataset
    (a few hundred people in classes, thousands of very sparse snapshots):
    n people in n_groups classes of near-equal size; a fixed pool of
    static_edges distinct pairs, round(within_frac * static_edges) of them
    inside a class (at most every such pair) and the rest between classes;
    snapshot t holds Poisson(contacts / T) pairs drawn from the pool without
    replacement, weight 1.  Returns (snapshots, class of every person)."""
    if n > 20000:
        raise ValueError("contact_temporal enumerates node pairs; keep n <= 20000")
    rng = np.random.default_rng(seed)
    group_of = rng.permutation(np.arange(n) % max(n_groups, 1))
    iu, ju = np.triu_indices(n, k=1)
    same = group_of[iu] == group_of[ju]
    within = np.flatnonzero(same)
    cross = np.flatnonzero(~same)
    m_in = min(int(round(within_frac * static_edges)), len(within))
    m_out = min(static_edges - m_in, len(cross))
    pick = np.concatenate([within[rng.choice(len(within), m_in, replace=False)] if m_in else np.zeros(0, np.int64),
                           cross[rng.choice(len(cross), m_out, replace=False)] if m_out else np.zeros(0, np.int64)])
    pu, pv = iu[pick].astype(np.int64), ju[pick].astype(np.int64)
    rate = contacts / max(T, 1)
    snaps = []
    for _ in range(T):
        k = min(int(rng.poisson(rate)), len(pick))
        idx = rng.choice(len(pick), k, replace=False) if k else np.zeros(0, np.int64)
        snaps.append(csr_from_edges(n, pu[idx], pv[idx], np.ones(k, np.int32)))
    return snaps, group_of


# Workload recipes.  Rationals are (numerator, denominator) pairs.
# Named recipes: a planted partition (T=4, n=1,000), the power-law temporal
# graph of the benchmark (T=16, n=100,000) and its large T=64, n=1,000,000
# form.
RECIPES = {
    "planted_t4_n1000": dict(kind="planted", n=1000, T=4, n_blocks=4, p_in=0.05, p_out=0.005, switch_frac=0.10,
            w_max=1, seed=1, gamma=(1, 1), omega=(1, 1)),
    "powerlaw_t16_n100k": dict(kind="dcsbm", n=100_000, T=16, deg_exp=2.5, mean_deg=20.0, size_exp=1.5, size_min=20,
            size_max=5000, mixing=0.3, churn=0.05, w_max=8, seed=2, gamma=(1, 1), omega=(1, 1)),
    "powerlaw_t64_n1m": dict(kind="dcsbm", n=1_000_000, T=64, deg_exp=2.3, mean_deg=16.0, size_exp=1.5, size_min=20,
            size_max=5000, mixing=0.4, churn=0.05, w_max=16, seed=4, gamma=(1, 1), omega=(1, 1)),
    # the shape of the paper's School contact dataset (Table 1: 327 people, 7,004 static and 188,508
    # temporal edges, 7,375 snapshots, 9 classes)
    "school_t7375_n327": dict(kind="contact", n=327, T=7375, n_groups=9, static_edges=7004, contacts=188508,
            within_frac=0.7, seed=6, gamma=(1, 1), omega=(1, 1)),
}


# Batched workload: 64 independent temporal planted-partition graphs (the
# planted-partition generator of planted_t4_n1000: 4 equal blocks, p_out = p_in / 10, 10% of the nodes
# switch block between snapshots), n log-uniform in [1k, 200k], T uniform in
# [2, 32], mean degree uniform in [8, 32], weights 1..8; every graph is solved
# at each (gamma, omega) of the grid below (1,152 solves).
BATCHED = dict(n_graphs=64, n_lo=1000, n_hi=200_000, T_lo=2, T_hi=32, deg_lo=8.0, deg_hi=32.0, w_max=8, seed=3)
BATCHED_GAMMAS = [(1, 2), (3, 4), (1, 1), (5, 4), (3, 2), (2, 1)]
BATCHED_OMEGAS = [(1, 10), (1, 1), (10, 1)]


def batched_specs(scale_n: float = 1.0, n_graphs: int | None = None):
    """(n, T, p_in, seed) of every graph of the batched workload (n scaled by
    scale_n, at least 8)."""
    c = BATCHED
    rng = np.random.default_rng(c["seed"])
    specs = []
    for g in range(c["n_graphs"] if n_graphs is None else n_graphs):
        n = float(np.exp(rng.uniform(np.log(c["n_lo"]), np.log(c["n_hi"]))))
        T = int(rng.integers(c["T_lo"], c["T_hi"] + 1))
        d = float(rng.uniform(c["deg_lo"], c["deg_hi"]))
        n = max(8, int(round(n * scale_n)))
        # expected degree with 4 equal blocks and p_out = p_in/10:
        # p_in (n/4 - 1) + (p_in/10)(3n/4)
        p_in = min(1.0, d / (n / 4 - 1 + 0.075 * n))
        specs.append((n, T, p_in, 1000 * c["seed"] + g))
    return specs


def batched_graph(spec):
    n, T, p_in, seed = spec
    snaps, _ = planted_partition_temporal(n, T, 4, p_in, p_in / 10, 0.10, None, BATCHED["w_max"], seed)
    return snaps


# Serving workload: 32 live temporal graphs (the planted-partition generator at
# mean degree 16), n log-uniform in
# [10k, 2M], each a stream of snapshots with 5% edge churn between
# consecutive ones, weights 1..8; windows of W = 8 slices; requests arrive
# as a Poisson process of 50 snapshots per second.
SERVING = dict(n_graphs=32, n_lo=10_000, n_hi=2_000_000, mean_deg=16.0, churn=0.05, w_max=8, window=8,
               rate_per_s=50.0, seed=5)


def serving_specs(scale_n: float = 1.0, n_graphs: int | None = None):
    """(n, p_in, seed) of every live graph of the serving workload."""
    c = SERVING
    rng = np.random.default_rng(c["seed"])
    specs = []
    for g in range(c["n_graphs"] if n_graphs is None else n_graphs):
        n = float(np.exp(rng.uniform(np.log(c["n_lo"]), np.log(c["n_hi"]))))
        n = max(8, int(round(n * scale_n)))
        p_in = min(1.0, c["mean_deg"] / (n / 4 - 1 + 0.075 * n))
        specs.append((n, p_in, 1000 * c["seed"] + g))
    return specs


def serving_stream(spec, steps: int):
    """The first `steps` snapshots of one live graph: 4 equal blocks,
    p_out = p_in / 10, 10% of the nodes switch block between snapshots and 5%
    of the edges are replaced."""
    n, p_in, seed = spec
    snaps, _ = planted_partition_temporal(n, steps, 4, p_in, p_in / 10, 0.10, SERVING["churn"], SERVING["w_max"],
                                          seed)
    return snaps


def recipe_graph(recipe: str | dict, scale_n: int | None = None, T: int | None = None):
    """Snapshots of a named recipe (or a recipe dict), optionally with n or T
    overridden."""
    c = dict(RECIPES[recipe]) if isinstance(recipe, str) else dict(recipe)
    n = scale_n if scale_n is not None else c["n"]
    TT = T if T is not None else c["T"]
    if c["kind"] == "contact":
        # fewer snapshots keep the contacts per snapshot
        snaps, _ = contact_temporal(n, TT, c["n_groups"], c["static_edges"], int(round(c["contacts"] * TT / c["T"])),
                                    c["within_frac"], c["seed"])
        return snaps
    if c["kind"] == "planted":
        snaps, _ = planted_partition_temporal(n, TT, c["n_blocks"], c["p_in"], c["p_out"], c["switch_frac"],
                                              c.get("churn"), c["w_max"], c["seed"])
    else:
        snaps, _ = dcsbm_powerlaw_temporal(n, TT, c["deg_exp"], c["mean_deg"], c["size_exp"], c["size_min"],
                                           c["size_max"], c["mixing"], c["churn"], c["w_max"], c["seed"])
    return snaps
