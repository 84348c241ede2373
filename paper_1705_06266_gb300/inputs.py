"""Seeded synthetic graphs and right-hand sides.

This module is the one piece shared by the oracle tests and the CUDA path's
tests and benchmark: it makes inputs and holds none of the solver's arithmetic.
Every graph comes out as a weighted, undirected, connected graph in CSR form:

* both directions of every edge are stored (the adjacency matrix ``A`` with
  ``A_ij = A_ji = w_ij``, Section 2.1 of the paper),
* rows are sorted by column, with no duplicates and no self-loops,
* weights are strictly positive,
* only the largest connected component is kept (the paper assumes a connected
  graph, Section 2.1) and its vertices are renumbered in ascending order.

Duplicate samples of an edge are merged and the weight of an edge is a
deterministic function of its unordered endpoint pair, so the result does not
depend on the order in which a sampler emitted the edge.

The workloads stand in for the paper's SNAP and UF graphs (social networks:
sparse, power-law degrees, low diameter, Section 2.1), which are not available
here: 2D/3D grids, Chung-Lu power-law graphs and R-MAT graphs.
"""

from __future__ import annotations

import dataclasses

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


@dataclasses.dataclass
class Graph:
    """A CSR graph: ``rowptr`` int64[n+1], ``col`` int32[nnz], ``w`` float64[nnz]."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def nnz_off(self) -> int:
        return int(self.rowptr[-1])

    @property
    def nnz(self) -> int:
        """nnz of the Laplacian L = D - A: the off-diagonal entries plus the diagonal."""
        return self.nnz_off + self.n

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _pair_weight(lo: np.ndarray, hi: np.ndarray, n: int, seed: int, wlo: float, whi: float) -> np.ndarray:
    """Weight in [wlo, whi) as a pure function of the unordered pair (lo, hi)."""
    with np.errstate(over="ignore"):
        key = lo.astype(np.uint64) * np.uint64(n) + hi.astype(np.uint64)
        z = np.uint64(seed) + (key + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return wlo + (whi - wlo) * u


def from_edges(n: int, u: np.ndarray, v: np.ndarray, *, weights: str = "unit", seed: int = 1,
               wlo: float = 0.5, whi: float = 1.5, keep_lcc: bool = True, name: str = "") -> Graph:
    """Build a clean CSR graph from sampled endpoint arrays.

    Self-loops are dropped, duplicate pairs merged, both directions stored and,
    with ``keep_lcc``, only the largest connected component kept.
    ``weights`` is ``"unit"`` or ``"uniform"`` (uniform in [wlo, whi)).
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = np.sort(lo * np.int64(n) + hi)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    lo = key // n
    hi = key % n
    if weights == "unit":
        wt = np.ones(lo.shape[0], dtype=np.float64)
    elif weights == "uniform":
        wt = _pair_weight(lo, hi, n, seed, wlo, whi)
    else:
        raise ValueError(f"unknown weights {weights!r}")

    if keep_lcc and lo.size:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import connected_components

        adj = sp.coo_matrix((np.ones(lo.size), (lo, hi)), shape=(n, n)).tocsr()
        ncomp, label = connected_components(adj, directed=False)
        if ncomp > 1:
            big = np.bincount(label).argmax()
            inside = label == big
            newid = np.cumsum(inside) - 1
            sel = inside[lo]  # both endpoints share the component
            lo, hi, wt = newid[lo[sel]], newid[hi[sel]], wt[sel]
            n = int(inside.sum())
    elif keep_lcc:
        n = 1

    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    ws = np.concatenate([wt, wt])
    order = np.argsort(rows * np.int64(n) + cols, kind="stable")
    rows, cols, ws = rows[order], cols[order], ws[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return Graph(n, rowptr, cols.astype(np.int32), np.ascontiguousarray(ws), name)


def grid2d(nx: int, ny: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    """2D 5-point grid graph, nx*ny vertices, vertex id = y*nx + x."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(nx * ny, u, v, weights=weights, seed=seed, name=f"grid2d_{nx}x{ny}")


def grid3d(nx: int, ny: int, nz: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    """3D 7-point grid graph, vertex id = (z*ny + y)*nx + x."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    u = np.concatenate([idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()])
    v = np.concatenate([idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()])
    return from_edges(nx * ny * nz, u, v, weights=weights, seed=seed, name=f"grid3d_{nx}x{ny}x{nz}")


def road_like(nx: int, ny: int, *, keep: float = 0.6, seed: int = 1) -> Graph:
    """A stand-in for road networks (long chains, low degree, large diameter):
    the 2D grid with each edge kept with probability ``keep`` (seeded), weights
    uniform in [0.5, 1.5), the largest component kept."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    rng = np.random.Generator(np.random.PCG64(seed))
    sel = rng.random(len(u)) < keep
    return from_edges(nx * ny, u[sel], v[sel], weights="uniform", seed=seed, name=f"road_like_{nx}x{ny}")


def chung_lu(n: int, *, exponent: float = 2.1, dmin: float = 1.0, dmax: float = 50000.0,
             m_target: int | None = None, seed: int = 1, weights: str = "uniform",
             wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """Chung-Lu power-law graph.

    Expected degrees are drawn i.i.d. from a Pareto density proportional to
    d^-exponent, truncated to [dmin, dmax]; ``m_target`` endpoint pairs are then
    drawn independently with probability proportional to the expected degree.
    Without ``m_target`` the number of pairs is half the sum of expected degrees.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = exponent - 1.0
    uu = rng.random(n)
    theta = dmin * (1.0 - uu * (1.0 - (dmin / dmax) ** a)) ** (-1.0 / a)
    if m_target is None:
        m_target = int(theta.sum() / 2)
    p = theta / theta.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    # Sorted queries make the search cache-friendly; shuffling one side keeps the
    # pairs independent draws.
    u = np.searchsorted(cdf, np.sort(rng.random(m_target)), side="right")
    v = np.searchsorted(cdf, np.sort(rng.random(m_target)), side="right")
    v = v[rng.permutation(m_target)]
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    return from_edges(n, u, v, weights=weights, seed=seed + 7, wlo=wlo, whi=whi,
                      name=f"chung_lu_{n}_{exponent}")


def rmat(scale: int, *, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, weights: str = "unit") -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale sampled edges (no noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale):
        r = rng.random(m)
        right = ((r >= a) & (r < ab)) | (r >= abc)  # quadrants b and d set the column bit
        down = r >= ab                               # quadrants c and d set the row bit
        u |= down.astype(np.int64) << bit
        v |= right.astype(np.int64) << bit
    return from_edges(n, u, v, weights=weights, seed=seed + 7, name=f"rmat_{scale}_{edge_factor}")


def _device_csr(n: int, key, *, weights: str, seed: int, device: str):
    """Deduplicated pair keys lo * n + hi (lo < hi) on a torch device -> the
    largest component as a symmetric CSR (n, rowptr int64, col int32, w
    float64), vertices renumbered in id order, rows sorted. Weights: "unit",
    or "uniform" in [0.5, 1.5) drawn by a seeded torch generator in key order."""
    import torch

    u, v = key // n, key % n
    if weights == "unit":
        wt = torch.ones(key.numel(), dtype=torch.float64, device=device)
    else:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        wt = 0.5 + torch.rand(key.numel(), generator=gen, device=device, dtype=torch.float64)
    del key
    # largest component: labels converge to the smallest id of each component
    label = torch.arange(n, dtype=torch.int64, device=device)
    while True:
        mn = torch.minimum(label[u], label[v])
        new = label.clone()
        new.scatter_reduce_(0, u, mn, reduce="amin")
        new.scatter_reduce_(0, v, mn, reduce="amin")
        del mn
        new = new[new]
        new = new[new]
        if torch.equal(new, label):
            break
        label = new
    root = torch.bincount(label, minlength=n).argmax()
    inc = label == root
    del label, new
    nid = torch.cumsum(inc.to(torch.int64), 0) - 1
    keep = inc[u]  # both ends of an edge share a component
    u, v, wt = nid[u[keep]], nid[v[keep]], wt[keep]
    nl = int(inc.sum())
    del nid, keep, inc
    rows = torch.cat([u, v])
    cols = torch.cat([v, u])
    ws = torch.cat([wt, wt])
    del u, v, wt
    order = torch.argsort(rows * nl + cols)
    rows, cols, ws = rows[order], cols[order].to(torch.int32), ws[order]
    del order
    rowptr = torch.zeros(nl + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(torch.bincount(rows, minlength=nl), 0)
    del rows
    if str(device).startswith("cuda"):
        torch.cuda.empty_cache()  # hand the temporaries' memory back for the solver's own allocations
    return nl, rowptr, cols, ws


def rmat_device(scale: int, *, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                seed: int = 1, device: str = "cuda", chunk: int = 1 << 27):
    """R-MAT (Chakrabarti, Zhan & Faloutsos 2004) generated on a torch device,
    for sizes whose host-side generation would be too slow (scale 26: 2^26
    vertices, 2^30 sampled edges). Edges are sampled in chunks from a seeded
    torch generator (one quadrant draw per bit), symmetrised, deduplicated,
    self-loops dropped, unit weights, and the largest connected component kept
    (min-label propagation with pointer jumping) and renumbered in id order.
    Returns (n, rowptr int64, col int32, w float64) on the device, rows sorted.
    Not bitwise the same graph as rmat() at equal seeds: another generator."""
    import torch

    n = 1 << scale
    m = edge_factor << scale
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    parts = []
    for start in range(0, m, chunk):
        cnt = min(chunk, m - start)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        for bit in range(scale - 1, -1, -1):
            r = torch.rand(cnt, generator=gen, device=device)
            u |= (r >= a + b).to(torch.int64) << bit
            v |= (((r >= a) & (r < a + b)) | (r >= a + b + c)).to(torch.int64) << bit
            del r
        lo, hi = torch.minimum(u, v), torch.maximum(u, v)
        del u, v
        keep = lo != hi
        parts.append(torch.unique(lo[keep] * n + hi[keep]))
        del lo, hi, keep
    key = torch.unique(torch.cat(parts))
    del parts
    return _device_csr(n, key, weights="unit", seed=seed, device=device)


def chung_lu_device(n: int, *, exponent: float = 2.1, dmin: float = 1.0, dmax: float = 50000.0,
                    m_target: int | None = None, seed: int = 1, device: str = "cuda"):
    """Chung-Lu power-law graph on a torch device (the recipe of chung_lu():
    expected degrees i.i.d. Pareto with the given exponent truncated to [dmin,
    dmax], m_target endpoint pairs drawn with probability proportional to the
    expected degree, self-loops dropped, pairs deduplicated, weights uniform in
    [0.5, 1.5), largest component). Another generator than chung_lu(): the
    same distribution, not the same graph at equal seeds."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    a = exponent - 1.0
    uu = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
    theta = dmin * (1.0 - uu * (1.0 - (dmin / dmax) ** a)) ** (-1.0 / a)
    if m_target is None:
        m_target = int(theta.sum().item() / 2)
    cdf = torch.cumsum(theta / theta.sum(), 0)
    cdf[-1] = 1.0
    u = torch.searchsorted(cdf, torch.rand(m_target, generator=gen, device=device, dtype=torch.float64), right=True)
    v = torch.searchsorted(cdf, torch.rand(m_target, generator=gen, device=device, dtype=torch.float64), right=True)
    u.clamp_(max=n - 1)
    v.clamp_(max=n - 1)
    lo, hi = torch.minimum(u, v), torch.maximum(u, v)
    del u, v
    keep = lo != hi
    key = torch.unique(lo[keep] * n + hi[keep])
    del lo, hi, keep
    return _device_csr(n, key, weights="uniform", seed=seed + 7, device=device)


def serving_mix_device(count: int, nmin: int, nmax: int, *, seed: int = 5, device: str = "cuda"):
    """The serving workload of serving_mix() (the same sizes and types, drawn
    from the same seed), with the power-law members generated on the device
    (chung_lu_device, rmat_device) so that hundreds of graphs up to millions of
    vertices are made in seconds. Returns [(name, n, rowptr, col, w)] with
    device tensors."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = int(rng.integers(0, 4))
        if kind in (0, 1):
            if kind == 0:
                side = max(2, int(round(math.sqrt(n))))
                g = grid2d(side, side)
            else:
                side = max(2, int(round(n ** (1.0 / 3.0))))
                g = grid3d(side, side, side)
            out.append((g.name, g.n, torch.from_numpy(g.rowptr).to(device), torch.from_numpy(g.col).to(device),
                        torch.from_numpy(g.w).to(device)))
        elif kind == 2:
            nl, rp, cl, w = chung_lu_device(n, m_target=5 * n, seed=1000 + q, device=device)
            out.append((f"chung_lu_{n}_2.1", nl, rp, cl, w))
        else:
            sc = max(6, int(round(math.log2(n))))
            nl, rp, cl, w = rmat_device(sc, seed=1000 + q, device=device)
            out.append((f"rmat_{sc}_16", nl, rp, cl, w))
    return out


def random_graph(n: int, avg_degree: float, *, seed: int = 1, weights: str = "uniform") -> Graph:
    """Small Erdos-Renyi style graph plus a spanning path, so it is connected."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(n * avg_degree / 2)
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    perm = rng.permutation(n)
    u = np.concatenate([u, perm[:-1]])
    v = np.concatenate([v, perm[1:]])
    return from_edges(n, u, v, weights=weights, seed=seed + 7, name=f"random_{n}_{avg_degree}")


def star(k: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    """Hub 0 joined to leaves 1..k."""
    leaves = np.arange(1, k + 1)
    return from_edges(k + 1, np.zeros(k, dtype=np.int64), leaves, weights=weights, seed=seed, name=f"star_{k}")


def path(n: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, weights=weights, seed=seed, name=f"path_{n}")


def cycle(n: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, weights=weights, seed=seed, name=f"cycle_{n}")


def complete(n: int, *, weights: str = "unit", seed: int = 1) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, weights=weights, seed=seed, name=f"complete_{n}")


def rhs(n: int, k: int = 1, *, seed: int = 2) -> np.ndarray:
    """Standard Gaussian right-hand side(s) with the constant vector projected out.

    Returns float64 [n] for k == 1, else [n][k] (row-major, one column per RHS).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.standard_normal((n, k))
    b -= b.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(b[:, 0]) if k == 1 else np.ascontiguousarray(b)


def serving_mix(count: int, nmin: int, nmax: int, *, seed: int = 5) -> list[Graph]:
    """Graphs of a serving workload: sizes log-uniform in [nmin, nmax] vertices,
    type uniform over 2D grid, 3D grid, Chung-Lu (exponent 2.1, 5 sampled edges
    per vertex) and R-MAT (edge factor 16, scale rounded to the size). Sizes
    are targets: grids round to whole sides, generated graphs keep their
    largest component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            side = max(2, int(round(math.sqrt(n))))
            out.append(grid2d(side, side))
        elif kind == 1:
            side = max(2, int(round(n ** (1.0 / 3.0))))
            out.append(grid3d(side, side, side))
        elif kind == 2:
            out.append(chung_lu(n, m_target=5 * n, seed=1000 + q))
        else:
            out.append(rmat(max(6, int(round(math.log2(n)))), seed=1000 + q))
    return out


# The workloads named by the benchmark, with their fixed seeds.
def workload(name: str) -> Graph:
    if name == "grid2d_64":
        return grid2d(64, 64)
    if name == "chung_lu_1m":
        return chung_lu(1_000_000, exponent=2.1, dmin=1.0, dmax=50000.0, m_target=10_000_000, seed=1)
    if name == "rmat_20":
        return rmat(20, edge_factor=16, seed=1)
    if name == "grid3d_128":
        return grid3d(128, 128, 128)
    raise KeyError(name)
