"""Seeded synthetic graphs shaped like Force2Vec's workloads.

This module holds input generation only: random graphs, their symmetric CSR
form and a held-out split for link prediction.  It contains none of the
embedding method's arithmetic, so the CUDA path and the CPU oracle can both
be fed from it.

Generators (numpy ``PCG64``, identical output on every platform for a seed):
  * ``erdos_renyi``   G(n, p) undirected graph.
  * ``rmat``          R-MAT (Chakrabarti, Zhan, Faloutsos, SDM'04) directed
                      edges with quadrant probabilities (a, b, c, 1-a-b-c),
                      then symmetrised, de-duplicated, self-loops dropped and
                      vertex ids randomly permuted.  Stands in for the paper's
                      scale-free graphs (Orkut, uk-2005, Table "dataset").
  * ``sbm``           stochastic block model with equal blocks, standing in
                      for graphs with community structure.
  * ``holdout``       removes a fraction of undirected edges (both directions)
                      for link prediction and draws as many non-edge pairs.
  * ``sbm_batch``     many SBM graphs of log-uniform size and random block
                      counts at once (the batched and served workloads), drawn
                      by the C helper gen/sbm.c (xoshiro256** per graph).

All graphs are returned as symmetric CSR with int32 ``row_ptr`` (n+1) and
``col_idx`` (nnz), each row sorted, no self-loops, no duplicates; the
adjacency is 0/1 as in Sec. II-A of the paper.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray            # int32, n + 1
    col_idx: np.ndarray            # int32, nnz
    test_pos: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    test_neg: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.size)

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an int64 array."""
    k = np.sort(np.asarray(keys, dtype=np.int64))
    if k.size:
        k = k[np.concatenate(([True], k[1:] != k[:-1]))]
    return k


def _keys_to_csr(n: int, keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sorted unique undirected keys u*n+v (u<v) -> symmetric CSR, rows sorted.

    Row r holds its smaller neighbours (from the reversed edges) followed by
    its larger ones (from the forward edges), so each row comes out sorted."""
    keys = np.asarray(keys, dtype=np.int64)
    u = keys // n
    v = keys % n
    cnt_f = np.bincount(u, minlength=n).astype(np.int64) if n else np.zeros(0, np.int64)
    cnt_r = np.bincount(v, minlength=n).astype(np.int64) if n else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_f + cnt_r, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    # forward entries (u -> v), already ordered by (u, v)
    fstart = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_f, out=fstart[1:])
    i = np.arange(keys.size, dtype=np.int64)
    col[row_ptr[u] + cnt_r[u] + (i - fstart[u])] = v
    # reversed entries (v -> u), ordered by (v, u)
    rkeys = np.sort(v * n + u)
    rv = rkeys // n
    ru = rkeys % n
    rstart = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_r, out=rstart[1:])
    col[row_ptr[rv] + (i - rstart[rv])] = ru
    return row_ptr.astype(np.int32), col


def _canonical_keys(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    u = u.astype(np.int64)
    v = v.astype(np.int64)
    keep = u != v
    lo = np.minimum(u[keep], v[keep])
    hi = np.maximum(u[keep], v[keep])
    return _sorted_unique(lo * n + hi)


def from_edges(n: int, u, v, name: str = "") -> Graph:
    """Symmetric CSR from an arbitrary edge list (loops and duplicates dropped)."""
    keys = _canonical_keys(n, np.asarray(u), np.asarray(v))
    rp, ci = _keys_to_csr(n, keys)
    return Graph(n, rp, ci, name=name)


def undirected_keys(g: Graph) -> np.ndarray:
    """Sorted keys u*n+v (u<v) of the undirected edges of g."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    dst = g.col_idx.astype(np.int64)
    m = src < dst
    return src[m] * g.n + dst[m]


def erdos_renyi(n: int, p: float | None = None, m: int | None = None, seed: int = 1) -> Graph:
    """G(n, p); if p is None it is chosen so the expected edge count is m."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if p is None:
        p = (m / total) if total else 0.0
    if n <= 20000:
        iu, ju = np.triu_indices(n, k=1)
        sel = rng.random(iu.size) < p
        keys = iu[sel].astype(np.int64) * n + ju[sel]
    else:
        cnt = rng.binomial(total, p)
        keys = np.zeros(0, np.int64)
        while keys.size < cnt:
            need = cnt - keys.size
            u = rng.integers(0, n, size=int(need * 1.1) + 16)
            v = rng.integers(0, n, size=u.size)
            keys = _sorted_unique(np.concatenate([keys, _canonical_keys(n, u, v)]))
        keys = np.sort(rng.permutation(keys)[:cnt])
    rp, ci = _keys_to_csr(n, np.sort(keys))
    return Graph(n, rp, ci, name=f"er-n{n}-p{p:.5f}-seed{seed}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, permute: bool = True,
         chunk: int = 1 << 22) -> Graph:
    """R-MAT graph with n = 2^scale and edge_factor * n directed edges, symmetrised."""
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    ab, abc = a + b, a + b + c
    parts = []
    for lo in range(0, m, chunk):
        cnt = min(chunk, m - lo)
        src = np.zeros(cnt, dtype=np.int64)
        dst = np.zeros(cnt, dtype=np.int64)
        for level in range(scale):
            r = rng.random(cnt)
            bit = np.int64(1) << (scale - 1 - level)
            src += (r >= ab) * bit
            dst += (((r >= a) & (r < ab)) | (r >= abc)) * bit
        keep = src != dst
        src, dst = src[keep], dst[keep]
        parts.append(_sorted_unique(np.minimum(src, dst) * n + np.maximum(src, dst)))
    keys = _sorted_unique(np.concatenate(parts)) if parts else np.zeros(0, np.int64)
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        u = perm[keys // n]
        v = perm[keys % n]
        keys = _sorted_unique(np.minimum(u, v) * n + np.maximum(u, v))
    rp, ci = _keys_to_csr(n, keys)
    return Graph(n, rp, ci, name=f"rmat-s{scale}-ef{edge_factor}-seed{seed}")


def sbm(n: int, blocks: int, p_in: float, p_out: float, seed: int = 1) -> Graph:
    """Stochastic block model: `blocks` near-equal blocks, edge probability
    p_in inside a block and p_out across blocks."""
    rng = np.random.default_rng(seed)
    bounds = np.linspace(0, n, blocks + 1).round().astype(np.int64)
    parts = []
    for i in range(blocks):
        for j in range(i, blocks):
            si = bounds[i + 1] - bounds[i]
            sj = bounds[j + 1] - bounds[j]
            if i == j:
                total = si * (si - 1) // 2
                p = p_in
            else:
                total = si * sj
                p = p_out
            if total <= 0 or p <= 0:
                continue
            cnt = int(rng.binomial(total, p))
            got = np.zeros(0, np.int64)
            while got.size < cnt:
                need = cnt - got.size
                k = int(need * 1.1) + 8
                u = rng.integers(bounds[i], bounds[i + 1], size=k)
                v = rng.integers(bounds[j], bounds[j + 1], size=k)
                got = _sorted_unique(np.concatenate([got, _canonical_keys(n, u, v)]))
            parts.append(rng.permutation(got)[:cnt])
    keys = _sorted_unique(np.concatenate(parts)) if parts else np.zeros(0, np.int64)
    rp, ci = _keys_to_csr(n, keys)
    return Graph(n, rp, ci, name=f"sbm-n{n}-B{blocks}-seed{seed}")


def holdout(g: Graph, frac: float = 0.05, seed: int = 7) -> Graph:
    """Removes `frac` of the undirected edges (both directions) for testing and
    draws the same number of uniform non-edge pairs u != v as negatives."""
    rng = np.random.default_rng(seed)
    keys = undirected_keys(g)
    n_test = int(round(frac * keys.size))
    perm = rng.permutation(keys.size)
    test_keys = np.sort(keys[perm[:n_test]])
    train_keys = np.sort(keys[perm[n_test:]])
    neg = np.zeros(0, np.int64)
    if g.n >= 2:
        while neg.size < n_test:
            need = n_test - neg.size
            u = rng.integers(0, g.n, size=int(need * 1.2) + 16)
            v = rng.integers(0, g.n, size=u.size)
            cand = _canonical_keys(g.n, u, v)
            pos = np.searchsorted(keys, cand)
            pos = np.minimum(pos, max(keys.size - 1, 0))
            is_edge = (keys.size > 0) & (keys[pos] == cand) if keys.size else np.zeros(cand.size, bool)
            cand = cand[~is_edge]
            neg = _sorted_unique(np.concatenate([neg, cand]))
        neg = np.sort(rng.permutation(neg)[:n_test])
    rp, ci = _keys_to_csr(g.n, train_keys)
    pos_pairs = np.stack([test_keys // g.n, test_keys % g.n], axis=1).astype(np.int32)
    neg_pairs = np.stack([neg // g.n, neg % g.n], axis=1).astype(np.int32)
    return Graph(g.n, rp, ci, pos_pairs, neg_pairs, name=g.name + f"-holdout{frac}")


def induced_subgraph(g: Graph, vertices: np.ndarray) -> Graph:
    """Subgraph induced by `vertices`, relabelled 0..len(vertices)-1 in the given order."""
    vertices = np.asarray(vertices, dtype=np.int64)
    remap = np.full(g.n, -1, dtype=np.int64)
    remap[vertices] = np.arange(vertices.size)
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    dst = g.col_idx.astype(np.int64)
    ms = remap[src]
    md = remap[dst]
    keep = (ms >= 0) & (md >= 0) & (ms < md)
    keys = _sorted_unique(ms[keep] * vertices.size + md[keep])
    rp, ci = _keys_to_csr(int(vertices.size), keys)
    return Graph(int(vertices.size), rp, ci, name=g.name + f"-sub{vertices.size}")


def star(n_leaves: int) -> Graph:
    """Vertex 0 joined to vertices 1..n_leaves (a hub row)."""
    u = np.zeros(n_leaves, np.int64)
    v = np.arange(1, n_leaves + 1, dtype=np.int64)
    return from_edges(n_leaves + 1, u, v, name=f"star-{n_leaves}")


def er1000_graph(seed: int = 1) -> Graph:
    """Erdos-Renyi n=1000 with p chosen for ~10,000 undirected edges."""
    return erdos_renyi(1000, m=10000, seed=seed)


def rmat_holdout_graph(seed: int = 1, scale: int = 20, frac: float = 0.05) -> Graph:
    """R-MAT scale-20 (16 * 2^20 directed edges, a=.57, b=c=.19), symmetrised,
    with `frac` of the undirected edges held out."""
    return holdout(rmat(scale, 16, seed=seed), frac=frac, seed=seed + 1000)


@dataclass
class GraphBatch:
    """Many graphs in the concatenated layout of include/f2v_batch.h."""
    n: np.ndarray          # int32 [G]
    d: np.ndarray          # int32 [G] row size of each graph's embedding
    blocks: np.ndarray     # int32 [G]
    seed: np.ndarray       # uint64 [G] embedding seeds
    row_ptr: np.ndarray    # int32, graph g's n[g]+1 entries after graph g-1's
    col_idx: np.ndarray    # int32, local ids
    row_off: np.ndarray = field(default=None)   # int64 [G+1]
    col_off: np.ndarray = field(default=None)   # int64 [G+1]
    name: str = ""

    @property
    def num_graphs(self) -> int:
        return int(self.n.size)

    def graph(self, g: int) -> Graph:
        rp = self.row_ptr[self.row_off[g]:self.row_off[g + 1]]
        ci = self.col_idx[self.col_off[g]:self.col_off[g + 1]]
        return Graph(int(self.n[g]), rp, ci, name=f"{self.name}[{g}]")

    @property
    def nnz(self) -> int:
        return int(self.col_idx.size)


_gen_lib = None


def _gen():
    global _gen_lib
    if _gen_lib is None:
        import ctypes
        from . import build
        lib = ctypes.CDLL(build.build_gen())
        lib.f2v_sbm_begin.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                      ctypes.c_void_p]
        lib.f2v_sbm_begin.restype = ctypes.c_void_p
        lib.f2v_sbm_finish.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.f2v_sbm_finish.restype = None
        _gen_lib = lib
    return _gen_lib


def sbm_graphs(n, blocks, p_in: float, p_out: float, seed: int = 1):
    """Symmetric CSRs of SBM graphs with the given sizes and block counts
    (concatenated layout); returns (row_ptr, col_idx, row_off, col_off)."""
    n = np.ascontiguousarray(n, np.int32)
    blocks = np.ascontiguousarray(blocks, np.int32)
    G = int(n.size)
    nnz = np.zeros(G, np.int64)
    lib = _gen()
    h = lib.f2v_sbm_begin(G, n.ctypes.data, blocks.ctypes.data, float(p_in), float(p_out),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, nnz.ctypes.data)
    if not h:
        raise MemoryError("graph generator out of memory")
    row_off = np.zeros(G + 1, np.int64)
    row_off[1:] = np.cumsum(n.astype(np.int64) + 1)
    col_off = np.zeros(G + 1, np.int64)
    col_off[1:] = np.cumsum(nnz)
    if col_off[-1] >= 2**31 * 64:
        raise ValueError("batch too large")
    row_ptr = np.empty(int(row_off[-1]), np.int32)
    col_idx = np.empty(max(int(col_off[-1]), 1), np.int32)
    lib.f2v_sbm_finish(h, row_ptr.ctypes.data, col_idx.ctypes.data)
    return row_ptr, col_idx[:int(col_off[-1])], row_off, col_off


def sbm_batch(num_graphs: int, seed: int = 1, n_range=(50, 20000), block_range=(2, 16),
              p_in: float = 0.05, p_out: float = 0.002, dims=(2, 16, 64)) -> GraphBatch:
    """The batched workload: `num_graphs` SBM graphs, n log-uniform in
    n_range, block counts uniform in block_range (inclusive), row sizes
    taken round-robin from `dims`, embedding seeds drawn per graph."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    n = np.exp(rng.uniform(lo, hi, num_graphs)).astype(np.int32)
    n = np.clip(n, n_range[0], n_range[1]).astype(np.int32)
    blocks = rng.integers(block_range[0], block_range[1] + 1, num_graphs).astype(np.int32)
    blocks = np.minimum(blocks, n).astype(np.int32)
    d = np.asarray([dims[i % len(dims)] for i in range(num_graphs)], np.int32)
    seeds = rng.integers(1, 2**63, num_graphs, dtype=np.int64).astype(np.uint64)
    rp, ci, roff, coff = sbm_graphs(n, blocks, p_in, p_out, seed=seed)
    return GraphBatch(n, d, blocks, seeds, rp, ci, roff, coff,
                      name=f"sbm-batch-G{num_graphs}-seed{seed}")
