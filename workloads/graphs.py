"""Graph generators for the synthetic workloads.

Edges are numbered in a fixed order; a site tensor holds its legs in ascending
incident-edge-id order (row-major, last leg fastest).  Every edge has dim 2.
"""
import numpy as np


def square_lattice(Lx: int, Ly: int):
    """Open Lx x Ly lattice.  Vertex id = x * Ly + y (x = row, y = column).

    Edges are enumerated vertex by vertex in id order: first the edge to the
    right neighbour (x, y+1), then the edge to the neighbour below (x+1, y).
    Returns (n_vertices, edges) with edges an (E, 2) int array, u < v.
    """
    edges = []
    for x in range(Lx):
        for y in range(Ly):
            v = x * Ly + y
            if y + 1 < Ly:
                edges.append((v, v + 1))
            if x + 1 < Lx:
                edges.append((v, v + Ly))
    return Lx * Ly, np.asarray(edges, dtype=np.int64).reshape(-1, 2)


def cubic_lattice(Lx: int, Ly: int, Lz: int):
    """Open Lx x Ly x Lz lattice.  Vertex id = (x * Ly + y) * Lz + z.

    Edges per vertex in id order: +z, then +y, then +x neighbour.
    """
    edges = []
    for x in range(Lx):
        for y in range(Ly):
            for z in range(Lz):
                v = (x * Ly + y) * Lz + z
                if z + 1 < Lz:
                    edges.append((v, v + 1))
                if y + 1 < Ly:
                    edges.append((v, v + Lz))
                if x + 1 < Lx:
                    edges.append((v, v + Ly * Lz))
    return Lx * Ly * Lz, np.asarray(edges, dtype=np.int64).reshape(-1, 2)


def incident_edges(n_vertices: int, edges: np.ndarray):
    """For every vertex, the ascending list of its incident edge ids."""
    inc = [[] for _ in range(n_vertices)]
    for e, (u, v) in enumerate(edges):
        inc[int(u)].append(e)
        inc[int(v)].append(e)
    return [sorted(lst) for lst in inc]


def random_regular(n: int, degree: int, seed: int, max_attempts: int = 10000):
    """Connected simple random ``degree``-regular graph on n vertices.

    Configuration model: the n * degree stubs are shuffled (Fisher-Yates driven
    by the counter-based generator, one block of uniforms per attempt) and
    paired in order; an attempt with a self loop, a repeated pair or more than
    one connected component is rejected and the next attempt draws again.
    Returns an (E, 2) int array, u < v, rows sorted.
    """
    from . import prng
    if (n * degree) % 2 or degree >= n:
        raise ValueError("need n * degree even and degree < n")
    m = n * degree
    for attempt in range(max_attempts):
        stubs = np.repeat(np.arange(n, dtype=np.int64), degree)
        u = prng.uniform(seed, m, offset=attempt * m)
        for i in range(m - 1, 0, -1):
            j = min(int(u[i] * (i + 1)), i)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        pairs = np.sort(stubs.reshape(-1, 2), axis=1)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        keyed = pairs[:, 0] * n + pairs[:, 1]
        if len(np.unique(keyed)) != len(keyed):
            continue
        if not _connected(n, pairs):
            continue
        order = np.lexsort((pairs[:, 1], pairs[:, 0]))
        return pairs[order]
    raise RuntimeError("no simple connected graph found")


def _connected(n: int, edges) -> bool:
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    seen = [False] * n
    stack = [0]
    seen[0] = True
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if not seen[y]:
                seen[y] = True
                stack.append(y)
    return all(seen)


def _bfs_order(adj, start, inside):
    """Breadth-first order from start within the vertex set ``inside``,
    neighbours taken in ascending id."""
    seen = {start}
    out = [start]
    head = 0
    while head < len(out):
        x = out[head]
        head += 1
        for y in adj[x]:
            if y in inside and y not in seen:
                seen.add(y)
                out.append(y)
    return out


def _bisect(adj, S):
    """Split the sorted vertex list S into halves (floor(|S|/2), rest) with a
    small cut: breadth-first growth from a pseudo-peripheral vertex, then
    Kernighan-Lin pair swaps while one strictly lowers the cut."""
    inside = set(S)
    start = S[0]
    for _ in range(2):                       # two sweeps to a far vertex
        bfs = _bfs_order(adj, start, inside)
        start = bfs[-1]
    bfs = _bfs_order(adj, start, inside)
    rest = [v for v in S if v not in set(bfs)]
    seq = bfs + rest
    half = len(S) // 2
    A, B = set(seq[:half]), set(seq[half:])
    for _ in range(4 * len(S)):
        def gain_of(x, own):
            ext = sum(1 for y in adj[x] if y in inside and y not in own)
            inn = sum(1 for y in adj[x] if y in own)
            return ext - inn
        gA = {a: gain_of(a, A) for a in A}
        gB = {b: gain_of(b, B) for b in B}
        best, pick = 0, None
        for a in sorted(A):
            for b in sorted(B):
                w = sum(1 for y in adj[a] if y == b)
                g = gA[a] + gB[b] - 2 * w
                if g > best:
                    best, pick = g, (a, b)
        if pick is None:
            break
        a, b = pick
        A.remove(a); B.add(a)
        B.remove(b); A.add(b)
    return sorted(A), sorted(B)


def bisection_order(n: int, edges):
    """Linear ordering of the vertices by recursive bisection (the heuristic
    the paper uses to order vertices of random regular graphs, Sec. 7.3)."""
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(edges):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    for lst in adj:
        lst.sort()

    def rec(S):
        if len(S) <= 2:
            return list(S)
        A, B = _bisect(adj, S)
        return rec(A) + rec(B)

    return rec(list(range(n)))


def relabel(edges, order):
    """Renumber vertices so that order[i] becomes vertex i; returns the edge
    array (u < v, rows sorted)."""
    new = np.empty(len(order), dtype=np.int64)
    new[np.asarray(order, dtype=np.int64)] = np.arange(len(order))
    e = new[np.asarray(edges, dtype=np.int64)]
    e = np.sort(e, axis=1)
    idx = np.lexsort((e[:, 1], e[:, 0]))
    return e[idx]
