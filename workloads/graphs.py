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
