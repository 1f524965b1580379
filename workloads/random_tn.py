"""Random tensor networks on the open square lattice (Sec. 7 workloads): every
site tensor entry is an i.i.d. uniform variable on [alpha, 1], alpha in [-1, 0].
Bond dimension 2, legs in ascending incident-edge-id order, vertex id x * Ly + y.
Entries come from the seeded counter-based generator, instance by instance.
"""
import numpy as np

from . import graphs, prng


def lattice2d(Lx: int, Ly: int, alpha: float, seed: int = 0):
    """dict(n, edges, alpha, Lx, Ly, tensors) with U[alpha, 1] entries."""
    if not -1.0 <= alpha <= 0.0:
        raise ValueError("alpha must lie in [-1, 0]")
    n, edges = graphs.square_lattice(Lx, Ly)
    inc = graphs.incident_edges(n, edges)
    tensors, off = [], 0
    for v in range(n):
        shape = (2,) * len(inc[v])
        size = int(np.prod(shape))
        u = prng.uniform(seed, size, off)
        off += size
        tensors.append((alpha + (1.0 - alpha) * u).reshape(shape))
    return dict(n=n, edges=edges, alpha=alpha, Lx=Lx, Ly=Ly, tensors=tensors)
