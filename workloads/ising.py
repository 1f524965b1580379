"""Ising-model tensor networks (the paper's Sec. 7.1 construction).

Z = sum over spins s in {+1,-1}^V of prod_{(i,j) in E} exp(beta * J_ij * s_i * s_j).
Spin index 0 is s = +1.  Each vertex v carries t_{E(v)} = sum_i prod_e W^{(v,e)}_{i, k_e}
with W the symmetric square root of the 2x2 bond matrix B(beta) (Sec. 7.1).

For a negative coupling (outside the paper, which uses J = 1) the lower-id end of
the edge takes W(beta|J|) and the higher-id end takes X W(beta|J|) (rows swapped),
so that W_u W_v^T = B(beta J) with a real square root.
"""
import numpy as np

from . import graphs, prng


def bond_sqrt(beta_j: float) -> np.ndarray:
    """Symmetric W with W W^T = [[e^{bJ}, e^{-bJ}], [e^{-bJ}, e^{bJ}]] for bJ >= 0."""
    c = np.sqrt(np.cosh(beta_j))
    s = np.sqrt(np.sinh(beta_j))
    return np.array([[c + s, c - s], [c - s, c + s]]) / np.sqrt(2.0)


def site_tensors(n_vertices: int, edges: np.ndarray, J: np.ndarray, beta: float):
    """Dense site tensors, legs in ascending incident-edge-id order, dims 2."""
    inc = graphs.incident_edges(n_vertices, edges)
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    out = []
    for v in range(n_vertices):
        mats = []
        for e in inc[v]:
            u, w = int(edges[e][0]), int(edges[e][1])
            W = bond_sqrt(beta * abs(float(J[e])))
            if J[e] < 0 and v == max(u, w):
                W = X @ W
            mats.append(W)
        t = np.zeros((2,) * len(mats))
        for i in range(2):
            term = np.ones(())
            for W in mats:
                term = np.multiply.outer(term, W[i])
            t = t + term
        out.append(t)
    return out


def lattice2d(Lx: int, Ly: int, beta: float, couplings: str = "ferro", seed: int = 0):
    """2D open lattice workload: returns dict(n, edges, J, beta, tensors)."""
    n, edges = graphs.square_lattice(Lx, Ly)
    if couplings == "ferro":
        J = np.ones(len(edges))
    elif couplings == "gauss":
        J = prng.normal(seed, len(edges))
    elif couplings == "pm1":
        J = np.where(prng.uniform(seed, len(edges)) < 0.5, 1.0, -1.0)
    else:
        raise ValueError(couplings)
    return dict(n=n, edges=edges, J=J, beta=beta, Lx=Lx, Ly=Ly,
                tensors=site_tensors(n, edges, J, beta))


# Workload recipes.  Config numbering follows the benchmark's list of configs.
CONFIG1 = dict(Lx=6, Ly=6, beta=0.44, couplings="ferro", chi=16)
CONFIG2 = dict(Lx=32, Ly=32, beta=0.5, couplings="gauss", chis=(32, 64))


def config2_instance(i: int, Lx: int = 32, Ly: int = 32):
    """Instance i of the 32x32 Gaussian spin glass (seed = 2 * 10**6 + i)."""
    return lattice2d(Lx, Ly, CONFIG2["beta"], "gauss", seed=2 * 10**6 + i)
