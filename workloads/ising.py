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


def graph_workload(n: int, edges, J, beta: float):
    """Ising workload on an arbitrary graph: dict(n, edges, J, beta, tensors)."""
    edges = np.asarray(edges, dtype=np.int64)
    return dict(n=n, edges=edges, J=np.asarray(J, dtype=np.float64), beta=beta,
                tensors=site_tensors(n, edges, np.asarray(J, dtype=np.float64), beta))


def cubic(Lx: int, Ly: int, Lz: int, beta: float):
    """Open Lx x Ly x Lz ferromagnet (J = 1).  Vertex id (x*Ly + y)*Lz + z, so
    the fibres along z are runs of Lz consecutive ids and a part of k fibres
    is a run of k*Lz ids (parts taken in id order: a row-wise traversal of the
    Lx x Ly array of fibres, Sec. 7.3)."""
    n, edges = graphs.cubic_lattice(Lx, Ly, Lz)
    w = graph_workload(n, edges, np.ones(len(edges)), beta)
    w.update(Lx=Lx, Ly=Ly, Lz=Lz)
    return w


def random_regular(n: int, degree: int, beta: float, seed: int):
    """Random regular graph with J = +-1 (equal probability), vertices
    renumbered along the recursive-bisection linear ordering (Sec. 7.3), so a
    part of k tensors is a run of k consecutive ids."""
    edges = graphs.random_regular(n, degree, seed)
    edges = graphs.relabel(edges, graphs.bisection_order(n, edges))
    J = np.where(prng.uniform(seed + 1, len(edges)) < 0.5, 1.0, -1.0)
    w = graph_workload(n, edges, J, beta)
    w.update(degree=degree)
    return w


CONFIG3 = dict(L=6, betas=(0.20, 0.2217, 0.25), chis=(16, 32, 64), fibres=(1, 2, 3))
CONFIG4 = dict(n_inst=256, n_range=(40, 200), degree=3, beta=0.3, chis=(16, 32, 48, 64))
CONFIG5 = dict(n_range=(100, 300), degree=4, beta=0.25, chi=32)


def config4_instance(i: int):
    """Instance i of the batched random 3-regular workload (seed 4*10**6 + i):
    n uniform in [40, 200] (rounded up to even), chi uniform in {16, 32, 48, 64}."""
    seed = 4 * 10**6 + i
    lo, hi = CONFIG4["n_range"]
    n = int(prng.randint(seed, 1, lo, hi, offset=0)[0])
    n += n % 2
    chi = int(CONFIG4["chis"][int(prng.randint(seed, 1, 0, 3, offset=1)[0])])
    w = random_regular(n, CONFIG4["degree"], CONFIG4["beta"], seed)
    w.update(chi=chi)
    return w


def config5_instance(i: int):
    """Instance i of the random 4-regular workload (seed 5*10**6 + i):
    n uniform in [100, 300]."""
    seed = 5 * 10**6 + i
    lo, hi = CONFIG5["n_range"]
    n = int(prng.randint(seed, 1, lo, hi, offset=0)[0])
    return random_regular(n, CONFIG5["degree"], CONFIG5["beta"], seed)
