"""q-state Potts tensor networks on the open square lattice: the construction of
Sec. 7.1 with q states per spin, so every bond has dimension q.

Z = sum over s in {0, .., q-1}^V of prod_{(i,j) in E} exp(beta * J_ij * [s_i == s_j]).
The bond matrix B = exp(beta J [s == s']) = (e^{beta J} - 1) I + 1 1^T is
positive definite for J >= 0; W is its symmetric square root and vertex v
carries t_{E(v)} = sum_i prod_e W^{(e)}_{i, k_e}, legs in ascending
incident-edge-id order.  Only couplings J >= 0 are generated.  These networks
exercise the paths for bond dimensions other than 2.
"""
import numpy as np

from . import graphs, prng


def bond_matrix(beta_j: float, q: int) -> np.ndarray:
    return (np.exp(beta_j) - 1.0) * np.eye(q) + np.ones((q, q))


def bond_sqrt(beta_j: float, q: int) -> np.ndarray:
    """Symmetric W with W W^T = bond_matrix(beta_j, q) (beta_j >= 0)."""
    lam, V = np.linalg.eigh(bond_matrix(beta_j, q))
    return (V * np.sqrt(np.clip(lam, 0.0, None))) @ V.T  # beta_j = 0: rank one


def site_tensors(n_vertices: int, edges: np.ndarray, J: np.ndarray, beta: float, q: int):
    inc = graphs.incident_edges(n_vertices, edges)
    out = []
    for v in range(n_vertices):
        mats = [bond_sqrt(beta * float(J[e]), q) for e in inc[v]]
        t = np.zeros((q,) * len(mats))
        for i in range(q):
            term = np.ones(())
            for W in mats:
                term = np.multiply.outer(term, W[i])
            t = t + term
        out.append(t)
    return out


def lattice2d(Lx: int, Ly: int, beta: float, q: int, couplings: str = "ferro", seed: int = 0):
    """Open Lx x Ly Potts lattice: dict(n, edges, J, beta, q, Lx, Ly, tensors).

    couplings: "ferro" (J = 1) or "uniform" (J ~ U[0.5, 1.5), seeded)."""
    n, edges = graphs.square_lattice(Lx, Ly)
    if couplings == "ferro":
        J = np.ones(len(edges))
    elif couplings == "uniform":
        J = 0.5 + prng.uniform(seed, len(edges))
    else:
        raise ValueError(couplings)
    return dict(n=n, edges=edges, J=J, beta=beta, q=q, Lx=Lx, Ly=Ly,
                tensors=site_tensors(n, edges, J, beta, q))
