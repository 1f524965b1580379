"""Exact partition functions and dense contractions (test infrastructure).

Plain definitions only:
  * Z of the Ising model as the spin sum of Sec. 7.1,
    Z = sum_s prod_{(i,j) in E} exp(beta J_ij s_i s_j)   (brute force),
  * Z of the q-state Potts model, sum_s prod exp(beta J_ij [s_i == s_j]) (brute force),
  * the row-to-row transfer matrix of an open Lx x Ly lattice (textbook),
  * closed forms for trees and cycles,
  * dense contraction of a whole tensor network with einsum (for tiny cases).
"""
import numpy as np


def ising_logz_bruteforce(n_vertices, edges, J, beta, chunk=1 << 18):
    """ln Z by summing all 2^n spin configurations (n <= 26)."""
    n = int(n_vertices)
    if n > 26:
        raise ValueError("brute force limited to 26 spins")
    edges = np.asarray(edges, dtype=np.int64)
    J = np.asarray(J, dtype=np.float64)
    total = 2 ** n
    parts = []
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        spins = 1.0 - 2.0 * ((idx[:, None] >> np.arange(n)[None, :]) & 1)
        energy = (spins[:, edges[:, 0]] * spins[:, edges[:, 1]]) @ J
        a = beta * energy
        m = a.max()
        parts.append(m + np.log(np.exp(a - m).sum()))
    parts = np.asarray(parts)
    m = parts.max()
    return float(m + np.log(np.exp(parts - m).sum()))


def potts_logz_bruteforce(n_vertices, edges, J, beta, q, chunk=1 << 17):
    """ln Z of the q-state Potts model by summing all q^n configurations."""
    n = int(n_vertices)
    if q ** n > 1 << 24:
        raise ValueError("brute force limited to 2^24 configurations")
    edges = np.asarray(edges, dtype=np.int64)
    J = np.asarray(J, dtype=np.float64)
    total = q ** n
    place = q ** np.arange(n, dtype=np.int64)
    parts = []
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        s = (idx[:, None] // place[None, :]) % q
        energy = (s[:, edges[:, 0]] == s[:, edges[:, 1]]).astype(np.float64) @ J
        a = beta * energy
        m = a.max()
        parts.append(m + np.log(np.exp(a - m).sum()))
    parts = np.asarray(parts)
    m = parts.max()
    return float(m + np.log(np.exp(parts - m).sum()))


def ising_logz_transfer_matrix(Lx, Ly, edges, J, beta):
    """ln Z of an open Lx x Ly lattice by row-to-row transfer matrices.

    Vertex id = x * Ly + y.  Works for any couplings (Ly <= 14).
    """
    if Ly > 14:
        raise ValueError("transfer matrix limited to width 14")
    Jh = np.zeros((Lx, max(Ly - 1, 0)))
    Jv = np.zeros((max(Lx - 1, 0), Ly))
    for e, (u, v) in enumerate(np.asarray(edges)):
        u, v = int(min(u, v)), int(max(u, v))
        x, y = divmod(u, Ly)
        if v == u + 1 and y + 1 < Ly:
            Jh[x, y] += J[e]
        elif v == u + Ly:
            Jv[x, y] += J[e]
        else:
            raise ValueError("edge is not a lattice edge")
    states = np.arange(2 ** Ly)
    s = 1.0 - 2.0 * ((states[:, None] >> np.arange(Ly)[None, :]) & 1)
    def row_log_weight(x):
        if Ly == 1:
            return np.zeros(len(states))
        return beta * (s[:, :-1] * s[:, 1:]) @ Jh[x]
    logscale = 0.0
    phi = np.exp(row_log_weight(0))
    for x in range(Lx - 1):
        V = np.exp(beta * (s * Jv[x][None, :]) @ s.T)
        phi = (phi @ V) * np.exp(row_log_weight(x + 1))
        m = phi.max()
        logscale += np.log(m)
        phi = phi / m
    return float(np.log(phi.sum()) + logscale)


def ising_logz_tree(J, beta):
    """Z = 2 prod_e 2 cosh(beta J_e) for any tree (n = |E| + 1 spins)."""
    J = np.asarray(J, dtype=np.float64)
    return float(np.log(2.0) + np.sum(np.log(2.0 * np.cosh(beta * J))))


def ising_logz_cycle(J, beta):
    """Z = 2^n (prod cosh(beta J_e) + prod sinh(beta J_e)) for an n-cycle."""
    J = np.asarray(J, dtype=np.float64)
    n = len(J)
    return float(n * np.log(2.0) + np.log(np.prod(np.cosh(beta * J)) + np.prod(np.sinh(beta * J))))


def contract_network(tensors, legs, open_order=None):
    """Dense contraction of a whole tensor network.

    tensors[i] has one axis per label in legs[i]; a label shared by two tensors
    is summed, a label that appears once is open.  The result has its open
    labels in ``open_order`` (default: ascending).  Only for tiny networks.
    """
    count = {}
    for ls in legs:
        for l in ls:
            count[l] = count.get(l, 0) + 1
    open_labels = sorted(l for l, c in count.items() if c == 1)
    if open_order is not None:
        if sorted(open_order) != open_labels:
            raise ValueError("open_order must list the open labels")
        open_labels = list(open_order)
    relabel = {l: i for i, l in enumerate(sorted(count))}
    args = []
    for t, ls in zip(tensors, legs):
        args.append(t)
        args.append([relabel[l] for l in ls])
    args.append([relabel[l] for l in open_labels])
    return np.einsum(*args, optimize="greedy")
