"""Exact partition functions and dense contractions (test infrastructure).

Plain definitions only:
  * Z of the Ising model as the spin sum of Sec. 7.1,
    Z = sum_s prod_{(i,j) in E} exp(beta J_ij s_i s_j)   (brute force),
  * Z of the q-state Potts model, sum_s prod exp(beta J_ij [s_i == s_j]) (brute force),
  * the row-to-row transfer matrix of an open Lx x Ly lattice (textbook),
  * closed forms for trees and cycles,
  * the Kac-Ward determinant of the open square lattice (any couplings, zero field),
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


def ising_logz_kac_ward(Lx, Ly, edges, J, beta):
    """ln Z of the zero-field Ising model on the open Lx x Ly lattice, any
    couplings, by the Kac-Ward determinant (Kac & Ward 1952; planar graph drawn
    with straight edges):  Z = 2^n prod_e cosh(beta J_e) det(I - T)^(1/2), where
    T is indexed by directed edges, T[(u->v), (v->w)] = tanh(beta J_vw) e^{i a/2}
    for w != u and a is the signed turning angle from u->v to v->w.  The root of
    the determinant is the generating function of the even subgraphs (the
    high-temperature expansion).  Vertex x * Ly + y is drawn at (y, x).
    """
    edges = np.asarray(edges, dtype=np.int64)
    J = np.asarray(J, dtype=np.float64)
    n, E = Lx * Ly, len(edges)
    pos = np.stack([np.arange(n) % Ly, np.arange(n) // Ly], axis=1).astype(np.float64)
    tail = np.empty(2 * E, dtype=np.int64)
    head = np.empty(2 * E, dtype=np.int64)
    tail[0::2], head[0::2] = edges[:, 0], edges[:, 1]
    tail[1::2], head[1::2] = edges[:, 1], edges[:, 0]
    leaving = [[] for _ in range(n)]
    for d in range(2 * E):
        leaving[int(tail[d])].append(d)
    t = np.tanh(beta * J)
    T = np.zeros((2 * E, 2 * E), dtype=np.complex128)
    for d in range(2 * E):
        u, v = int(tail[d]), int(head[d])
        a = pos[v] - pos[u]
        for d2 in leaving[v]:
            w = int(head[d2])
            if w == u:
                continue
            b = pos[w] - pos[v]
            ang = np.arctan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1])
            T[d, d2] = t[d2 // 2] * np.exp(0.5j * ang)
    sign, logabs = np.linalg.slogdet(np.eye(2 * E) - T)
    if abs(sign - 1.0) > 1e-8:
        raise ArithmeticError("Kac-Ward determinant is not real positive")
    return float(n * np.log(2.0) + np.sum(np.log(np.cosh(beta * J))) + 0.5 * logabs)


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
