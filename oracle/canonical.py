"""Canonicalisation-based truncation with the full environment (TEST INFRASTRUCTURE).

An independent algorithm used to PIN the density-matrix oracle below the exact
rank.  Sec. 2.2 (low-rank problem with an environment, and the MPO-MPS review)
states that the canonicalisation route and the density-matrix route give the
same output: the leading left singular vectors of E A B equal the leading
eigenvectors of the Gram matrix (E A B)(E A B)^T.

For every row contraction this module
  1. contracts the boundary tree TN with the next row column by column
     (the "application" step: an MPS whose bonds are the products of the
     boundary bond and the row's horizontal bond),
  2. orthogonalises every tensor towards the leftmost tree vertex with QR
     factorisations (canonical_form of Def. "Canonical form"),
  3. sweeps from the left: the rank-r truncated SVD of the non-orthogonal
     centre gives U_v and pushes S V^T into the next vertex
     (Algorithm canonize on the MPS tree, post-order = left to right).

It shares no code with ``dmtree``: its own tensor bookkeeping, no density
matrices and no eigensolver.  Rank per vertex: min(chi, rows, cols of the
centre, product of open-leg dims to the right).
"""
import numpy as np


def _row_tensors(workload):
    """Site tensors as arrays indexed [up, left, right, down] (dim 1 if absent),
    unit Frobenius norm; returns (T, sum of log norms)."""
    Lx, Ly, edges = workload["Lx"], workload["Ly"], np.asarray(workload["edges"])
    nbr = {}
    for e, (u, v) in enumerate(edges):
        nbr.setdefault(int(u), []).append((e, int(v)))
        nbr.setdefault(int(v), []).append((e, int(u)))
    T, lsum = {}, 0.0
    for v, t in enumerate(workload["tensors"]):
        x, y = divmod(v, Ly)
        where = {v - Ly: 0, v - 1: 1, v + 1: 2, v + Ly: 3}
        axes = [where[w] for _, w in sorted(nbr.get(v, []))]
        shape = [1, 1, 1, 1]
        for ax, slot in enumerate(axes):
            shape[slot] = t.shape[ax]
        order = sorted(range(len(axes)), key=lambda i: axes[i])
        t4 = np.transpose(np.asarray(t, float), order).reshape(shape)
        nrm = np.linalg.norm(t4)
        lsum += np.log(nrm)
        T[(x, y)] = t4 / nrm
    return T, lsum


def _apply_row(mps, row):
    """MPS sites (l, p, r) times row tensors (up, left, right, down) -> MPS
    with bonds (l*left, down, r*right)."""
    out = []
    for A, t in zip(mps, row):
        s = np.einsum("apb,plrd->aldbr", A, t)
        a, l, dd, b, r = s.shape
        out.append(s.reshape(a * l, dd, b * r))
    return out


def _truncate(mps, chi):
    """Canonicalise towards the left end, then truncate left to right.

    The leftmost tree vertex holds the two first legs, so the first two sites
    are merged before truncation; the result is returned in the same layout
    (site 0: (1, d0, d0) identity, site v: (r_{v-1}, d_v, r_v))."""
    n = len(mps)
    sites = [s.copy() for s in mps]
    # merge the first two sites: vertex 1 of the MPS tree holds x_0 and x_1
    a0, d0, _ = sites[0].shape
    _, d1, b1 = sites[1].shape
    first = np.einsum("aeb,bfc->aefc", sites[0], sites[1]).reshape(a0, d0 * d1, b1)
    sites = [first] + sites[2:]
    dims = [d0 * d1] + [s.shape[1] for s in sites[1:]]
    m = len(sites)
    # right-orthogonalise sites m-1..1 (QR of the transposed matricisation)
    for k in range(m - 1, 0, -1):
        A = sites[k]
        l, p, r = A.shape
        Q, R = np.linalg.qr(A.reshape(l, p * r).T)
        sites[k] = Q.T.reshape(Q.shape[1], p, r)
        sites[k - 1] = np.einsum("apb,cb->apc", sites[k - 1], R)
    # left-to-right truncated SVD
    out = []
    carry = np.ones((1, 1))
    for k in range(m - 1):
        C = np.einsum("ia,apb->ipb", carry, sites[k])
        i, p, b = C.shape
        C = C.reshape(i * p, b)
        beyond = int(np.prod(dims[k + 1:]))
        Uf, S, Vt = np.linalg.svd(C, full_matrices=False)
        r = min(chi, C.shape[0], C.shape[1], beyond, len(S))
        out.append(Uf[:, :r].reshape(i, p, r))
        carry = S[:r, None] * Vt[:r]
    root = np.einsum("ia,apb->ipb", carry, sites[m - 1])
    nrm = np.linalg.norm(root)
    out.append(root / nrm)
    # split vertex 1 back into an identity site and a (d0, d1, r) site
    U1 = out[0].reshape(d0, d1, -1)
    ident = np.eye(d0).reshape(1, d0, d0)
    return [ident, U1] + out[1:], float(np.log(nrm))


def partitioned_contract_rows_canonical(workload, chi):
    """ln Z of a 2D lattice network, rows as partitions, canonicalisation route."""
    Lx, Ly = workload["Lx"], workload["Ly"]
    T, logscale = _row_tensors(workload)
    # row 0 as an MPS: (left, down, right)
    mps = [np.transpose(T[(0, y)][0], (0, 2, 1)) for y in range(Ly)]
    for x in range(1, Lx):
        mps = _apply_row(mps, [T[(x, y)] for y in range(Ly)])
        if x == Lx - 1:
            vec = np.ones((1, 1))
            for A in mps:
                vec = vec @ A[:, 0, :]
                mx = np.max(np.abs(vec))
                logscale += np.log(mx)
                vec = vec / mx
            return float(np.log(vec[0, 0]) + logscale)
        mps, ln = _truncate(mps, chi)
        logscale += ln
