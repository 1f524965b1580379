"""FP64 oracle of the density-matrix tree approximation (TEST INFRASTRUCTURE).

Plain restatement of the paper's method for the boundary case used by the
lattice workloads:

  * partitioned_contract (Algorithm partitioned_contract, Sec. 3.2) with the
    partition V_i = row i of an open 2D lattice and the maximally unbalanced
    path ((V_1, V_2), V_3), ... (Sec. 7.3: lattices are contracted along a
    linear sequence of partitions).  Every contraction except the last one has
    open edges and is approximated; the last one closes the network.
  * approx_tensor_network (Algorithm approx_tensor_network, Sec. 6): for rows
    the edge-set ordering already equals the reference ordering, so the
    Kendall-Tau distance d is 0 and exactly one density-matrix pass runs.
  * density_matrix_alg (Algorithm density_matrix_alg, Sec. 5) on the MPS tree
    of Def. "MPS tree" (App. C): leaves x_0..x_{n-1} are the n open edges in
    column order; non-leaf vertex 1 joins x_0 and x_1, vertex v >= 2 joins
    vertex v-1 and x_v, vertex n-1 is the root.
  * the embedding phi puts the tensors of column c at tree vertex max(c, 1),
    i.e. "contract T(v) first" (Sec. 5.3, one valid contraction path).  By
    Def. "density matrix" each L_v is the whole current network matricised on
    A_v, so phi only changes the cost, never the result.
  * memoisation of Eq. (dm_cache): the root-side density matrices
    dm(v+1, v) are computed once, from the root end, and reused.

Readings where the paper is silent (each listed in the design notes):
  * rank: leading_eigenvectors(L_v, chi) keeps
        r_v = min(chi, dim A_v, dim B_v, prod of open-leg dims beyond v);
    the last three bound rank(L_v) structurally, so only exactly-zero
    eigenvalues are ever dropped beyond chi.
  * eigenvalues sorted descending; each kept eigenvector is signed so that its
    largest-magnitude entry (first on ties) is positive.
  * normalisation: every site tensor is scaled to unit Frobenius norm, every
    root tensor M_r is scaled to unit norm, the logs go to an FP64 log-scale;
    memoised density matrices are rescaled to max-abs 1 (eigenvectors are
    scale invariant).
  * branch: the direct branch when dim A_v <= dim B_v, else the QR-SVD branch
    (Algorithm density_matrix_alg, both are mathematically equal).
"""
import numpy as np



# ---------------------------------------------------------------- site tensors

def lattice_site_tensors(tensors, n_vertices, edges, Lx, Ly):
    """Return T[x][y] with legs (up, left, right, down), dim 1 where absent,
    each scaled to unit Frobenius norm, plus the summed log norms."""
    inc = [[] for _ in range(n_vertices)]
    for e, (u, v) in enumerate(np.asarray(edges)):
        inc[int(u)].append((e, int(v)))
        inc[int(v)].append((e, int(u)))
    logscale = 0.0
    T = [[None] * Ly for _ in range(Lx)]
    for x in range(Lx):
        for y in range(Ly):
            v = x * Ly + y
            legs = sorted(inc[v])                   # ascending edge id = axis order
            t = np.asarray(tensors[v], dtype=np.float64)
            role = []
            for _, w in legs:
                if w == v - Ly:
                    role.append(0)                  # up
                elif w == v - 1:
                    role.append(1)                  # left
                elif w == v + 1:
                    role.append(2)                  # right
                elif w == v + Ly:
                    role.append(3)                  # down
                else:
                    raise ValueError("not a square lattice")
            full = [1, 1, 1, 1]
            for ax, rl in enumerate(role):
                full[rl] = t.shape[ax]
            perm = np.argsort(role)
            t4 = np.transpose(t, perm).reshape(full)
            nrm = np.linalg.norm(t4)
            logscale += np.log(nrm)
            T[x][y] = t4 / nrm
    return T, logscale


# ------------------------------------------------------- density_matrix_alg

def _top_eigenvectors(L, r):
    """leading_eigenvectors(L, r): r eigenvectors of the largest eigenvalues
    (descending), each signed so that its largest-|.| entry is positive."""
    lam, V = np.linalg.eigh(L)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    V = V[:, order[:r]]
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return lam, V


def density_matrix_alg(blocks, chi, trace=None, force_branch=None):
    """Algorithm density_matrix_alg on an MPS tree with n leaves.

    ``blocks[v]`` (v = 1..n-1) is the contraction of the tensors embedded at
    tree vertex v (``blocks[0]`` is unused):
        blocks[1]    : (d_0, d_1, D_1)      rows: leaves x_0, x_1
        blocks[v]    : (D_{v-1}, d_v, D_v)  2 <= v <= n-2
        blocks[n-1]  : (D_{n-2}, d_{n-1}, 1)  (root, no parent)
    D_v is the dimension of the tree edge (v, v+1) before truncation.

    Returns (U, M_r, lognorm): U[v] (v = 1..n-2) are the orthonormal output
    tensors as matrices (dim A_v x r_v), M_r the unit-norm root tensor
    (r_{n-2} x d_{n-1}) and lognorm = ln ||M_r|| before scaling.
    """
    n = len(blocks)
    if n < 3:
        raise ValueError("need at least 3 open legs")
    d = [None] * n
    d[0], d[1] = blocks[1].shape[0], blocks[1].shape[1]
    for v in range(2, n):
        d[v] = blocks[v].shape[1]
    # Memoised root-side density matrices, Eq. (dm_cache):
    #   dm(v+1, v) = M^{(v+1)} (dm(v+2, v+1) (x) I_{x_{v+1}}) M^{(v+1)T},
    # with M^{(v+1)} the block at v+1 matricised with edge (v, v+1) as row.
    dm_parent = [None] * n
    dm_parent[n - 1] = np.ones((1, 1))               # nothing beyond the root
    for v in range(n - 2, 0, -1):
        Bk = blocks[v + 1]                           # (D_v, d_{v+1}, D_{v+1})
        env = dm_parent[v + 1]                       # dm(v+2, v+1): (D_{v+1}, D_{v+1})
        # the identity on leaf x_{v+1} in the Kronecker product = a sum over it
        L = sum(Bk[:, e, :] @ env @ Bk[:, e, :].T for e in range(Bk.shape[1]))
        dm_parent[v] = L / np.max(np.abs(L))
    # Post-order traversal of the MPS tree: vertices 1, 2, ..., n-2, then root.
    U = [None] * n
    P = None                                         # U_{v-1}^T folded into T'(v)
    for v in range(1, n - 1):
        # M_v: contraction of T'(v) with A_v (uncontracted edges) as rows and
        # B_v (the edge to the parent) as columns.
        if v == 1:
            M = blocks[1].reshape(d[0] * d[1], -1)
        else:
            M = np.tensordot(P, blocks[v], axes=(1, 0)).reshape(P.shape[0] * d[v], -1)
        dimA, dimB = M.shape
        beyond = int(np.prod(d[v + 1:]))             # open legs on the parent side
        chi_v = chi(v) if callable(chi) else chi     # per-edge ranks: chi(v)
        r = min(chi_v, dimA, dimB, beyond)
        env = dm_parent[v]                           # L_u = dm(parent(v), v)
        direct = dimA <= dimB if force_branch is None else force_branch == "direct"
        if direct:
            L = M @ env @ M.T                        # L_v = M_v L_u M_v^T
            L = 0.5 * (L + L.T)
            lam, Uv = _top_eigenvectors(L, r)
        else:
            # QR-SVD branch: M_v = Q_v R_v, leading singular vectors of
            # R_v L_u R_v^T, U_v = Q_v U_hat.
            Q, Rq = np.linalg.qr(M)
            Lhat = Rq @ env @ Rq.T
            Lhat = 0.5 * (Lhat + Lhat.T)
            lam, Uh = _top_eigenvectors(Lhat, r)
            Uv = Q @ Uh
            for j in range(Uv.shape[1]):
                i = int(np.argmax(np.abs(Uv[:, j])))
                if Uv[i, j] < 0:
                    Uv[:, j] = -Uv[:, j]
            L = None
        U[v] = Uv
        if trace is not None:
            trace.append(dict(v=v, M=M, env=env, L=L, lam=lam, U=Uv, r=r, direct=direct))
        # Fold T'(v) and U_v^T into the parent: the parent now sees P = U_v^T M_v.
        P = Uv.T @ M
    # Root: M_r = contraction of T'(root).
    Mr = np.tensordot(P, blocks[n - 1], axes=(1, 0)).reshape(P.shape[0], d[n - 1])
    nrm = np.linalg.norm(Mr)
    return U, Mr / nrm, float(np.log(nrm))


# ------------------------------------------------- partitioned_contract (rows)

def _blocks_first_pair(T0, T1):
    """Blocks for contracting rows 0 and 1 (the first contraction on the path).

    tn(V_1) is row 0 itself; its column-c tensor and the row-1 tensor of the
    same column are embedded at tree vertex max(c, 1).
    """
    Ly = len(T0)
    blocks = [None] * Ly
    # Column tensors of a row pair: S_c(hl, d, hr) = sum_p T0(1,hl0,hr0,p) T1(p,hl1,hr1,d)
    pair = []
    for c in range(Ly):
        a, b = T0[c][0], T1[c]                       # a: (hl0, hr0, p); b: (p, hl1, hr1, d)
        s = np.einsum("lrp,pmqd->lmdrq", a, b)       # (hl0, hl1, d, hr0, hr1)
        sh = s.shape
        pair.append(s.reshape(sh[0] * sh[1], sh[2], sh[3] * sh[4]))
    blocks[1] = np.einsum("xeb,bfc->efc", pair[0], pair[1])  # column 0 has left bond 1
    for c in range(2, Ly):
        blocks[c] = pair[c]
    return blocks


def _blocks_absorb_row(U, Mr, Trow):
    """Blocks for contracting the current tree TN {U_v, M_r} with one row.

    U[1] has legs (x_0 x_1, k_1); U[v] (x_v with k_{v-1} first: (k_{v-1} x_v, k_v));
    the row tensors of columns 0, 1 join U[1] at vertex 1, column c joins U[c].
    """
    Ly = len(Trow)
    blocks = [None] * Ly
    U1 = U[1].reshape(Trow[0].shape[0], Trow[1].shape[0], -1)         # (p0, p1, k1)
    t0, t1 = Trow[0][:, 0], Trow[1]                                  # t0: (p0, hr, d0)
    blk = np.einsum("pqk,prd,qrse->deks", U1, t0, t1)                # (d0, d1, k1, h12)
    sh = blk.shape
    blocks[1] = blk.reshape(sh[0], sh[1], sh[2] * sh[3])
    for c in range(2, Ly):
        if c < Ly - 1:
            Uc = U[c].reshape(-1, Trow[c].shape[0], U[c].shape[1])   # (k_{c-1}, p, k_c)
        else:
            Uc = Mr.reshape(Mr.shape[0], Trow[c].shape[0], 1)       # root: (k, p, 1)
        t = Trow[c]                                                  # (p, hl, hr, d)
        s = np.einsum("apb,plrd->aldbr", Uc, t)
        sh = s.shape
        blocks[c] = s.reshape(sh[0] * sh[1], sh[2], sh[3] * sh[4])
    return blocks


def _close_chain(blocks):
    """Exact scalar of the last contraction: every block has a phys dim 1."""
    vec = blocks[1].reshape(1, -1)
    logscale = 0.0
    for v in range(2, len(blocks)):
        vec = vec @ blocks[v][:, 0, :]
        m = np.max(np.abs(vec))
        logscale += np.log(m)
        vec = vec / m
    return float(vec.reshape(-1)[0]), logscale


def partitioned_contract_rows(workload, chi, trace=None, force_branch=None):
    """ln Z of a 2D lattice network by Algorithm partitioned_contract with rows
    as partitions, the linear path and the MPS ansatz.

    ``chi`` is one maximum rank, or a function chi(pass, v) giving the maximum
    rank of tree vertex v in DM pass ``pass`` (0-based, one pass per absorbed
    row) for per-edge ranks.

    Returns dict(logz, sign, logscale, steps) where steps lists the per-pass
    density_matrix_alg outputs when ``trace`` is a list (per-vertex records).
    """
    Lx, Ly = workload["Lx"], workload["Ly"]
    if Lx < 2 or Ly < 3:
        raise ValueError("need Lx >= 2 and Ly >= 3")
    T, logscale = lattice_site_tensors(workload["tensors"], workload["n"],
                                       workload["edges"], Lx, Ly)
    # First contraction on the path: rows 0 and 1.
    blocks = _blocks_first_pair(T[0], T[1])
    x = 1
    while True:
        last = (x == Lx - 1)
        if last:
            s, ls = _close_chain(blocks)
            if not s > 0:
                return dict(logz=float("nan"), sign=float(np.sign(s)), logscale=logscale)
            return dict(logz=float(np.log(s) + ls + logscale), sign=1.0, logscale=logscale)
        rec = [] if trace is not None else None
        chi_pass = (lambda v, p=x - 1: chi(p, v)) if callable(chi) else chi
        U, Mr, lognorm = density_matrix_alg(blocks, chi_pass, trace=rec, force_branch=force_branch)
        logscale += lognorm
        if trace is not None:
            trace.append(dict(row=x, vertices=rec, U=U, Mr=Mr, blocks=blocks))
        x += 1
        blocks = _blocks_absorb_row(U, Mr, T[x])
