"""FP64 reference of the learned per-edge rank part (TEST INFRASTRUCTURE).

The paper has no learned component; this module restates, plainly, what the
library's learned rank allocation computes, so the GPU kernels can be checked:

  * spectrum features of one density matrix L_v (descending eigenvalues lam,
    its order dim A_v, the vertex position and the pass index);
  * a 3-layer MLP (F -> 64 -> 64 -> 1, ReLU) forward pass and its gradient of
    the mean squared error, in FP64, with the weights given (the GPU rounds
    them to BF16 before use; pass the rounded weights here);
  * the budgeted rank decision of one edge from the MLP output;
  * the offline label: the allocation of a per-pass rank budget over the
    pass's edges that minimises the summed discarded weight
    sum_e sum_{i >= chi_e} lam_e,i / sum_i lam_e,i (greedy water-filling,
    optimal because each edge's discarded weight is convex in chi_e for
    descending eigenvalues).
Pinned in tests by finite differences (gradient) and brute force (allocation).
"""
import itertools

import numpy as np

N_FEATURES = 22
HIDDEN = 64
K_RATIOS = (2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128)
R_DISCARD = (8, 16, 24, 32, 48, 64)
FLOOR = 1e-12   # below the eigensolver's relative resolution


def features(lam, dim_a, vertex, n_legs, pass_index, n_passes, remaining, edges_left,
             uniform_rank):
    """Feature vector of one edge: spectrum shape of L_v (eigenvalue ratios and
    discarded shares, floored at FLOOR), dim A_v, position, pass, the budget
    left per edge left and the uniform method's rank."""
    lam = np.maximum(np.asarray(lam, dtype=np.float64)[:dim_a], 0.0)
    top = lam[0] if lam[0] > 0 else 1.0
    total = lam.sum() if lam.sum() > 0 else 1.0
    f = []
    for k in K_RATIOS:
        idx = min(k, dim_a) - 1
        f.append(np.log10(max(lam[idx] / top, FLOOR)) / 30.0)
    for r in R_DISCARD:
        disc = lam[r:].sum() / total if r < dim_a else 0.0
        f.append(np.log10(max(disc, FLOOR)) / 30.0)
    f.append(dim_a / 128.0)
    f.append(vertex / max(n_legs - 1, 1))
    f.append(pass_index / max(n_passes, 1))
    f.append(remaining / edges_left / 64.0)
    f.append(uniform_rank / 64.0)
    return np.asarray(f, dtype=np.float64)


def pass_budget(caps, chi_uniform):
    """Total rank of the uniform-chi method over one pass's edges."""
    return int(sum(min(chi_uniform, int(c)) for c in caps))


def budget_features(alloc, caps, chi_uniform):
    """Features 20 and 21 of each edge of one pass under allocation alloc."""
    rem = pass_budget(caps, chi_uniform)
    out = []
    for j, (a, c) in enumerate(zip(alloc, caps)):
        out.append((rem / (len(alloc) - j) / 64.0, min(chi_uniform, int(c)) / 64.0))
        rem -= a
    return out


def unpack(w):
    """Flat parameter vector -> (W1, b1, W2, b2, W3, b3)."""
    F, H = N_FEATURES, HIDDEN
    o = 0
    W1 = w[o:o + H * F].reshape(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o:o + 1]; o += 1
    assert o == len(w)
    return W1, b1, W2, b2, W3, b3


def n_params():
    return HIDDEN * N_FEATURES + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def forward(w, X):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(w, dtype=np.float64))
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ W3 + b3[0]
    return y, (Z1, H1, Z2, H2)


def loss_and_grad(w, X, t):
    """Mean squared error and its gradient with respect to the flat w."""
    w = np.asarray(w, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(w)
    y, (Z1, H1, Z2, H2) = forward(w, X)
    n = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3 = H2.T @ dy
    gb3 = np.array([dy.sum()])
    dH2 = np.outer(dy, W3) * (Z2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2) * (Z1 > 0)
    gW1 = dH1.T @ X
    gb1 = dH1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g


def numerical_rank(lam, dim_a):
    """Last position (1-based) whose eigenvalue exceeds FLOOR * lam_1; at least 1."""
    nr = 1
    for q in range(1, dim_a):
        if lam[q] > FLOOR * lam[0]:
            nr = q + 1
    return nr


def reserve_after(ranks_after):
    """Budget kept for the later edges of a pass: min(2, r_u) each."""
    return int(sum(min(2, int(r)) for r in ranks_after))


def select_rank(y, rk, n_rank, remaining, reserve):
    """Budgeted rank of one edge from the model output y: rint(64 y) (ties to
    even) clamped to [1, min(rk, n_rank)], then lowered to at most
    remaining - reserve (the budget the later edges keep), but not below 1.
    Returns (chi, remaining budget after this edge)."""
    pred = np.rint(64.0 * y)
    if not pred >= 1:
        pred = 1.0
    c = rk if pred > rk else int(pred)
    c = min(c, n_rank)
    c = min(c, remaining - reserve)
    c = max(c, 1)
    return c, remaining - c


def discarded(lam, chi):
    lam = np.maximum(np.asarray(lam, dtype=np.float64), 0.0)
    tot = lam.sum()
    return lam[chi:].sum() / tot if tot > 0 else 0.0


def water_fill(spectra, caps, budget):
    """Allocation chi_e in [1, caps[e]] with sum chi_e <= budget minimising
    sum_e discarded(lam_e, chi_e): start from 1 everywhere and repeatedly give
    one more rank to the edge whose next eigenvalue carries the largest share
    of its total (ties: lowest edge index)."""
    alloc = [1] * len(spectra)
    used = len(spectra)
    while used < budget:
        best, bi = -1.0, -1
        for e, lam in enumerate(spectra):
            if alloc[e] < caps[e] and alloc[e] < len(lam):
                lam_e = np.maximum(np.asarray(lam, dtype=np.float64), 0.0)
                tot = lam_e.sum()
                gain = lam_e[alloc[e]] / tot if tot > 0 else 0.0
                if gain > best:
                    best, bi = gain, e
        if bi < 0:
            break
        alloc[bi] += 1
        used += 1
    return alloc


def best_allocation_bruteforce(spectra, caps, budget):
    """Exhaustive minimum of the summed discarded weight (tiny cases only)."""
    best, arg = None, None
    for choice in itertools.product(*[range(1, c + 1) for c in caps]):
        if sum(choice) > budget:
            continue
        val = sum(discarded(l, c) for l, c in zip(spectra, choice))
        if best is None or val < best - 1e-15:
            best, arg = val, choice
    return list(arg), best
