"""Pins of the learned-rank reference (oracle/learned.py) and of per-edge
ranks in the oracle's density_matrix_alg, independent of the GPU path."""
import numpy as np
import pytest

from oracle import dmtree, exact
from oracle import learned as OL
from workloads import ising


def _spectra(rng, n_edges, length):
    out = []
    for _ in range(n_edges):
        lam = np.sort(rng.exponential(1.0, length) ** rng.uniform(1, 6))[::-1]
        out.append(lam / lam.sum())
    return out


@pytest.mark.parametrize("seed", range(6))
def test_water_fill_is_optimal(seed):
    """Greedy water-filling reaches the brute-force minimum of the summed
    discarded share (discarded share is convex in chi for descending spectra)."""
    rng = np.random.default_rng(seed)
    n_edges = int(rng.integers(2, 5))
    spectra = _spectra(rng, n_edges, 6)
    caps = [int(c) for c in rng.integers(1, 7, n_edges)]
    for budget in range(n_edges, sum(caps) + 2):
        alloc = OL.water_fill(spectra, caps, budget)
        assert all(1 <= a <= c for a, c in zip(alloc, caps))
        assert sum(alloc) <= max(budget, n_edges)
        _, best = OL.best_allocation_bruteforce(spectra, caps, budget)
        got = sum(OL.discarded(l, a) for l, a in zip(spectra, alloc))
        assert got == pytest.approx(best, abs=1e-14)


def test_water_fill_uses_budget_and_ties_low_index():
    spectra = [np.array([0.5, 0.25, 0.25]), np.array([0.5, 0.25, 0.25])]
    # equal gains: the lower edge index gets the rank first
    assert OL.water_fill(spectra, [3, 3], 3) == [2, 1]
    assert OL.water_fill(spectra, [3, 3], 6) == [3, 3]
    assert OL.water_fill(spectra, [3, 3], 9) == [3, 3]  # caps bind


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = rng.normal(0, 0.3, OL.n_params())
    X = rng.normal(0, 1, (37, OL.N_FEATURES))
    t = rng.uniform(0, 1, 37)
    loss, g = OL.loss_and_grad(w, X, t)
    assert g.shape == w.shape
    idx = rng.choice(len(w), 60, replace=False)
    h = 1e-6
    for q in idx:
        wp, wm = w.copy(), w.copy()
        wp[q] += h
        wm[q] -= h
        fd = (OL.loss_and_grad(wp, X, t)[0] - OL.loss_and_grad(wm, X, t)[0]) / (2 * h)
        assert fd == pytest.approx(g[q], rel=1e-5, abs=1e-8)
    # the loss is the mean squared error of the forward pass
    y, _ = OL.forward(w, X)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)


def test_forward_layer_layout():
    """A network that copies feature 3 through one hidden unit in each layer."""
    w = np.zeros(OL.n_params())
    W1, b1, W2, b2, W3, b3 = OL.unpack(w)   # views into w
    W1[5, 3] = 1.0
    W2[7, 5] = 2.0
    W3[7] = 0.5
    b3[0] = 0.125
    X = np.zeros((2, OL.N_FEATURES))
    X[0, 3], X[1, 3] = 0.75, -1.0
    y, _ = OL.forward(w, X)
    assert y.tolist() == [0.75 + 0.125, 0.125]   # ReLU clips the negative input


def test_features_of_a_geometric_spectrum():
    q, A = 0.5, 40
    lam = q ** np.arange(A)
    f = OL.features(lam, A, vertex=3, n_legs=13, pass_index=2, n_passes=8, remaining=30,
                    edges_left=8, uniform_rank=6)
    assert len(f) == OL.N_FEATURES == 22
    for j, k in enumerate(OL.K_RATIOS):
        kk = min(k, A)
        expect = max((kk - 1) * np.log10(q), -12.0) / 30.0
        assert f[j] == pytest.approx(expect, abs=1e-12)
    for j, r in enumerate(OL.R_DISCARD):
        share = (q ** r - q ** A) / (1 - q ** A) if r < A else 0.0
        expect = np.log10(max(share, 1e-12)) / 30.0
        assert f[len(OL.K_RATIOS) + j] == pytest.approx(expect, abs=1e-12)
    assert f[17] == A / 128 and f[18] == 3 / 12 and f[19] == 2 / 8
    assert f[20] == 30 / 8 / 64 and f[21] == 6 / 64


def test_budget_features():
    caps = [4, 8, 16, 2]
    assert OL.pass_budget(caps, 8) == 4 + 8 + 8 + 2
    bf = OL.budget_features([3, 9, 8, 2], caps, 8)
    assert bf == [(22 / 4 / 64, 4 / 64), (19 / 3 / 64, 8 / 64), (10 / 2 / 64, 8 / 64),
                  (2 / 1 / 64, 2 / 64)]


def test_select_rank_budget_rules():
    # rint ties to even, clamps to [1, min(rk, n_rank)]
    assert OL.select_rank(2.5 / 64, 10, 10, 100, 0) == (2, 98)
    assert OL.select_rank(3.5 / 64, 10, 10, 100, 0) == (4, 96)
    assert OL.select_rank(-1.0, 10, 10, 100, 0) == (1, 99)
    assert OL.select_rank(float("nan"), 10, 10, 100, 0) == (1, 99)
    assert OL.select_rank(1.0, 10, 10, 100, 0) == (10, 90)
    assert OL.select_rank(1.0, 10, 4, 100, 0) == (4, 96)
    # later edges keep their reserve
    assert OL.reserve_after([4, 1, 2, 8]) == 2 + 1 + 2 + 2
    assert OL.select_rank(1.0, 10, 10, 12, 5) == (7, 5)
    assert OL.select_rank(1.0, 10, 10, 5, 5) == (1, 4)


def test_numerical_rank():
    lam = np.array([1.0, 1e-3, 1e-11, 1e-13, 0.0])
    assert OL.numerical_rank(lam, 5) == 3
    assert OL.numerical_rank(lam, 2) == 2
    assert OL.numerical_rank(np.zeros(4), 4) == 1


def test_per_edge_ranks_at_the_cut_rank_are_exact():
    """Per-edge ranks chi(pass, v) = exact rank bound of the edge (2^min(v+1,
    n-1-v) on a row MPS of n legs) reproduce the transfer-matrix ln Z, while
    rank 1 on a single edge does not (so the per-edge rank reaches the cut)."""
    L, beta = 6, 0.8
    w = ising.lattice2d(L, L, beta, "gauss", seed=17)
    ex = exact.ising_logz_transfer_matrix(L, L, w["edges"], w["J"], beta)

    def cut(p, v):
        return 2 ** min(v + 1, L - 1 - v)

    r = dmtree.partitioned_contract_rows(w, cut)
    assert abs(r["logz"] - ex) <= 1e-12 * abs(ex)

    def short(p, v):
        return 1 if (p, v) == (1, 2) else cut(p, v)

    r2 = dmtree.partitioned_contract_rows(w, short)
    assert abs(r2["logz"] - ex) > 1e-6 * abs(ex)
