"""Pins of the CPU FP64 oracle against what the paper and mathematics fix.

Each test would fail under a plausible mistake in the oracle:
  * wrong W / sign convention      -> dense contraction != brute-force spin sum
  * wrong transfer matrix          -> != brute force, != closed forms
  * dropped/misindexed term in DM  -> != exact at chi >= exact rank,
                                      != canonicalisation route below it,
                                      != definition of the density matrix
  * transposed operand             -> breaks orthogonal-gauge invariance
"""
import os

import numpy as np
import pytest

from oracle import canonical, dmtree, exact
from workloads import graphs, ising

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "exact_logz.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, Lx, Ly, beta, cp, seed, method, z = line.split()
            rows.append((name, int(Lx), int(Ly), float(beta), cp, int(seed), method, float(z)))
    return rows


# ------------------------------------------------------------- exact layer

def test_bond_sqrt_squares_to_boltzmann_matrix():
    for bj in (0.0, 0.1, 0.44, 1.3):
        W = ising.bond_sqrt(bj)
        B = np.array([[np.exp(bj), np.exp(-bj)], [np.exp(-bj), np.exp(bj)]])
        np.testing.assert_allclose(W @ W.T, B, rtol=1e-14)


@pytest.mark.parametrize("cp,seed", [("ferro", 0), ("gauss", 7), ("pm1", 9)])
def test_tensor_network_equals_spin_sum(cp, seed):
    w = ising.lattice2d(3, 4, 0.9, cp, seed=seed)
    inc = graphs.incident_edges(w["n"], w["edges"])
    z = exact.contract_network(w["tensors"], inc)
    assert np.log(z) == pytest.approx(
        exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], 0.9), rel=1e-13)


def test_transfer_matrix_equals_bruteforce():
    for (Lx, Ly, cp, seed) in [(4, 4, "gauss", 3), (3, 5, "pm1", 5), (5, 3, "ferro", 0)]:
        w = ising.lattice2d(Lx, Ly, 0.6, cp, seed=seed)
        a = exact.ising_logz_transfer_matrix(Lx, Ly, w["edges"], w["J"], 0.6)
        b = exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], 0.6)
        assert a == pytest.approx(b, rel=1e-13)


def test_closed_forms():
    # 2x2 lattice = 4-cycle; 1 x n lattice = chain (a tree)
    beta = 0.44
    w = ising.lattice2d(2, 2, beta)
    closed = 4 * np.log(2) + np.log(np.cosh(beta) ** 4 + np.sinh(beta) ** 4)
    assert exact.ising_logz_cycle(w["J"], beta) == pytest.approx(closed, rel=1e-15)
    assert exact.ising_logz_bruteforce(4, w["edges"], w["J"], beta) == pytest.approx(closed, rel=1e-14)
    w = ising.lattice2d(1, 9, 0.7, "gauss", seed=1)
    assert exact.ising_logz_transfer_matrix(1, 9, w["edges"], w["J"], 0.7) == pytest.approx(
        exact.ising_logz_tree(w["J"], 0.7), rel=1e-14)


def test_kac_ward_equals_bruteforce_and_transfer_matrix():
    for (Lx, Ly, beta, cp, seed) in [(3, 3, 0.7, "gauss", 1), (3, 4, 1.1, "pm1", 2),
                                     (4, 4, 0.44, "ferro", 0), (2, 6, 2.0, "gauss", 4)]:
        w = ising.lattice2d(Lx, Ly, beta, cp, seed=seed)
        assert exact.ising_logz_kac_ward(Lx, Ly, w["edges"], w["J"], beta) == pytest.approx(
            exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], beta), rel=1e-13)
    w = ising.lattice2d(8, 10, 0.8, "gauss", seed=9)
    assert exact.ising_logz_kac_ward(8, 10, w["edges"], w["J"], 0.8) == pytest.approx(
        exact.ising_logz_transfer_matrix(8, 10, w["edges"], w["J"], 0.8), rel=1e-13)


def test_golden_values_reproduce():
    for name, Lx, Ly, beta, cp, seed, method, z in _golden():
        if method == "kw" and not name.endswith("_i0"):
            continue  # one 32 x 32 determinant is enough here
        w = ising.lattice2d(Lx, Ly, beta, cp, seed=seed)
        if method == "kw":
            val = exact.ising_logz_kac_ward(Lx, Ly, w["edges"], w["J"], beta)
        else:
            val = exact.ising_logz_transfer_matrix(Lx, Ly, w["edges"], w["J"], beta)
        assert val == pytest.approx(z, rel=1e-13), name
    assert _golden()[0][-1] == pytest.approx(31.564145959482058, rel=1e-15)


# --------------------------------------------------------- oracle (dmtree)

@pytest.mark.parametrize("name", ["config1_6x6_ferro", "glass_4x5_gauss_b0.5",
                                  "glass_6x6_gauss_b0.5", "glass_8x6_pm1_b0.7"])
def test_dm_is_exact_at_or_above_exact_rank(name):
    row = [r for r in _golden() if r[0] == name][0]
    _, Lx, Ly, beta, cp, seed, _, z = row
    w = ising.lattice2d(Lx, Ly, beta, cp, seed=seed)
    chi = 2 ** (Ly // 2)          # maximal bond rank of an MPS over Ly legs of dim 2
    got = dmtree.partitioned_contract_rows(w, chi)["logz"]
    assert abs(got - z) <= 1e-12 * abs(z)


@pytest.mark.parametrize("i", [0, 7])
def test_oracle_full_size_config2_matches_exact(i):
    """32 x 32 Gaussian spin glass at beta = 0.5, chi = 64: the oracle against the
    Kac-Ward value.  At this temperature the truncation error is below FP64
    rounding (measured <= 2.6e-13 relative over instances 0..7)."""
    row = [r for r in _golden() if r[0] == f"config2_32x32_gauss_i{i}"][0]
    _, Lx, Ly, beta, cp, seed, _, z = row
    w = ising.config2_instance(i)
    got = dmtree.partitioned_contract_rows(w, 64)["logz"]
    assert abs(got - z) <= 1e-11 * abs(z)


def test_config1_exact_at_chi16():
    w = ising.lattice2d(6, 6, 0.44)
    got = dmtree.partitioned_contract_rows(w, 16)["logz"]
    assert abs(got - 31.564145959482058) <= 1e-12 * 31.6


@pytest.mark.parametrize("Lx,Ly,beta,cp,seed,chi", [
    (5, 7, 0.8, "gauss", 3, 3), (6, 8, 0.44, "ferro", 0, 4), (7, 6, 1.0, "pm1", 4, 4),
    (6, 9, 0.5, "gauss", 2000001, 5), (4, 10, 0.3, "gauss", 8, 3)])
def test_dm_equals_canonicalisation_route_below_exact_rank(Lx, Ly, beta, cp, seed, chi):
    w = ising.lattice2d(Lx, Ly, beta, cp, seed=seed)
    a = dmtree.partitioned_contract_rows(w, chi)["logz"]
    b = canonical.partitioned_contract_rows_canonical(w, chi)
    ex = exact.ising_logz_transfer_matrix(Lx, Ly, w["edges"], w["J"], beta)
    assert abs(a - ex) > 1e-9            # truncation is really active
    assert abs(a - b) <= 1e-11 * abs(b)


def _dense_current_network(w, x, prev):
    """Dense tensor over the new open legs (columns in order) of the network
    tn(V_1 .. V_x) U (row x), built with exact.contract_network."""
    Lx, Ly = w["Lx"], w["Ly"]
    T, _ = dmtree.lattice_site_tensors(w["tensors"], w["n"], w["edges"], Lx, Ly)
    tensors, legs = [], []
    # labels: ("h", x, y) horizontal edge right of (x, y); ("v", x, y) edge below (x, y)
    def row_legs(xx, y):
        return [("v", xx - 1, y), ("h", xx, y - 1), ("h", xx, y), ("v", xx, y)]
    rows = range(0, x + 1) if prev is None else [x]
    for xx in rows:
        for y in range(Ly):
            t = T[xx][y]
            keep = [i for i in range(4) if t.shape[i] > 1]
            tensors.append(t.reshape([t.shape[i] for i in keep]))
            legs.append([row_legs(xx, y)[i] for i in keep])
    if prev is not None:
        U, Mr = prev
        tensors.append(U[1].reshape(2, 2, -1))
        legs.append([("v", x - 1, 0), ("v", x - 1, 1), ("k", 1)])
        for v in range(2, Ly - 1):
            tensors.append(U[v].reshape(-1, 2, U[v].shape[1]))
            legs.append([("k", v - 1), ("v", x - 1, v), ("k", v)])
        tensors.append(Mr)
        legs.append([("k", Ly - 2), ("v", x - 1, Ly - 1)])
    order = [("v", x, y) for y in range(Ly)]
    return exact.contract_network(tensors, legs, open_order=order)


def test_memoised_density_matrix_equals_definition():
    """Eq. (dm_cache) with the root-side memo == Def. "density matrix"."""
    w = ising.lattice2d(5, 6, 0.7, "gauss", seed=21)
    trace = []
    dmtree.partitioned_contract_rows(w, 3, trace=trace)
    Ly = w["Ly"]
    prev = None
    checked = 0
    for step in trace:
        x = step["row"]
        psi = _dense_current_network(w, x, prev)
        for rec in step["vertices"]:
            v = rec["v"]
            # fold U_1^T .. U_{v-1}^T into the first legs, as Algorithm
            # density_matrix_alg does, then matricise on A_v = (k_{v-1}, x_v)
            t = psi.reshape(4, -1)
            for u in range(1, v):
                t = step["U"][u].T @ t.reshape(step["U"][u].shape[0], -1)
                t = t.reshape(-1, 2 ** (Ly - u - 1))
            if v == 1:
                t = psi.reshape(4, -1)
            else:
                t = t.reshape(-1, 2 ** (Ly - v - 1))
            L_def = t @ t.T
            L_memo = rec["M"] @ rec["env"] @ rec["M"].T
            np.testing.assert_allclose(L_memo / np.linalg.norm(L_memo),
                                       L_def / np.linalg.norm(L_def), atol=1e-12)
            # discarded weight: ||T - U U^T T||^2 / ||T||^2 == sum_{k>r} lam / sum lam
            Uv = rec["U"]
            resid = np.linalg.norm(t - Uv @ (Uv.T @ t)) ** 2 / np.linalg.norm(t) ** 2
            lam = rec["lam"]
            assert resid == pytest.approx(lam[rec["r"]:].sum() / lam.sum(), abs=1e-12)
            checked += 1
        prev = (step["U"], step["Mr"])
    assert checked >= 10


def test_qrsvd_branch_equals_direct_branch():
    w = ising.lattice2d(6, 7, 0.6, "gauss", seed=33)
    a = dmtree.partitioned_contract_rows(w, 3, force_branch="direct")["logz"]
    b = dmtree.partitioned_contract_rows(w, 3, force_branch="qrsvd")["logz"]
    assert abs(a - b) <= 1e-11 * abs(a)


def test_orthogonal_gauge_invariance():
    """A random orthogonal gauge G G^T = I on every edge leaves the network,
    hence every density matrix spectrum and ln Z, unchanged."""
    w = ising.lattice2d(6, 7, 0.6, "gauss", seed=34)
    rng = np.random.default_rng(0)
    inc = graphs.incident_edges(w["n"], w["edges"])
    G = [np.linalg.qr(rng.standard_normal((2, 2)))[0] for _ in range(len(w["edges"]))]
    tens = []
    for v, t in enumerate(w["tensors"]):
        for ax, e in enumerate(inc[v]):
            t = np.moveaxis(np.tensordot(t, G[e], axes=([ax], [0])), -1, ax)
        tens.append(t)
    wg = dict(w, tensors=tens)
    for chi in (2, 3, 5):
        a = dmtree.partitioned_contract_rows(w, chi)["logz"]
        b = dmtree.partitioned_contract_rows(wg, chi)["logz"]
        assert abs(a - b) <= 1e-11 * abs(a)
