"""Pins of the q-state Potts workload (bond dimension q) and of the oracle on it.

  * wrong bond square root / leg order -> dense contraction != brute force
  * wrong Potts brute force            -> q = 2 != Ising at beta / 2 plus the constant
  * dimension-2 assumption in the DM   -> oracle at full rank != brute force
"""
import numpy as np
import pytest

from oracle import dmtree, exact
from workloads import graphs, ising, potts


def test_q2_potts_is_ising_at_half_beta():
    # [s == s'] = (1 + s s') / 2 for s in {+1, -1}
    beta = 0.8
    w = potts.lattice2d(3, 3, beta, 2, "uniform", seed=4)
    z_potts = exact.potts_logz_bruteforce(w["n"], w["edges"], w["J"], beta, 2)
    z_ising = exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], beta / 2)
    assert z_potts == pytest.approx(beta / 2 * w["J"].sum() + z_ising, rel=1e-14)


def test_bond_sqrt_squares_to_bond_matrix():
    for q in (2, 3, 4):
        for bj in (0.0, 0.3, 1.1):
            W = potts.bond_sqrt(bj, q)
            np.testing.assert_allclose(W, W.T, atol=1e-15)
            np.testing.assert_allclose(W @ W.T, potts.bond_matrix(bj, q), rtol=1e-13)


@pytest.mark.parametrize("q,Lx,Ly", [(3, 3, 3), (3, 2, 4), (4, 2, 3)])
def test_network_equals_configuration_sum(q, Lx, Ly):
    w = potts.lattice2d(Lx, Ly, 0.7, q, "uniform", seed=11)
    inc = graphs.incident_edges(w["n"], w["edges"])
    z = exact.contract_network(w["tensors"], inc)
    assert np.log(z) == pytest.approx(
        exact.potts_logz_bruteforce(w["n"], w["edges"], w["J"], 0.7, q), rel=1e-13)


@pytest.mark.parametrize("q,Lx,Ly", [(3, 4, 3), (3, 3, 4)])
def test_oracle_exact_at_full_rank(q, Lx, Ly):
    w = potts.lattice2d(Lx, Ly, 0.6, q, "uniform", seed=5)
    r = dmtree.partitioned_contract_rows(w, q ** Ly)
    assert r["logz"] == pytest.approx(
        exact.potts_logz_bruteforce(w["n"], w["edges"], w["J"], 0.6, q), rel=1e-12)
