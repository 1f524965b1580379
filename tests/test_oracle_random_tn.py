"""Pins of the random-tensor workload (entries uniform on [alpha, 1]) and of the
oracle on it: the oracle at full rank equals the dense contraction of the whole
network, and truncation moves the result (so the rank limit is active)."""
import numpy as np
import pytest

from oracle import dmtree, exact
from workloads import graphs, random_tn


def test_entries_lie_in_range_and_vary():
    w = random_tn.lattice2d(4, 5, -0.4, seed=3)
    allv = np.concatenate([t.reshape(-1) for t in w["tensors"]])
    assert allv.min() >= -0.4 and allv.max() <= 1.0
    assert allv.std() > 0.2
    w2 = random_tn.lattice2d(4, 5, -0.4, seed=4)
    assert not np.allclose(w["tensors"][0], w2["tensors"][0])


@pytest.mark.parametrize("Lx,Ly,alpha,seed", [(3, 4, 0.0, 1), (4, 4, -0.3, 2), (4, 5, -0.1, 5)])
def test_oracle_exact_at_full_rank(Lx, Ly, alpha, seed):
    w = random_tn.lattice2d(Lx, Ly, alpha, seed=seed)
    inc = graphs.incident_edges(w["n"], w["edges"])
    z = exact.contract_network(w["tensors"], inc)
    assert z > 0
    r = dmtree.partitioned_contract_rows(w, 2 ** Ly)
    assert r["logz"] == pytest.approx(np.log(z), rel=1e-12)


def test_truncation_is_active_below_exact_rank():
    w = random_tn.lattice2d(6, 8, 0.0, seed=7)
    full = dmtree.partitioned_contract_rows(w, 16)["logz"]
    low = dmtree.partitioned_contract_rows(w, 1)["logz"]
    assert abs(full - low) > 1e-6 * abs(full)
