"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/tn_dmtree.h declares, and the planner's shapes,
ranks, flop counts and error codes follow the method."""
import os
import re

import numpy as np
import pytest

from paper_2406_09769_gb300 import binding as B
from workloads import ising, potts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    B.lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "tn_dmtree.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert "tn_embed_tree" in names and "tn_contract_approx" in names and "tn_logz" in names
    lib = B.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == names


def _plan(Lx, Ly, chi, **kw):
    w = ising.lattice2d(Lx, Ly, 0.5)
    return B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=Ly, **kw), w


def test_plan_counts_and_offsets():
    p, w = _plan(6, 6, 16)
    info = p.info
    assert info["n_steps"] == 5 and info["n_dm_passes"] == 4 and info["max_legs"] == 6
    # site buffer: legs in ascending edge order, 2^degree entries per vertex
    sizes = [t.size for t in w["tensors"]]
    assert info["site_elems"] == sum(sizes)
    assert [p.site_offset(v) for v in range(36)] == list(np.cumsum([0] + sizes[:-1]))


def _expected_flops(Lx, Ly, chi, q=2):
    """Sec. 2.2 cost model over the shapes the row-partition method produces,
    written independently of the planner (2 flops per multiply-add); every bond
    of dimension q."""
    d = [q] * Ly
    bond = [q] * (Ly - 1)            # boundary MPS after row 0 (horizontal bonds)
    env = local = dens = proj = 0.0
    fac = kfac = svd = 0.0
    for _ in range(Lx - 2):
        D = [b * q for b in bond] + [1]
        r = [d[0]]
        for k in range(1, Ly - 1):
            r.append(min(chi, r[-1] * d[k], D[k], q ** (Ly - 1 - k)))
        for k in range(Ly - 1, 1, -1):
            env += 2.0 * D[k - 1] * d[k] * D[k] * D[k] + 2.0 * D[k - 1] ** 2 * d[k] * D[k]
        for k in range(1, Ly - 1):
            A = r[k - 1] * d[k]
            local += 2.0 * r[k - 1] * D[k - 1] * d[k] * D[k]
            dens += 2.0 * A * D[k] ** 2 + 2.0 * A * A * D[k]
            proj += 2.0 * r[k] * A * D[k]
            # factored form: Cholesky of R_k, K = M C, Golub-Kahan SVD of K
            # (4 m n^2 - 4 n^3 / 3 with m >= n the longer side) + back-transform
            fac += D[k] ** 3 / 3.0
            kfac += 2.0 * A * D[k] ** 2
            lo, hi = min(A, D[k]), max(A, D[k])
            svd += 4.0 * hi * lo ** 2 - 4.0 * lo ** 3 / 3.0 + 2.0 * A * A * r[k]
        proj += 2.0 * r[Ly - 2] * D[Ly - 2] * d[Ly - 1]
        bond = r[:Ly - 1]
    _expected_flops.factored = (fac, kfac, svd)
    return env, local, dens, proj


@pytest.mark.parametrize("Lx,Ly,chi", [(6, 6, 16), (32, 32, 64), (9, 13, 5)])
def test_plan_flops_match_cost_model(Lx, Ly, chi):
    p, _ = _plan(Lx, Ly, chi)
    info = p.info
    env, local, dens, proj = _expected_flops(Lx, Ly, chi)
    assert info["flops_env"] == pytest.approx(env)
    assert info["flops_local"] == pytest.approx(local)
    assert info["flops_density"] == pytest.approx(dens)
    assert info["flops_project"] == pytest.approx(proj)
    fac, kfac, svd = _expected_flops.factored
    assert info["flops_factor"] == pytest.approx(fac)
    assert info["flops_kfactor"] == pytest.approx(kfac)
    assert info["flops_svd"] == pytest.approx(svd)


def test_null_arguments_are_rejected_without_a_device():
    lib = B.lib()
    assert lib.tn_ctx_set_option(None, B.TN_OPT_EIG_ROUNDS, 9) == 1
    assert lib.tn_measure_peaks(0, None) == 1
    assert lib.tn_ctx_profile(None, None, None, 0) == 1


@pytest.mark.parametrize("Lx,Ly,chi,q", [(6, 6, 12, 3), (5, 7, 20, 3), (4, 5, 16, 4)])
def test_plan_with_bond_dimension_q(Lx, Ly, chi, q):
    """Potts networks: site buffer of q^degree entries per vertex and the cost
    model with every bond of dimension q."""
    w = potts.lattice2d(Lx, Ly, 0.6, q)
    p = B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), q), chi, env_size=Ly)
    sizes = [t.size for t in w["tensors"]]
    assert p.info["site_elems"] == sum(sizes)
    assert [p.site_offset(v) for v in range(w["n"])] == list(np.cumsum([0] + sizes[:-1]))
    env, local, dens, proj = _expected_flops(Lx, Ly, chi, q)
    assert p.info["flops_env"] == pytest.approx(env)
    assert p.info["flops_local"] == pytest.approx(local)
    assert p.info["flops_density"] == pytest.approx(dens)
    assert p.info["flops_project"] == pytest.approx(proj)


def test_plan_rejects_malformed_input():
    w = ising.lattice2d(4, 5, 0.5)
    dims = np.full(len(w["edges"]), 2)
    with pytest.raises(B.TNError) as e:
        B.tn_plan(w["n"], w["edges"], dims, 0, env_size=5)
    assert e.value.status == 1                       # chi < 1
    bad = w["edges"].copy()
    bad[0, 1] = 99
    with pytest.raises(B.TNError) as e:
        B.tn_plan(w["n"], bad, dims, 4, env_size=5)
    assert e.value.status == 1                       # endpoint out of range
    # parts that are not row paths: the general planner takes them
    assert B.tn_plan_query(B.tn_plan(w["n"], w["edges"], dims, 4, env_size=4))["general"] == 1
    with pytest.raises(B.TNError) as e:
        B.tn_plan(w["n"], w["edges"], dims, 4, env_size=5, planner=2)
    assert e.value.status == 1                       # unknown planner
    with pytest.raises(B.TNError) as e:
        B.tn_plan(w["n"], w["edges"], dims, 4, env_size=5, path=[0, 1, 1, 3])
    assert e.value.status == 1                       # path not a permutation
    with pytest.raises(B.TNError) as e:
        B.tn_plan(w["n"], w["edges"], dims, 4, env_size=5, ansatz=1)
    assert e.value.status == 8                       # comb ansatz not built


def test_plan_accepts_explicit_partition_and_reversed_path():
    w = ising.lattice2d(5, 4, 0.5)
    part = np.arange(20) // 4
    p = B.tn_plan(20, w["edges"], np.full(len(w["edges"]), 2), 8, partition=part,
                  path=[4, 3, 2, 1, 0])
    assert p.info["n_dm_passes"] == 3
