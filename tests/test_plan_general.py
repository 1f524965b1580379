"""Host-side checks of the general planner (no GPU): the library's plan of
every contraction -- leaf order of every density-matrix pass, untruncated
tree-edge dims, ranks, Kendall-Tau distance and number of swap passes -- is
identical to the oracle's independent restatement (oracle/general.py) on
random regular graphs, cubic lattices and 2D lattices."""
import numpy as np
import pytest

from oracle import general
from paper_2406_09769_gb300 import binding as B
from workloads import ising


def _oracle_steps(w, env, chi, swap):
    P = general.plan(w["n"], w["edges"], [2] * len(w["edges"]),
                     general.parts_from_env(w["n"], env), chi, swap)
    out = []
    for st in P["steps"]:
        if st["close"]:
            out.append(dict(kind=2, D=st["D"]))
        else:
            for p in st["passes"]:
                out.append(dict(kind=1, leaves=[l[1] for l in p["leaves"]], D=p["D"], r=p["r"],
                                n_kt=p["n_kt"]))
    return out


def _lib_steps(w, env, chi, swap, planner=1):
    plan = B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=env,
                     swap_batch=swap, planner=planner)
    return plan, B.tn_plan_steps(plan)


CASES = [
    ("rr3_40", lambda: ising.random_regular(40, 3, 0.3, 41), 1, 8, 0),
    ("rr3_40_swap1", lambda: ising.random_regular(40, 3, 0.3, 41), 1, 8, 1),
    ("rr3_60_env3_swap3", lambda: ising.random_regular(60, 3, 0.3, 31), 3, 16, 3),
    ("rr3_60_env6", lambda: ising.random_regular(60, 3, 0.3, 31), 6, 32, 32),
    ("rr4_30_env2", lambda: ising.random_regular(30, 4, 0.25, 42), 2, 16, 0),
    ("rr4_30_env2_swap2", lambda: ising.random_regular(30, 4, 0.25, 42), 2, 16, 2),
    ("cubic444_env2", lambda: ising.cubic(4, 4, 4, 0.2217), 2, 16, 0),
    ("cubic666_env3", lambda: ising.cubic(6, 6, 6, 0.2217), 3, 64, 0),
    ("lattice2d_rows", lambda: ising.lattice2d(6, 7, 0.5, "gauss", seed=7), 7, 4, 0),
    ("config4_0", lambda: ising.config4_instance(0), 6, 64, 32),
    ("config4_1", lambda: ising.config4_instance(1), 6, 48, 32),
]


@pytest.mark.parametrize("name,make,env,chi,swap", CASES, ids=[c[0] for c in CASES])
def test_plan_equals_oracle(name, make, env, chi, swap):
    w = make()
    ref = _oracle_steps(w, env, chi, swap)
    plan, got = _lib_steps(w, env, chi, swap)
    assert len(got) == len(ref)
    for a, b in zip(ref, got):
        assert b["general"] == 1
        assert a["kind"] == b["kind"]
        assert a["D"] == b["D"]
        if a["kind"] == 1:
            assert a["leaves"] == b["leaves"]
            assert a["r"] == b["r"]
            assert a["n_kt"] == b["n_kt"]
    info = B.tn_plan_query(plan)
    assert info["general"] == 1
    assert info["n_exec_steps"] == len(ref)
    assert info["n_dm_passes"] == sum(1 for s in ref if s["kind"] == 1)


def test_auto_planner_picks_boundary_for_rows_and_general_otherwise():
    w = ising.lattice2d(6, 7, 0.5, "gauss", seed=7)
    plan, steps = _lib_steps(w, 7, 8, 0, planner=0)
    assert B.tn_plan_query(plan)["general"] == 0
    assert steps[0]["kind"] == 0
    w = ising.random_regular(40, 3, 0.3, 41)
    plan, steps = _lib_steps(w, 2, 8, 0, planner=0)
    assert B.tn_plan_query(plan)["general"] == 1


def test_swap_batches_split_the_reordering():
    """ceil(d / r) passes per contraction (Algorithm approx_tensor_network)."""
    w = ising.random_regular(40, 3, 0.3, 41)
    _, one = _lib_steps(w, 1, 8, 0)
    _, many = _lib_steps(w, 1, 8, 1)
    kts = [s["n_kt"] for s in one if s["kind"] == 1]
    assert sum(max(1, d) for d in kts) == sum(1 for s in many if s["kind"] == 1)
    assert any(d > 1 for d in kts)


def test_oversized_cut_is_rejected():
    w = ising.cubic(6, 6, 6, 0.2217)
    with pytest.raises(B.TNError) as e:
        _lib_steps(w, 12, 64, 0)
    assert e.value.status == 8


def test_explicit_partition_fibre_portions_equals_oracle():
    """An explicit partition (the 5x5x5 lattice with every z-fibre cut into
    portions of 3 and 2 sites, as the paper's parts of 3 on that lattice): no
    part spans two fibres, and the library's plan equals the oracle's."""
    import bench
    w = ising.cubic(5, 5, 5, 0.3)
    part = bench._fibre_parts(5, 3)
    parts = [list(np.where(part == p)[0]) for p in range(part.max() + 1)]
    for vs in parts:
        assert len({v // 5 for v in vs}) == 1 and len(vs) in (2, 3)
    P = general.plan(w["n"], w["edges"], [2] * len(w["edges"]), parts, 16, 32)
    ref = []
    for st in P["steps"]:
        if st["close"]:
            ref.append(dict(kind=2, D=st["D"]))
        else:
            for p in st["passes"]:
                ref.append(dict(kind=1, leaves=[l[1] for l in p["leaves"]], D=p["D"], r=p["r"]))
    plan = B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), 16, env_size=0,
                     partition=part, swap_batch=32)
    got = B.tn_plan_steps(plan)
    assert len(got) == len(ref)
    for a, b in zip(ref, got):
        assert a["kind"] == b["kind"] and a["D"] == b["D"]
        if a["kind"] == 1:
            assert a["leaves"] == b["leaves"] and a["r"] == b["r"]
