"""GPU parity of general plans (random regular graphs, cubic lattices, any
partition, swap passes) against the FP64 oracle of oracle/general.py, through
the C ABI.

Tolerances: FP64 path 1e-10 relative ln Z (as for the lattice plans); the
factored mixed path (TN_PREC_TF32) 1e-6 relative; ln Z at chi above every cut
rank within 1e-12 of the brute-force spin sum.
"""
import numpy as np
import pytest

from oracle import exact, general
from paper_2406_09769_gb300 import binding as B
from workloads import ising

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL_FP64 = 1e-10
RTOL_TF32 = 1e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    return B.tn_ctx_create(0)


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _plan(w, env, chi, swap, planner=1):
    return B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=env,
                     swap_batch=swap, planner=planner)


def _run(ctx, ws, plans, precision=B.TN_PREC_FP64):
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], precision, 0, _stream())
    return B.tn_logz(ctx, len(plans))


def _oracle(w, env, chi, swap):
    return general.partitioned_contract_graph(w, general.parts_from_env(w["n"], env), chi,
                                              swap)["logz"]


CASES = [
    ("rr3_40_env1", lambda: ising.random_regular(40, 3, 0.3, 41), 1, 8, 0),
    ("rr3_40_env1_swap1", lambda: ising.random_regular(40, 3, 0.3, 41), 1, 8, 1),
    ("rr3_60_env3_swap3", lambda: ising.random_regular(60, 3, 0.3, 31), 3, 16, 3),
    ("rr3_60_env6_chi32", lambda: ising.random_regular(60, 3, 0.3, 31), 6, 32, 32),
    ("rr4_30_env2", lambda: ising.random_regular(30, 4, 0.25, 42), 2, 16, 0),
    ("cubic444_env2", lambda: ising.cubic(4, 4, 4, 0.2217), 2, 16, 0),
    ("cubic666_env3_chi16", lambda: ising.cubic(6, 6, 6, 0.2217), 3, 16, 0),
]


@pytest.mark.parametrize("name,make,env,chi,swap", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle(ctx, name, make, env, chi, swap):
    w = make()
    ref = _oracle(w, env, chi, swap)
    logz, status = _run(ctx, [w], [_plan(w, env, chi, swap)])
    assert status[0] == 0
    assert abs(logz[0] - ref) / abs(ref) < RTOL_FP64


def test_exact_at_full_rank(ctx):
    w = ising.random_regular(20, 3, 0.4, 12)
    ex = exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], w["beta"])
    for env, swap in ((1, 0), (3, 1)):
        logz, status = _run(ctx, [w], [_plan(w, env, 1024, swap)])
        assert status[0] == 0 and abs(logz[0] - ex) / abs(ex) < 1e-12


def test_rows_general_equals_boundary_plan(ctx):
    """The general planner on a 2D lattice with rows as parts computes the
    same ln Z as the boundary-absorption plan (same tree, different blocks)."""
    w = ising.lattice2d(8, 9, 0.5, "gauss", seed=77)
    a, sa = _run(ctx, [w], [_plan(w, 9, 6, 0, planner=1)])
    b, sb = _run(ctx, [w], [_plan(w, 9, 6, 0, planner=0)])
    assert sa[0] == 0 and sb[0] == 0
    # same tree and ranks; only the rounding order of the blocks differs
    assert abs(a[0] - b[0]) / abs(b[0]) < RTOL_FP64


def test_heterogeneous_random_graph_batch(ctx):
    """Random 3-regular instances of different sizes and chi (the batched
    workload's recipe) in one call, each against the oracle."""
    ws = [ising.config4_instance(i) for i in range(6)]
    ws = [w for w in ws if w["n"] <= 120][:4]
    plans = [_plan(w, 6, w["chi"], 32) for w in ws]
    logz, status = _run(ctx, ws, plans)
    for i, w in enumerate(ws):
        ref = _oracle(w, 6, w["chi"], 32)
        assert status[i] == 0
        assert abs(logz[i] - ref) / abs(ref) < RTOL_FP64


TF32_CASES = [CASES[0], CASES[2], CASES[5], CASES[6]]


@pytest.mark.parametrize("name,make,env,chi,swap", TF32_CASES, ids=[c[0] for c in TF32_CASES])
def test_tf32_matches_oracle(ctx, name, make, env, chi, swap):
    w = make()
    ref = _oracle(w, env, chi, swap)
    logz, status = _run(ctx, [w], [_plan(w, env, chi, swap)], B.TN_PREC_TF32)
    assert status[0] == 0
    assert abs(logz[0] - ref) / abs(ref) < RTOL_TF32


def test_tf32_passes_beyond_factored_shapes_run_in_gram_form(ctx):
    """Passes with tree edges above 128 (4-regular graph, parts of 2) run in
    the compensated Gram form; the result still matches the oracle to the
    Gram form's resolution of L_v (eigen-directions down to ~1e-7)."""
    name, make, env, chi, swap = CASES[4]
    w = make()
    plan = _plan(w, env, chi, swap)
    assert B.tn_plan_query(plan)["max_bond"] > 128
    ref = _oracle(w, env, chi, swap)
    logz, status = _run(ctx, [w], [plan], B.TN_PREC_TF32)
    assert status[0] == 0
    assert abs(logz[0] - ref) / abs(ref) < 1e-5
