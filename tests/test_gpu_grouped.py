"""GPU checks of the grouped executor: a mixed-precision batch of more than
eight plan structures (random 3-regular graphs of different sizes and chi,
the batched workload's recipe) runs as one launch sequence in which every
operation covers the problems of all instances.

  * every instance matches the FP64 oracle (oracle/general.py) within the
    mixed path's 1e-6 relative ln Z;
  * the grouped and the per-bucket executors agree within 1e-6;
  * a captured graph of the grouped batch replays to the same bits;
  * the range-guard diagnostic (every global access checked against the
    batch's allocations) records no access outside them.
"""
import os

import numpy as np
import pytest

from oracle import general
from paper_2406_09769_gb300 import binding as B
from workloads import ising

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL_TF32 = 1e-6
ENV, SWAP = 3, 4


def _instances():
    out = []
    i = 0
    while len(out) < 12:
        w = ising.config4_instance(i)
        if w["n"] <= 80:
            out.append(w)
        i += 1
    return out


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    ws = _instances()
    plans = [B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), w["chi"],
                       env_size=ENV, swap_batch=SWAP) for w in ws]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    ctx = B.tn_ctx_create(0)
    return ws, plans, bufs, ctx


def _run(batch, grouped):
    ws, plans, bufs, ctx = batch
    B.tn_ctx_set_option(ctx, B.TN_OPT_GROUPED, grouped)
    try:
        B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32, 0,
                             torch.cuda.current_stream().cuda_stream)
        return B.tn_logz(ctx, len(plans))
    finally:
        B.tn_ctx_set_option(ctx, B.TN_OPT_GROUPED, 1)


def test_batch_has_more_plan_structures_than_streams(batch):
    ws, plans, _, _ = batch
    sizes = {(w["n"], w["chi"]) for w in ws}
    assert len(sizes) > 8  # distinct plans: the grouped executor engages


def test_grouped_matches_oracle(batch):
    ws = batch[0]
    logz, status = _run(batch, 1)
    assert (status == 0).all()
    for i, w in enumerate(ws):
        ref = general.partitioned_contract_graph(w, general.parts_from_env(w["n"], ENV),
                                                 w["chi"], SWAP)["logz"]
        assert abs(logz[i] - ref) / abs(ref) < RTOL_TF32, (i, w["n"], w["chi"])


def test_grouped_equals_bucketed(batch):
    a, sa = _run(batch, 1)
    b, sb = _run(batch, 0)
    assert (sa == 0).all() and (sb == 0).all()
    assert (np.abs(a - b) / np.abs(b)).max() < RTOL_TF32


def test_graph_replay_of_grouped_batch(batch):
    ws, plans, bufs, ctx = batch
    eager, _ = _run(batch, 1)
    g = B.Graph(ctx, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32)
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        g.launch(st)
    torch.cuda.synchronize()
    logz, status = g.logz()
    assert (status == 0).all()
    assert np.array_equal(logz, eager)


def test_range_guard_records_nothing(batch, monkeypatch):
    monkeypatch.setenv("TN_GROUPED_GUARD", "1")
    logz, status = _run(batch, 1)
    assert (status == 0).all()
    monkeypatch.delenv("TN_GROUPED_GUARD")
    ref, _ = _run(batch, 1)
    assert np.array_equal(logz, ref)
