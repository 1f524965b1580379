"""Batching support: heterogeneous batches (different lattice sizes and chi in
one tn_contract_approx), a batch captured once into a CUDA graph and
replayed, and autotuned tensor-core tiles.  Every instance is checked against
the FP64 oracle; the batched, replayed and tuned runs must also equal the
plain single-instance runs bit for bit (the arithmetic of an instance does
not depend on its batch, and every tile candidate computes the same values)."""
import os

import numpy as np
import pytest

from oracle import dmtree
from paper_2406_09769_gb300 import binding as B
from workloads import ising

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (Lx, Ly, beta, chi): four plan structures, one of them twice
MIX = [(6, 6, 0.6, 8), (8, 7, 0.5, 16), (5, 9, 0.7, 4), (6, 6, 0.6, 8), (7, 7, 0.8, 6),
       (9, 6, 0.5, 12)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    return B.tn_ctx_create(0)


@pytest.fixture(scope="module")
def mix():
    ws, plans, bufs, refs = [], [], [], []
    for i, (Lx, Ly, beta, chi) in enumerate(MIX):
        w = ising.lattice2d(Lx, Ly, beta, "gauss", seed=6000 + i)
        p = B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=Ly)
        ws.append(w)
        plans.append(p)
        bufs.append(torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda())
        refs.append(dmtree.partitioned_contract_rows(w, chi)["logz"])
    return ws, plans, bufs, np.array(refs)


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _run(ctx, plans, bufs, prec):
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], prec, 0, _stream())
    return B.tn_logz(ctx, len(plans))


@pytest.mark.parametrize("prec,tol", [(B.TN_PREC_FP64, 1e-10), (B.TN_PREC_TF32, 1e-6)])
def test_heterogeneous_batch_matches_oracle_and_single_runs(ctx, mix, prec, tol):
    _, plans, bufs, refs = mix
    logz, status = _run(ctx, plans, bufs, prec)
    assert list(status) == [0] * len(plans)
    assert np.max(np.abs(logz - refs) / np.abs(refs)) <= tol
    single = np.array([_run(ctx, [p], [b], prec)[0][0] for p, b in zip(plans, bufs)])
    assert np.array_equal(logz, single)


def test_heterogeneous_batch_from_host_buffers(ctx, mix):
    ws, plans, _, refs = mix
    host = [np.ascontiguousarray(B.pack_sites(p, w["tensors"])) for p, w in zip(plans, ws)]
    logz, status = B.tn_contract_approx_host(ctx, plans, [h.ctypes.data for h in host],
                                             B.TN_PREC_TF32, 0, _stream())
    assert list(status) == [0] * len(plans)
    assert np.max(np.abs(logz - refs) / np.abs(refs)) <= 1e-6


def test_batch_graph_replays_the_batch_and_follows_the_site_buffers(ctx, mix):
    ws, plans, bufs, refs = mix
    eager, _ = _run(ctx, plans, bufs, B.TN_PREC_TF32)
    g = B.Graph(ctx, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32)
    for _ in range(2):
        g.launch(_stream())
        logz, status = g.logz()
        assert list(status) == [0] * len(plans)
        assert np.array_equal(logz, eager)
    # scaling every site tensor of instance 1 by 2 multiplies its Z by 2^|V|
    saved = bufs[1].clone()
    bufs[1].mul_(2.0)
    torch.cuda.synchronize()
    g.launch(_stream())
    logz2, status2 = g.logz()
    bufs[1].copy_(saved)
    torch.cuda.synchronize()
    assert list(status2) == [0] * len(plans)
    nv = ws[1]["n"]
    assert abs(logz2[1] - (eager[1] + nv * np.log(2.0))) <= 1e-6 * abs(logz2[1])
    assert np.array_equal(np.delete(logz2, 1), np.delete(eager, 1))
    # the ctx itself is free for other batches meanwhile
    logz3, _ = _run(ctx, plans[:2], bufs[:2], B.TN_PREC_TF32)
    assert np.array_equal(logz3, eager[:2])
    del g


def test_autotuned_tiles_keep_results_and_round_trip_through_the_cache(mix, tmp_path):
    _, plans, bufs, refs = mix
    c1 = B.tn_ctx_create(0)
    base, _ = _run(c1, plans, bufs, B.TN_PREC_TF32)
    cache = str(tmp_path / "tiles.json")
    n = B.tn_autotune(c1, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32, cache)
    assert n > 0 and os.path.exists(cache)
    tuned, status = _run(c1, plans, bufs, B.TN_PREC_TF32)
    assert list(status) == [0] * len(plans)
    assert np.array_equal(tuned, base)
    c2 = B.tn_ctx_create(0)
    assert B.tn_autotune(c2, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32, cache) == n
    again, _ = _run(c2, plans, bufs, B.TN_PREC_TF32)
    assert np.array_equal(again, base)
    text = open(cache).read()
    assert '"entries"' in text and '"BN"' in text
