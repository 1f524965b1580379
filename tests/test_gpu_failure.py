"""Failure paths, exercised without a GPU fault: an injected host-side
allocation failure (TN_FAULT_ALLOC_AT), an eigensolver whose search is cut
short (TN_OPT_EIG_ROUNDS: per-instance TN_ERR_EIG_NOCONV) and a bounded device
wait that runs out on a flag nothing sets (TN_OPT_WAIT_PROBE: TN_ERR_TIMEOUT).
After each, the same ctx must produce correct results again."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import dmtree
from paper_2406_09769_gb300 import binding as B
from workloads import ising

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    return B.tn_ctx_create(0)


def _batch(n=3, Lx=6, Ly=6, beta=0.6, chi=8):
    ws = [ising.lattice2d(Lx, Ly, beta, "gauss", seed=4000 + i) for i in range(n)]
    plans = [B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=Ly)
             for w in ws]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    refs = [dmtree.partitioned_contract_rows(w, chi)["logz"] for w in ws]
    return plans, bufs, np.array(refs)


def _run(ctx, plans, bufs, prec):
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], prec, 0,
                         torch.cuda.current_stream().cuda_stream)
    return B.tn_logz(ctx, len(plans))


_ALLOC_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_2406_09769_gb300 import binding as B
from workloads import ising
w = ising.lattice2d(6, 6, 0.6, "gauss", seed=4100)
plan = B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), 8, env_size=6)
sites = torch.from_numpy(B.pack_sites(plan, w["tensors"])).cuda()
# a first ctx loads the library's kernels and makes three device allocations
warm = B.tn_ctx_create(0)
B.tn_contract_approx(warm, [plan], [sites.data_ptr()], {prec}, 0, 0)
B.tn_logz(warm, 1)
B.tn_ctx_destroy(warm)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
ctx = B.tn_ctx_create(0)
out = {{}}
try:
    B.tn_contract_approx(ctx, [plan], [sites.data_ptr()], {prec}, 0, 0)
    out["first"] = 0
except B.TNError as e:
    out["first"] = e.status
B.tn_contract_approx(ctx, [plan], [sites.data_ptr()], {prec}, 0, 0)
lz, st = B.tn_logz(ctx, 1)
out["second_status"] = int(st[0])
out["logz"] = float(lz[0])
B.tn_ctx_destroy(ctx)
torch.cuda.synchronize()
out["leak_bytes"] = int(free0 - torch.cuda.mem_get_info()[0])
print(json.dumps(out))
"""


@pytest.mark.parametrize("prec", [B.TN_PREC_FP64, B.TN_PREC_TF32])
def test_injected_allocation_failure_reports_oom_and_ctx_recovers(prec):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    # allocations 1-3 belong to the warm-up ctx; the test ctx's second (its
    # workspace arena) is the fifth of the process and fails
    env = dict(os.environ, TN_FAULT_ALLOC_AT="5")
    r = subprocess.run([sys.executable, "-c", _ALLOC_SCRIPT.format(root=ROOT, prec=prec)],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["first"] == 2                       # TN_ERR_OOM
    assert out["second_status"] == 0
    w = ising.lattice2d(6, 6, 0.6, "gauss", seed=4100)
    ref = dmtree.partitioned_contract_rows(w, 8)["logz"]
    tol = 1e-10 if prec == B.TN_PREC_FP64 else 1e-6
    assert abs(out["logz"] - ref) <= tol * abs(ref)
    assert abs(out["leak_bytes"]) <= 8 << 20       # the ctx's workspace went back


def test_eigensolver_cut_short_reports_noconv_per_instance(ctx):
    plans, bufs, refs = _batch()
    B.tn_ctx_set_option(ctx, B.TN_OPT_EIG_ROUNDS, 1)
    try:
        _, status = _run(ctx, plans, bufs, B.TN_PREC_TF32)
    finally:
        B.tn_ctx_set_option(ctx, B.TN_OPT_EIG_ROUNDS, 9)
    assert list(status) == [7] * len(plans)       # TN_ERR_EIG_NOCONV
    logz, status = _run(ctx, plans, bufs, B.TN_PREC_TF32)
    assert list(status) == [0] * len(plans)
    assert np.max(np.abs(logz - refs) / np.abs(refs)) <= 1e-6


def test_expired_device_wait_reports_timeout_and_ctx_recovers(ctx):
    plans, bufs, refs = _batch()
    B.tn_ctx_set_option(ctx, B.TN_OPT_WAIT_PROBE, 1)
    logz, status = _run(ctx, plans, bufs, B.TN_PREC_TF32)
    assert list(status) == [6] * len(plans)       # TN_ERR_TIMEOUT
    assert np.all(np.isnan(logz))
    # the probe applies to one batch only; the ctx is usable afterwards
    logz, status = _run(ctx, plans, bufs, B.TN_PREC_TF32)
    assert list(status) == [0] * len(plans)
    assert np.max(np.abs(logz - refs) / np.abs(refs)) <= 1e-6


def test_rejected_option_values(ctx):
    with pytest.raises(B.TNError) as e:
        B.tn_ctx_set_option(ctx, B.TN_OPT_EIG_ROUNDS, 0)
    assert e.value.status == 1
    with pytest.raises(B.TNError) as e:
        B.tn_ctx_set_option(ctx, 99, 1)
    assert e.value.status == 1
