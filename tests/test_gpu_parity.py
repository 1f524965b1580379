"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerance (FP64 path): relative ln Z error <= 1e-10; per-tensor entries of one
density-matrix pass within 1e-9 absolute (unit-norm tensors, FP64 rounding of
a few hundred flops per entry, amplified by at most 1/gap of the spectra the
seeded inputs produce).
"""
import numpy as np
import pytest

from oracle import dmtree
from paper_2406_09769_gb300 import binding as B
from workloads import ising, prng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL_LOGZ = 1e-10


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


def _plan(w, chi):
    return B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=w["Ly"])


def _run(ctx, workloads, chi, precision=B.TN_PREC_FP64):
    plans = [_plan(w, chi) for w in workloads]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, workloads)]
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], precision, 0, _stream())
    return B.tn_logz(ctx, len(plans))


# ------------------------------------------------------------ one DM pass

def _random_chain(seed, d, D):
    n = len(d)
    shapes = [(1, d[0], D[0])] + [(D[k - 1], d[k], D[k]) for k in range(1, n - 1)] + \
             [(D[n - 2], d[n - 1], 1)]
    blocks, off = [], 0
    for s in shapes:
        size = int(np.prod(s))
        blocks.append((prng.uniform(seed, size, off) - 0.3).reshape(s))
        off += size
    return blocks


@pytest.mark.parametrize("d,D,chi", [
    ([2] * 8, [4, 8, 16, 16, 16, 8, 4], 5),
    ([2, 3, 2, 4, 2, 2, 3, 2, 2], [6, 12, 20, 24, 24, 20, 12, 6], 7),
    ([2] * 12, [4, 8, 16, 32, 64, 64, 64, 32, 16, 8, 4], 32),
    ([2] * 3, [4, 4], 1),
])
def test_embed_tree_matches_oracle(ctx, d, D, chi):
    n = len(d)
    n_inst = 3
    chains = [_random_chain(100 + i, d, D) for i in range(n_inst)]
    dev_in = [torch.from_numpy(np.concatenate([b.reshape(-1) for b in ch])).cuda() for ch in chains]
    ref, traces = [], []
    for ch in chains:
        blocks = [None, np.einsum("xeb,bfc->efc", ch[0], ch[1])] + ch[2:]
        tr = []
        ref.append(dmtree.density_matrix_alg(blocks, chi, trace=tr))
        traces.append(tr)
    r = [d[0]]
    for k in range(1, n - 1):
        r.append(min(chi, r[-1] * d[k], D[k], int(np.prod(d[k + 1:]))))
    sizes = [d[0] * d[1] * r[1]] + [r[k - 1] * d[k] * r[k] for k in range(2, n - 1)] + \
            [r[n - 2] * d[n - 1]]
    outs = [torch.full((sum(sizes),), np.nan, dtype=torch.float64, device="cuda")
            for _ in range(n_inst)]
    lognorm = torch.zeros(n_inst, dtype=torch.float64, device="cuda")
    status = torch.full((n_inst,), -1, dtype=torch.int32, device="cuda")
    ranks = B.tn_embed_tree(ctx, [x.data_ptr() for x in dev_in], d, D, chi,
                            [o.data_ptr() for o in outs], lognorm.data_ptr(), status.data_ptr(),
                            stream=_stream())
    torch.cuda.synchronize()
    assert list(ranks) == r
    assert status.cpu().tolist() == [0] * n_inst
    for i in range(n_inst):
        U_ref, Mr_ref, ln_ref = ref[i]
        got = outs[i].cpu().numpy()
        pos = 0
        compared = 0
        for v in range(1, n - 1):
            Ug = got[pos:pos + sizes[v - 1]].reshape(U_ref[v].shape)
            pos += sizes[v - 1]
            np.testing.assert_allclose(Ug.T @ Ug, np.eye(Ug.shape[1]), atol=1e-12)
            # An eigenvector is determined to ~eps ||L|| / gap (absolute
            # accuracy of any backward-stable solver): compare each column
            # with that bound, and the kept subspace when its gap is clear.
            lam = traces[i][v - 1]["lam"]
            rk = Ug.shape[1]
            for j in range(rk):
                gaps = [abs(lam[j] - lam[k]) for k in (j - 1, j + 1) if 0 <= k < len(lam)]
                relgap = (min(gaps) if gaps else lam[0]) / lam[0]
                if relgap > 1e-6:
                    np.testing.assert_allclose(Ug[:, j], U_ref[v][:, j],
                                               atol=1e-9 + 1e-13 / relgap)
                    compared += 1
            if rk < len(lam) and (lam[rk - 1] - lam[rk]) / lam[0] > 1e-8:
                np.testing.assert_allclose(Ug @ Ug.T, U_ref[v] @ U_ref[v].T, atol=1e-8)
        assert compared >= n - 2
        Mg = got[pos:].reshape(Mr_ref.shape)
        # gauge-invariant on the root's tree bond
        np.testing.assert_allclose(Mg.T @ Mg, Mr_ref.T @ Mr_ref, atol=1e-9)
        assert lognorm[i].item() == pytest.approx(ln_ref, abs=1e-11)


# ------------------------------------------------------- whole contraction

def test_config1_exact(ctx):
    w = ising.lattice2d(6, 6, 0.44)
    logz, status = _run(ctx, [w], 16)
    assert status[0] == 0
    assert abs(logz[0] - 31.564145959482058) <= RTOL_LOGZ * 31.6
    assert abs(logz[0] - dmtree.partitioned_contract_rows(w, 16)["logz"]) <= RTOL_LOGZ * 31.6


@pytest.mark.parametrize("Lx,Ly,beta,cp,chi", [
    (6, 9, 0.8, "gauss", 4), (8, 8, 0.5, "gauss", 6), (7, 10, 1.0, "pm1", 5),
    (3, 11, 0.6, "gauss", 3), (2, 7, 0.5, "gauss", 4), (7, 3, 0.9, "gauss", 1),
    (5, 5, 0.44, "ferro", 100), (12, 14, 0.7, "gauss", 17)])
def test_contract_matches_oracle(ctx, Lx, Ly, beta, cp, chi):
    ws = [ising.lattice2d(Lx, Ly, beta, cp, seed=1000 * Lx + Ly + i) for i in range(5)]
    logz, status = _run(ctx, ws, chi)
    assert list(status) == [0] * 5
    for i, w in enumerate(ws):
        ref = dmtree.partitioned_contract_rows(w, chi)["logz"]
        assert abs(logz[i] - ref) <= RTOL_LOGZ * abs(ref), (i, logz[i], ref)


def test_full_size_config2_sampled(ctx):
    """32x32 spin glass, chi = 64, in a batch; instances 0 and last sampled."""
    n_inst = 8
    ws = [ising.config2_instance(i) for i in range(n_inst)]
    logz, status = _run(ctx, ws, 64)
    assert list(status) == [0] * n_inst
    for i in (0, n_inst - 1):
        ref = dmtree.partitioned_contract_rows(ws[i], 64)["logz"]
        assert abs(logz[i] - ref) <= RTOL_LOGZ * abs(ref), (i, logz[i], ref)


def test_nonfinite_instance_is_isolated(ctx):
    ws = [ising.lattice2d(6, 7, 0.6, "gauss", seed=s) for s in range(3)]
    bad = dict(ws[1])
    bad["tensors"] = [t.copy() for t in ws[1]["tensors"]]
    bad["tensors"][10][0, 0, 0, 0] = np.nan
    logz, status = _run(ctx, [ws[0], bad, ws[2]], 4)
    assert list(status) == [0, 4, 0]
    assert np.isnan(logz[1])
    for i in (0, 2):
        ref = dmtree.partitioned_contract_rows(ws[i], 4)["logz"]
        assert abs(logz[i] - ref) <= RTOL_LOGZ * abs(ref)


def test_nonpositive_result_reported(ctx):
    w = ising.lattice2d(5, 6, 0.5)
    neg = dict(w)
    neg["tensors"] = [t.copy() for t in w["tensors"]]
    neg["tensors"][7] = -neg["tensors"][7]          # Z -> -Z exactly
    logz, status = _run(ctx, [w, neg], 8)
    assert list(status) == [0, 5]
    assert dmtree.partitioned_contract_rows(neg, 8)["sign"] < 0


def test_host_entry_point_equals_device_path(ctx):
    ws = [ising.lattice2d(9, 8, 0.7, "gauss", seed=s) for s in range(4)]
    plans = [_plan(w, 6) for w in ws]
    host = [B.pack_sites(p, w["tensors"]) for p, w in zip(plans, ws)]
    pinned = [torch.from_numpy(h).pin_memory() for h in host]
    logz_h, st_h = B.tn_contract_approx_host(ctx, plans, [t.data_ptr() for t in pinned],
                                             B.TN_PREC_FP64, 0, _stream())
    logz_d, st_d = _run(ctx, ws, 6)
    assert list(st_h) == [0] * 4 and list(st_d) == [0] * 4
    assert np.array_equal(logz_h, logz_d)            # same kernels, same inputs: bitwise


def test_repeatable_bitwise(ctx):
    ws = [ising.lattice2d(10, 10, 0.6, "gauss", seed=s) for s in range(3)]
    a, _ = _run(ctx, ws, 8)
    b, _ = _run(ctx, ws, 8)
    assert np.array_equal(a, b)
