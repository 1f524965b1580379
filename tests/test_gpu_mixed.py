"""GPU parity of the mixed-precision (TF32 tensor-core) path against the FP64
oracle.  Bar: relative ln Z error <= 1e-6 with the same chi (the truncation is
the oracle's, so this is the error the mixed precision adds beyond it), on
every case, including truncations far below the largest eigenvalue: the
default mixed mode never forms L_v, it takes the leading left singular
vectors of K_v = M_v C_v with R_v = C_v C_v^T."""
import numpy as np
import pytest

from oracle import dmtree
from paper_2406_09769_gb300 import binding as B
from workloads import ising, potts, random_tn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    return B.tn_ctx_create(0)


def _exact_config2(n_inst):
    """Kac-Ward ln Z of config-2 instances 0..n_inst-1 (tests/golden/exact_logz.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "exact_logz.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("config2_32x32_gauss_i"):
                parts = line.split()
                vals[int(parts[0].rsplit("_i", 1)[1])] = float(parts[-1])
    return np.array([vals[i] for i in range(n_inst)])


def _run(ctx, ws, chi, precision):
    plans = [B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), 2), chi, env_size=w["Ly"])
             for w in ws]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], precision, 0,
                         torch.cuda.current_stream().cuda_stream)
    return B.tn_logz(ctx, len(plans))


def test_tf32_config1_exact(ctx):
    w = ising.lattice2d(6, 6, 0.44)
    logz, status = _run(ctx, [w], 16, B.TN_PREC_TF32)
    assert status[0] == 0
    assert abs(logz[0] - 31.564145959482058) <= RTOL_MIXED * 31.6


def _oracle(w, chi):
    return dmtree.partitioned_contract_rows(w, chi)["logz"]


@pytest.mark.parametrize("Lx,Ly,beta,cp,chi", [
    (6, 9, 0.8, "gauss", 4), (8, 8, 0.5, "gauss", 6), (7, 10, 1.0, "pm1", 5),
    (3, 11, 0.6, "gauss", 3), (2, 7, 0.5, "gauss", 4), (7, 3, 0.9, "gauss", 1),
    (12, 14, 0.7, "gauss", 17), (16, 16, 0.5, "gauss", 32)])
def test_tf32_matches_oracle(ctx, Lx, Ly, beta, cp, chi):
    ws = [ising.lattice2d(Lx, Ly, beta, cp, seed=500 * Lx + Ly + i) for i in range(6)]
    logz, status = _run(ctx, ws, chi, B.TN_PREC_TF32)
    assert list(status) == [0] * len(ws)
    for i, w in enumerate(ws):
        ref = _oracle(w, chi)
        assert abs(logz[i] - ref) <= RTOL_MIXED * abs(ref), (i, logz[i], ref)


@pytest.mark.parametrize("q,Lx,Ly,chi", [(3, 6, 6, 12), (3, 5, 7, 20), (4, 4, 5, 16)])
def test_tf32_potts_matches_oracle(ctx, q, Lx, Ly, chi):
    """Bond dimension q != 2 (q-state Potts): every row takes the general
    fusion kernel, and contraction shapes that are not multiples of four take
    the plain-FMA fallback."""
    ws = [potts.lattice2d(Lx, Ly, 0.6, q, "uniform", seed=300 + 10 * q + i) for i in range(3)]
    plans = [B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), q), chi, env_size=w["Ly"])
             for w in ws]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], B.TN_PREC_TF32, 0,
                         torch.cuda.current_stream().cuda_stream)
    logz, status = B.tn_logz(ctx, len(plans))
    assert list(status) == [0] * len(ws)
    for i, w in enumerate(ws):
        ref = _oracle(w, chi)
        assert abs(logz[i] - ref) <= RTOL_MIXED * abs(ref), (i, logz[i], ref)


@pytest.mark.parametrize("L,alpha,chi", [(8, 0.0, 8), (28, 0.0, 32)])
def test_tf32_random_tensors_match_oracle(ctx, L, alpha, chi):
    """Random tensor networks with entries uniform on [0, 1], including the
    paper's 28 x 28 lattice size."""
    ws = [random_tn.lattice2d(L, L, alpha, seed=900 + 7 * L + i) for i in range(3)]
    logz, status = _run(ctx, ws, chi, B.TN_PREC_TF32)
    assert list(status) == [0] * len(ws)
    for i, w in enumerate(ws):
        ref = _oracle(w, chi)
        assert abs(logz[i] - ref) <= RTOL_MIXED * abs(ref), (i, logz[i], ref)


@pytest.mark.parametrize("chi", [32, 64])
def test_tf32_full_size_config2_sampled(ctx, chi):
    n_inst = 8
    ws = [ising.config2_instance(i) for i in range(n_inst)]
    logz, status = _run(ctx, ws, chi, B.TN_PREC_TF32)
    fp64, st64 = _run(ctx, ws, chi, B.TN_PREC_FP64)
    assert list(status) == [0] * n_inst and list(st64) == [0] * n_inst
    assert np.max(np.abs(logz - fp64) / np.abs(fp64)) <= RTOL_MIXED
    for i in (0, n_inst - 1):
        ref = dmtree.partitioned_contract_rows(ws[i], chi)["logz"]
        assert abs(logz[i] - ref) <= RTOL_MIXED * abs(ref), (i, logz[i], ref)
    # every instance against the exact (Kac-Ward) value, which the method
    # reaches at this temperature to FP64 rounding
    ex = _exact_config2(n_inst)
    assert np.max(np.abs(logz - ex) / np.abs(ex)) <= RTOL_MIXED


def test_tf32_nonfinite_instance_is_isolated(ctx):
    ws = [ising.lattice2d(6, 8, 0.6, "gauss", seed=s) for s in range(3)]
    bad = dict(ws[2])
    bad["tensors"] = [t.copy() for t in ws[2]["tensors"]]
    bad["tensors"][5].flat[3] = np.inf
    logz, status = _run(ctx, [ws[0], ws[1], bad], 4, B.TN_PREC_TF32)
    assert list(status) == [0, 0, 4]
    for i in (0, 1):
        ref = dmtree.partitioned_contract_rows(ws[i], 4)["logz"]
        assert abs(logz[i] - ref) <= RTOL_MIXED * abs(ref)


def test_tf32_fast_mode_error_is_bounded(ctx):
    """Plain TF32 on the density-matrix side: directions below ~1e-3 of the
    top eigenvalue are resolved only to TF32 noise; the measured cost on the
    32x32 chi=64 workload is a few 1e-6 relative in ln Z (bound 2e-5 here).
    A fast mode with a stated error, not the default."""
    ws = [ising.config2_instance(i) for i in range(4)]
    fast, st = _run(ctx, ws, 64, B.TN_PREC_TF32_FAST)
    fp64, st64 = _run(ctx, ws, 64, B.TN_PREC_FP64)
    assert list(st) == [0] * 4 and list(st64) == [0] * 4
    assert np.max(np.abs(fast - fp64) / np.abs(fp64)) <= 2e-5


def test_tf32_gram_mode_error_is_bounded(ctx):
    """L_v formed in FP32 (compensated products) with an FP32 eigensolver:
    eigen-directions below ~1e-7 of the top eigenvalue are noise.  On the
    32x32 chi=64 workload the cost stays below 1e-6 relative; on strongly
    truncated runs it reaches a few 1e-6 (measured), which is why it is not
    the default."""
    ws = [ising.config2_instance(i) for i in range(4)]
    gram, st = _run(ctx, ws, 64, B.TN_PREC_TF32_GRAM)
    fp64, st64 = _run(ctx, ws, 64, B.TN_PREC_FP64)
    assert list(st) == [0] * 4 and list(st64) == [0] * 4
    assert np.max(np.abs(gram - fp64) / np.abs(fp64)) <= 1e-6


def test_unsupported_precision_is_reported(ctx):
    w = ising.lattice2d(4, 4, 0.5)
    with pytest.raises(B.TNError) as e:
        _run(ctx, [w], 4, B.TN_PREC_BF16)
    assert e.value.status == 8


# ------------------------------------------------------ one pass, per edge

def _chain(seed, d, D):
    from workloads import prng
    n = len(d)
    shapes = [(1, d[0], D[0])] + [(D[k - 1], d[k], D[k]) for k in range(1, n - 1)] + \
             [(D[n - 2], d[n - 1], 1)]
    blocks, off = [], 0
    for s in shapes:
        size = int(np.prod(s))
        blocks.append((prng.uniform(seed, size, off) - 0.3).reshape(s))
        off += size
    return blocks


def _isometries(U, d, n):
    """B_v = U_1 ... U_v as (prod of leaf dims) x r_v matrices."""
    out = [None] * n
    Bv = U[1]
    out[1] = Bv
    for v in range(2, n - 1):
        r = U[v].shape[1]
        Bv = (Bv.reshape(-1, U[v].shape[0] // d[v]) @ U[v].reshape(-1, d[v] * r)).reshape(-1, r)
        out[v] = Bv
    return out


@pytest.mark.parametrize("d,D,chi", [
    ([2] * 8, [4, 8, 16, 16, 16, 8, 4], 5),
    ([2, 3, 2, 4, 2, 2, 3, 2, 2], [6, 12, 20, 24, 24, 20, 12, 6], 7),
    ([2] * 12, [4, 8, 16, 32, 64, 64, 64, 32, 16, 8, 4], 32),
])
def test_tf32_embed_tree_per_edge_matches_oracle(ctx, d, D, chi):
    """One factored mixed-precision pass (tn_embed_tree, TN_PREC_TF32) on
    explicit blocks, edge by edge: orthonormal tree tensors, the kept
    subspaces (projectors of the isometries B_v) where the singular-value gap
    at the cut resolves them in FP32, the tensor the tree represents and its
    log-norm, against the FP64 oracle."""
    n = len(d)
    n_inst = 3
    chains = [_chain(200 + i, d, D) for i in range(n_inst)]
    dev_in = [torch.from_numpy(np.concatenate([b.reshape(-1) for b in ch])).cuda() for ch in chains]
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
                            precision=B.TN_PREC_TF32,
                            stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert list(ranks) == r
    assert status.cpu().tolist() == [0] * n_inst
    for i, ch in enumerate(chains):
        blocks = [None, np.einsum("xeb,bfc->efc", ch[0], ch[1])] + ch[2:]
        tr = []
        U_ref, Mr_ref, ln_ref = dmtree.density_matrix_alg(blocks, chi, trace=tr)
        got = outs[i].cpu().numpy()
        assert np.all(np.isfinite(got))
        Ug, pos = [None] * n, 0
        for v in range(1, n - 1):
            Ug[v] = got[pos:pos + sizes[v - 1]].reshape(U_ref[v].shape)
            pos += sizes[v - 1]
            np.testing.assert_allclose(Ug[v].T @ Ug[v], np.eye(Ug[v].shape[1]), atol=2e-6)
        Mg = got[pos:].reshape(Mr_ref.shape)
        Bg, Br = _isometries(Ug, d, n), _isometries(U_ref, d, n)
        gapmin = 1.0  # smallest relative singular-value gap at a cut so far
        for v in range(1, n - 1):
            s = np.sqrt(np.maximum(tr[v - 1]["lam"], 0.0))
            rk = Ug[v].shape[1]
            if rk < len(s):
                gapmin = min(gapmin, (s[rk - 1] - s[rk]) / s[0])
            if gapmin > 1e-3:
                # Davis-Kahan: subspace error <= backward error / gap, with the
                # FP32 SVD's backward error a few eps_32 of ||K_v|| (2e-7)
                np.testing.assert_allclose(Bg[v] @ Bg[v].T, Br[v] @ Br[v].T,
                                           atol=2e-6 + 2e-7 / gapmin)
        psi_g = (Bg[n - 2].reshape(-1, Mg.shape[0]) @ Mg).reshape(-1)
        psi_r = (Br[n - 2].reshape(-1, Mr_ref.shape[0]) @ Mr_ref).reshape(-1)
        np.testing.assert_allclose(psi_g, psi_r, atol=2e-5)
        # the mixed path's bar: 1e-6 relative (absolute below a log-norm of 1)
        assert lognorm[i].item() == pytest.approx(ln_ref, abs=1e-6 * max(1.0, abs(ln_ref)))


def test_tf32_embed_tree_on_spin_glass_blocks(ctx):
    """The factored pass on the blocks of a real row absorption (kept spectrum
    spanning many decades): the represented tensor and its log-norm."""
    w = ising.lattice2d(8, 14, 0.7, "gauss", seed=77)
    trace = []
    dmtree.partitioned_contract_rows(w, 12, trace=trace)
    blocks = trace[3]["blocks"]
    n = len(blocks)
    b1 = blocks[1]
    d0 = b1.shape[0]
    Y = [np.eye(d0).reshape(1, d0, d0), b1.reshape(d0, b1.shape[1], b1.shape[2])] + blocks[2:]
    d = [y.shape[1] for y in Y]
    D = [y.shape[2] for y in Y[:-1]]
    dev_in = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y])).cuda()
    out = torch.zeros(1 << 20, dtype=torch.float64, device="cuda")
    lognorm = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ranks = B.tn_embed_tree(ctx, [dev_in.data_ptr()], d, D, 12, [out.data_ptr()],
                            lognorm.data_ptr(), status.data_ptr(), precision=B.TN_PREC_TF32,
                            stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert status.item() == 0
    U_ref, Mr_ref, ln_ref = dmtree.density_matrix_alg(blocks, 12)
    got = out.cpu().numpy()
    pos, Ug = 0, [None] * n
    for v in range(1, n - 1):
        size = U_ref[v].shape[0] * ranks[v]
        Ug[v] = got[pos:pos + size].reshape(U_ref[v].shape)
        pos += size
    Mg = got[pos:pos + Mr_ref.size].reshape(Mr_ref.shape)
    Bg, Br = _isometries(Ug, d, n), _isometries(U_ref, d, n)
    psi_g = (Bg[n - 2] @ Mg).reshape(-1)
    psi_r = (Br[n - 2] @ Mr_ref).reshape(-1)
    np.testing.assert_allclose(psi_g, psi_r, atol=2e-5)
    assert lognorm.item() == pytest.approx(ln_ref, abs=1e-6 * max(1.0, abs(ln_ref)))
