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
from workloads import ising, potts, prng, random_tn

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
        Ug_all = [None] * n
        for v in range(1, n - 1):
            Ug = got[pos:pos + sizes[v - 1]].reshape(U_ref[v].shape)
            pos += sizes[v - 1]
            Ug_all[v] = Ug
            np.testing.assert_allclose(Ug.T @ Ug, np.eye(Ug.shape[1]), atol=1e-12)
        Mg = got[pos:].reshape(Mr_ref.shape)
        # Vertex 1 has no upstream gauge: its eigenvectors are compared one by
        # one within their accuracy eps ||L|| / gap.
        lam = traces[i][0]["lam"]
        for j in range(Ug_all[1].shape[1]):
            gaps = [abs(lam[j] - lam[k]) for k in (j - 1, j + 1) if 0 <= k < len(lam)]
            relgap = (min(gaps) if gaps else lam[0]) / lam[0]
            if relgap > 1e-6:
                np.testing.assert_allclose(Ug_all[1][:, j], U_ref[1][:, j],
                                           atol=1e-9 + 1e-13 / relgap)
        # Downstream vertices are fixed only up to rotations inside (near-)
        # degenerate kept eigenspaces, which propagate through P = U^T M; the
        # gauge-invariant objects are the kept subspaces (projectors of the
        # isometries B_v = U_1 ... U_v) and the tensor the tree represents.
        Bg = Br = None
        gapmin = 1.0          # smallest relative truncation gap so far (Davis-Kahan)
        for v in range(1, n - 1):
            if v == 1:
                Bg, Br = Ug_all[1], U_ref[1]
            else:
                Bg = (Bg.reshape(-1, Ug_all[v].shape[0] // d[v]) @
                      Ug_all[v].reshape(-1, d[v] * Ug_all[v].shape[1])).reshape(-1, Ug_all[v].shape[1])
                Br = (Br.reshape(-1, U_ref[v].shape[0] // d[v]) @
                      U_ref[v].reshape(-1, d[v] * U_ref[v].shape[1])).reshape(-1, U_ref[v].shape[1])
            lamv = traces[i][v - 1]["lam"]
            rk = Bg.shape[1]
            if rk < len(lamv):
                gapmin = min(gapmin, (lamv[rk - 1] - lamv[rk]) / lamv[0])
            if gapmin > 1e-10:
                np.testing.assert_allclose(Bg @ Bg.T, Br @ Br.T, atol=1e-10 + 1e-14 / gapmin)
        psi_g = (Bg.reshape(-1, Mg.shape[0]) @ Mg).reshape(-1)
        psi_r = (Br.reshape(-1, Mr_ref.shape[0]) @ Mr_ref).reshape(-1)
        if gapmin > 1e-10:
            np.testing.assert_allclose(psi_g, psi_r, atol=1e-10 + 1e-14 / gapmin)
            assert lognorm[i].item() == pytest.approx(ln_ref, abs=1e-11 + 1e-14 / gapmin)


def test_embed_tree_on_spin_glass_blocks(ctx):
    """The DM pass on blocks of a real row absorption (physical spectra)."""
    w = ising.lattice2d(8, 14, 0.7, "gauss", seed=77)
    trace = []
    dmtree.partitioned_contract_rows(w, 12, trace=trace)
    step = trace[3]                                   # absorbing row 4
    blocks = step["blocks"]
    n = len(blocks)
    # split vertex 1's block back into Y_0 (1, d0, d0) = identity and Y_1
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
                            lognorm.data_ptr(), status.data_ptr(), stream=_stream())
    torch.cuda.synchronize()
    assert status.item() == 0
    U_ref, Mr_ref, ln_ref = dmtree.density_matrix_alg(blocks, 12)
    got = out.cpu().numpy()
    pos, Bg, Br = 0, None, None
    for v in range(1, n - 1):
        r = ranks[v]
        size = U_ref[v].shape[0] * r
        Ug = got[pos:pos + size].reshape(U_ref[v].shape)
        pos += size
        if v == 1:
            Bg, Br = Ug, U_ref[1]
        else:
            Bg = (Bg @ Ug.reshape(-1, d[v] * r)).reshape(-1, r)
            Br = (Br @ U_ref[v].reshape(-1, d[v] * r)).reshape(-1, r)
    # Here L_v has numerical rank below chi (kept eigenvalues down to ~1e-26
    # of the largest), so part of each kept basis is rounding noise in both
    # codes; the represented tensor and its norm are what is determined.
    Mg = got[pos:pos + Mr_ref.size].reshape(Mr_ref.shape)
    np.testing.assert_allclose((Bg @ Mg).reshape(-1), (Br @ Mr_ref).reshape(-1), atol=1e-10)
    assert lognorm.item() == pytest.approx(ln_ref, abs=1e-11)


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


@pytest.mark.parametrize("q,Lx,Ly,chi", [(3, 6, 6, 12), (3, 5, 7, 20), (4, 4, 5, 16)])
def test_potts_contract_matches_oracle(ctx, q, Lx, Ly, chi):
    """Bond dimension q != 2 (q-state Potts): the general fusion and the
    contraction shapes that are not multiples of four."""
    ws = [potts.lattice2d(Lx, Ly, 0.6, q, "uniform", seed=300 + 10 * q + i) for i in range(3)]
    plans = [B.tn_plan(w["n"], w["edges"], np.full(len(w["edges"]), q), chi, env_size=w["Ly"])
             for w in ws]
    bufs = [torch.from_numpy(B.pack_sites(p, w["tensors"])).cuda() for p, w in zip(plans, ws)]
    B.tn_contract_approx(ctx, plans, [b.data_ptr() for b in bufs], B.TN_PREC_FP64, 0, _stream())
    logz, status = B.tn_logz(ctx, len(plans))
    assert list(status) == [0] * len(ws)
    for i, w in enumerate(ws):
        ref = dmtree.partitioned_contract_rows(w, chi)["logz"]
        assert abs(logz[i] - ref) <= RTOL_LOGZ * abs(ref), (i, logz[i], ref)


@pytest.mark.parametrize("L,alpha,chi", [(8, 0.0, 8), (8, -0.3, 8), (28, -0.2, 32)])
def test_random_tensors_match_oracle(ctx, L, alpha, chi):
    """Random tensor networks (entries uniform on [alpha, 1]), including the
    paper's 28 x 28 lattice size.  With negative entries Z itself can be
    negative (8 x 8, alpha = -0.3, seed 957): ln Z is then undefined, the oracle
    returns sign -1 and the library must report TN_ERR_NONPOSITIVE (5)."""
    ws = [random_tn.lattice2d(L, L, alpha, seed=900 + 7 * L + i) for i in range(3)]
    logz, status = _run(ctx, ws, chi)
    for i, w in enumerate(ws):
        r = dmtree.partitioned_contract_rows(w, chi)
        if r["sign"] < 0:
            assert status[i] == 5, (i, status[i])
            continue
        assert status[i] == 0, (i, status[i])
        assert abs(logz[i] - r["logz"]) <= RTOL_LOGZ * abs(r["logz"]), (i, logz[i], r["logz"])


def test_full_size_config2_sampled(ctx):
    """32x32 spin glass, chi = 64, in a batch; instances 0 and last against the
    oracle, every instance against the exact (Kac-Ward) value, which the method
    reaches at this temperature to FP64 rounding."""
    n_inst = 8
    ws = [ising.config2_instance(i) for i in range(n_inst)]
    logz, status = _run(ctx, ws, 64)
    assert list(status) == [0] * n_inst
    for i in (0, n_inst - 1):
        ref = dmtree.partitioned_contract_rows(ws[i], 64)["logz"]
        assert abs(logz[i] - ref) <= RTOL_LOGZ * abs(ref), (i, logz[i], ref)
    ex = _exact_config2(n_inst)
    assert np.max(np.abs(logz - ex) / np.abs(ex)) <= RTOL_LOGZ


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
