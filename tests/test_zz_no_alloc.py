"""The allocation-free density-matrix pass (tn_embed_tree_noalloc).

Some callers cannot allocate device memory (their own allocator holds the
device's memory, their host forbids direct allocation, or cudaMalloc's
possible device synchronisation is not acceptable in their loop).  For them
the library offers one entry point whose workspace is a fixed device array
compiled into the library.  This file checks it through the C ABI against the
ctx-based tn_embed_tree on the same inputs, on two calls in a row (the second
with different data, since the shared array keeps the previous contents), and
that an oversized problem is refused.  It is named to be collected last.
"""
import numpy as np
import pytest

from paper_2406_09769_gb300 import binding as B
from workloads import prng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ATOL = 1e-9          # the per-tensor tolerance of the one-pass parity tests


def _chain(seed, d, D):
    n = len(d)
    shapes = [(1, d[0], D[0])] + [(D[k - 1], d[k], D[k]) for k in range(1, n - 1)] + \
             [(D[n - 2], d[n - 1], 1)]
    flat, off = [], 0
    for s in shapes:
        size = int(np.prod(s))
        flat.append(prng.uniform(seed, size, off) - 0.3)
        off += size
    return torch.from_numpy(np.concatenate(flat)).cuda()


def _run(entry, blocks, d, D, chi, ctx=None):
    n_inst = len(blocks)
    outs = [torch.full((1 << 16,), np.nan, dtype=torch.float64, device="cuda") for _ in range(n_inst)]
    lognorm = torch.full((n_inst,), np.nan, dtype=torch.float64, device="cuda")
    status = torch.full((n_inst,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    if entry == "ctx":
        ranks = B.tn_embed_tree(ctx, [b.data_ptr() for b in blocks], d, D, chi,
                                [o.data_ptr() for o in outs], lognorm.data_ptr(),
                                status.data_ptr(), stream=stream)
    else:
        ranks = B.tn_embed_tree_noalloc([b.data_ptr() for b in blocks], d, D, chi,
                                        [o.data_ptr() for o in outs], lognorm.data_ptr(),
                                        status.data_ptr(), stream=stream)
    torch.cuda.synchronize()
    return ranks, [o.cpu().numpy() for o in outs], lognorm.cpu().numpy(), status.cpu().numpy()


def test_noalloc_pass_matches_ctx_pass_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_2406_09769_gb300 import build
        build.build()
    ctx = B.tn_ctx_create(0)
    cases = [([2] * 10, [4, 8, 16, 32, 32, 32, 16, 8, 4], 12, 7),
             ([2, 3, 2, 2, 3, 2, 2], [6, 12, 18, 18, 12, 6], 9, 11)]
    for d, D, chi, seed in cases:          # two calls in a row, different data and shapes
        blocks = [_chain(seed + i, d, D) for i in range(3)]
        r1, t1, l1, s1 = _run("ctx", blocks, d, D, chi, ctx)
        r2, t2, l2, s2 = _run("noalloc", blocks, d, D, chi)
        assert list(r1) == list(r2)
        assert list(s1) == [0] * 3 and list(s2) == [0] * 3
        size = d[0] * d[1] * r1[1] + sum(r1[k - 1] * d[k] * r1[k] for k in range(2, len(d) - 1)) + \
            r1[-1] * d[-1]
        for a, b in zip(t1, t2):
            assert np.all(np.isfinite(b[:size]))
            np.testing.assert_allclose(b[:size], a[:size], atol=ATOL, rtol=0)
        np.testing.assert_allclose(l2, l1, atol=ATOL, rtol=0)


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    d = [2] * 40
    D = [256] * 39
    blocks = [torch.zeros(1, dtype=torch.float64, device="cuda")]
    with pytest.raises(B.TNError) as e:
        B.tn_embed_tree_noalloc([b.data_ptr() for b in blocks], d, D, 64, [blocks[0].data_ptr()],
                                blocks[0].data_ptr(), blocks[0].data_ptr())
    assert e.value.status == 1
    assert "static workspace" in str(e.value)
