"""Learned per-edge ranks: record spectra, make labels, train, contract.

The paper truncates every tree edge to one maximum rank chi.  This module
drives the library's learned alternative (declared in include/tn_dmtree.h
under "learned ranks"): a small MLP, run on the GPU after each eigensolve,
spends the rank budget of the uniform-chi method unevenly over the edges of
each density-matrix pass.  Every numerical step runs in the library's
kernels; this module only allocates device buffers (PyTorch) and sequences
the calls:

  1. ``record``: a batch at the maximum rank chi_max with spectrum recording
     (features, eigenvalues, plan ranks) of every edge;
  2. ``labels``: greedy water-filling of each pass's budget
     sum_e min(chi_uniform, r_e) over the recorded spectra (kernel);
  3. ``train``: Adam on the mean squared error of chi_e / 64 (forward and
     backward kernels);
  4. ``contract``: a batch with learned ranks, optionally judged per
     instance against the uniform-chi method by the summed discarded share
     of the spectra (the smaller one's ln Z is returned).
"""
import numpy as np
import torch

from . import binding as B

N_FEATURES = 22
MAX_SPEC = 128


def _dev(x, dtype, device):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).to(device)


def n_params():
    return B.tn_rank_model_params()


def init_weights(seed):
    """He-initialised FP32 parameters [W1, b1, W2, b2, W3, b3] (host array)."""
    rng = np.random.default_rng(seed)
    H, F = 64, N_FEATURES
    parts = [rng.normal(0.0, np.sqrt(2.0 / F), H * F), np.zeros(H),
             rng.normal(0.0, np.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0.0, np.sqrt(1.0 / H), H), np.array([0.25])]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == n_params()
    return w


class Record:
    """Spectrum records of one batch (device tensors, edge-major: [e, i, ...])."""

    def __init__(self, feat, spec, chi, acc, logz, status, n_passes):
        self.feat, self.spec, self.chi, self.acc = feat, spec, chi, acc
        self.logz, self.status = logz, status
        self.n_edges, self.n_inst = chi.shape
        # DM pass of each edge: the pass feature (pass / passes) of instance 0
        pid = np.rint(feat[:, 0, 19].double().cpu().numpy() * n_passes).astype(np.int64)
        starts = [0] + [e for e in range(1, self.n_edges) if pid[e] != pid[e - 1]]
        self.pass_start = np.array(starts + [self.n_edges], dtype=np.int32)


def record(ctx, plans, sites_dev, precision, learned=False, device="cuda"):
    """Run one batch with recording on; returns a Record."""
    info = plans[0].info
    n_edges, n_inst = int(info["n_eig"]), len(plans)
    feat = torch.zeros(n_edges, n_inst, N_FEATURES, dtype=torch.float32, device=device)
    spec = torch.zeros(n_edges, n_inst, MAX_SPEC, dtype=torch.float64, device=device)
    chi = torch.zeros(n_edges, n_inst, dtype=torch.int32, device=device)
    acc = torch.zeros(n_inst, dtype=torch.float64, device=device)
    B.tn_rank_record(ctx, feat.data_ptr(), spec.data_ptr(), chi.data_ptr(), acc.data_ptr(),
                     n_edges)
    try:
        B.tn_contract_approx(ctx, plans, sites_dev, precision, learned_chi=int(learned),
                             stream=torch.cuda.current_stream().cuda_stream)
        logz, status = B.tn_logz(ctx, n_inst)
    finally:
        B.tn_rank_record(ctx)
    return Record(feat, spec, chi, acc, logz, status, int(info["n_dm_passes"]))


def pass_budgets(caps, pass_start, chi_uniform):
    """Per-pass rank budget of the uniform-chi method: sum_e min(chi_u, r_e)."""
    return np.array([int(np.minimum(caps[a:b], chi_uniform).sum())
                     for a, b in zip(pass_start[:-1], pass_start[1:])], dtype=np.int32)


def labels(ctx, rec, chi_uniform):
    """Water-filling labels (device int32 [e, i]) for a record taken at the
    plan ranks (rec.chi holds r_e there); rewrites the record's budget
    features (20, 21) for the labelled allocation."""
    caps = rec.chi[:, 0].cpu().numpy().astype(np.int32)
    out = torch.zeros_like(rec.chi)
    B.tn_rank_labels(ctx, rec.spec.data_ptr(), rec.n_inst, caps, rec.pass_start, chi_uniform,
                     out.data_ptr(), rec.feat.data_ptr(),
                     stream=torch.cuda.current_stream().cuda_stream)
    return out


def train(ctx, X, y, steps, batch, lr, seed, w0=None):
    """Adam on the MSE of the model over (X [n, 22], y [n]) device tensors.
    Returns (FP32 weights as a host array, per-step minibatch losses)."""
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    idx = _dev(rng.integers(0, n, size=steps * batch), torch.int32, X.device)
    w = _dev(init_weights(seed) if w0 is None else w0, torch.float32, X.device)
    loss = torch.zeros(steps, dtype=torch.float32, device=X.device)
    B.tn_rank_model_train(ctx, X.data_ptr(), y.data_ptr(), idx.data_ptr(), steps, batch, lr,
                          w.data_ptr(), loss.data_ptr(),
                          stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return w.cpu().numpy(), loss.cpu().numpy()


def fit(ctx, plans_max, sites_dev, chi_uniform, precision=B.TN_PREC_FP64, steps=2000,
        batch=256, lr=3e-3, seed=0):
    """Record spectra at chi_max, label them, train; returns (weights, losses)."""
    rec = record(ctx, plans_max, sites_dev, precision)
    lab = labels(ctx, rec, chi_uniform)
    X = rec.feat.reshape(-1, N_FEATURES).contiguous()
    y = (lab.reshape(-1).float() / 64.0).contiguous()
    return train(ctx, X, y, steps, batch, lr, seed)


def contract(ctx, plans_max, sites_dev, weights, chi_uniform, precision=B.TN_PREC_FP64,
             judged=True):
    """ln Z with learned ranks; with judged (the default) the library also runs
    the uniform chi_uniform ranks and keeps, per instance, the run with the
    smaller summed discarded share (tn_contract_approx with learned_chi = 2).
    Returns (logz, status, used_learned)."""
    B.tn_rank_model_load(ctx, weights, chi_uniform)
    ptrs = [int(p) for p in sites_dev]
    B.tn_contract_approx(ctx, plans_max, ptrs, precision, 2 if judged else 1,
                         torch.cuda.current_stream().cuda_stream)
    logz, status = B.tn_logz(ctx, len(plans_max))
    if judged:
        used = B.tn_rank_judged(ctx, len(plans_max)).astype(bool)
    else:
        used = np.ones(len(plans_max), dtype=bool)
    return logz, status, used
