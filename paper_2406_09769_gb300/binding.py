"""Thin ctypes binding of libtn_dmtree.so (declared in include/tn_dmtree.h).

Functions carry the C names and do argument marshalling only: every step of
the contraction runs in the library's CUDA kernels.  Device buffers are plain
integer addresses (e.g. ``torch.Tensor.data_ptr()``); streams are integer
``cudaStream_t`` handles (e.g. ``torch.cuda.current_stream().cuda_stream``).
Loading fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtn_dmtree.so")

TN_OK = 0
STATUS_NAMES = {0: "TN_OK", 1: "TN_ERR_INVALID", 2: "TN_ERR_OOM", 3: "TN_ERR_CUDA",
                4: "TN_ERR_NONFINITE", 5: "TN_ERR_NONPOSITIVE", 6: "TN_ERR_TIMEOUT",
                7: "TN_ERR_EIG_NOCONV", 8: "TN_ERR_UNSUPPORTED"}
TN_PREC_FP64, TN_PREC_BF16, TN_PREC_TF32, TN_PREC_TF32_FAST, TN_PREC_TF32_GRAM = 0, 1, 2, 3, 4

_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class tn_graph(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("edge_u", _i32p), ("edge_v", _i32p), ("edge_dim", _i32p)]


class tn_plan_opts(ctypes.Structure):
    _fields_ = [("chi_max", ctypes.c_int32), ("env_size", ctypes.c_int32),
                ("partition", _i32p), ("path", _i32p), ("n_path", ctypes.c_int32),
                ("ansatz", ctypes.c_int32), ("swap_batch", ctypes.c_int32),
                ("planner", ctypes.c_int32)]


class tn_plan_info(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("n_dm_passes", ctypes.c_int32),
                ("max_legs", ctypes.c_int32), ("max_bond", ctypes.c_int32),
                ("max_eig_n", ctypes.c_int32), ("site_elems", ctypes.c_int64),
                ("flops_env", ctypes.c_double), ("flops_local", ctypes.c_double),
                ("flops_density", ctypes.c_double), ("flops_project", ctypes.c_double),
                ("flops_eig", ctypes.c_double), ("n_eig", ctypes.c_int64),
                ("flops_factor", ctypes.c_double), ("flops_kfactor", ctypes.c_double),
                ("flops_svd", ctypes.c_double), ("n_exec_steps", ctypes.c_int32),
                ("general", ctypes.c_int32)]


class tn_plan_step(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("n_kt", ctypes.c_int32),
                ("general", ctypes.c_int32)]


class TNError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

# Every symbol include/tn_dmtree.h declares.
EXPORTS = ("tn_plan", "tn_plan_destroy", "tn_plan_query", "tn_plan_step_query",
           "tn_plan_site_offset",
           "tn_ctx_create", "tn_ctx_destroy", "tn_embed_tree", "tn_contract_approx",
           "tn_logz", "tn_contract_approx_host", "tn_embed_tree_noalloc",
           "tn_rank_model_params", "tn_rank_model_load", "tn_rank_record", "tn_rank_labels",
           "tn_rank_model_grad", "tn_rank_model_train", "tn_rank_judged",
           "tn_ctx_set_option", "tn_ctx_set_profiling", "tn_ctx_profile", "tn_measure_peaks",
           "tn_autotune", "tn_autotune_entries", "tn_batch_graph_capture", "tn_batch_graph_launch",
           "tn_batch_graph_logz", "tn_batch_graph_destroy", "tn_last_error")

KERNEL_CLASSES = ("norm", "fuse", "env", "local", "density", "eig", "project", "root", "close",
                  "factor")


def lib():
    """Load the shared library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA extension not built: {LIB_PATH} is missing "
                           "(run python -m paper_2406_09769_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    L.tn_plan.argtypes = [ctypes.POINTER(tn_graph), ctypes.POINTER(tn_plan_opts), ctypes.POINTER(_vp)]
    L.tn_plan_destroy.argtypes = [_vp]
    L.tn_plan_query.argtypes = [_vp, ctypes.POINTER(tn_plan_info)]
    L.tn_plan_site_offset.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    L.tn_plan_step_query.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(tn_plan_step), _i32p,
                                     _i32p, _i32p, _i32p]
    L.tn_ctx_create.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp)]
    L.tn_ctx_destroy.argtypes = [_vp]
    L.tn_embed_tree.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                ctypes.POINTER(_vp), ctypes.c_int32, _i32p, ctypes.c_int32,
                                ctypes.POINTER(_vp), _vp, _vp, _i32p, _vp]
    L.tn_contract_approx.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                                     ctypes.c_int32, ctypes.c_int32, _vp]
    L.tn_logz.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), _i32p, ctypes.c_int32]
    L.tn_contract_approx_host.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int32,
                                          ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), _i32p, _vp]
    L.tn_embed_tree_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                        ctypes.POINTER(_vp), ctypes.c_int32, _i32p,
                                        ctypes.POINTER(_vp), _vp, _vp, _i32p, _vp]
    _f32p = ctypes.POINTER(ctypes.c_float)
    L.tn_rank_model_params.argtypes = []
    L.tn_rank_model_load.argtypes = [_vp, _f32p, ctypes.c_int32, ctypes.c_int32]
    L.tn_rank_record.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64]
    L.tn_rank_labels.argtypes = [_vp, _vp, ctypes.c_int32, _i32p, _i32p, ctypes.c_int32,
                                 ctypes.c_int32, _vp, _vp, _vp]
    L.tn_rank_model_grad.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
    L.tn_rank_model_train.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_float, _vp, _vp, _vp]
    L.tn_ctx_set_option.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64]
    L.tn_rank_judged.argtypes = [_vp, _i32p, ctypes.c_int32]
    L.tn_autotune.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                              ctypes.c_int32, ctypes.c_char_p]
    L.tn_autotune_entries.argtypes = [_vp, _i32p]
    L.tn_batch_graph_capture.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                                   ctypes.c_int32, ctypes.POINTER(_vp)]
    L.tn_batch_graph_launch.argtypes = [_vp, _vp]
    L.tn_batch_graph_logz.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), _i32p, ctypes.c_int32]
    L.tn_batch_graph_destroy.argtypes = [_vp]
    L.tn_ctx_set_profiling.argtypes = [_vp, ctypes.c_int32]
    L.tn_ctx_profile.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    L.tn_measure_peaks.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.tn_measure_peaks.restype = ctypes.c_int
    L.tn_last_error.argtypes = [_vp]
    L.tn_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "tn_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def tn_last_error(ctx=None):
    msg = lib().tn_last_error(ctx.handle if ctx is not None else None)
    return msg.decode() if msg else ""


def _check(status, ctx=None):
    if status != TN_OK:
        raise TNError(status, tn_last_error(ctx))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


class Plan:
    """Owns a tn_plan_t*; released by tn_plan_destroy."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_plan_destroy(self.handle)
            self.handle = None

    @property
    def info(self):
        return tn_plan_query(self)

    def site_offset(self, v):
        return tn_plan_site_offset(self, v)


class Ctx:
    """Owns a tn_ctx_t*; released by tn_ctx_destroy."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_ctx_destroy(self.handle)
            self.handle = None


def tn_plan(n_vertices, edges, edge_dim, chi, env_size=0, partition=None, path=None,
            ansatz=0, swap_batch=32, planner=0):
    edges = np.asarray(edges).reshape(-1, 2)
    u, up = _i32(edges[:, 0])
    v, vp = _i32(edges[:, 1])
    dm, dp = _i32(edge_dim)
    g = tn_graph(int(n_vertices), len(edges), up, vp, dp)
    keep = [u, v, dm]
    part_p = path_p = None
    n_path = 0
    if partition is not None:
        pa, part_p = _i32(partition)
        keep.append(pa)
    if path is not None:
        pt, path_p = _i32(path)
        keep.append(pt)
        n_path = len(pt)
    o = tn_plan_opts(int(chi), int(env_size), part_p, path_p, n_path, int(ansatz), int(swap_batch),
                     int(planner))
    h = _vp()
    _check(lib().tn_plan(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)))
    return Plan(h, None)


def tn_plan_query(plan):
    info = tn_plan_info()
    _check(lib().tn_plan_query(plan.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in tn_plan_info._fields_}


def tn_plan_step_query(plan, step):
    """dict(kind, n, n_kt, general, leaves, d, D, r) of executed step `step`."""
    info = tn_plan_step()
    _check(lib().tn_plan_step_query(plan.handle, int(step), ctypes.byref(info), None, None, None,
                                    None))
    n = info.n
    leaves = np.zeros(n, np.int32)
    d = np.zeros(n, np.int32)
    D = np.zeros(n, np.int32)
    r = np.zeros(max(n - 1, 1), np.int32)
    ptr = lambda a: a.ctypes.data_as(_i32p)
    _check(lib().tn_plan_step_query(plan.handle, int(step), ctypes.byref(info), ptr(leaves),
                                    ptr(d), ptr(D), ptr(r)))
    return dict(kind=info.kind, n=n, n_kt=info.n_kt, general=info.general,
                leaves=leaves.tolist(), d=d.tolist(), D=D.tolist(),
                r=r[:n - 1].tolist() if info.kind == 1 else [])


def tn_plan_steps(plan):
    """Every executed step of a plan (tn_plan_step_query in order)."""
    return [tn_plan_step_query(plan, s) for s in range(tn_plan_query(plan)["n_exec_steps"])]


def tn_plan_site_offset(plan, vertex):
    off = ctypes.c_int64()
    _check(lib().tn_plan_site_offset(plan.handle, int(vertex), ctypes.byref(off)))
    return off.value


def tn_ctx_create(device=0):
    h = _vp()
    _check(lib().tn_ctx_create(int(device), ctypes.byref(h)))
    return Ctx(h)


def tn_ctx_destroy(ctx):
    _check(lib().tn_ctx_destroy(ctx.handle))
    ctx.handle = None


def _ptrs(addrs):
    arr = (_vp * len(addrs))(*[int(a) for a in addrs])
    return arr


def tn_embed_tree(ctx, blocks_dev, leg_dim, bond_dim, chi, tree_dev, lognorm_dev, status_dev,
                  chi_per_edge=None, precision=TN_PREC_FP64, stream=0):
    """One density_matrix_alg pass; returns the ranks r_0..r_{n-2}."""
    n = len(leg_dim)
    ld, ldp = _i32(leg_dim)
    bd, bdp = _i32(bond_dim)
    cpe = cpep = None
    if chi_per_edge is not None:
        cpe, cpep = _i32(chi_per_edge)
    ranks = np.zeros(n - 1, dtype=np.int32)
    st = lib().tn_embed_tree(ctx.handle, len(blocks_dev), n, ldp, bdp, _ptrs(blocks_dev), int(chi),
                             cpep, int(precision), _ptrs(tree_dev), _vp(int(lognorm_dev)),
                             _vp(int(status_dev)), ranks.ctypes.data_as(_i32p), _vp(int(stream)))
    _check(st, ctx)
    return ranks


def tn_embed_tree_noalloc(blocks_dev, leg_dim, bond_dim, chi, tree_dev, lognorm_dev, status_dev,
                          chi_per_edge=None, stream=0):
    """Allocation-free FP64 density-matrix pass (no ctx; static device workspace).

    For callers that cannot allocate device memory; see include/tn_dmtree.h.
    Returns the ranks r_0..r_{n-2}.
    """
    n = len(leg_dim)
    ld, ldp = _i32(leg_dim)
    bd, bdp = _i32(bond_dim)
    cpe = cpep = None
    if chi_per_edge is not None:
        cpe, cpep = _i32(chi_per_edge)
    ranks = np.zeros(n - 1, dtype=np.int32)
    st = lib().tn_embed_tree_noalloc(len(blocks_dev), n, ldp, bdp, _ptrs(blocks_dev), int(chi),
                                     cpep, _ptrs(tree_dev), _vp(int(lognorm_dev)),
                                     _vp(int(status_dev)), ranks.ctypes.data_as(_i32p),
                                     _vp(int(stream)))
    _check(st)
    return ranks


def tn_contract_approx(ctx, plans, sites_dev, precision=TN_PREC_FP64, learned_chi=0, stream=0):
    hs = _ptrs([p.handle.value for p in plans])
    st = lib().tn_contract_approx(ctx.handle, hs, len(plans), _ptrs(sites_dev), int(precision),
                                  int(learned_chi), _vp(int(stream)))
    _check(st, ctx)


def tn_logz(ctx, n_inst, raise_on_error=False):
    """Returns (logz float64[n_inst], status int32[n_inst])."""
    logz = np.empty(n_inst, dtype=np.float64)
    status = np.empty(n_inst, dtype=np.int32)
    st = lib().tn_logz(ctx.handle, logz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       status.ctypes.data_as(_i32p), int(n_inst))
    # per-instance outcomes (non-finite, non-positive, timeout, no convergence)
    # come back in status; anything else raises
    if st != TN_OK and (raise_on_error or st not in (4, 5, 6, 7)):
        _check(st, ctx)
    return logz, status


def tn_contract_approx_host(ctx, plans, sites_host, precision=TN_PREC_FP64, learned_chi=0,
                            stream=0, raise_on_error=False):
    """End-to-end call from host buffers (addresses of FP64 arrays)."""
    n = len(plans)
    logz = np.empty(n, dtype=np.float64)
    status = np.empty(n, dtype=np.int32)
    hs = _ptrs([p.handle.value for p in plans])
    st = lib().tn_contract_approx_host(ctx.handle, hs, n, _ptrs(sites_host), int(precision),
                                       int(learned_chi),
                                       logz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       status.ctypes.data_as(_i32p), _vp(int(stream)))
    # per-instance outcomes (non-finite, non-positive, timeout, no convergence)
    # come back in status; anything else raises
    if st != TN_OK and (raise_on_error or st not in (4, 5, 6, 7)):
        _check(st, ctx)
    return logz, status


def tn_rank_model_params():
    return int(lib().tn_rank_model_params())


def tn_rank_model_load(ctx, weights, chi_uniform):
    """Load FP32 rank-model parameters (host array) or unload them (weights=None)."""
    if weights is None:
        _check(lib().tn_rank_model_load(ctx.handle, None, 0, int(chi_uniform)), ctx)
        return
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(lib().tn_rank_model_load(ctx.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    len(w), int(chi_uniform)), ctx)


def tn_rank_record(ctx, feat_dev=0, spec_dev=0, chi_dev=0, acc_dev=0, cap_edges=0):
    """Set (device addresses) or clear (all 0) the spectrum records of later batches."""
    _check(lib().tn_rank_record(ctx.handle, _vp(int(feat_dev) or None), _vp(int(spec_dev) or None),
                                _vp(int(chi_dev) or None), _vp(int(acc_dev) or None),
                                int(cap_edges)), ctx)


def tn_rank_labels(ctx, spec_dev, n_inst, cap, pass_start, chi_uniform, chi_dev, feat_dev=0,
                   stream=0):
    c, cp = _i32(cap)
    ps, psp = _i32(pass_start)
    _check(lib().tn_rank_labels(ctx.handle, _vp(int(spec_dev)), int(n_inst), cp, psp,
                                len(ps) - 1, int(chi_uniform), _vp(int(chi_dev)),
                                _vp(int(feat_dev) or None), _vp(int(stream))), ctx)


def tn_rank_model_grad(ctx, X_dev, y_dev, n, w_dev, grad_dev, loss_dev, idx_dev=0, stream=0):
    _check(lib().tn_rank_model_grad(ctx.handle, _vp(int(X_dev)), _vp(int(y_dev)),
                                    _vp(int(idx_dev) or None), int(n), _vp(int(w_dev)),
                                    _vp(int(grad_dev)), _vp(int(loss_dev)), _vp(int(stream))), ctx)


def tn_rank_model_train(ctx, X_dev, y_dev, idx_dev, steps, batch, lr, w_dev, loss_dev, stream=0):
    _check(lib().tn_rank_model_train(ctx.handle, _vp(int(X_dev)), _vp(int(y_dev)),
                                     _vp(int(idx_dev)), int(steps), int(batch), float(lr),
                                     _vp(int(w_dev)), _vp(int(loss_dev)), _vp(int(stream))), ctx)


def tn_ctx_set_profiling(ctx, on):
    _check(lib().tn_ctx_set_profiling(ctx.handle, int(bool(on))), ctx)


def tn_ctx_profile(ctx):
    """Returns {class: (launches, ms)} since the last call (ms = 0 unless profiling)."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(lib().tn_ctx_profile(ctx.handle, ms, cnt, n), ctx)
    return {k: (int(cnt[i]), float(ms[i])) for i, k in enumerate(KERNEL_CLASSES)}


TN_OPT_EIG_ROUNDS, TN_OPT_WAIT_PROBE, TN_OPT_VALUE_PATH, TN_OPT_GROUPED = 1, 2, 3, 4


def tn_rank_judged(ctx, n_inst):
    """Which run each instance of the last judged batch kept (1 = learned)."""
    used = np.empty(n_inst, dtype=np.int32)
    _check(lib().tn_rank_judged(ctx.handle, used.ctypes.data_as(_i32p), int(n_inst)), ctx)
    return used


def tn_autotune(ctx, plans, sites_dev, precision=TN_PREC_TF32, cache_path=None):
    """Tune the tensor-core tiles of ctx on this batch (or load cache_path)."""
    hs = _ptrs([p.handle.value for p in plans])
    cp = cache_path.encode() if cache_path else None
    _check(lib().tn_autotune(ctx.handle, hs, len(plans), _ptrs(sites_dev), int(precision), cp),
           ctx)
    n = ctypes.c_int32()
    _check(lib().tn_autotune_entries(ctx.handle, ctypes.byref(n)), ctx)
    return n.value


class Graph:
    """A captured batch (tn_batch_graph_capture); replay with launch(), read with logz()."""

    def __init__(self, ctx, plans, sites_dev, precision=TN_PREC_TF32):
        self.handle = _vp()
        self.n = len(plans)
        self._plans = plans  # the graph reads the plans' tables only at capture
        hs = _ptrs([p.handle.value for p in plans])
        _check(lib().tn_batch_graph_capture(ctx.handle, hs, len(plans), _ptrs(sites_dev),
                                      int(precision), ctypes.byref(self.handle)), ctx)

    def launch(self, stream=0):
        _check(lib().tn_batch_graph_launch(self.handle, _vp(stream)))

    def logz(self):
        logz = np.empty(self.n, dtype=np.float64)
        status = np.empty(self.n, dtype=np.int32)
        st = lib().tn_batch_graph_logz(self.handle, logz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 status.ctypes.data_as(_i32p), self.n)
        if st != TN_OK and st not in (4, 5, 6, 7):
            _check(st)
        return logz, status

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.tn_batch_graph_destroy(self.handle)
            self.handle = _vp()


def tn_ctx_set_option(ctx, option, value):
    _check(lib().tn_ctx_set_option(ctx.handle, int(option), int(value)), ctx)


def tn_measure_peaks(device=0):
    """Measured arithmetic peaks of the device in TFLOP/s: FP32 FMA, packed FP32x2
    FMA, FP64 FMA and the tcgen05 tensor pipe in kind::tf32."""
    out = (ctypes.c_double * 4)()
    st = lib().tn_measure_peaks(int(device), out)
    if st != 0:
        raise TNError(st, f"tn_measure_peaks failed with status {st}")
    return {"fp32": out[0], "fp32x2": out[1], "fp64": out[2], "tf32": out[3]}


def pack_sites(plan, tensors):
    """Pack per-vertex tensors (legs in ascending edge id) into one FP64 buffer."""
    info = tn_plan_query(plan)
    buf = np.empty(info["site_elems"], dtype=np.float64)
    for v, t in enumerate(tensors):
        off = tn_plan_site_offset(plan, v)
        flat = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
        buf[off:off + flat.size] = flat
    return buf
