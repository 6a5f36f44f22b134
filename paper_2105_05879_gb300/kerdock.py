"""Thin Python binding of libkerdock.so (ctypes).

The functions below carry the C-ABI names of ``include/kerdock.h`` and only
marshal arguments; every step of the transform runs in the library's CUDA
kernels.  ``KerdockPlan`` adds convenience on top: it lets PyTorch allocate the
device buffers the library asks for and passes torch's current CUDA stream.

There is no fallback: if the library cannot be loaded, importing the binding
works but the first call raises ``KerdockError``.
"""
import ctypes
import os

import numpy as np

KERDOCK_OK = 0
KERDOCK_F32 = 0
KERDOCK_BF16 = 1
KERDOCK_FLAG_FULL_OUTPUT = 1

_ERRORS = {
    -1: "KERDOCK_ERR_INVALID_ARG", -2: "KERDOCK_ERR_UNSUPPORTED", -3: "KERDOCK_ERR_NOT_BOUND",
    -4: "KERDOCK_ERR_NOT_PREPROCESSED", -5: "KERDOCK_ERR_CAPACITY", -6: "KERDOCK_ERR_CUDA",
    -7: "KERDOCK_ERR_DEVICE_TIMEOUT", -8: "KERDOCK_ERR_ALIGNMENT",
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkerdock.so")

# Every symbol include/kerdock.h declares.
EXPORTED = [
    "kerdock_plan_create", "kerdock_plan_info", "kerdock_plan_bind", "kerdock_set_stream",
    "kerdock_preprocess", "kerdock_apply_workspace_bytes", "kerdock_apply",
    "kerdock_apply_debug", "kerdock_sync", "kerdock_debug_signs", "kerdock_plan_destroy",
    "kerdock_strerror", "kerdock_version", "kerdock_apply_noalloc",
    "kerdock_batch_workspace_bytes", "kerdock_batch_create", "kerdock_batch_launch",
    "kerdock_batch_set_tuning", "kerdock_batch_set_costs", "kerdock_batch_ctas",
    "kerdock_batch_set_schedule", "kerdock_debug_batch_schedule", "kerdock_batch_tune",
    "kerdock_batch_sync",
    "kerdock_batch_destroy", "kerdock_plan_set_tuning", "kerdock_plan_tune",
    "kerdock_mlp_create", "kerdock_mlp_sizes", "kerdock_mlp_bind", "kerdock_mlp_pointers",
    "kerdock_mlp_sync_weights", "kerdock_mlp_init", "kerdock_mlp_forward", "kerdock_mlp_backward",
    "kerdock_mlp_loss", "kerdock_mlp_adamw", "kerdock_mlp_destroy", "kerdock_refine_scores",
    "kerdock_plan_clone", "kerdock_mlp_set_input", "kerdock_debug_wait_timeout",
    "kerdock_mlp_set_skip", "kerdock_theory_parameters", "kerdock_apply_shared_workspace_bytes",
    "kerdock_apply_shared", "kerdock_apply_shared_scores", "kerdock_debug_gemm",
    "kerdock_debug_set_poll_limit",
    "kerdock_check_reconstruction", "kerdock_check_tight_frame",
]

KERDOCK_MLP_INPUT_LINEAR = 0
KERDOCK_MLP_INPUT_ABS = 1

KERDOCK_BATCH_GRAPH = 1


class KerdockError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        name = _ERRORS.get(code, str(code))
        text = ""
        if _lib is not None:
            text = _lib.kerdock_strerror(code).decode()
        super().__init__(f"{where}: {name} ({text})")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32),
        ("dtype", ctypes.c_int32), ("d", ctypes.c_int64), ("num_bases", ctypes.c_int64),
        ("L", ctypes.c_int64), ("ldr", ctypes.c_int64), ("J", ctypes.c_int32),
        ("K", ctypes.c_int32), ("S", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("repr_bytes", ctypes.c_size_t), ("table_bytes", ctypes.c_size_t),
    ]


class Query(ctypes.Structure):
    """Mirror of kerdock_query_t."""
    _fields_ = [
        ("plan", ctypes.c_void_p), ("x", ctypes.c_void_p), ("J", ctypes.c_int32),
        ("K", ctypes.c_int32), ("S", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("eps", ctypes.c_float), ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("index", ctypes.c_int64), ("out_idx", ctypes.c_void_p), ("out_val", ctypes.c_void_p),
        ("out_count", ctypes.c_void_p),
    ]


_lib = None


def load_library(path=None):
    """Load libkerdock.so (built by ``paper_2105_05879_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise KerdockError(-6, f"libkerdock.so not found at {path}; run the build first")
    lib = ctypes.CDLL(path)
    c_i64, c_i32, c_vp, c_sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.c_void_p
    sig = {
        "kerdock_plan_create": (ctypes.c_int, [ctypes.POINTER(P), c_i64, c_i64, c_i32, c_i32, c_i32, c_i32]),
        "kerdock_plan_info": (ctypes.c_int, [P, ctypes.POINTER(PlanInfo)]),
        "kerdock_plan_bind": (ctypes.c_int, [P, c_vp, c_sz, c_vp, c_sz, c_vp]),
        "kerdock_set_stream": (ctypes.c_int, [P, c_vp]),
        "kerdock_preprocess": (ctypes.c_int, [P, c_vp, c_i64]),
        "kerdock_apply_workspace_bytes": (c_sz, [P, c_i64]),
        "kerdock_apply": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_float, ctypes.c_uint64,
                                         c_i32, c_vp, c_vp, c_vp, c_vp, c_sz]),
        "kerdock_apply_debug": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_float,
                                               ctypes.c_uint64, c_i32, c_vp, c_vp, c_vp, c_vp,
                                               c_sz, c_vp, c_vp, c_vp]),
        "kerdock_apply_noalloc": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_float,
                                                 ctypes.c_uint64, c_i32, c_vp, c_vp, c_vp]),
        "kerdock_batch_workspace_bytes": (c_sz, [ctypes.POINTER(Query), c_i64]),
        "kerdock_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(Query), c_i64,
                                                c_vp, c_sz, c_vp, c_i32]),
        "kerdock_batch_launch": (ctypes.c_int, [P]),
        "kerdock_batch_set_tuning": (ctypes.c_int, [P, c_i32, c_i32]),
        "kerdock_batch_set_costs": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double), c_i64]),
        "kerdock_batch_ctas": (c_i32, [P]),
        "kerdock_debug_batch_schedule": (ctypes.c_int, [ctypes.POINTER(c_vp),
                                                        ctypes.POINTER(ctypes.c_uint32),
                                                        ctypes.POINTER(ctypes.c_double), c_i64,
                                                        c_i32, ctypes.POINTER(c_i32),
                                                        ctypes.POINTER(c_i64)]),
        "kerdock_batch_set_schedule": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32),
                                                      ctypes.POINTER(c_i64), c_i32]),
        "kerdock_batch_tune": (ctypes.c_int, [P, c_i32, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_float)]),
        "kerdock_batch_sync": (ctypes.c_int, [P]),
        "kerdock_batch_destroy": (ctypes.c_int, [P]),
        "kerdock_plan_set_tuning": (ctypes.c_int, [P, c_i32, c_i32]),
        "kerdock_plan_tune": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_float,
                                             ctypes.c_uint64, c_vp, c_vp, c_vp, c_vp, c_sz, c_i32,
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_float)]),
        "kerdock_mlp_create": (ctypes.c_int, [ctypes.POINTER(P), c_i32, c_i32, c_i32, c_i32]),
        "kerdock_mlp_sizes": (ctypes.c_int, [P, ctypes.POINTER(c_sz), ctypes.POINTER(c_sz),
                                             ctypes.POINTER(c_i64)]),
        "kerdock_mlp_bind": (ctypes.c_int, [P, c_vp, c_sz, c_vp, c_sz, c_vp]),
        "kerdock_mlp_pointers": (ctypes.c_int, [P, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp),
                                                ctypes.POINTER(c_i64)]),
        "kerdock_mlp_sync_weights": (ctypes.c_int, [P]),
        "kerdock_mlp_init": (ctypes.c_int, [P, ctypes.c_uint64]),
        "kerdock_mlp_set_input": (ctypes.c_int, [P, c_i32]),
        "kerdock_mlp_set_skip": (ctypes.c_int, [P, ctypes.c_float]),
        "kerdock_mlp_forward": (ctypes.c_int, [P, c_vp, c_i32, ctypes.c_float, c_vp]),
        "kerdock_mlp_backward": (ctypes.c_int, [P, c_vp, c_vp, c_i32, ctypes.c_float,
                                                ctypes.c_float]),
        "kerdock_mlp_loss": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float)]),
        "kerdock_mlp_adamw": (ctypes.c_int, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float]),
        "kerdock_mlp_destroy": (ctypes.c_int, [P]),
        "kerdock_refine_scores": (ctypes.c_int, [P, c_vp, c_i64, c_i64, c_vp, c_i32,
                                                 ctypes.c_float, c_i32, c_vp, c_vp, c_vp]),
        "kerdock_apply_shared_workspace_bytes": (c_sz, [P, c_i64]),
        "kerdock_apply_shared": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_float, ctypes.c_uint64,
                                                c_i32, c_vp, c_vp, c_vp, c_vp, c_sz]),
        "kerdock_apply_shared_scores": (ctypes.c_int, [P, c_vp, c_i64, c_i64, ctypes.c_uint64,
                                                       c_vp, c_vp, c_sz]),
        "kerdock_theory_parameters": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, c_i64, ctypes.POINTER(c_i32),
                                                     ctypes.POINTER(c_i32)]),
        "kerdock_plan_clone": (ctypes.c_int, [ctypes.POINTER(P), P, c_i32, c_i32, c_i32]),
        "kerdock_debug_wait_timeout": (ctypes.c_int, [P, c_i32]),
        "kerdock_debug_set_poll_limit": (ctypes.c_int, [P, ctypes.c_uint32]),
        "kerdock_check_reconstruction": (ctypes.c_int, [P, c_i64, c_i64, c_vp]),
        "kerdock_check_tight_frame": (ctypes.c_int, [P, c_vp, c_i32, c_i64, c_i64, c_vp, c_vp]),
        "kerdock_debug_gemm": (ctypes.c_int, [c_vp, c_i64, c_i64, c_vp, c_i64, c_i64, c_i32,
                                                   c_i32, c_i32, c_i32, c_vp, c_i64, c_vp]),
        "kerdock_sync": (ctypes.c_int, [P]),
        "kerdock_debug_signs": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint32), c_sz]),
        "kerdock_plan_destroy": (ctypes.c_int, [P]),
        "kerdock_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "kerdock_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, where):
    if rc != KERDOCK_OK:
        raise KerdockError(rc, where)


# --- C-ABI mirrors -----------------------------------------------------------

def kerdock_plan_create(m, n, dtype, J, K, S):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.kerdock_plan_create(ctypes.byref(h), m, n, dtype, J, K, S), "kerdock_plan_create")
    return h


def kerdock_plan_info(plan):
    info = PlanInfo()
    _check(load_library().kerdock_plan_info(plan, ctypes.byref(info)), "kerdock_plan_info")
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_ if f != "reserved"}


def kerdock_plan_bind(plan, repr_ptr, repr_bytes, table_ptr, table_bytes, stream):
    _check(load_library().kerdock_plan_bind(plan, repr_ptr, repr_bytes, table_ptr, table_bytes,
                                            stream), "kerdock_plan_bind")


def kerdock_apply_shared(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr, val_ptr, cnt_ptr, ws_ptr,
                         ws_bytes):
    _check(load_library().kerdock_apply_shared(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr,
                                               val_ptr, cnt_ptr, ws_ptr, ws_bytes),
           "kerdock_apply_shared")


def kerdock_apply_shared_scores(plan, X_ptr, q, ldx, seed, scores_ptr, ws_ptr, ws_bytes):
    _check(load_library().kerdock_apply_shared_scores(plan, X_ptr, q, ldx, seed, scores_ptr,
                                                      ws_ptr, ws_bytes),
           "kerdock_apply_shared_scores")


def kerdock_theory_parameters(a_row_norm_max, eps, delta, eta, m):
    """(J, K) of Theorem 3 for ||mu - Ax||_inf < (eps - delta)/2 w.p. >= 1 - eta.
    Raises for invalid arguments and for (J, K) beyond the library's limits."""
    J, K = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load_library().kerdock_theory_parameters(float(a_row_norm_max), float(eps), float(delta),
                                                     float(eta), int(m), ctypes.byref(J),
                                                     ctypes.byref(K)), "kerdock_theory_parameters")
    return J.value, K.value


def kerdock_set_stream(plan, stream):
    _check(load_library().kerdock_set_stream(plan, stream), "kerdock_set_stream")


def kerdock_preprocess(plan, A_ptr, lda):
    _check(load_library().kerdock_preprocess(plan, A_ptr, lda), "kerdock_preprocess")


def kerdock_apply_workspace_bytes(plan, q):
    return load_library().kerdock_apply_workspace_bytes(plan, q)


def kerdock_apply(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr, val_ptr, cnt_ptr, ws_ptr, ws_bytes):
    _check(load_library().kerdock_apply(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr, val_ptr,
                                        cnt_ptr, ws_ptr, ws_bytes), "kerdock_apply")


def kerdock_apply_debug(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr, val_ptr, cnt_ptr, ws_ptr,
                        ws_bytes, mu_ptr, ells_ptr, coef_ptr):
    _check(load_library().kerdock_apply_debug(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr,
                                              val_ptr, cnt_ptr, ws_ptr, ws_bytes, mu_ptr,
                                              ells_ptr, coef_ptr), "kerdock_apply_debug")


def kerdock_apply_noalloc(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr, val_ptr, cnt_ptr):
    """kerdock_apply without a workspace: for callers that cannot allocate device
    memory; the scratch is a fixed array inside the library (see kerdock.h)."""
    _check(load_library().kerdock_apply_noalloc(plan, X_ptr, q, ldx, eps, seed, flags, idx_ptr,
                                                val_ptr, cnt_ptr), "kerdock_apply_noalloc")


def kerdock_batch_workspace_bytes(queries):
    arr = (Query * len(queries))(*queries)
    return load_library().kerdock_batch_workspace_bytes(arr, len(queries))


def kerdock_batch_create(queries, ws_ptr, ws_bytes, stream, options):
    arr = (Query * len(queries))(*queries)
    h = ctypes.c_void_p()
    _check(load_library().kerdock_batch_create(ctypes.byref(h), arr, len(queries), ws_ptr,
                                               ws_bytes, stream, options), "kerdock_batch_create")
    return h


def kerdock_batch_launch(batch):
    _check(load_library().kerdock_batch_launch(batch), "kerdock_batch_launch")


def kerdock_batch_set_tuning(batch, ring_kb, crows):
    _check(load_library().kerdock_batch_set_tuning(batch, ring_kb, crows),
           "kerdock_batch_set_tuning")


def kerdock_batch_set_costs(batch, costs):
    c = np.ascontiguousarray(costs, dtype=np.float64)
    _check(load_library().kerdock_batch_set_costs(
        batch, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), c.size), "kerdock_batch_set_costs")


def kerdock_debug_batch_schedule(plan_ids, row_bytes, costs, grid):
    """The library's batch schedule for these queries (host only): a list of
    per-CTA lists of query indices."""
    n = len(costs)
    ids = (ctypes.c_void_p * n)(*[int(p) for p in plan_ids])
    rb = np.ascontiguousarray(row_bytes, dtype=np.uint32)
    c = np.ascontiguousarray(costs, dtype=np.float64)
    order = np.zeros(max(n, 1), dtype=np.int32)
    start = np.zeros(max(grid, 0) + 1, dtype=np.int64)
    _check(load_library().kerdock_debug_batch_schedule(
        ids, rb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, grid,
        order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        start.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "kerdock_debug_batch_schedule")
    return [order[start[g]:start[g + 1]].tolist() for g in range(grid)]


def kerdock_batch_ctas(batch):
    return int(load_library().kerdock_batch_ctas(batch))


def kerdock_batch_set_schedule(batch, lists):
    """lists[c] = the creation-list indices CTA c runs, in order."""
    order = np.ascontiguousarray(np.concatenate([np.asarray(l, dtype=np.int32) for l in lists])
                                 if lists else np.zeros(0, np.int32), dtype=np.int32)
    start = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(l) for l in lists])]),
                                 dtype=np.int64)
    _check(load_library().kerdock_batch_set_schedule(
        batch, order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        start.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(lists)),
        "kerdock_batch_set_schedule")


def kerdock_batch_tune(batch, reps):
    rk, cr, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load_library().kerdock_batch_tune(batch, reps, ctypes.byref(rk), ctypes.byref(cr),
                                             ctypes.byref(ms)), "kerdock_batch_tune")
    return rk.value, cr.value, ms.value


def kerdock_batch_sync(batch):
    _check(load_library().kerdock_batch_sync(batch), "kerdock_batch_sync")


def kerdock_batch_destroy(batch):
    if batch is not None:
        load_library().kerdock_batch_destroy(batch)


def kerdock_plan_set_tuning(plan, ring_kb, crows):
    _check(load_library().kerdock_plan_set_tuning(plan, ring_kb, crows), "kerdock_plan_set_tuning")


def kerdock_plan_tune(plan, X_ptr, q, ldx, eps, seed, idx_ptr, val_ptr, cnt_ptr, ws_ptr, ws_bytes,
                      reps):
    rk, cr, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load_library().kerdock_plan_tune(plan, X_ptr, q, ldx, eps, seed, idx_ptr, val_ptr,
                                            cnt_ptr, ws_ptr, ws_bytes, reps, ctypes.byref(rk),
                                            ctypes.byref(cr), ctypes.byref(ms)),
           "kerdock_plan_tune")
    return rk.value, cr.value, ms.value


def kerdock_plan_clone(plan, J, K, S):
    h = ctypes.c_void_p()
    _check(load_library().kerdock_plan_clone(ctypes.byref(h), plan, J, K, S), "kerdock_plan_clone")
    return h


def kerdock_refine_scores(plan, X_ptr, q, ldx, scores_ptr, S, eps, flags, idx_ptr, val_ptr, cnt_ptr):
    _check(load_library().kerdock_refine_scores(plan, X_ptr, q, ldx, scores_ptr, S, eps, flags,
                                                idx_ptr, val_ptr, cnt_ptr), "kerdock_refine_scores")


def kerdock_mlp_create(in_dim, hidden, out_dim, max_batch):
    h = ctypes.c_void_p()
    _check(load_library().kerdock_mlp_create(ctypes.byref(h), in_dim, hidden, out_dim, max_batch),
           "kerdock_mlp_create")
    return h


def kerdock_mlp_sizes(mlp):
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
    _check(load_library().kerdock_mlp_sizes(mlp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "kerdock_mlp_sizes")
    return a.value, b.value, c.value


def kerdock_mlp_bind(mlp, state_ptr, state_bytes, work_ptr, work_bytes, stream):
    _check(load_library().kerdock_mlp_bind(mlp, state_ptr, state_bytes, work_ptr, work_bytes, stream),
           "kerdock_mlp_bind")


def kerdock_mlp_pointers(mlp):
    p, g = ctypes.c_void_p(), ctypes.c_void_p()
    off = (ctypes.c_int64 * 7)()
    _check(load_library().kerdock_mlp_pointers(mlp, ctypes.byref(p), ctypes.byref(g), off),
           "kerdock_mlp_pointers")
    return p.value, g.value, list(off)


def kerdock_mlp_sync_weights(mlp):
    _check(load_library().kerdock_mlp_sync_weights(mlp), "kerdock_mlp_sync_weights")


def kerdock_mlp_set_input(mlp, mode):
    _check(load_library().kerdock_mlp_set_input(mlp, mode), "kerdock_mlp_set_input")


def kerdock_mlp_set_skip(mlp, skip):
    _check(load_library().kerdock_mlp_set_skip(mlp, skip), "kerdock_mlp_set_skip")


def kerdock_mlp_init(mlp, seed):
    _check(load_library().kerdock_mlp_init(mlp, seed), "kerdock_mlp_init")


def kerdock_mlp_forward(mlp, feats_ptr, B, scale, logits_ptr):
    _check(load_library().kerdock_mlp_forward(mlp, feats_ptr, B, scale, logits_ptr),
           "kerdock_mlp_forward")


def kerdock_mlp_backward(mlp, feats_ptr, labels_ptr, B, scale, pos_weight):
    _check(load_library().kerdock_mlp_backward(mlp, feats_ptr, labels_ptr, B, scale, pos_weight),
           "kerdock_mlp_backward")


def kerdock_mlp_loss(mlp):
    v = ctypes.c_float()
    _check(load_library().kerdock_mlp_loss(mlp, ctypes.byref(v)), "kerdock_mlp_loss")
    return v.value


def kerdock_mlp_adamw(mlp, lr, beta1, beta2, eps, wd):
    _check(load_library().kerdock_mlp_adamw(mlp, lr, beta1, beta2, eps, wd), "kerdock_mlp_adamw")


def kerdock_mlp_destroy(mlp):
    if mlp is not None:
        load_library().kerdock_mlp_destroy(mlp)


def kerdock_debug_wait_timeout(plan, max_polls):
    _check(load_library().kerdock_debug_wait_timeout(plan, max_polls), "kerdock_debug_wait_timeout")


def kerdock_debug_set_poll_limit(plan, max_polls):
    _check(load_library().kerdock_debug_set_poll_limit(plan, max_polls),
           "kerdock_debug_set_poll_limit")


def kerdock_check_reconstruction(plan, b0, nb, err_dev):
    _check(load_library().kerdock_check_reconstruction(plan, b0, nb, err_dev),
           "kerdock_check_reconstruction")


def kerdock_check_tight_frame(plan, Y_dev, P, b0, nb, frame_dev, ref_dev):
    _check(load_library().kerdock_check_tight_frame(plan, Y_dev, P, b0, nb, frame_dev, ref_dev),
           "kerdock_check_tight_frame")


def kerdock_debug_gemm(A, sAm, sAk, B, sBn, sBk, M, N, K, kc, C, ldc, stream=None):
    _check(load_library().kerdock_debug_gemm(A, sAm, sAk, B, sBn, sBk, M, N, K, kc, C, ldc,
                                                  stream), "kerdock_debug_gemm")


def kerdock_sync(plan):
    _check(load_library().kerdock_sync(plan), "kerdock_sync")


def kerdock_debug_signs(plan):
    info = kerdock_plan_info(plan)
    words = max(4, info["d"] // 32)
    out = np.zeros((info["d"] // 2, words), dtype=np.uint32)
    _check(load_library().kerdock_debug_signs(
        plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), out.size), "kerdock_debug_signs")
    return out


def kerdock_plan_destroy(plan):
    if plan is not None and load_library() is not None:
        _lib.kerdock_plan_destroy(plan)


def kerdock_strerror(code):
    return load_library().kerdock_strerror(code).decode()


def kerdock_version():
    return load_library().kerdock_version()


# --- torch convenience ---------------------------------------------------------

class KerdockPlan:
    """A plan whose device buffers PyTorch allocates.

    >>> plan = KerdockPlan(m, n, J=375, K=2, S=160, dtype="f32")
    >>> plan.preprocess(A)                        # A: (m, n) float32 CUDA tensor
    >>> idx, val, cnt = plan.apply(X, eps, seed)  # X: (q, n) float32 CUDA tensor
    """

    def __init__(self, m, n, J, K, S, dtype="f32", device=None, stream=None):
        import torch
        self.torch = torch
        self.dtype = KERDOCK_BF16 if dtype in ("bf16", KERDOCK_BF16) else KERDOCK_F32
        self.device = torch.device(device or "cuda")
        self.handle = kerdock_plan_create(m, n, self.dtype, J, K, S)
        self.info = kerdock_plan_info(self.handle)
        self.repr = torch.empty(self.info["repr_bytes"], dtype=torch.uint8, device=self.device)
        self.table = torch.empty(self.info["table_bytes"], dtype=torch.uint8, device=self.device)
        self._stream = stream
        kerdock_plan_bind(self.handle, self.repr.data_ptr(), self.repr.numel(),
                          self.table.data_ptr(), self.table.numel(), self._stream_ptr())
        self.A = None
        self._ws = None
        self._ws_shared = None

    def _stream_ptr(self):
        s = self._stream if self._stream is not None else self.torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def _sync_stream(self):
        kerdock_set_stream(self.handle, self._stream_ptr())

    @property
    def S(self):
        return self.info["S"]

    @property
    def N(self):
        return self.info["J"] * self.info["K"]

    def representation(self):
        """R as a (num_bases, d, ldr) tensor view (float32 or bfloat16)."""
        t = self.torch
        dt = t.bfloat16 if self.dtype == KERDOCK_BF16 else t.float32
        i = self.info
        return self.repr.view(dt).view(i["num_bases"], i["d"], i["ldr"])

    def preprocess(self, A):
        t = self.torch
        assert A.dtype == t.float32 and A.is_cuda and A.dim() == 2 and A.stride(1) == 1
        self._sync_stream()
        self.A = A  # the library reads rows of A in kerdock_apply
        kerdock_preprocess(self.handle, A.data_ptr(), A.stride(0))

    def workspace(self, q):
        nb = kerdock_apply_workspace_bytes(self.handle, q)
        if nb == 0:
            return None
        if self._ws is None or self._ws.numel() < nb:
            if self._ws is not None:
                self.sync()  # the plan's stream may still read the old buffer
            self._ws = self.torch.empty(nb, dtype=self.torch.uint8, device=self.device)
        return self._ws

    def shared_workspace(self, q):
        """Workspace of kerdock_apply_shared for q queries, kept by the plan
        (the library's kernels read it after the call returns)."""
        nb = load_library().kerdock_apply_shared_workspace_bytes(self.handle, q)
        if self._ws_shared is None or self._ws_shared.numel() < nb:
            if self._ws_shared is not None:
                self.sync()
            self._ws_shared = self.torch.empty(max(nb, 1), dtype=self.torch.uint8,
                                               device=self.device)
        return self._ws_shared, nb

    def alloc_outputs(self, q):
        t = self.torch
        S = self.S
        return (t.empty((q, S), dtype=t.int32, device=self.device),
                t.empty((q, S), dtype=t.float32, device=self.device),
                t.empty((q,), dtype=t.int32, device=self.device))

    def apply(self, X, eps, seed, flags=0, out=None, debug=False):
        t = self.torch
        assert X.dtype == t.float32 and X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        q = X.shape[0]
        idx, val, cnt = out if out is not None else self.alloc_outputs(q)
        ws = self.workspace(q)
        wsp, wsb = (ws.data_ptr(), ws.numel()) if ws is not None else (None, 0)
        self._sync_stream()
        if not debug:
            kerdock_apply(self.handle, X.data_ptr(), q, X.stride(0), float(eps), int(seed), flags,
                          idx.data_ptr(), val.data_ptr(), cnt.data_ptr(), wsp, wsb)
            return idx, val, cnt
        m = self.info["m"]
        mu = t.empty((q, m), dtype=t.float32, device=self.device)
        ells = t.empty((q, self.N), dtype=t.int64, device=self.device)
        coef = t.empty((q, self.N), dtype=t.float32, device=self.device)
        kerdock_apply_debug(self.handle, X.data_ptr(), q, X.stride(0), float(eps), int(seed), flags,
                            idx.data_ptr(), val.data_ptr(), cnt.data_ptr(), wsp, wsb,
                            mu.data_ptr(), ells.data_ptr(), coef.data_ptr())
        return idx, val, cnt, mu, ells, coef

    def sync(self):
        kerdock_sync(self.handle)

    def shared_scores(self, X, seed, out=None):
        """|mu| of every query with the shared sample set (q x m float32),
        the scores kerdock_apply_shared ranks (kerdock_apply_shared_scores)."""
        t = self.torch
        assert X.dtype == t.float32 and X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        q = X.shape[0]
        out = out if out is not None else t.empty((q, self.info["m"]), dtype=t.float32,
                                                  device=self.device)
        ws, nb = self.shared_workspace(q)
        self._sync_stream()
        kerdock_apply_shared_scores(self.handle, X.data_ptr(), q, X.stride(0), int(seed),
                                    out.data_ptr(), ws.data_ptr(), nb)
        return out

    def apply_shared(self, X, eps, seed, flags=0, out=None):
        """All rows of X share one sample set (kerdock_apply_shared)."""
        t = self.torch
        assert X.dtype == t.float32 and X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        q = X.shape[0]
        idx, val, cnt = out if out is not None else self.alloc_outputs(q)
        ws, nb = self.shared_workspace(q)
        self._sync_stream()
        kerdock_apply_shared(self.handle, X.data_ptr(), q, X.stride(0), float(eps), int(seed), flags,
                             idx.data_ptr(), val.data_ptr(), cnt.data_ptr(), ws.data_ptr(), nb)
        return idx, val, cnt

    def check_reconstruction(self, b0=0, nb=None):
        """Float64 reconstruction error per basis (kerdock_check_reconstruction),
        as a float64 CUDA tensor of nb entries."""
        t = self.torch
        nb = self.info["num_bases"] - b0 if nb is None else nb
        err = t.empty(nb, dtype=t.float64, device=self.device)
        self._sync_stream()
        kerdock_check_reconstruction(self.handle, b0, nb, err.data_ptr())
        return err

    def check_tight_frame(self, Y, b0=0, nb=None):
        """(frame, ref) of kerdock_check_tight_frame for the probes Y (P x m
        float64 CUDA tensor, P <= 4)."""
        t = self.torch
        assert Y.dtype == t.float64 and Y.is_cuda and Y.is_contiguous() and Y.dim() == 2
        nb = self.info["num_bases"] - b0 if nb is None else nb
        frame = t.empty_like(Y)
        ref = t.empty_like(Y)
        self._sync_stream()
        kerdock_check_tight_frame(self.handle, Y.data_ptr(), Y.shape[0], b0, nb, frame.data_ptr(),
                                  ref.data_ptr())
        return frame, ref

    def clone(self, J, K, S):
        """A plan over the same representation with other (J, K, S)."""
        c = KerdockPlan.__new__(KerdockPlan)
        c.torch, c.dtype, c.device = self.torch, self.dtype, self.device
        c.handle = kerdock_plan_clone(self.handle, J, K, S)
        c.info = kerdock_plan_info(c.handle)
        c.repr, c.table, c._stream, c.A, c._ws = self.repr, self.table, self._stream, self.A, None
        c._ws_shared = None
        c._parent = self
        return c

    def refine_scores(self, X, scores, S, eps, flags=0, out=None):
        """Top-S of scores (q x m), exact A_S x, threshold (Algorithm 1's last step)."""
        t = self.torch
        q = X.shape[0]
        if out is None:
            out = (t.empty((q, S), dtype=t.int32, device=self.device),
                   t.empty((q, S), dtype=t.float32, device=self.device),
                   t.empty((q,), dtype=t.int32, device=self.device))
        idx, val, cnt = out
        self._sync_stream()
        kerdock_refine_scores(self.handle, X.data_ptr(), q, X.stride(0), scores.data_ptr(), S,
                              float(eps), flags, idx.data_ptr(), val.data_ptr(), cnt.data_ptr())
        return idx, val, cnt

    def signs(self):
        return kerdock_debug_signs(self.handle)

    def close(self):
        if self.handle is not None:
            kerdock_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KerdockBatch:
    """Queries over several KerdockPlans answered by one persistent launch
    (optionally a replayed CUDA graph).  ``specs`` is a list of dicts with
    keys plan, x (1-D CUDA float32 tensor, n floats), J, K, S, eps, seed,
    index and optionally flags.  Outputs are allocated here."""

    def __init__(self, specs, graph=True, stream=None):
        import torch
        self.torch = torch
        self.specs = specs
        dev = specs[0]["plan"].device
        self.outputs = []
        queries = []
        for sp in specs:
            S = int(sp["S"])
            idx = torch.empty(S, dtype=torch.int32, device=dev)
            val = torch.empty(S, dtype=torch.float32, device=dev)
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            self.outputs.append((idx, val, cnt))
            x = sp["x"]
            assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
            queries.append(Query(plan=sp["plan"].handle.value, x=x.data_ptr(), J=int(sp["J"]),
                                 K=int(sp["K"]), S=S, flags=int(sp.get("flags", 0)),
                                 eps=float(sp["eps"]), reserved=0, seed=int(sp["seed"]),
                                 index=int(sp["index"]), out_idx=idx.data_ptr(),
                                 out_val=val.data_ptr(), out_count=cnt.data_ptr()))
        self.queries = queries
        nb = kerdock_batch_workspace_bytes(queries)
        if nb == 0:
            raise KerdockError(-1, "kerdock_batch_workspace_bytes")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.handle = kerdock_batch_create(queries, self.ws.data_ptr(), nb, self.stream.cuda_stream,
                                           KERDOCK_BATCH_GRAPH if graph else 0)

    def launch(self):
        kerdock_batch_launch(self.handle)

    def tune(self, reps=3):
        return kerdock_batch_tune(self.handle, reps)

    def set_tuning(self, ring_kb, crows):
        kerdock_batch_set_tuning(self.handle, ring_kb, crows)

    def set_costs(self, costs):
        """Re-deal the queries to the CTAs by these per-query cost estimates."""
        kerdock_batch_set_costs(self.handle, costs)

    @property
    def ctas(self):
        return kerdock_batch_ctas(self.handle)

    def set_schedule(self, lists):
        """Run lists[c] (indices into specs, in order) on CTA c."""
        kerdock_batch_set_schedule(self.handle, lists)

    def sync(self):
        kerdock_batch_sync(self.handle)

    def results(self):
        out = []
        for idx, val, cnt in self.outputs:
            c = int(cnt.item())
            out.append((idx[:c].cpu().numpy().astype(np.int64), val[:c].cpu().numpy().astype(np.float64)))
        return out

    def close(self):
        if getattr(self, "handle", None) is not None:
            kerdock_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KerdockMLP:
    """The learned-proposal network with PyTorch-allocated device buffers."""

    def __init__(self, in_dim, hidden, out_dim, max_batch, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.handle = kerdock_mlp_create(in_dim, hidden, out_dim, max_batch)
        sb, wb, self.count = kerdock_mlp_sizes(self.handle)
        self.state = torch.empty(sb, dtype=torch.uint8, device=self.device)
        self.work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        kerdock_mlp_bind(self.handle, self.state.data_ptr(), sb, self.work.data_ptr(), wb,
                         s.cuda_stream)
        self.dims = (in_dim, hidden, out_dim)
        self.max_batch = max_batch
        p, g, self.offsets = kerdock_mlp_pointers(self.handle)
        self.params = self._view(p)
        self.grads = self._view(g)

    def _view(self, ptr):
        # a float32 tensor over the library's parameter/gradient block
        t = self.torch
        base = self.state.data_ptr()
        off = (ptr - base) // 4
        return self.state.view(t.float32)[off:off + self.count]

    def tensors(self, flat):
        i, h, o = self.dims
        shapes = [(h, i), (h,), (h, h), (h,), (o, h), (o,)]
        return [flat[self.offsets[k]:self.offsets[k + 1]].view(*shapes[k]) for k in range(6)]

    def init(self, seed):
        kerdock_mlp_init(self.handle, seed)

    def set_input(self, mode):
        kerdock_mlp_set_input(self.handle, mode)

    def set_skip(self, skip):
        kerdock_mlp_set_skip(self.handle, float(skip))

    def forward(self, feats, scale, out=None):
        t = self.torch
        B = feats.shape[0]
        out = out if out is not None else t.empty((B, self.dims[2]), dtype=t.float32, device=self.device)
        kerdock_mlp_forward(self.handle, feats.data_ptr(), B, float(scale), out.data_ptr())
        return out

    def backward(self, feats, labels, scale, pos_weight):
        kerdock_mlp_backward(self.handle, feats.data_ptr(), labels.data_ptr(), feats.shape[0],
                             float(scale), float(pos_weight))

    def loss(self):
        return kerdock_mlp_loss(self.handle)

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
        kerdock_mlp_adamw(self.handle, lr, beta1, beta2, eps, wd)

    def sync_weights(self):
        kerdock_mlp_sync_weights(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            kerdock_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def results_to_lists(idx, val, cnt):
    """Host lists [(indices, values)] per query from the output tensors."""
    idx = idx.cpu().numpy()
    val = val.cpu().numpy()
    cnt = cnt.cpu().numpy()
    return [(idx[r, :cnt[r]].astype(np.int64), val[r, :cnt[r]].astype(np.float64))
            for r in range(len(cnt))]
