"""Expected Force (EF_2) on GB300: Python binding of libef.so.

The binding only marshals arguments: every step of the computation runs in
the library's sm_103a CUDA kernels behind the C ABI of ``include/ef.h``.
PyTorch provides device memory and streams.  There is no CPU path: if
``libef.so`` has not been built, or no CUDA device is present, every call
raises ``EfError``.

Functions carry the C names (``ef_ctx_create``, ``ef_compute``,
``ef_compute_ex``, ...); ``Context`` is a small convenience wrapper.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libef.so")

EF_OK, EF_ERR_ARG, EF_ERR_GRAPH, EF_ERR_OOM, EF_ERR_CUDA, EF_ERR_TIMEOUT, EF_ERR_MODEL, EF_ERR_UNSUPPORTED = range(8)
EF_PREC_FP64, EF_PREC_FP32C = 0, 1
EF_MAX_DEGREE = 1 << 20   # largest maximum degree a validated call accepts (include/ef.h)
PRECISIONS = {"fp64": EF_PREC_FP64, "fp32c": EF_PREC_FP32C}

# Every symbol include/ef.h declares (checked by the CPU test of the ABI).
EXPORTED = ("ef_ctx_create", "ef_ctx_set_memory_limit", "ef_ctx_destroy", "ef_last_error", "ef_sync", "ef_get_stats",
            "ef_compute", "ef_compute_ex", "ef_compute_batched", "ef_get_tuning", "ef_set_tuning", "ef_autotune",
            "ef_compute_nodes", "ef_features", "ef_model_create", "ef_model_destroy", "ef_model_get", "ef_model_set",
            "ef_model_feature_mode", "ef_model_save", "ef_model_load", "ef_mlp_forward", "ef_mlp_grad",
            "ef_surrogate_train", "ef_surrogate_rank", "ef_compute_static", "ef_compute_shard",
            "ef_finalize_partials", "ef_sir_run")
MODEL_PARAMS = 5313
MODEL_FLOATS = MODEL_PARAMS + 32


class EfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libef error {code}: {msg}")
        self.code = code


class ef_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class ef_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("trust_input", ctypes.c_int32), ("host_io", ctypes.c_int32),
                ("async_", ctypes.c_int32), ("profile", ctypes.c_int32), ("wedge_mode", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("device_check", ctypes.c_int32)]


class ef_outputs(ctypes.Structure):
    _fields_ = [("ef", ctypes.c_void_p), ("n_clusters", ctypes.c_void_p), ("s", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("triangles", ctypes.c_void_p), ("flag", ctypes.c_void_p)]


class ef_partials(ctypes.Structure):
    _fields_ = [("t", ctypes.c_void_p), ("q", ctypes.c_void_p), ("triangles", ctypes.c_void_p),
                ("n_clusters", ctypes.c_void_p), ("s_open", ctypes.c_void_p)]


PARTIALS = ("t", "q", "triangles", "n_clusters", "s_open")   # float64, then int64 x4


class ef_sir_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("sim_base", ctypes.c_int64), ("max_steps", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("spread_min_size", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ef_sir_outputs(ctypes.Structure):
    _fields_ = [("final_size", ctypes.c_void_p), ("length", ctypes.c_void_p), ("peak_infected", ctypes.c_void_p),
                ("peak_step", ctypes.c_void_p), ("truncated", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("spread", ctypes.c_void_p), ("spread_sims", ctypes.c_void_p)]


class ef_stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("prep_ms", ctypes.c_double), ("orient_ms", ctypes.c_double),
                ("wedge_small_ms", ctypes.c_double), ("wedge_big_ms", ctypes.c_double),
                ("tri_hash_ms", ctypes.c_double), ("tri_pairs_ms", ctypes.c_double),
                ("finalize_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("kernels", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ef_train_options(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("pad", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class ef_train_stats(ctypes.Structure):
    _fields_ = [("first_loss", ctypes.c_float), ("last_loss", ctypes.c_float), ("ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ef_rank_stats(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("n_audit", ctypes.c_int32), ("n_top", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("spearman_audit", ctypes.c_double), ("max_abs_err_audit", ctypes.c_double),
                ("features_ms", ctypes.c_double), ("infer_ms", ctypes.c_double), ("select_ms", ctypes.c_double),
                ("exact_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("exact_tri_ms", ctypes.c_double),
                ("exact_wedge_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ef_tuning(ctypes.Structure):
    _fields_ = [("row_thread_max", ctypes.c_int32), ("hub_min", ctypes.c_int32), ("tri_variant", ctypes.c_int32),
                ("grid_per_sm", ctypes.c_int32), ("layout", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libef.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise EfError(EF_ERR_CUDA, f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.ef_ctx_create.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.ef_ctx_destroy.argtypes = [vp]
    lib.ef_ctx_set_memory_limit.argtypes = [vp, ctypes.c_uint64]
    lib.ef_last_error.argtypes = [vp]
    lib.ef_last_error.restype = ctypes.c_char_p
    lib.ef_sync.argtypes = [vp]
    lib.ef_get_stats.argtypes = [vp, ctypes.POINTER(ef_stats), ctypes.c_int]
    lib.ef_compute.argtypes = [ctypes.POINTER(ef_csr), i32, i64, vp]
    lib.ef_compute_ex.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, ctypes.POINTER(ef_options),
                                  ctypes.POINTER(ef_outputs)]
    lib.ef_compute_batched.argtypes = [vp, ctypes.POINTER(ef_csr), i64, ctypes.POINTER(ctypes.c_int64), i32,
                                       ctypes.POINTER(ef_options), ctypes.POINTER(ef_outputs)]
    lib.ef_get_tuning.argtypes = [vp, ctypes.POINTER(ef_tuning)]
    lib.ef_set_tuning.argtypes = [vp, ctypes.POINTER(ef_tuning)]
    lib.ef_autotune.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, ctypes.POINTER(ef_options), i32,
                                ctypes.POINTER(ef_tuning)]
    lib.ef_compute_nodes.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, vp, i32, ctypes.POINTER(ef_options),
                                     ctypes.POINTER(ef_outputs)]
    lib.ef_features.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, i32, ctypes.POINTER(ef_options), vp]
    lib.ef_model_create.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(vp)]
    lib.ef_model_destroy.argtypes = [vp]
    lib.ef_model_get.argtypes = [vp, vp]
    lib.ef_model_set.argtypes = [vp, vp]
    lib.ef_model_feature_mode.argtypes = [vp]
    lib.ef_model_save.argtypes = [vp, ctypes.c_char_p]
    lib.ef_model_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(vp)]
    lib.ef_mlp_forward.argtypes = [vp, vp, vp, i32, vp]
    lib.ef_mlp_grad.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(ctypes.c_float), vp]
    lib.ef_surrogate_train.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(ef_train_options),
                                       ctypes.POINTER(ef_train_stats)]
    lib.ef_surrogate_rank.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, vp, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ef_options), vp, vp, vp,
                                      ctypes.POINTER(ef_rank_stats)]
    lib.ef_compute_static.argtypes = [ctypes.POINTER(ef_csr), i32, i64, i32, vp, vp]
    lib.ef_compute_shard.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, i32, i32, ctypes.POINTER(ef_options),
                                     ctypes.POINTER(ef_partials), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]
    lib.ef_finalize_partials.argtypes = [vp, i32, ctypes.POINTER(ef_partials), i32, ctypes.POINTER(ef_options),
                                         ctypes.POINTER(ef_outputs)]
    lib.ef_sir_run.argtypes = [vp, ctypes.POINTER(ef_csr), i32, i64, vp, i32, vp, i32, vp,
                               ctypes.POINTER(ef_sir_params), ctypes.POINTER(ef_options), ctypes.POINTER(ef_sir_outputs)]
    for name in EXPORTED:
        if name != "ef_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != EF_OK:
        msg = load_library().ef_last_error(ctx)
        raise EfError(rc, (msg or b"").decode(errors="replace"))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ------------------------------------------------------------- C-named calls

def ef_ctx_create(device: int = 0, stream: int | None = None) -> int:
    """Create a context on `device` issuing on `stream` (a cudaStream_t handle, None = default)."""
    h = ctypes.c_void_p()
    _check(load_library().ef_ctx_create(device, stream or None, ctypes.byref(h)))
    return h.value


def ef_ctx_set_memory_limit(ctx: int, nbytes: int) -> None:
    """Cap the device bytes the context's working buffers may hold (0 = no cap)."""
    _check(load_library().ef_ctx_set_memory_limit(ctx, int(nbytes)), ctx)


def ef_ctx_destroy(ctx: int) -> None:
    _check(load_library().ef_ctx_destroy(ctx), ctx)


def ef_last_error(ctx: int | None = None) -> str:
    return (load_library().ef_last_error(ctx) or b"").decode(errors="replace")


def ef_sync(ctx: int) -> None:
    _check(load_library().ef_sync(ctx), ctx)


def ef_get_stats(ctx: int, reset: bool = False) -> dict:
    st = ef_stats()
    _check(load_library().ef_get_stats(ctx, ctypes.byref(st), int(reset)), ctx)
    return st.as_dict()


def ef_compute(row_ptr, col_idx, out_ef) -> None:
    """EF of every node; CUDA tensors (int32 CSR, float64 output), FP64 path, synchronous."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    _check(load_library().ef_compute(ctypes.byref(g), n, int(col_idx.shape[0]), _ptr(out_ef)))


def _options(precision, trust_input, host_io, async_, profile, wedge_mode, graph, device_check=False) -> ef_options:
    return ef_options(PRECISIONS[precision], int(trust_input), int(host_io), int(async_), int(profile),
                      int(wedge_mode), int(graph), int(device_check))


def ef_compute_ex(ctx: int, row_ptr, col_idx, *, precision: str = "fp64", ef=None, n_clusters=None, s=None,
                  t=None, triangles=None, flag=None, trust_input: bool = False, host_io: bool = False,
                  async_: bool = False, profile: bool = False, wedge_mode: int = 0, graph: bool = False,
                  device_check: bool = False) -> None:
    """Full-control EF: writes whichever output buffers are given (device, or host with host_io)."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, host_io, async_, profile, wedge_mode, graph, device_check)
    out = ef_outputs(_ptr(ef), _ptr(n_clusters), _ptr(s), _ptr(t), _ptr(triangles), _ptr(flag))
    _check(load_library().ef_compute_ex(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), ctypes.byref(o),
                                        ctypes.byref(out)), ctx)


def ef_compute_batched(ctx: int, row_ptr, col_idx, graph_off, *, precision: str = "fp64", ef=None,
                       n_clusters=None, s=None, t=None, triangles=None, flag=None, trust_input: bool = False,
                       host_io: bool = False, async_: bool = False, profile: bool = False, wedge_mode: int = 0,
                       graph: bool = True, device_check: bool = False) -> None:
    """EF of every node of a batch of graphs given as one disjoint-union CSR; graph_off is a host int64
    array of num_graphs + 1 node offsets."""
    off = np.ascontiguousarray(np.asarray(graph_off, dtype=np.int64))
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, host_io, async_, profile, wedge_mode, graph, device_check)
    out = ef_outputs(_ptr(ef), _ptr(n_clusters), _ptr(s), _ptr(t), _ptr(triangles), _ptr(flag))
    _check(load_library().ef_compute_batched(ctx, ctypes.byref(g), int(col_idx.shape[0]),
                                             off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1,
                                             ctypes.byref(o), ctypes.byref(out)), ctx)


def ef_get_tuning(ctx: int) -> dict:
    t = ef_tuning()
    _check(load_library().ef_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t.as_dict()


def ef_set_tuning(ctx: int, tuning: dict | None = None) -> None:
    """Set the context's launch parameters (None restores the defaults)."""
    if tuning is None:
        _check(load_library().ef_set_tuning(ctx, None), ctx)
        return
    t = ef_tuning(**tuning)
    _check(load_library().ef_set_tuning(ctx, ctypes.byref(t)), ctx)


def ef_autotune(ctx: int, row_ptr, col_idx, *, precision: str = "fp32c", reps: int = 3,
                trust_input: bool = False, wedge_mode: int = 0) -> dict:
    """Time candidate launch parameters on this graph; keeps the fastest on the context and returns it."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, False, False, False, wedge_mode, False)
    t = ef_tuning()
    _check(load_library().ef_autotune(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), ctypes.byref(o), int(reps),
                                      ctypes.byref(t)), ctx)
    return t.as_dict()


def ef_compute_static(row_ptr, col_idx, out_ef, precision: str = "fp64", stream: int | None = None) -> None:
    """EF of every node with no allocation (fixed 32 MiB library scratch); CUDA tensors, synchronous."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    _check(load_library().ef_compute_static(ctypes.byref(g), n, int(col_idx.shape[0]), PRECISIONS[precision],
                                            _ptr(out_ef), stream or None))


def ef_compute_nodes(ctx: int, row_ptr, col_idx, nodes, *, precision: str = "fp64", ef=None, n_clusters=None,
                     s=None, t=None, triangles=None, flag=None, trust_input: bool = False) -> None:
    """Exact EF of the listed nodes only (device tensors; outputs of length len(nodes))."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, False, False, False, 0, False)
    out = ef_outputs(_ptr(ef), _ptr(n_clusters), _ptr(s), _ptr(t), _ptr(triangles), _ptr(flag))
    _check(load_library().ef_compute_nodes(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), _ptr(nodes),
                                           int(nodes.shape[0]), ctypes.byref(o), ctypes.byref(out)), ctx)


def empty_partials(n: int, device) -> dict:
    """Device buffers for one shard's partials (the five arrays of ef_partials)."""
    import torch
    return {k: torch.empty(n, dtype=torch.float64 if k == "t" else torch.int64, device=device) for k in PARTIALS}


def ef_compute_shard(ctx: int, row_ptr, col_idx, shard: int, num_shards: int, parts: dict, *,
                     precision: str = "fp64", trust_input: bool = False, wedge_mode: int = 0) -> tuple:
    """Partials of one shard into ``parts`` (the five device tensors of
    ``empty_partials``).  Returns (frac_bits, (lo, hi)): the fixed-point scale
    of q and the shard's node range."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, False, False, False, wedge_mode, False)
    p = ef_partials(*(_ptr(parts.get(k)) for k in PARTIALS))
    frac = ctypes.c_int32()
    rng = (ctypes.c_int32 * 2)()
    _check(load_library().ef_compute_shard(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), int(shard),
                                           int(num_shards), ctypes.byref(o), ctypes.byref(p), ctypes.byref(frac),
                                           rng), ctx)
    return frac.value, tuple(rng)


def ef_finalize_partials(ctx: int, parts: dict, frac_bits: int, *, precision: str = "fp64", ef=None,
                         n_clusters=None, s=None, t=None, triangles=None, flag=None) -> None:
    """EF from partials summed over every shard of one graph (device tensors; no graph input)."""
    n = int(parts["t"].shape[0])
    o = _options(precision, False, False, False, False, 0, False)
    p = ef_partials(*(_ptr(parts.get(k)) for k in PARTIALS))
    out = ef_outputs(_ptr(ef), _ptr(n_clusters), _ptr(s), _ptr(t), _ptr(triangles), _ptr(flag))
    _check(load_library().ef_finalize_partials(ctx, n, ctypes.byref(p), int(frac_bits), ctypes.byref(o),
                                               ctypes.byref(out)), ctx)


def allreduce_partials(parts: dict, group=None) -> None:
    """The one exchange of a sharded computation: element-wise sums over the
    ranks of ``group`` (torch.distributed, in place, 40 bytes per node).  T
    is summed in FP64; the other four arrays are integers and sum exactly."""
    import torch.distributed as dist
    for k in PARTIALS:
        dist.all_reduce(parts[k], op=dist.ReduceOp.SUM, group=group)


def shard_ranges(node_range, group=None) -> list:
    """Every rank's node range [lo, hi), from each rank's own (as ef_compute_shard
    reported it): one all-gather of two integers per rank."""
    import torch
    import torch.distributed as dist
    mine = torch.tensor(list(node_range), dtype=torch.int64)
    allr = [torch.zeros(2, dtype=torch.int64) for _ in range(dist.get_world_size(group))]
    dist.all_gather(allr, mine, group=group)
    return [tuple(int(x) for x in r) for r in allr]


def reduce_scatter_partials(parts: dict, ranges: list, group=None) -> None:
    """The exchange by node range: rank r receives, in place in its own
    ``parts``, the sums over all ranks of the partials of its nodes
    ranges[r] = [lo, hi) (the other slices of ``parts`` are left undefined).
    Each node's sums reach only the rank that finalizes it: (R - 1) / R of
    the 40 bytes per node leave each rank, half of what an all-reduce moves."""
    import torch.distributed as dist
    ranks = dist.get_process_group_ranks(group) if group is not None else list(range(dist.get_world_size()))
    for r, (lo, hi) in enumerate(ranges):
        if hi <= lo:
            continue
        for k in PARTIALS:
            dist.reduce(parts[k][lo:hi], dst=ranks[r], op=dist.ReduceOp.SUM, group=group)


def partials_slice(parts: dict, lo: int, hi: int) -> dict:
    """The partials of nodes [lo, hi) (views, no copy)."""
    return {k: v[lo:hi] for k, v in parts.items()}


def compute_sharded(ctx: int, row_ptr, col_idx, rank: int, world: int, *, group=None, precision: str = "fp64",
                    outputs=("ef",), trust_input: bool = False, exchange: str = "allreduce") -> dict:
    """EF with the cluster loop split over ``world`` ranks.

    Each rank holds the whole CSR (device tensors) and computes shard
    ``rank``.  exchange="allreduce": ``allreduce_partials`` (skipped when
    world == 1), then every rank finalizes every node and returns the full
    outputs.  exchange="reduce_scatter": ``reduce_scatter_partials``, then
    each rank finalizes only its own node range and returns those outputs
    (length hi - lo) with the key "range" = (lo, hi).  The exchange runs on
    the partials' device (the process group's backend must support it).
    """
    import torch
    n = int(row_ptr.shape[0]) - 1
    dev = row_ptr.device
    parts = empty_partials(n, dev)
    frac, rng = ef_compute_shard(ctx, row_ptr, col_idx, rank, world, parts, precision=precision,
                                 trust_input=trust_input)
    dt = dict(ef=torch.float64, n_clusters=torch.int64, s=torch.int64, t=torch.float64, triangles=torch.int64,
              flag=torch.uint8)
    if exchange == "allreduce":
        if world > 1:
            allreduce_partials(parts, group)
        res = {k: torch.empty(n, dtype=dt[k], device=dev) for k in outputs}
        ef_finalize_partials(ctx, parts, frac, precision=precision, **res)
        return res
    if exchange != "reduce_scatter":
        raise ValueError(f"exchange must be 'allreduce' or 'reduce_scatter', not {exchange!r}")
    ranges = shard_ranges(rng, group) if world > 1 else [rng]
    if world > 1:
        reduce_scatter_partials(parts, ranges, group)
    lo, hi = rng
    res = {k: torch.empty(hi - lo, dtype=dt[k], device=dev) for k in outputs}
    if hi > lo:
        ef_finalize_partials(ctx, partials_slice(parts, lo, hi), frac, precision=precision, **res)
    res["range"] = (lo, hi)
    return res


SIR_OUTPUTS = ("final_size", "length", "peak_infected", "peak_step", "truncated", "parent", "spread",
               "spread_sims")


def ef_sir_run(ctx: int, row_ptr, col_idx, index_cases, *, beta: float, gamma: float, seed: int, sim_base: int = 0,
               max_steps: int = 100000, depth: int = 4, spread_min_size: int = 0, immune=None, immune_set=None,
               trust_input: bool = False, **outputs) -> None:
    """SIR simulations from the given index cases (device tensors); writes the
    ef_sir_outputs members passed by name (device tensors)."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options("fp64", trust_input, False, False, False, 0, False)
    p = ef_sir_params(float(beta), float(gamma), int(seed) & (2 ** 64 - 1), int(sim_base), int(max_steps), int(depth),
                      int(spread_min_size), 0)
    bad = set(outputs) - set(SIR_OUTPUTS)
    if bad:
        raise TypeError(f"unknown SIR outputs {sorted(bad)}")
    out = ef_sir_outputs(*(_ptr(outputs.get(k)) for k in SIR_OUTPUTS))
    nsets = 0 if immune is None else int(immune.shape[0])
    _check(load_library().ef_sir_run(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), _ptr(index_cases),
                                     int(index_cases.shape[0]), _ptr(immune), nsets, _ptr(immune_set),
                                     ctypes.byref(p), ctypes.byref(o), ctypes.byref(out)), ctx)


def ef_features(ctx: int, row_ptr, col_idx, x, *, mode: int = 0, trust_input: bool = False) -> None:
    """The 16 learned-path features of every node into x (device float32 [n, 16])."""
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options("fp64", trust_input, False, False, False, 0, False)
    _check(load_library().ef_features(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), int(mode), ctypes.byref(o),
                                      _ptr(x)), ctx)


def ef_model_create(ctx: int, seed: int = 0, feature_mode: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load_library().ef_model_create(ctx, int(seed), int(feature_mode), ctypes.byref(h)), ctx)
    return h.value


def ef_model_destroy(model: int) -> None:
    _check(load_library().ef_model_destroy(model))


def ef_model_get(model: int) -> np.ndarray:
    h = np.zeros(MODEL_FLOATS, dtype=np.float32)
    _check(load_library().ef_model_get(model, h.ctypes.data))
    return h


def ef_model_set(model: int, flat) -> None:
    h = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
    if h.shape != (MODEL_FLOATS,):
        raise EfError(EF_ERR_ARG, f"expected {MODEL_FLOATS} floats")
    _check(load_library().ef_model_set(model, h.ctypes.data))


def ef_model_feature_mode(model: int) -> int:
    return load_library().ef_model_feature_mode(model)


def ef_model_save(model: int, path: str) -> None:
    _check(load_library().ef_model_save(model, str(path).encode()))


def ef_model_load(ctx: int, path: str) -> int:
    h = ctypes.c_void_p()
    _check(load_library().ef_model_load(ctx, str(path).encode(), ctypes.byref(h)), ctx)
    return h.value


def ef_mlp_forward(ctx: int, model: int, x, out) -> None:
    _check(load_library().ef_mlp_forward(ctx, model, _ptr(x), int(x.shape[0]), _ptr(out)), ctx)


def ef_mlp_grad(ctx: int, model: int, x, y) -> tuple[float, np.ndarray]:
    g = np.zeros(MODEL_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load_library().ef_mlp_grad(ctx, model, _ptr(x), _ptr(y), int(x.shape[0]), ctypes.byref(loss),
                                      g.ctypes.data), ctx)
    return float(loss.value), g


def ef_surrogate_train(ctx: int, model: int, x, y, *, steps: int, batch: int = 4096, lr: float = 1e-3,
                       seed: int = 1) -> dict:
    o = ef_train_options(int(steps), int(batch), float(lr), 0, int(seed))
    st = ef_train_stats()
    _check(load_library().ef_surrogate_train(ctx, model, _ptr(x), _ptr(y), int(x.shape[0]), ctypes.byref(o),
                                             ctypes.byref(st)), ctx)
    return st.as_dict()


def ef_surrogate_rank(ctx: int, model: int, row_ptr, col_idx, out_idx, out_ef, *, top_frac: float = 0.01,
                      cand_frac: float = 0.02, audit_frac: float = 0.001, seed: int = 7, precision: str = "fp32c",
                      out_score=None, trust_input: bool = False) -> dict:
    n = int(row_ptr.shape[0]) - 1
    g = ef_csr(_ptr(row_ptr), _ptr(col_idx))
    o = _options(precision, trust_input, False, False, False, 0, False)
    st = ef_rank_stats()
    _check(load_library().ef_surrogate_rank(ctx, ctypes.byref(g), n, int(col_idx.shape[0]), model, float(top_frac),
                                            float(cand_frac), float(audit_frac), int(seed), ctypes.byref(o),
                                            _ptr(out_idx), _ptr(out_ef), _ptr(out_score), ctypes.byref(st)), ctx)
    return st.as_dict()


class Model:
    """A surrogate network on the device of a context (wraps ef_model_*)."""

    def __init__(self, ctx: int, seed: int = 0, feature_mode: int = 0, handle: int | None = None):
        self.ctx = ctx
        self.handle = ef_model_create(ctx, seed, feature_mode) if handle is None else handle

    @classmethod
    def load(cls, ctx: int, path: str) -> "Model":
        return cls(ctx, handle=ef_model_load(ctx, path))

    def close(self):
        if self.handle:
            ef_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def feature_mode(self) -> int:
        return ef_model_feature_mode(self.handle)

    def get(self) -> np.ndarray:
        return ef_model_get(self.handle)

    def set(self, flat) -> None:
        ef_model_set(self.handle, flat)

    def save(self, path: str) -> None:
        ef_model_save(self.handle, path)

    def forward(self, x, out) -> None:
        ef_mlp_forward(self.ctx, self.handle, x, out)

    def grad(self, x, y) -> tuple[float, np.ndarray]:
        return ef_mlp_grad(self.ctx, self.handle, x, y)

    def train(self, x, y, **kw) -> dict:
        return ef_surrogate_train(self.ctx, self.handle, x, y, **kw)

    def rank(self, row_ptr, col_idx, out_idx, out_ef, **kw) -> dict:
        return ef_surrogate_rank(self.ctx, self.handle, row_ptr, col_idx, out_idx, out_ef, **kw)


# ---------------------------------------------------------------- convenience

class Context:
    """A libef context bound to one CUDA device and the torch stream current at creation."""

    def __init__(self, device: int | None = None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise EfError(EF_ERR_CUDA, "no CUDA device")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = ef_ctx_create(self.device, self.stream.cuda_stream)

    def close(self):
        if self.handle:
            ef_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, row_ptr, col_idx, precision: str = "fp64", outputs=("ef",), **kw) -> dict:
        """Allocate the requested outputs on the device and run ef_compute_ex."""
        import torch
        n = int(row_ptr.shape[0]) - 1
        dev = torch.device("cuda", self.device)
        dt = dict(ef=torch.float64, n_clusters=torch.int64, s=torch.int64, t=torch.float64,
                  triangles=torch.int64, flag=torch.uint8)
        res = {k: torch.empty(n, dtype=dt[k], device=dev) for k in outputs}
        ef_compute_ex(self.handle, row_ptr, col_idx, precision=precision, **res, **kw)
        return res

    def stats(self, reset: bool = False) -> dict:
        return ef_get_stats(self.handle, reset)

    def set_memory_limit(self, nbytes: int) -> None:
        ef_ctx_set_memory_limit(self.handle, nbytes)

    def sir(self, row_ptr, col_idx, index_cases, *, outputs=("final_size", "length", "peak_infected", "peak_step"),
            depth: int = 4, **kw) -> dict:
        """Allocate the requested SIR outputs on the device and run ef_sir_run."""
        import torch
        n = int(row_ptr.shape[0]) - 1
        B = int(index_cases.shape[0])
        dev = torch.device("cuda", self.device)
        shape = dict(final_size=(B,), length=(B,), peak_infected=(B,), peak_step=(B,), truncated=(B,),
                     parent=(B, n), spread=(depth, n), spread_sims=(n,))
        dt = dict(final_size=torch.int32, length=torch.int32, peak_infected=torch.int32, peak_step=torch.int32,
                  truncated=torch.uint8, parent=torch.int32, spread=torch.int64, spread_sims=torch.int64)
        res = {k: torch.empty(shape[k], dtype=dt[k], device=dev) for k in outputs}
        ef_sir_run(self.handle, row_ptr, col_idx, index_cases, depth=depth, **kw, **res)
        return res
