"""ctypes binding of the C ABI in include/rg.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: GEMMs, sweeps, plan tables and statistics all run in
librg.so.  Device buffers are passed as integers (``tensor.data_ptr()``) or
as objects with a ``data_ptr()`` method; streams as ``torch.cuda.Stream``,
raw ``cudaStream_t`` integers or None (legacy default stream).

If librg.so is missing the import fails loudly: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# RG_LIBRARY may name another build of the same library (for example the phase-timer build,
# librg_timers.so, next to librg.so); by default the in-tree librg.so.
_LIB_PATH = os.environ.get("RG_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "librg.so")

RG_OK = 0
RG_ERR_INVALID = -1
RG_ERR_ALIGN = -2
RG_ERR_SHAPE = -3
RG_ERR_OOM = -4
RG_ERR_CUDA = -5
RG_ERR_TIMEOUT = -6
RG_ERR_PLAN_MISMATCH = -7
RG_ERR_ADMISSION = -8
RG_ERR_NO_DEVICE = -9

RG_T_UNMEASURED = 1 << 60
RG_T_OTHER_SHARD = 0
RG_NUM_TILES = 8
RG_NUM_PAPER_TILES = 6                # tiles 0..5: the paper's six (best-of-6)
RG_NUM_SPLITS = 4
PAIR_TILES = [4, 5, 7]                # 256x128, 256x256, 256x192: also run as cta_group::2 pairs
RG_NUM_VARIANTS = RG_NUM_TILES * RG_NUM_SPLITS + RG_NUM_TILES + len(PAIR_TILES) * (RG_NUM_SPLITS + 1)
TILES = [(128, 64), (128, 128), (128, 256), (256, 64), (256, 128), (256, 256), (128, 192), (256, 192)]
SPLITS = [1, 2, 4, 8]
SK = "SK"
TWO_SM = "2SM"
TWO_SM_SK = "2SM-SK"
_BASE_2SM = RG_NUM_TILES * RG_NUM_SPLITS + RG_NUM_TILES
_BASE_2SM_SK = _BASE_2SM + len(PAIR_TILES) * RG_NUM_SPLITS


def variant(tile: int, split=1) -> int:
    """Variant id of a tile with split factor 1/2/4/8, split="SK" for stream-K, "2SM" / ("2SM", S)
    for the cta_group::2 pair with split factor S, or "2SM-SK" for the cta_group::2 stream-K form
    (the last three for the pair tiles 256x128, 256x256 and 256x192 only)."""
    if split == TWO_SM_SK or split == TWO_SM or (isinstance(split, tuple) and split[0] == TWO_SM):
        if tile not in PAIR_TILES:
            raise ValueError("the 2-SM variants exist for the 256x128, 256x256 and 256x192 tiles only")
        i = PAIR_TILES.index(tile)
        if split == TWO_SM_SK:
            return _BASE_2SM_SK + i
        s = 1 if split == TWO_SM else split[1]
        return _BASE_2SM + i * RG_NUM_SPLITS + SPLITS.index(s)
    if split == SK:
        return RG_NUM_TILES * RG_NUM_SPLITS + tile
    return tile * RG_NUM_SPLITS + SPLITS.index(split)


def variant_tile(v: int) -> int:
    """Tile index (0..7) of a variant id."""
    n = RG_NUM_TILES * RG_NUM_SPLITS
    if v >= _BASE_2SM_SK:
        return PAIR_TILES[v - _BASE_2SM_SK]
    if v >= _BASE_2SM:
        return PAIR_TILES[(v - _BASE_2SM) // RG_NUM_SPLITS]
    return v - n if v >= n else v // RG_NUM_SPLITS


def variant_name(v: int) -> str:
    if v >= _BASE_2SM_SK:
        bm, bn = TILES[variant_tile(v)]
        return f"{bm}x{bn}/2SM-SK"
    if v >= _BASE_2SM:
        bm, bn = TILES[variant_tile(v)]
        s = SPLITS[(v - _BASE_2SM) % RG_NUM_SPLITS]
        return f"{bm}x{bn}/2SM" + ("" if s == 1 else f"-S{s}")
    if v >= RG_NUM_TILES * RG_NUM_SPLITS:
        bm, bn = TILES[v - RG_NUM_TILES * RG_NUM_SPLITS]
        return f"{bm}x{bn}/SK"
    bm, bn = TILES[v // RG_NUM_SPLITS]
    return f"{bm}x{bn}/S{SPLITS[v % RG_NUM_SPLITS]}"


class rg_axis(C.Structure):
    _fields_ = [("start", C.c_int32), ("step", C.c_int32), ("count", C.c_int32)]


class rg_grid(C.Structure):
    _fields_ = [("m", rg_axis), ("n", rg_axis), ("k", rg_axis)]


class rg_leaf(C.Structure):
    _fields_ = [("variant", C.c_int32), ("beta", C.c_int32), ("phase", C.c_int32), ("reserved", C.c_int32),
                ("m0", C.c_int64), ("n0", C.c_int64), ("k0", C.c_int64),
                ("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int64),
                ("pm", C.c_int64), ("pn", C.c_int64), ("pk", C.c_int64)]


class rg_sweep_opts(C.Structure):
    _fields_ = [("reps", C.c_int32), ("warmup", C.c_int32), ("global_warmup", C.c_int32),
                ("shuffle", C.c_int32), ("seed", C.c_uint64), ("spin_ns", C.c_int64),
                ("prune_splits", C.c_int32), ("shard_index", C.c_int32), ("shard_count", C.c_int32),
                ("reserved", C.c_int32)]


class rg_group_problem(C.Structure):
    _fields_ = [("M", C.c_int64), ("N", C.c_int64), ("K", C.c_int64), ("A", C.c_void_p), ("lda", C.c_int64),
                ("B", C.c_void_p), ("ldb", C.c_int64), ("C", C.c_void_p), ("ldc", C.c_int64),
                ("pm", C.c_int64), ("pn", C.c_int64), ("pk", C.c_int64), ("beta", C.c_int32),
                ("variant", C.c_int32)]


class rg_serve_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_batch", C.c_int32), ("max_inflight", C.c_int32),
                ("tile", C.c_int32), ("workspace_mib", C.c_int32), ("fp8_plan", C.c_void_p)]


RG_DTYPE_BF16 = 0
RG_DTYPE_FP8 = 1


class rg_serve_request(C.Structure):
    _fields_ = [("M", C.c_int64), ("N", C.c_int64), ("K", C.c_int64), ("A", C.c_void_p), ("lda", C.c_int64),
                ("B", C.c_void_p), ("ldb", C.c_int64), ("C", C.c_void_p), ("ldc", C.c_int64),
                ("arrival_ns", C.c_int64), ("dtype", C.c_int32), ("reserved", C.c_int32),
                ("sA", C.c_void_p), ("lds_a", C.c_int64), ("sB", C.c_void_p), ("lds_b", C.c_int64)]


def serve_request(M, N, K, A, lda, B, ldb, Cp, ldc, arrival_ns=0, fp8=None) -> rg_serve_request:
    """One request; fp8 = (sA, lds_a, sB, lds_b) makes it an FP8 request (A, B are e4m3 codes)."""
    if fp8 is None:
        return rg_serve_request(M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, int(arrival_ns), RG_DTYPE_BF16,
                                0, None, 0, None, 0)
    sA, lds_a, sB, lds_b = fp8
    return rg_serve_request(M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, int(arrival_ns), RG_DTYPE_FP8, 0,
                            _ptr(sA), lds_a, _ptr(sB), lds_b)


class rg_serve_result(C.Structure):
    _fields_ = [("admitted_ns", C.c_int64), ("launched_ns", C.c_int64), ("done_ns", C.c_int64),
                ("batch", C.c_int32), ("status", C.c_int32)]


class rg_serve_stats(C.Structure):
    _fields_ = [("requests", C.c_int64), ("batches", C.c_int64), ("admission_stalls", C.c_int64),
                ("wall_s", C.c_double), ("p50_latency_us", C.c_double), ("p99_latency_us", C.c_double),
                ("mean_latency_us", C.c_double), ("tflops", C.c_double)]


class RGError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


if not os.path.exists(_LIB_PATH):
    raise ImportError(f"librg.so not built ({_LIB_PATH}); run __graft_entry__.build() or "
                      f"python -m paper_2605_29752_gb300.build")
_lib = C.CDLL(_LIB_PATH)

_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_sigs = {
    "rg_version": (C.c_char_p, []),
    "rg_strerror": (C.c_char_p, [C.c_int]),
    "rg_last_error": (C.c_char_p, []),
    "rg_sweep_opts_default": (None, [C.POINTER(rg_sweep_opts)]),
    "rg_init": (C.c_int, [C.c_int, _I64, C.POINTER(_P)]),
    "rg_destroy": (None, [_P]),
    "rg_sm_count": (C.c_int, [_P, C.POINTER(_I32)]),
    "rg_check": (C.c_int, [_P, _P]),
    "rg_set_timeout_cycles": (C.c_int, [_P, _I64]),
    "rg_set_static_operands": (C.c_int, [_P, _I32]),
    "rg_gemm": (C.c_int, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I32, _I32, _I64, _I64, _I64, _P]),
    "rg_plan_build": (C.c_int, [C.POINTER(rg_grid), _P, _I32, _P, C.POINTER(_P)]),
    "rg_plan_build_ex": (C.c_int, [C.POINTER(rg_grid), _P, _I32, _P, _I32, C.POINTER(_P)]),
    "rg_launch_count": (C.c_int, [_P, C.POINTER(_I64)]),
    "rg_set_test_stall": (C.c_int, [_P, _I32]),
    "rg_group_create": (C.c_int, [_P, _I32, _I32, _I64, C.POINTER(_P)]),
    "rg_group_destroy": (None, [_P]),
    "rg_gemm_grouped": (C.c_int, [_P, C.POINTER(rg_group_problem), _I32, _P]),
    "rg_serve_opts_default": (None, [C.POINTER(rg_serve_opts)]),
    "rg_serve": (C.c_int, [_P, _P, C.POINTER(rg_serve_opts), C.POINTER(rg_serve_request), _I32,
                           C.POINTER(rg_serve_result), C.POINTER(rg_serve_stats)]),
    "rg_serve_start": (C.c_int, [_P, _P, C.POINTER(rg_serve_opts), C.POINTER(_P)]),
    "rg_serve_submit": (C.c_int, [_P, C.POINTER(rg_serve_request), C.POINTER(_I64)]),
    "rg_serve_poll": (C.c_int, [_P, _I64, C.POINTER(rg_serve_result), C.POINTER(_I32)]),
    "rg_serve_wait": (C.c_int, [_P, _I64, C.POINTER(rg_serve_result)]),
    "rg_serve_stop": (C.c_int, [_P, C.POINTER(rg_serve_stats)]),
    "rg_fp8_quantize": (C.c_int, [_P, _P, _I64, _I64, _I64, _P, _I64, _P, _P]),
    "rg_gemm_fp8": (C.c_int, [_P, _I64, _I64, _I64, _P, _I64, _P, _P, _I64, _P, _P, _I64, _P]),
    "rg_gemm_fp8_ex": (C.c_int, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _I32, _I32,
                                 _I64, _I64, _I64, _P]),
    "rg_gemm_fp8_plan": (C.c_int, [_P, _P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rg_sweep_fp8": (C.c_int, [_P, C.POINTER(rg_grid), _I32, _P, _P, _P, _P, _P, _P, _P, C.POINTER(rg_sweep_opts), _P,
                               _P, _P, _P]),
    "rg_landscape": (C.c_int, [C.POINTER(rg_grid), _I32, C.c_double, _I32, C.c_double, _I32, _P, _I32, _I32, _P]),
    "rg_kol": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, _P, _P]),
    "rg_gemm_noalloc": (C.c_int, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I32, _I32, _P]),
    "rg_noalloc_check": (C.c_int, [_P]),
    "rg_phase_trace": (C.c_int, [_P, _I32]),
    "rg_phase_trace_read": (C.c_int, [_P, _P, _I32, C.POINTER(_I32)]),
    "rg_plan_free": (None, [_P]),
    "rg_plan_grid": (C.c_int, [_P, C.POINTER(rg_grid)]),
    "rg_plan_tables": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "rg_plan_lookup": (C.c_int, [_P, _I64, _I64, _I64, C.POINTER(C.POINTER(rg_leaf)), C.POINTER(_I32),
                                 C.POINTER(_I64)]),
    "rg_gemm_plan": (C.c_int, [_P, _P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rg_gemm_plan_host": (C.c_int, [_P, _P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rg_plan_save": (C.c_int, [_P, _P, C.c_char_p]),
    "rg_plan_load": (C.c_int, [C.c_char_p, _P, C.POINTER(_P)]),
    "rg_surface_stats": (C.c_int, [C.POINTER(rg_grid), _P, _P, _P, _P]),
    "rg_variant_desc": (C.c_int, [_I32, _P]),
    "rg_streamk_geometry": (C.c_int, [_I64, _I64, _I64, _P]),
    "rg_sweep": (C.c_int, [_P, C.POINTER(rg_grid), _I32, _P, _P, _P, _P, _P, C.POINTER(rg_sweep_opts), _P, _P, _P,
                           _P]),
    "rg_gemm_memtwin": (C.c_int, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I32, _P]),
    "rg_sweep_memtwin": (C.c_int, [_P, C.POINTER(rg_grid), _I32, _P, _P, _P, _P, C.POINTER(rg_sweep_opts), _P,
                                   _P]),
    "rg_decompose": (C.c_int, [C.POINTER(rg_grid), _P, _P, C.c_double, _P, _P, _P]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

HEADER_SYMBOLS = tuple(_sigs)


def lib_path() -> str:
    return _LIB_PATH


def library():
    return _lib


def _check(code: int, where: str) -> int:
    if code != RG_OK:
        raise RGError(code, where, _lib.rg_last_error().decode() or _lib.rg_strerror(code).decode())
    return code


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError(f"not a stream: {type(s)}")


def make_grid(m, n=None, k=None) -> rg_grid:
    """Grid from (start, step, count) triples; n and k default to m."""
    n = n or m
    k = k or m
    return rg_grid(rg_axis(*m), rg_axis(*n), rg_axis(*k))


def grid_cells(g: rg_grid) -> int:
    return g.m.count * g.n.count * g.k.count


# ------------------------------------------------------------------ entry points

def rg_version() -> str:
    return _lib.rg_version().decode()


def rg_strerror(code: int) -> str:
    return _lib.rg_strerror(code).decode()


def rg_init(device: int = 0, workspace_bytes: int = 0) -> int:
    h = _P()
    _check(_lib.rg_init(device, workspace_bytes, C.byref(h)), "rg_init")
    return h.value


def rg_destroy(ctx: int) -> None:
    _lib.rg_destroy(ctx)


def rg_sm_count(ctx: int) -> int:
    v = _I32()
    _check(_lib.rg_sm_count(ctx, C.byref(v)), "rg_sm_count")
    return v.value


def rg_check(ctx: int, stream=None) -> None:
    _check(_lib.rg_check(ctx, _stream(stream)), "rg_check")


def rg_check_status(ctx: int, stream=None) -> int:
    return _lib.rg_check(ctx, _stream(stream))


def rg_set_timeout_cycles(ctx: int, cycles: int) -> None:
    _check(_lib.rg_set_timeout_cycles(ctx, cycles), "rg_set_timeout_cycles")


def rg_set_static_operands(ctx, enable: bool) -> None:
    """Declare that A and B are not written by earlier work on the stream (see include/rg.h)."""
    _check(_lib.rg_set_static_operands(ctx, 1 if enable else 0), "rg_set_static_operands")


def rg_gemm(ctx, M, N, K, A, lda, B, ldb, Cp, ldc, variant_id, beta=0, pm=0, pn=0, pk=0, stream=None) -> None:
    _check(_lib.rg_gemm(ctx, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, variant_id, beta, pm, pn, pk,
                        _stream(stream)), "rg_gemm")


def rg_gemm_status(ctx, M, N, K, A, lda, B, ldb, Cp, ldc, variant_id, beta=0, pm=0, pn=0, pk=0, stream=None) -> int:
    """rg_gemm returning the status code instead of raising (for error-path tests)."""
    return _lib.rg_gemm(ctx, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, variant_id, beta, pm, pn, pk,
                        _stream(stream))


RG_PLAN_PAD_ONLY = 1


def rg_plan_build(grid: rg_grid, T0_ns: np.ndarray, variant_ids) -> int:
    T0 = np.ascontiguousarray(T0_ns, dtype=np.int64).reshape(len(variant_ids), -1)
    vids = np.ascontiguousarray(variant_ids, dtype=np.int32)
    h = _P()
    _check(_lib.rg_plan_build(C.byref(grid), T0.ctypes.data, len(vids), vids.ctypes.data, C.byref(h)),
           "rg_plan_build")
    return h.value


def rg_plan_build_ex(grid: rg_grid, T0_ns: np.ndarray, variant_ids, flags: int) -> int:
    T0 = np.ascontiguousarray(T0_ns, dtype=np.int64).reshape(len(variant_ids), -1)
    vids = np.ascontiguousarray(variant_ids, dtype=np.int32)
    h = _P()
    _check(_lib.rg_plan_build_ex(C.byref(grid), T0.ctypes.data, len(vids), vids.ctypes.data, flags, C.byref(h)),
           "rg_plan_build_ex")
    return h.value


def rg_set_test_stall(ctx: int, enable: bool) -> None:
    _check(_lib.rg_set_test_stall(ctx, 1 if enable else 0), "rg_set_test_stall")


def rg_launch_count(ctx: int) -> int:
    v = _I64()
    _check(_lib.rg_launch_count(ctx, C.byref(v)), "rg_launch_count")
    return v.value


def rg_plan_free(plan: int) -> None:
    _lib.rg_plan_free(plan)


def rg_plan_grid(plan: int) -> rg_grid:
    g = rg_grid()
    _check(_lib.rg_plan_grid(plan, C.byref(g)), "rg_plan_grid")
    return g


def rg_plan_tables(plan: int) -> dict:
    g = rg_plan_grid(plan)
    n = grid_cells(g)
    t = {"T0s": np.zeros(n, np.int64), "vstar": np.zeros(n, np.int32), "T1": np.zeros(n, np.int64),
         "target": np.zeros(3 * n, np.int32), "T2": np.zeros(n, np.int64), "action": np.zeros(n, np.int32),
         "q": np.zeros(n, np.int32)}
    _check(_lib.rg_plan_tables(plan, t["T0s"].ctypes.data, t["vstar"].ctypes.data, t["T1"].ctypes.data,
                               t["target"].ctypes.data, t["T2"].ctypes.data, t["action"].ctypes.data,
                               t["q"].ctypes.data), "rg_plan_tables")
    shape = (g.m.count, g.n.count, g.k.count)
    out = {k: v.reshape(shape) for k, v in t.items() if k != "target"}
    out["target"] = t["target"].reshape(shape + (3,))
    return out


def rg_plan_lookup(plan: int, M: int, N: int, K: int):
    """(list of leaf tuples (variant, beta, phase, m0, n0, k0, m, n, k, pm, pn, pk), T2 ns)."""
    lp = C.POINTER(rg_leaf)()
    n = _I32()
    t2 = _I64()
    _check(_lib.rg_plan_lookup(plan, M, N, K, C.byref(lp), C.byref(n), C.byref(t2)), "rg_plan_lookup")
    leaves = []
    for i in range(n.value):
        L = lp[i]
        leaves.append((L.variant, L.beta, L.phase, L.m0, L.n0, L.k0, L.m, L.n, L.k, L.pm, L.pn, L.pk))
    return leaves, t2.value


def rg_gemm_plan(ctx, plan, M, N, K, A, lda, B, ldb, Cp, ldc, stream=None) -> None:
    _check(_lib.rg_gemm_plan(ctx, plan, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, _stream(stream)),
           "rg_gemm_plan")


def rg_gemm_plan_host(ctx, plan, M, N, K, A, lda, B, ldb, Cp, ldc, stream=None) -> None:
    """Plan GEMM on host buffers (numpy arrays, pinned tensors or raw host addresses): copies in,
    executes, copies out and synchronises inside the library."""
    _check(_lib.rg_gemm_plan_host(ctx, plan, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, _stream(stream)),
           "rg_gemm_plan_host")


def rg_plan_save(plan: int, path: str, ctx: int | None = None) -> None:
    _check(_lib.rg_plan_save(plan, ctx, path.encode()), "rg_plan_save")


def rg_plan_load(path: str, ctx: int | None = None) -> int:
    h = _P()
    _check(_lib.rg_plan_load(path.encode(), ctx, C.byref(h)), "rg_plan_load")
    return h.value


def rg_plan_load_status(path: str, ctx: int | None = None) -> int:
    h = _P()
    code = _lib.rg_plan_load(path.encode(), ctx, C.byref(h))
    if code == RG_OK:
        _lib.rg_plan_free(h.value)
    return code


def rg_variant_desc(v: int) -> dict:
    """The library's description of BF16 variant v (host)."""
    out = np.zeros(6, np.int32)
    _check(_lib.rg_variant_desc(v, out.ctypes.data), "rg_variant_desc")
    return dict(zip(("tile", "split", "streamk", "two_sm", "bm", "bn"), (int(x) for x in out)))


def rg_streamk_geometry(tiles: int, kblocks: int, units: int) -> dict:
    """The stream-K schedule the library launches for `tiles` tiles of `kblocks` K blocks on `units` CTAs."""
    out = np.zeros(4, np.int64)
    _check(_lib.rg_streamk_geometry(tiles, kblocks, units, out.ctypes.data), "rg_streamk_geometry")
    return dict(zip(("grid", "dp_tiles", "tail_ctas", "max_pieces"), (int(x) for x in out)))


def rg_surface_stats(grid: rg_grid, t_ns: np.ndarray):
    """(tflops surface [cells], {R_M, R_N, R_K, R_3D, R_N_slice}, mean TFLOP/s)."""
    t = np.ascontiguousarray(t_ns, dtype=np.int64).ravel()
    tf = np.zeros(t.size, np.float64)
    r = np.zeros(5, np.float64)
    mean = C.c_double()
    _check(_lib.rg_surface_stats(C.byref(grid), t.ctypes.data, tf.ctypes.data, r.ctypes.data, C.byref(mean)),
           "rg_surface_stats")
    keys = ("R_M", "R_N", "R_K", "R_3D", "R_N_slice")
    return tf, dict(zip(keys, (float(x) for x in r))), mean.value


def rg_sweep_opts_default() -> rg_sweep_opts:
    o = rg_sweep_opts()
    _lib.rg_sweep_opts_default(C.byref(o))
    return o


def rg_sweep(ctx, grid: rg_grid, variant_ids, A, B, Cp, opts: rg_sweep_opts | None = None, plan: int | None = None,
             stream=None) -> np.ndarray:
    """t_ns[len(variant_ids)][cells] (or [1][cells] for a plan sweep)."""
    return rg_sweep_surfaces(ctx, grid, variant_ids, A, B, Cp, opts, plan, stream)[0]


SWEEP_STATS = ("R_M", "R_N", "R_K", "R_3D", "R_N_slice", "mean_tflops")


def rg_sweep_surfaces(ctx, grid: rg_grid, variant_ids, A, B, Cp, opts: rg_sweep_opts | None = None,
                      plan: int | None = None, stream=None):
    """(t_ns[rows][cells], tflops[rows][cells], stats[rows][6]) from one rg_sweep call; the stats
    columns are SWEEP_STATS (NaN for a row the pruning left incomplete)."""
    vids = np.ascontiguousarray(variant_ids if plan is None else [0], dtype=np.int32)
    out = np.zeros((len(vids), grid_cells(grid)), np.int64)
    tf = np.zeros((len(vids), grid_cells(grid)), np.float64)
    st = np.zeros((len(vids), 6), np.float64)
    o = opts or rg_sweep_opts_default()
    _check(_lib.rg_sweep(ctx, C.byref(grid), len(vids), vids.ctypes.data, plan, _ptr(A), _ptr(B), _ptr(Cp),
                         C.byref(o), out.ctypes.data, tf.ctypes.data, st.ctypes.data, _stream(stream)), "rg_sweep")
    return out, tf, st


def rg_gemm_memtwin(ctx, M, N, K, A, lda, B, ldb, Cp, ldc, tile, stream=None) -> None:
    """One launch of a tile's memory twin (loads and stores, no MMA; C gets undefined values)."""
    _check(_lib.rg_gemm_memtwin(ctx, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, tile, _stream(stream)),
           "rg_gemm_memtwin")


def rg_sweep_memtwin(ctx, grid: rg_grid, tile_ids, A, B, Cp, opts: rg_sweep_opts | None = None,
                     stream=None) -> np.ndarray:
    """t_ns[len(tile_ids)][cells] of the tiles' memory twins under the sweep protocol."""
    tids = np.ascontiguousarray(tile_ids, dtype=np.int32)
    out = np.zeros((len(tids), grid_cells(grid)), np.int64)
    o = opts or rg_sweep_opts_default()
    _check(_lib.rg_sweep_memtwin(ctx, C.byref(grid), len(tids), tids.ctypes.data, _ptr(A), _ptr(B), _ptr(Cp),
                                 C.byref(o), out.ctypes.data, _stream(stream)), "rg_sweep_memtwin")
    return out


def rg_decompose(grid: rg_grid, t_gemm_ns, t_mem_ns, p_tflops: float):
    """(compute_ns[cells], overhead_ns[cells], stats[4]) of the four-surface decomposition."""
    tg = np.ascontiguousarray(t_gemm_ns, dtype=np.int64).reshape(-1)
    tm = np.ascontiguousarray(t_mem_ns, dtype=np.int64).reshape(-1)
    n = grid_cells(grid)
    if tg.size != n or tm.size != n:
        raise ValueError("time surfaces must have one entry per grid cell")
    comp = np.zeros(n, np.float64)
    over = np.zeros(n, np.float64)
    st = np.zeros(4, np.float64)
    _check(_lib.rg_decompose(C.byref(grid), tg.ctypes.data, tm.ctypes.data, p_tflops, comp.ctypes.data,
                             over.ctypes.data, st.ctypes.data), "rg_decompose")
    return comp, over, st


def rg_group_create(ctx: int, tile: int, max_items: int, workspace_bytes: int = 64 << 20) -> int:
    h = _P()
    _check(_lib.rg_group_create(ctx, tile, max_items, workspace_bytes, C.byref(h)), "rg_group_create")
    return h.value


def rg_group_destroy(group: int) -> None:
    _lib.rg_group_destroy(group)


def group_problems(items) -> "C.Array":
    """items: iterables (M, N, K, A, lda, B, ldb, C, ldc[, beta[, pm, pn, pk[, variant]]]) with pointers or
    tensors; variant -1 (the default) runs the group's tile with split 1."""
    arr = (rg_group_problem * max(1, len(items)))()
    for i, it in enumerate(items):
        M, N, K, A, lda, B, ldb, Cp, ldc = it[:9]
        beta = it[9] if len(it) > 9 else 0
        pm, pn, pk = it[10:13] if len(it) > 12 else (0, 0, 0)
        v = it[13] if len(it) > 13 else -1
        arr[i] = rg_group_problem(M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, pm, pn, pk, beta, v)
    return arr


def rg_gemm_grouped(group: int, problems, n: int | None = None, stream=None) -> None:
    arr = problems if isinstance(problems, C.Array) else group_problems(problems)
    count = len(problems) if n is None else n
    _check(_lib.rg_gemm_grouped(group, arr, count, _stream(stream)), "rg_gemm_grouped")


def rg_serve_opts_default() -> rg_serve_opts:
    o = rg_serve_opts()
    _lib.rg_serve_opts_default(C.byref(o))
    return o


def rg_serve(ctx, plan, opts: rg_serve_opts, requests):
    """requests: iterables (M, N, K, A, lda, B, ldb, C or None, ldc, arrival_ns[, (sA, lds_a, sB, lds_b)])
    -- the optional last item makes an FP8 request.  Returns (list of result dicts, stats dict)."""
    n = len(requests)
    arr = (rg_serve_request * max(1, n))()
    for i, r in enumerate(requests):
        arr[i] = serve_request(*r[:10], fp8=r[10] if len(r) > 10 else None)
    res = (rg_serve_result * max(1, n))()
    st = rg_serve_stats()
    _check(_lib.rg_serve(ctx, plan, C.byref(opts), arr, n, res, C.byref(st)), "rg_serve")
    results = [{"admitted_ns": r.admitted_ns, "launched_ns": r.launched_ns, "done_ns": r.done_ns,
                "batch": r.batch, "status": r.status} for r in res[:n]]
    stats = {k: getattr(st, k) for k, _ in rg_serve_stats._fields_}
    return results, stats


def _result_dict(r) -> dict:
    return {"admitted_ns": r.admitted_ns, "launched_ns": r.launched_ns, "done_ns": r.done_ns,
            "batch": r.batch, "status": r.status}


def rg_serve_start(ctx, plan, opts: rg_serve_opts) -> int:
    """Start an online server (a worker thread running the serving engine); returns its handle."""
    h = _P()
    _check(_lib.rg_serve_start(ctx, plan, C.byref(opts), C.byref(h)), "rg_serve_start")
    return h.value


def rg_serve_submit(server, M, N, K, A, lda, B, ldb, Cp, ldc, fp8=None) -> int:
    """Submit one request (fp8 = (sA, lds_a, sB, lds_b) for an FP8 one); returns its id."""
    req = serve_request(M, N, K, A, lda, B, ldb, Cp, ldc, 0, fp8)
    i = _I64()
    _check(_lib.rg_serve_submit(server, C.byref(req), C.byref(i)), "rg_serve_submit")
    return i.value


def rg_serve_poll(server, rid: int):
    """None while the request runs, else its result dict."""
    r = rg_serve_result()
    d = _I32()
    _check(_lib.rg_serve_poll(server, rid, C.byref(r), C.byref(d)), "rg_serve_poll")
    return _result_dict(r) if d.value else None


def rg_serve_wait(server, rid: int) -> dict:
    r = rg_serve_result()
    _check(_lib.rg_serve_wait(server, rid, C.byref(r)), "rg_serve_wait")
    return _result_dict(r)


def rg_serve_stop(server) -> dict:
    st = rg_serve_stats()
    _check(_lib.rg_serve_stop(server, C.byref(st)), "rg_serve_stop")
    return {k: getattr(st, k) for k, _ in rg_serve_stats._fields_}


def rg_fp8_quantize(ctx, X, rows, cols, ldx, Q, ldq, scales, stream=None) -> None:
    _check(_lib.rg_fp8_quantize(ctx, _ptr(X), rows, cols, ldx, _ptr(Q), ldq, _ptr(scales), _stream(stream)),
           "rg_fp8_quantize")


def rg_gemm_fp8(ctx, M, N, K, qA, lda, sA, qB, ldb, sB, Cp, ldc, stream=None) -> None:
    _check(_lib.rg_gemm_fp8(ctx, M, N, K, _ptr(qA), lda, _ptr(sA), _ptr(qB), ldb, _ptr(sB), _ptr(Cp), ldc,
                            _stream(stream)), "rg_gemm_fp8")


RG_FP8_VARIANT_BASE = 64
RG_FP8_NUM_TILES = 3
RG_FP8_NUM_VARIANTS = RG_FP8_NUM_TILES * RG_NUM_SPLITS
FP8_TILES = [(128, 256), (128, 128), (256, 256)]
FP8_PAIR_TILE = 2                    # the 256x256 tile runs as a cta_group::2 pair


def fp8_variant(tile: int, split: int = 1) -> int:
    """FP8 variant id: tile 0 = 128x256, 1 = 128x128, 2 = 256x256 cta_group::2 pair; split-K 1/2/4/8."""
    return RG_FP8_VARIANT_BASE + tile * RG_NUM_SPLITS + SPLITS.index(split)


def fp8_variant_name(v: int) -> str:
    t, s = divmod(v - RG_FP8_VARIANT_BASE, RG_NUM_SPLITS)
    bm, bn = FP8_TILES[t]
    pair = "/2SM" if t == FP8_PAIR_TILE else ""
    return f"fp8 {bm}x{bn}{pair}/S{SPLITS[s]}"


def rg_gemm_fp8_ex(ctx, M, N, K, qA, lda, sA, lds_a, qB, ldb, sB, lds_b, Cp, ldc, variant_id, beta=0, pm=0, pn=0,
                   pk=0, stream=None) -> None:
    _check(_lib.rg_gemm_fp8_ex(ctx, M, N, K, _ptr(qA), lda, _ptr(sA), lds_a, _ptr(qB), ldb, _ptr(sB), lds_b,
                               _ptr(Cp), ldc, variant_id, beta, pm, pn, pk, _stream(stream)), "rg_gemm_fp8_ex")


def rg_gemm_fp8_plan(ctx, plan, M, N, K, qA, lda, sA, lds_a, qB, ldb, sB, lds_b, Cp, ldc, stream=None) -> None:
    _check(_lib.rg_gemm_fp8_plan(ctx, plan, M, N, K, _ptr(qA), lda, _ptr(sA), lds_a, _ptr(qB), ldb, _ptr(sB), lds_b,
                                 _ptr(Cp), ldc, _stream(stream)), "rg_gemm_fp8_plan")


def rg_sweep_fp8_surfaces(ctx, grid: rg_grid, variant_ids, qA, sA, qB, sB, Cp, opts: rg_sweep_opts | None = None,
                          plan: int | None = None, stream=None):
    """(t_ns[rows][cells], tflops[rows][cells], stats[rows][6]) of an FP8 sweep (variants or a plan)."""
    vids = np.ascontiguousarray(variant_ids if plan is None else [0], dtype=np.int32)
    out = np.zeros((len(vids), grid_cells(grid)), np.int64)
    tf = np.zeros((len(vids), grid_cells(grid)), np.float64)
    st = np.zeros((len(vids), 6), np.float64)
    o = opts or rg_sweep_opts_default()
    _check(_lib.rg_sweep_fp8(ctx, C.byref(grid), len(vids), vids.ctypes.data, plan, _ptr(qA), _ptr(sA), _ptr(qB),
                             _ptr(sB), _ptr(Cp), C.byref(o), out.ctypes.data, tf.ctypes.data, st.ctypes.data,
                             _stream(stream)), "rg_sweep_fp8")
    return out, tf, st


def rg_sweep_fp8(ctx, grid: rg_grid, qA, sA, qB, sB, Cp, opts: rg_sweep_opts | None = None, stream=None,
                 variant_ids=None, plan: int | None = None) -> np.ndarray:
    """t_ns[cells] of the default FP8 variant (or t_ns[rows][cells] when variant_ids or a plan is given)."""
    vids = [fp8_variant(0, 1)] if variant_ids is None else variant_ids
    t = rg_sweep_fp8_surfaces(ctx, grid, vids, qA, sA, qB, sB, Cp, opts, plan, stream)[0]
    return t[0] if variant_ids is None and plan is None else t


RG_LANDSCAPE_IDEAL = 0
RG_LANDSCAPE_OPTIMAL = 1


def rg_landscape(grid: rg_grid, mode: int, p_tflops: float, c_units: int, bw_gbs: float, tiles,
                 channels: int = 0, interleave: int = 256) -> np.ndarray:
    """First-principles TFLOP/s surface [cells] (RG_LANDSCAPE_IDEAL or RG_LANDSCAPE_OPTIMAL)."""
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(grid_cells(grid), np.float64)
    _check(_lib.rg_landscape(C.byref(grid), mode, p_tflops, c_units, bw_gbs, len(t), t.ctypes.data, channels,
                             interleave, out.ctypes.data), "rg_landscape")
    return out


def rg_kol(mean_a: float, mean_o: float, r_a: float, r_o: float) -> dict:
    o = np.zeros(2, np.float64)
    b = np.zeros(3, np.int32)
    _check(_lib.rg_kol(mean_a, mean_o, r_a, r_o, o.ctypes.data, b.ctypes.data), "rg_kol")
    return {"tau": float(o[0]), "rho": float(o[1]), "T": int(b[0]), "S": int(b[1]), "L": int(b[2])}


RG_NOALLOC_PARTIAL_BYTES = 16 << 20
RG_NOALLOC_MAX_TILES = 4096


def rg_gemm_noalloc(M, N, K, A, lda, B, ldb, Cp, ldc, variant_id, beta=0, stream=None) -> int:
    """GEMM that allocates no device memory (scratch in a fixed array inside the
    library); returns the status code.  See include/rg.h for its limits."""
    return _lib.rg_gemm_noalloc(M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(Cp), ldc, variant_id, beta,
                                _stream(stream))


def rg_noalloc_check(stream=None) -> int:
    """Status of the rg_gemm_noalloc work enqueued so far on the current device (synchronises the
    stream): RG_OK, or RG_ERR_TIMEOUT if a bounded wait expired (the scratch is then cleared)."""
    return _lib.rg_noalloc_check(_stream(stream))


RG_TRACE_FIELDS = 12
TRACE_FIELDS = ("gt_entry_ns", "gt_exit_ns", "exit", "dep_wait", "first_stage", "last_mma_commit",
                "first_acc_ready", "epilogue_done", "fixup_start", "fixup_end", "units", "reserved")


def rg_phase_trace(ctx, enable: bool) -> None:
    """Enable the per-CTA phase stamps of a phase-timer build (RG_PHASE_TIMERS=1)."""
    _check(_lib.rg_phase_trace(ctx, 1 if enable else 0), "rg_phase_trace")


def rg_phase_trace_read(ctx, max_ctas: int = 1024) -> np.ndarray:
    """uint64[n_ctas][RG_TRACE_FIELDS] stamps of the last traced launch (see include/rg.h)."""
    out = np.zeros((max_ctas, RG_TRACE_FIELDS), np.uint64)
    n = _I32()
    _check(_lib.rg_phase_trace_read(ctx, out.ctypes.data, max_ctas, C.byref(n)), "rg_phase_trace_read")
    return out[:n.value]
