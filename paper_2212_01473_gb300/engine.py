"""ctypes binding of the engine's C ABI (include/mce.h), same names as the C calls.

Argument marshalling only: every step of the enumeration runs in the CUDA
library libmce.so. PyTorch supplies device memory (through the caching
allocator, passed to the library as its allocator) and the CUDA stream.
There is no CPU fallback: if the library is missing, the calls raise.
"""
import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmce.so")

MCE_OK, MCE_EINVAL, MCE_ENOMEM, MCE_ECUDA, MCE_ETIMEOUT, MCE_ERANGE, MCE_EUNSUPPORTED, MCE_EBUDGET = range(8)
MCE_FLAG_DEVICE_PTRS = 1
MCE_PIVOT_AUTO, MCE_PIVOT_IP, MCE_PIVOT_IPX = 0, 1, 2
MCE_ORDER_PLAIN, MCE_ORDER_PRIORITY = 0, 1
MCE_DONATE_PAPER, MCE_DONATE_EITHER, MCE_DONATE_ANY = 0, 1, 2
MCE_MAX_DEGENERACY = 4096

_NAMES = {MCE_EINVAL: "MCE_EINVAL", MCE_ENOMEM: "MCE_ENOMEM", MCE_ECUDA: "MCE_ECUDA",
          MCE_ETIMEOUT: "MCE_ETIMEOUT", MCE_ERANGE: "MCE_ERANGE", MCE_EUNSUPPORTED: "MCE_EUNSUPPORTED",
          MCE_EBUDGET: "MCE_EBUDGET"}


class MCEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_NAMES.get(code, str(code)), msg))
        self.code = code


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class mce_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class mce_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("pivot", ctypes.c_int32), ("order", ctypes.c_int32),
                ("worker_list", ctypes.c_int32), ("donate_min_p", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("donate_policy", ctypes.c_int32), ("stats", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int64), ("root_count", ctypes.c_void_p),
                ("root_hash", ctypes.c_void_p), ("root_nodes", ctypes.c_void_p),
                ("root_priority", ctypes.c_void_p), ("roots", ctypes.c_void_p),
                ("n_roots", ctypes.c_int64), ("tuned", ctypes.c_int32), ("subtree_level", ctypes.c_int32),
                ("run_budget_ms", ctypes.c_int64), ("merge_wp", ctypes.c_int32), ("block_warps", ctypes.c_int32)]


class mce_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("hash", ctypes.c_uint64), ("max_size", ctypes.c_int32),
                ("degeneracy", ctypes.c_int32), ("tree_nodes", ctypes.c_uint64),
                ("donations", ctypes.c_uint64), ("ms_prep", ctypes.c_double),
                ("ms_traverse", ctypes.c_double)]


class mce_stats(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("class_wp", ctypes.c_int32 * 16), ("class_roots", ctypes.c_int32 * 16),
                ("class_rows", ctypes.c_int32 * 16), ("class_blocks", ctypes.c_int32 * 16),
                ("class_groups", ctypes.c_int32 * 16), ("class_group_warps", ctypes.c_int32 * 16),
                ("class_ms", ctypes.c_double * 16), ("kernel_launches", ctypes.c_uint64),
                ("peel_rounds", ctypes.c_int64), ("phase_cycles", ctypes.c_uint64 * 9),
                ("phase_counts", ctypes.c_uint64 * 9), ("class_wp_min", ctypes.c_int32 * 16),
                ("peel_stage_ms", ctypes.c_double * 3), ("peel_stage_rounds", ctypes.c_int32 * 3),
                ("peel_cluster", ctypes.c_int32)]


PHASES = ["setup", "pivot", "branch", "leaf", "partition", "donate", "idle", "backtrack", "compact_entry"]

_lib = None


def library():
    """Load libmce.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmce.so is not built (run paper_2212_01473_gb300/build.py); "
                              "the engine has no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        i32p, u64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64)
        lib.mce_default_opts.argtypes = [ctypes.POINTER(mce_opts)]
        lib.mce_default_opts.restype = None
        lib.mce_create.argtypes = [vp, vp, i32, i64, u32, ctypes.POINTER(mce_allocator), vp,
                                   ctypes.POINTER(vp)]
        lib.mce_batch_create.argtypes = [vp, i32, vp, vp, i32, i64, u32,
                                         ctypes.POINTER(mce_allocator), vp, ctypes.POINTER(vp)]
        lib.mce_run.argtypes = [vp, ctypes.POINTER(mce_opts), ctypes.POINTER(mce_result), u64p, i32]
        lib.mce_run_batch.argtypes = [vp, ctypes.POINTER(mce_opts), ctypes.POINTER(mce_result), u64p, i32,
                                      ctypes.POINTER(mce_result)]
        lib.mce_graph_info.argtypes = [vp, i32p, ctypes.POINTER(ctypes.c_int64), i32p, i32p, i32p]
        lib.mce_get_order.argtypes = [vp, i32p, i32p, i32p]
        lib.mce_get_stats.argtypes = [vp, ctypes.POINTER(mce_stats)]
        lib.mce_autotune.argtypes = [vp, ctypes.POINTER(mce_opts), ctypes.c_double]
        lib.mce_get_tuning.argtypes = [vp, i32p, i32p, i32p, i32p, i32p]
        lib.mce_prepare.argtypes = [vp, ctypes.POINTER(mce_opts)]
        lib.mce_run_prepared.argtypes = [vp, ctypes.POINTER(mce_result), u64p, i32, ctypes.POINTER(mce_result)]
        lib.mce_peel_noalloc.argtypes = [vp, vp, i32, i64, vp, vp, vp, vp]
        lib.mce_selftest_waits.argtypes = [i32, i64, vp]
        dp = ctypes.POINTER(ctypes.c_double)
        lib.mce_microbench.argtypes = [i32, dp, dp, dp, vp]
        f32p = ctypes.POINTER(ctypes.c_float)
        lib.mce_root_features.argtypes = [vp, vp, vp]
        lib.mce_model_create.argtypes = [f32p, ctypes.POINTER(mce_allocator), vp, ctypes.POINTER(vp)]
        lib.mce_model_get_params.argtypes = [vp, f32p]
        lib.mce_model_predict.argtypes = [vp, vp, i64, vp]
        lib.mce_model_gradient.argtypes = [vp, vp, vp, i32, f32p, f32p]
        lib.mce_model_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, f32p]
        lib.mce_predict_priority.argtypes = [vp, vp, i32, vp]
        lib.mce_run_list.argtypes = [vp, ctypes.POINTER(mce_opts), vp, i64, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(mce_result)]
        lib.mce_model_destroy.argtypes = [vp]
        lib.mce_model_destroy.restype = None
        lib.mce_destroy.argtypes = [vp]
        lib.mce_destroy.restype = None
        lib.mce_last_error.argtypes = []
        lib.mce_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != MCE_OK:
        raise MCEError(rc, library().mce_last_error().decode(errors="replace"))


# ------------------------------------------------------------ torch plumbing

class _TorchAllocator:
    """Routes the library's device allocations to the PyTorch caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, ctx):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None

        def _free(ptr, ctx):
            if ptr:
                self._torch.cuda.caching_allocator_delete(int(ptr))

        self.c_alloc = ALLOC_FN(_alloc)
        self.c_free = FREE_FN(_free)
        self.struct = mce_allocator(self.c_alloc, self.c_free, None)


def _as_int32_buffer(a):
    """(pointer, keepalive, is_device) for a numpy array or torch tensor of int32."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.int32:
                a = a.to(torch.int32)
            a = a.contiguous()
            return ctypes.c_void_p(a.data_ptr()), a, a.is_cuda
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.int32)
    return ctypes.c_void_p(arr.ctypes.data), arr, False


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream, torch.cuda.current_device()


@dataclass
class Result:
    count: int
    hash: int
    max_size: int
    degeneracy: int
    tree_nodes: int
    donations: int
    ms_prep: float
    ms_traverse: float
    hist: Optional[np.ndarray] = None


def _result(r: mce_result, hist=None) -> Result:
    return Result(int(r.count), int(r.hash), int(r.max_size), int(r.degeneracy), int(r.tree_nodes),
                  int(r.donations), float(r.ms_prep), float(r.ms_traverse), hist)


class Handle:
    """Owns an mce_graph* and the allocator callbacks it uses."""

    def __init__(self, ptr: ctypes.c_void_p, allocator, n: int, G: int):
        self.ptr = ptr
        self._allocator = allocator
        self.n = n
        self.G = G

    def __del__(self):
        try:
            mce_destroy(self)
        except Exception:
            pass


def mce_default_opts(**kw) -> mce_opts:
    o = mce_opts()
    library().mce_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError("mce_opts has no field %r" % k)
        setattr(o, k, v)
    return o


def _create(graph_ptr, row_ptr, col, stream, use_torch_allocator):
    lib = library()
    rp, rp_keep, rp_dev = _as_int32_buffer(row_ptr)
    cp, cp_keep, cp_dev = _as_int32_buffer(col if len(col) else np.zeros(1, np.int32))
    n = int(len(rp_keep)) - 1
    m = int(len(col)) // 2
    flags = MCE_FLAG_DEVICE_PTRS if rp_dev else 0
    if rp_dev != cp_dev:
        raise ValueError("row_ptr and col must both be host or both be device buffers")
    s, dev = (stream, None) if stream is not None else _current_stream()
    if dev is None:
        import torch
        dev = torch.cuda.current_device()
    alloc = _TorchAllocator(dev, s) if use_torch_allocator else None
    out = ctypes.c_void_p()
    if graph_ptr is None:
        rc = lib.mce_create(rp, cp, n, m, flags, ctypes.byref(alloc.struct) if alloc else None,
                            ctypes.c_void_p(s), ctypes.byref(out))
        G = 1
    else:
        gp, gp_keep, gp_dev = _as_int32_buffer(graph_ptr)
        if gp_dev != rp_dev:
            raise ValueError("graph_ptr must live where row_ptr lives")
        G = int(len(gp_keep)) - 1
        rc = lib.mce_batch_create(gp, G, rp, cp, n, m, flags,
                                  ctypes.byref(alloc.struct) if alloc else None, ctypes.c_void_p(s),
                                  ctypes.byref(out))
    _check(rc)
    return Handle(out, alloc, n, G)


def mce_create(row_ptr, col, stream: Optional[int] = None, use_torch_allocator: bool = True) -> Handle:
    """Build a handle from a canonical CSR (numpy / CPU tensor = host, CUDA tensor = device)."""
    return _create(None, row_ptr, col, stream, use_torch_allocator)


def mce_batch_create(graph_ptr, row_ptr, col, stream: Optional[int] = None,
                     use_torch_allocator: bool = True) -> Handle:
    return _create(graph_ptr, row_ptr, col, stream, use_torch_allocator)


def mce_run(h: Handle, opts: Optional[mce_opts] = None, hist_len: Optional[int] = None) -> Result:
    lib = library()
    if hist_len is None:
        d = mce_graph_info(h)["degeneracy"]
        hist_len = d + 2
    hist = np.zeros(max(hist_len, 1), np.uint64)
    r = mce_result()
    _check(lib.mce_run(h.ptr, ctypes.byref(opts) if opts is not None else None, ctypes.byref(r),
                       hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), hist_len))
    return _result(r, hist[: r.max_size + 1].copy())


def mce_run_batch(h: Handle, opts: Optional[mce_opts] = None, hist_len: Optional[int] = None):
    """(per-graph results, hist [G, hist_len], total)."""
    lib = library()
    if hist_len is None:
        hist_len = mce_graph_info(h)["degeneracy"] + 2
    per = (mce_result * h.G)()
    hist = np.zeros((h.G, max(hist_len, 1)), np.uint64)
    tot = mce_result()
    _check(lib.mce_run_batch(h.ptr, ctypes.byref(opts) if opts is not None else None, per,
                             hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), hist_len,
                             ctypes.byref(tot)))
    return [_result(per[i]) for i in range(h.G)], hist, _result(tot)


def mce_autotune(h: Handle, opts: Optional[mce_opts] = None, budget_ms: float = 5000.0) -> dict:
    """Pick launch settings per width class (see include/mce.h); returns them."""
    _check(library().mce_autotune(h.ptr, ctypes.byref(opts) if opts is not None else None, budget_ms))
    d, p, b, w = ((ctypes.c_int32 * 9)() for _ in range(4))
    mw = ctypes.c_int32()
    _check(library().mce_get_tuning(h.ptr, d, p, b, w, ctypes.byref(mw)))
    return {"donate_min_p": list(d), "donate_policy": list(p), "blocks": list(b), "warps": list(w),
            "merge_wp": mw.value}


def mce_prepare(h: Handle, opts: Optional[mce_opts] = None):
    """Capture one run into a CUDA graph kept by the handle."""
    h._prepared_opts = opts  # the opts' device buffers must outlive the capture
    _check(library().mce_prepare(h.ptr, ctypes.byref(opts) if opts is not None else None))


def mce_run_prepared(h: Handle, hist_len: Optional[int] = None):
    """Replay the captured run: (per-graph results, hist [G, hist_len], total)."""
    if hist_len is None:
        hist_len = mce_graph_info(h)["degeneracy"] + 2
    per = (mce_result * h.G)()
    hist = np.zeros((h.G, max(hist_len, 1)), np.uint64)
    tot = mce_result()
    _check(library().mce_run_prepared(h.ptr, per, hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      hist_len, ctypes.byref(tot)))
    return [_result(per[i]) for i in range(h.G)], hist, _result(tot)


def mce_graph_info(h: Handle) -> dict:
    n, G, d, md = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    m = ctypes.c_int64()
    _check(library().mce_graph_info(h.ptr, ctypes.byref(n), ctypes.byref(m), ctypes.byref(G),
                                    ctypes.byref(d), ctypes.byref(md)))
    return {"n": n.value, "m": m.value, "G": G.value, "degeneracy": d.value, "max_degree": md.value}


def mce_get_order(h: Handle):
    """(core, rank, out_degree) numpy int32 arrays indexed by input vertex id."""
    n = h.n
    core = np.zeros(max(n, 1), np.int32)
    rank = np.zeros(max(n, 1), np.int32)
    outd = np.zeros(max(n, 1), np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    _check(library().mce_get_order(h.ptr, core.ctypes.data_as(P), rank.ctypes.data_as(P),
                                   outd.ctypes.data_as(P)))
    return core[:n], rank[:n], outd[:n]


def mce_get_stats(h: Handle) -> dict:
    """Launch facts (per width class) and optional phase counters of the last run."""
    st = mce_stats()
    st.struct_size = ctypes.sizeof(mce_stats)
    _check(library().mce_get_stats(h.ptr, ctypes.byref(st)))
    k = st.n_classes
    return {
        "classes": [{"wp": st.class_wp[i], "wp_min": st.class_wp_min[i], "roots": st.class_roots[i], "rows": st.class_rows[i],
                     "blocks": st.class_blocks[i], "groups": st.class_groups[i],
                     "group_warps": st.class_group_warps[i], "ms": st.class_ms[i]} for i in range(k)],
        "kernel_launches": int(st.kernel_launches),
        "peel_rounds": int(st.peel_rounds),
        "peel_stage_ms": [float(x) for x in st.peel_stage_ms],
        "peel_stage_rounds": [int(x) for x in st.peel_stage_rounds],
        "peel_cluster": int(st.peel_cluster),
        "phase_cycles": {PHASES[i]: int(st.phase_cycles[i]) for i in range(len(PHASES))},
        "phase_counts": {PHASES[i]: int(st.phase_counts[i]) for i in range(len(PHASES))},
    }


def mce_peel_noalloc(row_ptr, col, core, rank, order, stream: Optional[int] = None):
    """Degeneracy peel into caller-owned CUDA int32 tensors, allocating nothing
    (see include/mce.h): core and rank by input id, order[r] = vertex of rank r."""
    import torch
    for t in (row_ptr, col, core, rank, order):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise TypeError("mce_peel_noalloc takes contiguous CUDA int32 tensors")
    n = row_ptr.numel() - 1
    if min(core.numel(), rank.numel(), order.numel()) < n:
        raise ValueError("output tensors shorter than n")
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(library().mce_peel_noalloc(ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                      n, col.numel() // 2, ctypes.c_void_p(core.data_ptr()),
                                      ctypes.c_void_p(rank.data_ptr()), ctypes.c_void_p(order.data_ptr()),
                                      ctypes.c_void_p(s)))


MCE_NUM_FEATURES = 16
MCE_MODEL_PARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 + 16 + 16


def mce_selftest_waits(which: int, timeout_ms: int = 100, stream: Optional[int] = None) -> int:
    """Run one of the engine's device-side waits on its own (include/mce.h):
    returns the MCE_* status it ends with (MCE_ETIMEOUT for which 0 and 1,
    MCE_OK for which 2) instead of raising."""
    s = _current_stream()[0] if stream is None else stream
    return int(library().mce_selftest_waits(int(which), int(timeout_ms), ctypes.c_void_p(s)))


def mce_microbench(which: int, stream: Optional[int] = None) -> dict:
    """One of the roofline microbenchmarks (include/mce.h): 0 word-ops/s,
    1 LOP3 ops/s, 2 L2 read bytes/s; with the SM clock seen meanwhile."""
    s = _current_stream()[0] if stream is None else stream
    rate, mhz, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(library().mce_microbench(int(which), ctypes.byref(rate), ctypes.byref(mhz), ctypes.byref(ms),
                                    ctypes.c_void_p(s)))
    return {"rate": rate.value, "sm_mhz": mhz.value, "ms": ms.value}


def mce_root_features(h: Handle, raw: bool = False):
    """Root features as CUDA tensors [n, 16] indexed by input id: float32
    log2(1 + value), or int32 raw values with raw=True."""
    import torch
    n = max(h.n, 1)
    if raw:
        t = torch.empty((n, MCE_NUM_FEATURES), dtype=torch.int32, device="cuda")
        _check(library().mce_root_features(h.ptr, ctypes.c_void_p(t.data_ptr()), None))
    else:
        t = torch.empty((n, MCE_NUM_FEATURES), dtype=torch.float32, device="cuda")
        _check(library().mce_root_features(h.ptr, None, ctypes.c_void_p(t.data_ptr())))
    return t[: h.n]


class Model:
    """mce_model: the work estimator's parameters (FP32 master, BF16 in use) and Adam state."""

    def __init__(self, params, stream: Optional[int] = None, use_torch_allocator: bool = True):
        import torch
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MCE_MODEL_PARAMS,):
            raise ValueError("need %d parameters" % MCE_MODEL_PARAMS)
        s, dev = (stream, torch.cuda.current_device()) if stream is not None else _current_stream()
        self._alloc = _TorchAllocator(dev, s) if use_torch_allocator else None
        self.ptr = ctypes.c_void_p()
        _check(library().mce_model_create(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          ctypes.byref(self._alloc.struct) if self._alloc else None,
                                          ctypes.c_void_p(s), ctypes.byref(self.ptr)))

    def params(self) -> np.ndarray:
        out = np.zeros(MCE_MODEL_PARAMS, np.float32)
        _check(library().mce_model_get_params(self.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def predict(self, feat):
        import torch
        feat = feat.contiguous()
        out = torch.empty(feat.shape[0], dtype=torch.float32, device="cuda")
        _check(library().mce_model_predict(self.ptr, ctypes.c_void_p(feat.data_ptr()), feat.shape[0],
                                           ctypes.c_void_p(out.data_ptr())))
        return out

    def gradient(self, feat, label):
        g = np.zeros(MCE_MODEL_PARAMS, np.float32)
        loss = ctypes.c_float()
        feat, label = feat.contiguous(), label.contiguous()
        _check(library().mce_model_gradient(self.ptr, ctypes.c_void_p(feat.data_ptr()),
                                            ctypes.c_void_p(label.data_ptr()), feat.shape[0],
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
        return g, float(loss.value)

    def train_step(self, feat, label, lr: float, want_loss: bool = False):
        loss = ctypes.c_float()
        _check(library().mce_model_train_step(self.ptr, ctypes.c_void_p(feat.data_ptr()),
                                              ctypes.c_void_p(label.data_ptr()), feat.shape[0], lr,
                                              ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def close(self):
        if self.ptr:
            library().mce_model_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mce_predict_priority(h: Handle, model: "Model", min_p: int = 33):
    """Predicted log2 subtree size per root (CUDA float32 [n] by input id);
    roots with |P0| < min_p get -1 (see include/mce.h)."""
    import torch
    out = torch.empty(max(h.n, 1), dtype=torch.float32, device="cuda")
    _check(library().mce_predict_priority(h.ptr, model.ptr, min_p, ctypes.c_void_p(out.data_ptr())))
    return out[: h.n]


def mce_destroy(h: Handle):
    if h is not None and h.ptr:
        library().mce_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


def mce_run_list(h: Handle, buf=None, opts: Optional[mce_opts] = None):
    """List the maximal cliques into `buf` (a CUDA int32 tensor; None: only
    size the list) as records [k, id_1, ..., id_k] (see include/mce.h).
    Returns (Result, words needed). Raises MCEError(MCE_ERANGE) when the list
    does not fit; the records that fit are written."""
    lib = library()
    words = ctypes.c_int64(0)
    r = mce_result()
    if buf is not None:
        import torch
        if not (isinstance(buf, torch.Tensor) and buf.is_cuda and buf.dtype == torch.int32 and buf.is_contiguous()):
            raise TypeError("buf must be a contiguous CUDA int32 tensor")
        ptr, cap = buf.data_ptr(), buf.numel()
    else:
        ptr, cap = None, 0
    _check(lib.mce_run_list(h.ptr, ctypes.byref(opts) if opts is not None else None, ptr, cap,
                            ctypes.byref(words), ctypes.byref(r)))
    return _result(r), int(words.value)


def decode_clique_records(flat) -> List[np.ndarray]:
    """Split a list of records [k, id_1, ..., id_k] (numpy int32) into arrays.

    Raises ValueError on a record of size < 1 or one that runs past the end:
    every record mce_run_list writes holds a clique of at least one vertex."""
    out, i, n = [], 0, len(flat)
    while i < n:
        k = int(flat[i])
        if k < 1 or i + 1 + k > n:
            raise ValueError("malformed clique record at word %d (size %d, %d words left)" % (i, k, n - i - 1))
        out.append(np.asarray(flat[i + 1:i + 1 + k]))
        i += 1 + k
    return out


def list_maximal_cliques(row_ptr, col, max_words: int = 1 << 26, **opt_fields) -> List[np.ndarray]:
    """One-shot listing of every maximal clique (input vertex ids), produced
    root subset by root subset so that no buffer exceeds max_words words."""
    import torch
    h = mce_create(row_ptr, col)
    try:
        _, need = mce_run_list(h, None, mce_default_opts(**opt_fields))
        pieces = []

        def go(roots):
            opts = mce_default_opts(**opt_fields)
            keep = None
            if roots is not None:
                keep = torch.as_tensor(np.ascontiguousarray(roots, dtype=np.int32)).cuda()
                opts.roots = keep.data_ptr()
                opts.n_roots = len(keep)
            _, w = mce_run_list(h, None, opts)
            if w <= max_words or (roots is not None and len(roots) == 1):
                buf = torch.empty(max(w, 1), dtype=torch.int32, device="cuda")
                _, w2 = mce_run_list(h, buf, opts)
                pieces.extend(decode_clique_records(buf[:w2].cpu().numpy()))
                return
            ids = np.arange(h.n, dtype=np.int32) if roots is None else np.asarray(roots)
            half = len(ids) // 2
            go(ids[:half])
            go(ids[half:])

        go(None if need <= max_words else np.arange(h.n, dtype=np.int32))
        return pieces
    finally:
        mce_destroy(h)


def enumerate_maximal_cliques(row_ptr, col, per_root: bool = False, roots=None, **opt_fields):
    """One-shot convenience: create, run, destroy. With per_root, also returns
    per-vertex subtree (count, hash, nodes) as numpy uint64 arrays. `roots`
    (input vertex ids) restricts the enumeration to those first-level subtrees."""
    import torch
    h = mce_create(row_ptr, col)
    try:
        opts = mce_default_opts(**opt_fields)
        keep = []
        if roots is not None:
            rt = torch.as_tensor(np.ascontiguousarray(roots, dtype=np.int32)).cuda()
            keep_roots = rt
            opts.roots = rt.data_ptr() if len(rt) else torch.zeros(1, dtype=torch.int32, device="cuda").data_ptr()
            opts.n_roots = len(rt)
        if per_root:
            n = max(h.n, 1)
            for name in ("root_count", "root_hash", "root_nodes"):
                t = torch.zeros(n, dtype=torch.int64, device="cuda")
                keep.append(t)
                setattr(opts, name, t.data_ptr())
        res = mce_run(h, opts)
        if per_root:
            torch.cuda.current_stream().synchronize()
            arrs = [t.cpu().numpy().view(np.uint64)[: h.n] for t in keep]
            return res, arrs
        return res
    finally:
        mce_destroy(h)
