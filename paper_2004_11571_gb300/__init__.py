"""Python binding of libpolyeval (partial modular polynomial evaluation on GB300).

Argument marshalling only: every step of the evaluation runs in the library's
CUDA kernels.  PyTorch supplies device buffers and streams.  If the compiled
library is missing the import of any entry point raises; there is no CPU
fallback.

Entry points mirror include/poly_eval.h:
  Poly(p, coeffs, exps, variant)        poly_eval_create
  Poly.groups() / Poly.G                poly_eval_groups
  Poly.run(beta, T, t0, out, stream)    poly_eval_run
  Poly.set_tiles / Poly.plan_info       poly_eval_set_tiles / poly_eval_plan_info
  Batch(jobs) / Batch.launch            poly_eval_batch_plan / _launch
  tune(poly, T)                         poly_eval_tune
  Server(...)                           poly_eval_server_*
  modmul_peak(variant, p)               poly_eval_modmul_peak
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpolyeval.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "poly_eval.h")

VARIANTS = {"auto": 0, "mont64": 1, "fp64": 2, "barrett64": 3, "barrett32": 4}
STATUS = {0: "PE_OK", 1: "PE_ERR_ARG", 2: "PE_ERR_PRIME", 3: "PE_ERR_NOT_REDUCED", 4: "PE_ERR_EXP_RANGE",
          5: "PE_ERR_NOMEM", 6: "PE_ERR_ADMISSION", 7: "PE_ERR_CUDA", 8: "PE_ERR_TIMEOUT", 9: "PE_PENDING",
          10: "PE_ERR_NOT_FOUND", 11: "PE_ERR_SINGULAR"}
PE_OK, PE_PENDING, PE_ERR_TIMEOUT, PE_ERR_ADMISSION = 0, 9, 8, 6
PE_ERR_NOT_REDUCED, PE_ERR_SINGULAR = 3, 11
FLAG_DEVICE_PTRS, FLAG_SORTED, FLAG_BORROW = 0x1, 0x2, 0x4


class PolyEvalError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint64), ("n", ctypes.c_uint32), ("exp_bytes", ctypes.c_uint32),
                ("s", ctypes.c_uint64), ("coeffs", ctypes.c_void_p), ("exps", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("variant", ctypes.c_int)]


class _Tiles(ctypes.Structure):
    _fields_ = [("K", ctypes.c_uint32), ("slabs", ctypes.c_uint32), ("tchunk", ctypes.c_uint32),
                ("warps_per_block", ctypes.c_uint32), ("tail", ctypes.c_uint32)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("tiles", _Tiles), ("variant", ctypes.c_int), ("chunks", ctypes.c_uint64),
                ("items", ctypes.c_uint64), ("spans", ctypes.c_uint64), ("padded_terms", ctypes.c_uint64),
                ("tail_points", ctypes.c_uint64), ("method", ctypes.c_uint32)]


class _Job(ctypes.Structure):
    _fields_ = [("poly", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("T", ctypes.c_uint64),
                ("t0", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class _ServerCfg(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_uint64), ("max_queue", ctypes.c_uint32),
                ("max_epoch_jobs", ctypes.c_uint32), ("streams", ctypes.c_uint32)]


class _Request(ctypes.Structure):
    _fields_ = [("poly_desc", ctypes.c_void_p), ("resident_id", ctypes.c_uint64), ("beta", ctypes.c_void_p),
                ("T", ctypes.c_uint64), ("t0", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("new_resident_id", ctypes.c_void_p)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("epochs", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("term_points", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("resident_bytes", ctypes.c_uint64), ("resident_polys", ctypes.c_uint64),
                ("evictions", ctypes.c_uint64), ("upload_s", ctypes.c_double), ("plan_s", ctypes.c_double),
                ("launch_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_vp, _u64, _u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32


def declared_functions() -> list:
    """Names of the functions declared in include/poly_eval.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(poly_eval_\w+)\s*\(", text)))


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpolyeval.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        sig = {
            "poly_eval_create": (st, [ctypes.POINTER(_Desc), ctypes.POINTER(_vp)]),
            "poly_eval_groups": (st, [_vp, ctypes.POINTER(_u64), _vp]),
            "poly_eval_run": (st, [_vp, _vp, _u64, _u64, _vp, _vp]),
            "poly_eval_destroy": (None, [_vp]),
            "poly_eval_last_error": (ctypes.c_char_p, []),
            "poly_eval_set_tiles": (st, [_vp, ctypes.POINTER(_Tiles)]),
            "poly_eval_plan_info": (st, [_vp, _u64, ctypes.POINTER(_PlanInfo)]),
            "poly_eval_launches_per_run": (st, [_vp, _u64, ctypes.POINTER(_u32)]),
            "poly_eval_set_timing": (st, [_vp, ctypes.c_int]),
            "poly_eval_kernel_times": (st, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u64)]),
            "poly_eval_batch_plan": (st, [_vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
            "poly_eval_batch_launch": (st, [_vp, _vp]),
            "poly_eval_batch_set_beta": (st, [_vp, ctypes.c_size_t, _vp]),
            "poly_eval_batch_launches": (st, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
            "poly_eval_batch_destroy": (None, [_vp]),
            "poly_eval_batch": (st, [_vp, ctypes.c_size_t, _vp]),
            "poly_eval_tune": (st, [_vp, _u64, ctypes.POINTER(_Tiles), ctypes.POINTER(ctypes.c_double)]),
            "poly_eval_tune_save": (st, [ctypes.c_char_p]),
            "poly_eval_tune_load": (st, [ctypes.c_char_p]),
            "poly_eval_server_create": (st, [ctypes.POINTER(_ServerCfg), ctypes.POINTER(_vp)]),
            "poly_eval_server_register": (st, [_vp, ctypes.POINTER(_Desc), ctypes.POINTER(_u64)]),
            "poly_eval_server_submit": (st, [_vp, ctypes.POINTER(_Request), ctypes.POINTER(_u64)]),
            "poly_eval_server_poll": (st, [_vp, _u64, ctypes.c_int64]),
            "poly_eval_server_stats": (st, [_vp, ctypes.POINTER(_ServerStats)]),
            "poly_eval_server_destroy": (None, [_vp]),
            "poly_eval_server_pause": (st, [_vp, ctypes.c_int]),
            "poly_eval_modmul_peak": (st, [ctypes.c_int, _u64, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
            "poly_eval_int_pipe_rates": (st, [ctypes.POINTER(ctypes.c_double)]),
            "poly_eval_fp64_pipe_rates": (st, [ctypes.POINTER(ctypes.c_double)]),
            "poly_eval_num_sms": (st, [ctypes.POINTER(ctypes.c_uint32)]),
            "poly_eval_compact": (st, [_vp, _u64, _u64, _vp, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp]),
            "poly_eval_monomials": (st, [_vp, _vp, _vp, _vp, _vp]),
            "poly_eval_create_like": (st, [_vp, _u64, _vp, _u32, ctypes.c_int, ctypes.POINTER(_vp)]),
            "poly_eval_run_fast": (st, [_vp, _vp, _u64, _u64, _vp, _vp]),
            "poly_eval_debug_fail_alloc": (st, [_u32]),
            "poly_eval_vandermonde_solve": (st, [_u64, _u64, _vp, _vp, _vp, _u64, _u64, _u64, _vp, _vp]),
            "poly_eval_vandermonde_timing": (st, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
            "poly_eval_stepb_noalloc": (st, [_u64, _u64, _u64, _vp, _vp, _vp, _u64, _u64, _vp, _vp]),
            "poly_eval_stepb_noalloc_shape": (st, [_u64, _u64, ctypes.POINTER(ctypes.c_uint32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int):
    if status != PE_OK:
        msg = lib().poly_eval_last_error()
        raise PolyEvalError(status, msg.decode() if msg else "")


def _variant(v) -> int:
    return VARIANTS[v] if isinstance(v, str) else int(v)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _make_desc(p, coeffs, exps, variant, sorted_hint):
    """Builds a descriptor; returns (desc, keepalive)."""
    if _is_torch(coeffs):
        import torch
        if not coeffs.is_cuda:
            coeffs = coeffs.numpy()
            exps = exps.numpy()
    if _is_torch(coeffs):
        exps_t = exps.contiguous()
        coeffs_t = coeffs.contiguous()
        s, n = exps_t.shape
        eb = exps_t.element_size()
        desc = _Desc(p, n, eb, s, coeffs_t.data_ptr(), exps_t.data_ptr(),
                     FLAG_DEVICE_PTRS | (FLAG_SORTED if sorted_hint else 0), _variant(variant))
        return desc, (coeffs_t, exps_t)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64)
    exps = np.asarray(exps)
    if exps.dtype not in (np.uint8, np.uint16, np.uint32):
        exps = exps.astype(np.uint32)
    exps = np.ascontiguousarray(exps)
    s = coeffs.shape[0]
    n = exps.shape[1] if exps.ndim == 2 else 0
    desc = _Desc(p, n, exps.dtype.itemsize, s, coeffs.ctypes.data, exps.ctypes.data,
                 FLAG_SORTED if sorted_hint else 0, _variant(variant))
    return desc, (coeffs, exps)


class Poly:
    """A polynomial resident on the current CUDA device (poly_eval_create)."""

    def __init__(self, p: int, coeffs, exps, variant="auto", sorted_hint: bool = False):
        L = lib()
        desc, keep = _make_desc(int(p), coeffs, exps, variant, sorted_hint)
        h = ctypes.c_void_p()
        _check(L.poly_eval_create(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.p = int(p)
        self.n = int(desc.n)
        self.s = int(desc.s)
        G = ctypes.c_uint64()
        _check(L.poly_eval_groups(h, ctypes.byref(G), None))
        self.G = int(G.value)

    @classmethod
    def from_workload(cls, w, variant="auto"):
        return cls(w.p, w.coeffs, w.exps, variant=variant)

    def like(self, p: int, coeffs, variant="auto"):
        """The same terms modulo another prime p (coefficients reduced mod p, in
        the order given to this polynomial's constructor); shares the device
        exponents (poly_eval_create_like)."""
        if _is_torch(coeffs):
            ptr, flags, keep = coeffs.data_ptr(), FLAG_DEVICE_PTRS, coeffs
        else:
            keep = np.ascontiguousarray(np.asarray(coeffs, dtype=np.uint64).reshape(-1))
            ptr, flags = keep.ctypes.data, 0
        h = ctypes.c_void_p()
        _check(lib().poly_eval_create_like(self._h, int(p), ptr, flags, _variant(variant), ctypes.byref(h)))
        q = Poly.__new__(Poly)
        q._h, q.p, q.n, q.s, q.G = h, int(p), self.n, self.s, self.G
        return q

    @property
    def handle(self):
        return self._h

    def groups(self) -> np.ndarray:
        keys = np.zeros((max(self.G, 1), 2), np.uint32)
        G = ctypes.c_uint64()
        _check(lib().poly_eval_groups(self._h, ctypes.byref(G), keys.ctypes.data))
        return keys[: self.G].copy()

    def run(self, beta: Sequence[int], T: int, t0: int = 1, out=None, stream=None):
        """Evaluates T images; returns `out` (a new int64 CUDA tensor of shape (T, G) when None)."""
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
        if out is None:
            import torch
            out = torch.empty((int(T), self.G), dtype=torch.int64, device="cuda")
        ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
        bptr = b.ctypes.data if b.size else None
        _check(lib().poly_eval_run(self._h, bptr, int(T), int(t0), ptr, _stream_ptr(stream)))
        return out

    def monomials(self, beta: Sequence[int], stream=None):
        """(z, off): the monomial values M_i(beta) as an int64 CUDA tensor of s
        uint64 values in the library's term order (stable sort by (d, e)
        descending), and the G+1 term offsets of the image columns (numpy)."""
        import torch
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
        z = torch.empty(max(self.s, 1), dtype=torch.int64, device="cuda")
        off = np.zeros(self.G + 1, np.uint64)
        _check(lib().poly_eval_monomials(self._h, b.ctypes.data if b.size else None, z.data_ptr(),
                                         off.ctypes.data, _stream_ptr(stream)))
        return z[: self.s], off

    def run_fast(self, beta: Sequence[int], T: int, t0: int = 1, out=None, stream=None):
        """The same images by the fast method (poly_eval_run_fast; NTT-friendly p, T <= 4096)."""
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
        if out is None:
            import torch
            out = torch.empty((int(T), self.G), dtype=torch.int64, device="cuda")
        ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
        _check(lib().poly_eval_run_fast(self._h, b.ctypes.data if b.size else None, int(T), int(t0), ptr,
                                        _stream_ptr(stream)))
        return out

    def set_tiles(self, K=0, slabs=0, tchunk=0, warps_per_block=0, tail=0):
        t = _Tiles(K, slabs, tchunk, warps_per_block, tail)
        _check(lib().poly_eval_set_tiles(self._h, ctypes.byref(t)))

    def plan_info(self, T: int) -> dict:
        info = _PlanInfo()
        _check(lib().poly_eval_plan_info(self._h, int(T), ctypes.byref(info)))
        return {"K": info.tiles.K, "slabs": info.tiles.slabs, "tchunk": info.tiles.tchunk,
                "warps_per_block": info.tiles.warps_per_block, "variant": info.variant,
                "chunks": info.chunks, "items": info.items, "spans": info.spans,
                "padded_terms": info.padded_terms, "tail_points": info.tail_points,
                "method": "fast" if info.method == 1 else "matrix"}

    def launches_per_run(self, T: int) -> int:
        n = ctypes.c_uint32()
        _check(lib().poly_eval_launches_per_run(self._h, int(T), ctypes.byref(n)))
        return int(n.value)

    def set_timing(self, enable: bool = True):
        _check(lib().poly_eval_set_timing(self._h, 1 if enable else 0))

    def kernel_times(self):
        """(ms power tables, ms Step A, ms Step B, runs) summed since the last call."""
        ms = (ctypes.c_double * 3)()
        runs = ctypes.c_uint64()
        _check(lib().poly_eval_kernel_times(self._h, ms, ctypes.byref(runs)))
        return ms[0], ms[1], ms[2], int(runs.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().poly_eval_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A planned batch (poly_eval_batch_plan): one CUDA graph running every job's
    power tables and a persistent Step A+B kernel over a shared work queue;
    jobs of at least 2^28 term-points run as plain runs after it.

    jobs: sequence of (poly, beta, T, t0, out) with `out` a CUDA tensor (T x G)."""

    def __init__(self, jobs):
        L = lib()
        n = len(jobs)
        arr = (_Job * max(n, 1))()
        self._keep = []
        for i, (poly, beta, T, t0, out) in enumerate(jobs):
            b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
            self._keep.append(b)
            arr[i] = _Job(poly.handle.value, b.ctypes.data if b.size else None, int(T), int(t0), out.data_ptr())
        self._keep.append(arr)
        self.polys = [j[0] for j in jobs]
        h = ctypes.c_void_p()
        _check(L.poly_eval_batch_plan(arr, n, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().poly_eval_batch_launch(self._h, _stream_ptr(stream)))

    def set_beta(self, j: int, beta):
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
        _check(lib().poly_eval_batch_set_beta(self._h, int(j), b.ctypes.data if b.size else None))

    def launches(self) -> dict:
        """Kernel launches per launch() and the number of plain-run jobs."""
        k, n = _u32(), _u32()
        _check(lib().poly_eval_batch_launches(self._h, ctypes.byref(k), ctypes.byref(n)))
        return {"kernels": k.value, "plain_jobs": n.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().poly_eval_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (poly_eval_server_*).

    submit() returns a ticket; results land in the caller's host buffer `out`
    (T x G uint64; page-locked buffers take the asynchronous path)."""

    def __init__(self, mem_cap_bytes: int = 40 << 30, max_queue: int = 4096, max_epoch_jobs: int = 256,
                 streams: int = 4):
        cfg = _ServerCfg(int(mem_cap_bytes), int(max_queue), int(max_epoch_jobs), int(streams))
        h = ctypes.c_void_p()
        _check(lib().poly_eval_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def register(self, p: int, coeffs, exps, variant="auto") -> int:
        desc, keep = _make_desc(int(p), coeffs, exps, variant, False)
        rid = ctypes.c_uint64()
        _check(lib().poly_eval_server_register(self._h, ctypes.byref(desc), ctypes.byref(rid)))
        return int(rid.value)

    def submit(self, beta, T: int, out: np.ndarray, t0: int = 1, poly=None, resident_id: int = 0,
               variant="auto", borrow: bool = False):
        """poly = (p, coeffs, exps) uploads a new polynomial; returns (ticket, new_resident_id).
        borrow=True: the arrays are not copied and must stay unchanged until the ticket completes."""
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(-1))
        new_id = ctypes.c_uint64(0)
        desc_ref = None
        keep = None
        if poly is not None:
            desc, keep = _make_desc(int(poly[0]), poly[1], poly[2], variant, False)
            if borrow:
                desc.flags |= FLAG_BORROW
            desc_ref = ctypes.addressof(desc)
        req = _Request(desc_ref, int(resident_id), b.ctypes.data if b.size else None, int(T), int(t0),
                       out.ctypes.data, ctypes.addressof(new_id))
        t = ctypes.c_uint64()
        _check(lib().poly_eval_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        del desc_ref
        self._keep[int(t.value)] = (out, keep) if borrow else out
        return int(t.value), int(new_id.value)

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        """Status code: 0 done, 9 pending (timeout 0), 8 timed out; errors raise."""
        st = lib().poly_eval_server_poll(self._h, int(ticket), int(timeout_us))
        if st in (PE_OK, PE_PENDING, PE_ERR_TIMEOUT):
            if st == PE_OK:
                self._keep.pop(int(ticket), None)
            return st
        self._keep.pop(int(ticket), None)
        _check(st)

    def pause(self, paused: bool = True):
        _check(lib().poly_eval_server_pause(self._h, 1 if paused else 0))

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib().poly_eval_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().poly_eval_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune(poly: "Poly", T: int):
    """Autotunes the tile shape and modular product for poly's shape bucket;
    returns (tiles dict, milliseconds per run)."""
    t = _Tiles()
    ms = ctypes.c_double()
    _check(lib().poly_eval_tune(poly.handle, int(T), ctypes.byref(t), ctypes.byref(ms)))
    return {"K": t.K, "slabs": t.slabs, "tchunk": t.tchunk, "warps_per_block": t.warps_per_block}, ms.value


def tune_save(path: str):
    _check(lib().poly_eval_tune_save(path.encode()))


def tune_load(path: str):
    _check(lib().poly_eval_tune_load(path.encode()))


def stepb_noalloc(p: int, coeffs, m, group_off, T: int, t0: int, out, stream=None):
    """poly_eval_stepb_noalloc on CUDA tensors: coeffs, m (int64 views of
    uint64), group_off (int32 view of uint32, G+1 entries) and out (T x G)."""
    L = lib()
    fn = L.poly_eval_stepb_noalloc
    s, G = int(coeffs.shape[0]), int(group_off.shape[0]) - 1
    _check(fn(int(p), s, G, coeffs.data_ptr(), m.data_ptr(), group_off.data_ptr(), int(T), int(t0),
              out.data_ptr(), _stream_ptr(stream)))
    return out


def stepb_noalloc_shape(s: int, T: int) -> dict:
    """The work decomposition stepb_noalloc uses for s terms and T points
    (poly_eval_stepb_noalloc_shape): units, T-chunks, points per chunk, slabs per unit."""
    sh = (ctypes.c_uint32 * 4)()
    _check(lib().poly_eval_stepb_noalloc_shape(int(s), int(T), sh))
    return {"units": sh[0], "tchunks": sh[1], "tchunk": sh[2], "kslabs": sh[3]}


def modmul_peak(variant="barrett64", p: int = (1 << 61) - 1):
    """(term-points/s, SM MHz) of the register-only Step B inner loop."""
    tps, mhz = ctypes.c_double(), ctypes.c_double()
    _check(lib().poly_eval_modmul_peak(_variant(variant), int(p), ctypes.byref(tps), ctypes.byref(mhz)))
    return tps.value, mhz.value


def compact(dense, stream=None):
    """Sparse images from a dense (T, G) CUDA tensor: (row_ptr[T+1], cols, vals)
    as CUDA tensors (int64, int32, int64 views of uint64 / uint32)."""
    import torch
    T, G = int(dense.shape[0]), int(dense.shape[1])
    row_ptr = torch.empty(T + 1, dtype=torch.int64, device=dense.device)
    cap = T * G
    cols = torch.empty(max(cap, 1), dtype=torch.int32, device=dense.device)
    vals = torch.empty(max(cap, 1), dtype=torch.int64, device=dense.device)
    nnz = ctypes.c_uint64()
    _check(lib().poly_eval_compact(dense.data_ptr(), T, G, row_ptr.data_ptr(), cols.data_ptr(), vals.data_ptr(),
                                   cap, ctypes.byref(nnz), _stream_ptr(stream)))
    n = int(nnz.value)
    return row_ptr, cols[:n], vals[:n]


def vandermonde_solve(p: int, off, z, images, t0: int = 1, out=None, stream=None):
    """Coefficients c (int64 CUDA tensor of off[-1] uint64 values) with
    sum_i c[off[g]+i] z[off[g]+i]^(t0+k) = images[k, g] for k < off[g+1]-off[g]:
    interpolation of every image column from its monomial values (Sect. 1).
    `z` and `images` are int64 CUDA tensors (uint64 values); `off` is host."""
    import torch
    off = np.ascontiguousarray(np.asarray(off, dtype=np.uint64).reshape(-1))
    G = off.shape[0] - 1
    s = int(off[-1]) if G >= 0 and off.size else 0
    if out is None:
        out = torch.empty(max(s, 1), dtype=torch.int64, device=z.device if _is_torch(z) else "cuda")
    rows, lda = (int(images.shape[0]), int(images.stride(0))) if images.dim() == 2 else (0, G)
    _check(lib().poly_eval_vandermonde_solve(int(p), G, off.ctypes.data, z.data_ptr(), images.data_ptr(), rows,
                                             lda, int(t0), out.data_ptr(), _stream_ptr(stream)))
    return out[:s]


def vandermonde_timing(enable=None) -> dict:
    """Kernel milliseconds of the latest timed vandermonde_solve on this thread;
    enable=True/False switches timing for later calls."""
    ms = (ctypes.c_double * 4)()
    _check(lib().poly_eval_vandermonde_timing(-1 if enable is None else int(bool(enable)), ms))
    return {"leaves": ms[0], "tree": ms[1], "correlation": ms[2], "horner": ms[3]}


def debug_fail_alloc(nth: int):
    """Make the nth device allocation of the library from now fail (0 cancels);
    a testing aid for failure paths (poly_eval_debug_fail_alloc)."""
    _check(lib().poly_eval_debug_fail_alloc(int(nth)))


def int_pipe_rates() -> dict:
    """Thread operations per SM per clock of mad.lo / mad.hi / mad.wide / add (u32)."""
    r = (ctypes.c_double * 4)()
    _check(lib().poly_eval_int_pipe_rates(r))
    return {"mad_lo": r[0], "mad_hi": r[1], "mad_wide": r[2], "add": r[3]}


def fp64_pipe_rates() -> dict:
    """Thread operations per SM per clock of fma.rn.f64 / add.rn.f64."""
    r = (ctypes.c_double * 2)()
    _check(lib().poly_eval_fp64_pipe_rates(r))
    return {"fma": r[0], "add": r[1]}


def num_sms() -> int:
    """Streaming multiprocessors of the current device (poly_eval_num_sms)."""
    n = ctypes.c_uint32()
    _check(lib().poly_eval_num_sms(ctypes.byref(n)))
    return int(n.value)


def to_u64(t) -> np.ndarray:
    """A (T, G) int64 CUDA tensor or numpy array viewed as uint64 on the host."""
    if _is_torch(t):
        t = t.cpu().numpy()
    return np.ascontiguousarray(t).view(np.uint64)
