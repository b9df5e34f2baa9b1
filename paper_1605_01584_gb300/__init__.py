"""Python binding of libpcc.so (include/pcc.h): all-pairs Pearson correlation
on GB300 tensor cores.

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory (tensors) and streams.  The names follow the
C ABI; each function raises PccError when the library returns a status
other than PCC_OK.  There is no CPU fallback: if the library is not built,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpcc.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "pcc.h")

# pcc_status
PCC_OK = 0
PCC_ERR_INVALID_ARG = 1
PCC_ERR_CUDA = 2
PCC_ERR_OOM = 3
PCC_ERR_CAPACITY = 4
PCC_ERR_TIMEOUT = 5
PCC_ERR_UNSUPPORTED = 6
PCC_ERR_ABORTED = 7
# pcc_dtype
PCC_F32 = 0
PCC_F64 = 1
# pcc_prec
PCC_PREC_FP64 = 0
PCC_PREC_FP32 = 1
PCC_PREC_BF16X3 = 2
PCC_PREC_FP16X3S = 3
PCC_PREC_BF16X4 = 4
PCC_PREC_BF16X1 = 5
PCC_PREC_AUTO = 6
PCC_PERM_SMEM = 0
PCC_PERM_WORKSPACE = 1
PCC_PERM_TRANSPOSED = 2

PREC_NAMES = {"fp64": PCC_PREC_FP64, "fp32": PCC_PREC_FP32,
              "bf16x3": PCC_PREC_BF16X3, "fp16x3s": PCC_PREC_FP16X3S,
              "bf16x4": PCC_PREC_BF16X4, "bf16x1": PCC_PREC_BF16X1,
              "auto": PCC_PREC_AUTO}

EDGE_BYTES = 12  # pcc_edge {u32 i, u32 j, f32 r}

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U64 = ctypes.c_uint64
_ST = ctypes.c_int


class PccError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = _lib.pcc_status_string(self.status).decode() if _lib else ""
        super().__init__(f"{where}: {msg} (status {self.status})")


def header_functions() -> list[str]:
    """Names of the functions declared in include/pcc.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pcc_[a-z0-9_]+)\s*\(", txt)))


_SINK = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_int64, ctypes.c_void_p)


def load(path: str | None = None):
    """Load libpcc.so; raise if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(p)
    sig = {
        "pcc_standardize": (_ST, [_P, _I32, _I64, _I64, _I64, _I32,
                                  ctypes.POINTER(_P), _P]),
        "pcc_standardize_host": (_ST, [_P, _I32, _I64, _I64, _I64, _I32,
                                       ctypes.POINTER(_P), _P]),
        "pcc_edges_copy_host": (_ST, [_P, _P, _U64, _P, _P, _P]),
        "pcc_zmat_destroy": (_ST, [_P]),
        "pcc_standardize_batched": (_ST, [_P, _P, _P, _P, _I32, _I32, _P,
                                          _P]),
        "pcc_zmat_info": (_ST, [_P, _P, _P, _P, _P, _P]),
        "pcc_zmat_buffers": (_ST, [_P, _P, _P, _P, _P]),
        "pcc_num_tiles": (_I64, [_P]),
        "pcc_allpairs_upper": (_ST, [_P, _P, _I32, _I64, _I64, _P]),
        "pcc_threshold_edges": (_ST, [_P, ctypes.c_float, _P, _U64, _P, _P,
                                      _P]),
        "pcc_cross_num_tiles": (_I64, [_P, _P]),
        "pcc_cross_allpairs": (_ST, [_P, _P, _P, _I32, _I64, _I64, _I64, _P]),
        "pcc_cross_edges": (_ST, [_P, _P, ctypes.c_float, _P, _U64, _P, _P,
                                  _I64, _P]),
        "pcc_allpairs_upper_host": (_ST, [_P, _P, _I32, _I64, _SINK, _P,
                                          _P]),
        "pcc_cross_allpairs_host": (_ST, [_P, _P, _P, _I32, _I64, _I64,
                                          _SINK, _P, _P]),
        "pcc_threshold_edges_host": (_ST, [_P, ctypes.c_float, _P, _U64, _P,
                                           _P, _I64, _SINK, _P, _P]),
        "pcc_perm_test": (_ST, [_P, _P, _I32, _I32, _I32, _P, _P]),
        "pcc_allpairs_upper_batched": (_ST, [_P, _I32, _P, _P]),
        "pcc_allpairs_upper_batched_tuned": (_ST, [_P, _I32, _P, _P, _P,
                                                   _P]),
        "pcc_sync_status": (_ST, [_P, _P]),
        "pcc_allpairs_upper_noalloc": (_ST, [_P, _I64, _I64, _I64, _I32, _P,
                                             _P, _P]),
        "pcc_set_wait_limit_ns": (_ST, [_U64]),
        "pcc_debug_drop_loads": (_ST, [_I32]),
        "pcc_set_tuning": (_ST, [_I32, _I32, _I32, ctypes.c_double,
                                 ctypes.c_double]),
        "pcc_get_tuning": (_ST, [_P, _P, _P, _P, _P]),
        "pcc_set_pair_mma": (_ST, [_I32]),
        "pcc_measure_fp32_fma": (_ST, [_P, _P]),
        "pcc_get_pair_mma": (_I32, []),
        "pcc_set_perm_form": (_ST, [_I32]),
        "pcc_get_perm_form": (_I32, []),
        "pcc_num_pairs": (_I64, [_I64]),
        "pcc_pair_index": (_I64, [_I64, _I64, _I64]),
        "pcc_pair_coords": (_ST, [_I64, _I64, _P, _P]),
        "pcc_tile_coords": (_ST, [_I64, _I64, _P, _P]),
        "pcc_schedule_num_tiles": (_I64, [_I64, _I32]),
        "pcc_schedule_tile_rect": (_ST, [_I64, _I32, _I64, _P, _P, _P, _P]),
        "pcc_status_string": (ctypes.c_char_p, [_ST]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(st: int, where: str):
    if st != PCC_OK:
        raise PccError(st, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _prec(p):
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


class Zmat:
    """Owner of a library-allocated pcc_zmat (freed on close/garbage)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def info(self):
        n, l, lpad = _I64(), _I64(), _I64()
        prec, s = _I32(), _I32()
        _check(load().pcc_zmat_info(self.handle, ctypes.byref(n),
                                    ctypes.byref(l), ctypes.byref(lpad),
                                    ctypes.byref(prec), ctypes.byref(s)),
               "pcc_zmat_info")
        return dict(n=n.value, l=l.value, lpad=lpad.value, prec=prec.value,
                    scale_exp=s.value)

    def buffers(self):
        hi, lo, z, fl = _P(), _P(), _P(), _P()
        _check(load().pcc_zmat_buffers(self.handle, ctypes.byref(hi),
                                       ctypes.byref(lo), ctypes.byref(z),
                                       ctypes.byref(fl)), "pcc_zmat_buffers")
        return dict(hi=hi.value, lo=lo.value, z=z.value, flags=fl.value)

    def num_tiles(self) -> int:
        return int(load().pcc_num_tiles(self.handle))

    def close(self):
        if self.handle and self.handle.value and _lib is not None:
            _lib.pcc_zmat_destroy(self.handle)
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcc_standardize(X, prec="auto", Z: Zmat | None = None, stream=None,
                    n=None, l=None, ldx=None) -> Zmat:
    """Eq. (5): standardize the rows of the device matrix X (float32/64,
    2-D with unit inner stride).  Reuses Z when its shape/precision match."""
    import torch
    L = load()
    assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
    xt = {torch.float32: PCC_F32, torch.float64: PCC_F64}[X.dtype]
    n = X.shape[0] if n is None else n
    l = X.shape[1] if l is None else l
    ldx = X.stride(0) if ldx is None else ldx
    h = ctypes.c_void_p(Z.handle.value if Z is not None else None)
    _check(L.pcc_standardize(_ptr(X), xt, n, l, ldx, _prec(prec),
                             ctypes.byref(h), _stream(stream)),
           "pcc_standardize")
    if Z is not None and h.value == Z.handle.value:
        return Z
    return Zmat(h.value)


def pcc_standardize_host(X, prec="auto", Z: Zmat | None = None,
                         stream=None) -> Zmat:
    """Eq. (5) from a HOST matrix (torch CPU tensor, float32/64, 2-D with
    unit inner stride; pin it for an asynchronous copy): the library copies
    it to the device and standardizes it.  Reuses Z when it matches."""
    import torch
    assert not X.is_cuda and X.dim() == 2 and X.stride(1) == 1
    xt = {torch.float32: PCC_F32, torch.float64: PCC_F64}[X.dtype]
    h = ctypes.c_void_p(Z.handle.value if Z is not None else None)
    _check(load().pcc_standardize_host(
        _ptr(X), xt, X.shape[0], X.shape[1], X.stride(0), _prec(prec),
        ctypes.byref(h), _stream(stream)), "pcc_standardize_host")
    if Z is not None and h.value == Z.handle.value:
        return Z
    return Zmat(h.value)


def pcc_edges_copy_host(edges, d_count, capacity: int, edges_host,
                        stream=None) -> int:
    """Copy the device edge list (uint8 buffer of pcc_edge records) and its
    count to host memory (edges_host: CPU uint8 tensor of >= capacity*12
    bytes); returns the count (PCC_ERR_CAPACITY raises)."""
    c = _U64()
    _check(load().pcc_edges_copy_host(_ptr(edges), _ptr(d_count),
                                      int(capacity), _ptr(edges_host),
                                      ctypes.byref(c), _stream(stream)),
           "pcc_edges_copy_host")
    return int(c.value)


def pcc_standardize_batched(Xs, prec="auto", Zs=None, stream=None):
    """pcc_standardize for many FP32 device matrices in one launch per
    stored form.  Zs (optional): matching Zmats are reused in place; returns
    the list of Zmats (new ones where a shape or form changed)."""
    import torch
    B = len(Xs)
    for X in Xs:
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        assert X.dtype == torch.float32
    xs = (_P * B)(*[X.data_ptr() for X in Xs])
    ns = (_I64 * B)(*[X.shape[0] for X in Xs])
    ls = (_I64 * B)(*[X.shape[1] for X in Xs])
    lds = (_I64 * B)(*[X.stride(0) for X in Xs])
    old = list(Zs) if Zs is not None else [None] * B
    hs = (_P * B)(*[z.handle.value if z is not None else None for z in old])
    _check(load().pcc_standardize_batched(xs, ns, ls, lds, B, _prec(prec),
                                          hs, _stream(stream)),
           "pcc_standardize_batched")
    out = []
    for z, h in zip(old, hs):
        out.append(z if z is not None and h == z.handle.value else Zmat(h))
    return out


def pcc_allpairs_upper(Z: Zmat, R, tile_begin: int = 0, tile_end: int = -1,
                       stream=None):
    import torch
    rt = PCC_F64 if R.dtype == torch.float64 else PCC_F32
    _check(load().pcc_allpairs_upper(Z.handle, _ptr(R), rt, tile_begin,
                                     tile_end, _stream(stream)),
           "pcc_allpairs_upper")
    return R


def pcc_threshold_edges(Z: Zmat, tau: float, edges, capacity: int, d_count,
                        R=None, stream=None):
    """edges: device buffer of >= capacity*12 bytes (or None); d_count: a
    device int64/uint64 scalar tensor, added to."""
    _check(load().pcc_threshold_edges(Z.handle, float(tau), _ptr(edges),
                                      int(capacity), _ptr(d_count), _ptr(R),
                                      _stream(stream)),
           "pcc_threshold_edges")


def pcc_cross_num_tiles(ZX: Zmat, ZY: Zmat) -> int:
    return int(load().pcc_cross_num_tiles(ZX.handle, ZY.handle))


def pcc_cross_allpairs(ZX: Zmat, ZY: Zmat, R, ldr: int | None = None,
                       tile_begin: int = 0, tile_end: int = -1, stream=None):
    """R[i * ldr + j] = r(x_i, y_j) (Eq. (7)-(8)); R a device float32 (or
    float64 for the FP64 form) buffer of nx rows of ldr (default ny)."""
    import torch
    rt = PCC_F64 if R.dtype == torch.float64 else PCC_F32
    if ldr is None:
        ldr = R.stride(0) if R.dim() == 2 else ZY.info()["n"]
    _check(load().pcc_cross_allpairs(ZX.handle, ZY.handle, _ptr(R), rt,
                                     int(ldr), tile_begin, tile_end,
                                     _stream(stream)), "pcc_cross_allpairs")
    return R


def pcc_cross_edges(ZX: Zmat, ZY: Zmat, tau: float, edges, capacity: int,
                    d_count, R=None, ldr: int | None = None, stream=None):
    """Edges {i in X, j in Y, r} with |r| >= tau; optional dense FP32 R."""
    if ldr is None:
        ldr = (R.stride(0) if R is not None and R.dim() == 2
               else ZY.info()["n"])
    _check(load().pcc_cross_edges(ZX.handle, ZY.handle, float(tau),
                                  _ptr(edges), int(capacity), _ptr(d_count),
                                  _ptr(R), int(ldr), _stream(stream)),
           "pcc_cross_edges")


def _host_buffer(R_host):
    """(pointer, is_float64, elements) of a contiguous host buffer given as
    a numpy array or a CPU torch tensor (pinned for overlapped copies)."""
    import numpy as np
    if R_host is None:
        return None, False, 0
    if hasattr(R_host, "data_ptr"):
        import torch
        assert not R_host.is_cuda and R_host.is_contiguous()
        return (ctypes.c_void_p(R_host.data_ptr()),
                R_host.dtype == torch.float64, R_host.numel())
    assert R_host.flags.c_contiguous
    return (ctypes.c_void_p(R_host.ctypes.data), R_host.dtype == np.float64,
            R_host.size)


def _host_stream(call, n_rows_elems, esize, sink):
    """Run a host-streaming entry point with a Python sink(r0, r1, view)."""
    import numpy as np
    err = []
    cb = None
    if sink is not None:
        dt = np.float64 if esize == 8 else np.float32

        def _cb(user, r0, r1, ptr):
            try:
                cnt = n_rows_elems(r0, r1)
                buf = (ctypes.c_char * (cnt * esize)).from_address(ptr)
                sink(r0, r1, np.frombuffer(buf, dtype=dt, count=cnt))
                return 0
            except BaseException as e:  # re-raised after the call returns
                err.append(e)
                return 1
        cb = _SINK(_cb)
    st = call(cb if cb is not None else _SINK())
    if err:
        raise err[0]
    return st


def pcc_allpairs_upper_host(Z: Zmat, R_host=None, device_bytes: int = 0,
                            sink=None, stream=None):
    """The packed triangle into host memory in overlapped passes; R_host a
    numpy float32 array of n(n-1)/2 (float64 for the FP64 form) or None
    with a sink(row_begin, row_end, slice) taking each packed slice."""
    info = Z.info()
    n = info["n"]
    hp, f64, size = _host_buffer(R_host)
    rt = PCC_F64 if f64 else PCC_F32
    if R_host is not None:
        assert size == n * (n - 1) // 2

    def elems(r0, r1):
        return r1 * (2 * n - r1 - 1) // 2 - r0 * (2 * n - r0 - 1) // 2

    st = _host_stream(
        lambda cb: load().pcc_allpairs_upper_host(
            Z.handle, hp, rt, int(device_bytes), cb, None, _stream(stream)),
        elems, 8 if f64 else 4, sink)
    _check(st, "pcc_allpairs_upper_host")
    return R_host


def pcc_threshold_edges_host(Z: Zmat, tau: float, edges, capacity: int,
                             d_count, R_host=None, device_bytes: int = 0,
                             sink=None, stream=None):
    """pcc_threshold_edges with the packed FP32 triangle delivered to host
    memory in overlapped passes (R_host: numpy/pinned float32 of n(n-1)/2,
    or a tensor on the host; None with a sink)."""
    n = Z.info()["n"]

    def elems(r0, r1):
        return r1 * (2 * n - r1 - 1) // 2 - r0 * (2 * n - r0 - 1) // 2

    hp, _, _ = _host_buffer(R_host)
    st = _host_stream(
        lambda cb: load().pcc_threshold_edges_host(
            Z.handle, float(tau), _ptr(edges), int(capacity), _ptr(d_count),
            hp, int(device_bytes), cb, None, _stream(stream)),
        elems, 4, sink)
    _check(st, "pcc_threshold_edges_host")
    return R_host


def pcc_cross_allpairs_host(ZX: Zmat, ZY: Zmat, R_host=None,
                            device_bytes: int = 0, sink=None, stream=None):
    """Dense cross matrix into host memory in overlapped passes; R_host a
    2-D numpy array (nx x >= ny, unit inner stride) or None with a sink."""
    ny = ZY.info()["n"]
    hp, f64, _ = (_host_buffer(R_host) if R_host is None
                  or hasattr(R_host, "data_ptr") else
                  (ctypes.c_void_p(R_host.ctypes.data),
                   R_host.dtype.itemsize == 8, R_host.size))
    rt = PCC_F64 if f64 else PCC_F32
    esize = 8 if f64 else 4
    if R_host is None:
        ldr = ny
    elif hasattr(R_host, "data_ptr"):
        ldr = R_host.stride(0)
    else:
        ldr = R_host.strides[0] // esize
    st = _host_stream(
        lambda cb: load().pcc_cross_allpairs_host(
            ZX.handle, ZY.handle, hp, rt, int(ldr), int(device_bytes), cb,
            None, _stream(stream)),
        lambda r0, r1: (r1 - r0) * ldr if R_host is not None
        else (r1 - r0) * ny, esize, sink)
    _check(st, "pcc_cross_allpairs_host")
    return R_host


def pcc_perm_test(Z: Zmat, d_perms, P: int, k0: int, k1: int, d_counts,
                  stream=None):
    _check(load().pcc_perm_test(Z.handle, _ptr(d_perms), int(P), int(k0),
                                int(k1), _ptr(d_counts), _stream(stream)),
           "pcc_perm_test")


_FORM_NAMES = {PCC_PREC_BF16X3: "bf16x3", PCC_PREC_FP16X3S: "fp16x3s",
               PCC_PREC_BF16X4: "bf16x4", PCC_PREC_BF16X1: "bf16x1"}


def pcc_allpairs_upper_batched(Zs, Rs, stream=None, choices="auto",
                               cache=None):
    """All pairs of many standardized matrices (pcc.h).  choices:
      "auto"  (default) each matrix gets the tuner's best CTA form and band
              rows for its shape when the tune cache (autotune.cache_path()
              or `cache`, a path or a loaded dict) has an entry for it; the
              others run under the current knobs;
      None    every matrix under the current knobs;
      a list  (pair, band_rows) per matrix.
    Returns the list of (pair, band_rows) used per matrix."""
    B = len(Zs)
    harr = (ctypes.c_void_p * B)(*[z.handle.value for z in Zs])
    rarr = (ctypes.c_void_p * B)(*[r.data_ptr() for r in Rs])
    t = pcc_get_tuning()
    default = (1 if t["pair_mma"] and t["cluster"] == 2 else 0,
               t["band_rows"])
    if choices is None:
        used = [default] * B
    elif isinstance(choices, str) and choices == "auto":
        from . import autotune
        c = autotune.load_cache(cache) if cache is None or \
            isinstance(cache, str) else cache
        used = []
        for z in Zs:
            info = z.info()
            form = _FORM_NAMES.get(info["prec"])  # others: rejected below
            b = None if form is None else autotune.lookup_batched(
                info["n"], info["l"], form, c, stage_k=t["stage_k"])
            used.append(b if b is not None else default)
    else:
        used = [(int(p), int(g)) for p, g in choices]
        if len(used) != B:
            raise ValueError("one (pair, band_rows) per matrix")
    pa = (_I32 * B)(*[u[0] for u in used])
    ga = (_I32 * B)(*[u[1] for u in used])
    _check(load().pcc_allpairs_upper_batched_tuned(harr, B, rarr, pa, ga,
                                                   _stream(stream)),
           "pcc_allpairs_upper_batched_tuned")
    return used


def pcc_allpairs_upper_noalloc(X, R, prec="auto", d_status=None,
                               stream=None):
    """All pairs of the device FP32 matrix X into R without any device
    allocation (the standardized matrix lives in the library's fixed 32 MiB
    device array); see include/pcc.h for the size limit."""
    assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
    _check(load().pcc_allpairs_upper_noalloc(
        _ptr(X), X.shape[0], X.shape[1], X.stride(0), _prec(prec), _ptr(R),
        _ptr(d_status), _stream(stream)), "pcc_allpairs_upper_noalloc")
    return R


def pcc_sync_status(Z: Zmat, stream=None) -> int:
    return int(load().pcc_sync_status(Z.handle, _stream(stream)))


def pcc_set_wait_limit_ns(ns: int):
    _check(load().pcc_set_wait_limit_ns(int(ns)), "pcc_set_wait_limit_ns")


def pcc_debug_drop_loads(enable):
    """Test hook: make the pair kernel's operand waits run out (see pcc.h).
    True/1: no producer issues loads; 2 / 3: only the odd / even CTA of each
    CTA pair issues none."""
    _check(load().pcc_debug_drop_loads(int(enable)), "pcc_debug_drop_loads")


def pcc_set_tuning(stage_k=0, cluster=0, band_rows=0, cost_c0=0.0,
                   cost_c1=0.0, pair_mma=None, perm_form=None):
    """Zeros (and None) keep a value; pair_mma 1/0 selects CTA pairs running
    one 2-SM MMA or independent CTAs (pcc_set_pair_mma); perm_form selects
    the form of the permutation test (pcc_set_perm_form):
    PCC_PERM_TRANSPOSED (the default), PCC_PERM_WORKSPACE or
    PCC_PERM_SMEM."""
    _check(load().pcc_set_tuning(int(stage_k), int(cluster), int(band_rows),
                                 float(cost_c0), float(cost_c1)),
           "pcc_set_tuning")
    if pair_mma is not None:
        _check(load().pcc_set_pair_mma(int(pair_mma)), "pcc_set_pair_mma")
    if perm_form is not None:
        _check(load().pcc_set_perm_form(int(perm_form)),
               "pcc_set_perm_form")


def pcc_measure_fp32_fma(stream=None) -> float:
    """Measured FP32 FMA rate of the device's CUDA cores, TFLOP/s."""
    v = ctypes.c_double()
    _check(load().pcc_measure_fp32_fma(ctypes.byref(v), _stream(stream)),
           "pcc_measure_fp32_fma")
    return v.value


def pcc_get_tuning() -> dict:
    k, c, b = _I32(), _I32(), _I32()
    c0, c1 = ctypes.c_double(), ctypes.c_double()
    _check(load().pcc_get_tuning(ctypes.byref(k), ctypes.byref(c),
                                 ctypes.byref(b), ctypes.byref(c0),
                                 ctypes.byref(c1)), "pcc_get_tuning")
    return dict(stage_k=k.value, cluster=c.value, band_rows=b.value,
                cost_c0=c0.value, cost_c1=c1.value,
                pair_mma=int(load().pcc_get_pair_mma()),
                perm_form=int(load().pcc_get_perm_form()))


def pcc_num_pairs(n: int) -> int:
    return int(load().pcc_num_pairs(n))


def pcc_pair_index(n: int, i: int, j: int) -> int:
    return int(load().pcc_pair_index(n, i, j))


def pcc_pair_coords(n: int, J: int):
    i, j = _I64(), _I64()
    _check(load().pcc_pair_coords(n, J, ctypes.byref(i), ctypes.byref(j)),
           "pcc_pair_coords")
    return i.value, j.value


def pcc_tile_coords(m: int, Jt: int):
    y, x = _I64(), _I64()
    _check(load().pcc_tile_coords(m, Jt, ctypes.byref(y), ctypes.byref(x)),
           "pcc_tile_coords")
    return y.value, x.value


def pcc_schedule_num_tiles(n: int, prec="auto") -> int:
    return int(load().pcc_schedule_num_tiles(int(n), _prec(prec)))


def pcc_schedule_tile_rect(n: int, prec, tile: int):
    """(row0, row1, col0, col1) of a tile of the pair schedule (host)."""
    v = [_I64() for _ in range(4)]
    _check(load().pcc_schedule_tile_rect(int(n), _prec(prec), int(tile),
                                         *[ctypes.byref(x) for x in v]),
           "pcc_schedule_tile_rect")
    return tuple(x.value for x in v)


def pcc_status_string(s: int) -> str:
    return load().pcc_status_string(int(s)).decode()


def edges_view(edges_u8, count: int):
    """Split a pcc_edge byte buffer (torch uint8, on any device) into (i, j,
    r) numpy arrays of the first `count` records."""
    import numpy as np
    raw = edges_u8[:count * EDGE_BYTES].cpu().numpy().view(np.uint8)
    rec = raw.view(np.dtype([("i", "<u4"), ("j", "<u4"), ("r", "<f4")]))
    return (rec["i"].astype(np.int64), rec["j"].astype(np.int64),
            rec["r"].astype(np.float32))
