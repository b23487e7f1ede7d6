"""GB300 OptA template search: Python binding of libopta.so.

Thin marshalling layer over the C ABI declared in include/opta.h (same
names).  Images and templates may be numpy arrays (host) or torch tensors
(host or CUDA); streams are torch.cuda.Stream objects, raw cudaStream_t
integers or None (the current torch stream when torch has CUDA, else the
legacy default stream).  Nothing here computes any part of the search.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_float, c_int32, c_int64, c_size_t, c_void_p

from . import _lib
from ._lib import OptaImage, OptaParams, OptaResult, OptaSizeInfo, OptaTemplate, STATUS

__all__ = [
    "OptaError", "opta_params_default", "optA_prepare", "optA_search", "zncc_full",
    "zncc_full_noalloc",
    "optA_debug_bounds", "optA_size_info", "optA_memory_bytes", "optA_destroy",
    "optA_debug_maps", "opta_dbg_window_stats", "opta_dbg_blur", "opta_dbg_blur_corr", "opta_dbg_i64_to_f32",
    "opta_dbg_survivors", "opta_dbg_survivor_lane_min",
    "opta_dbg_rho_co", "opta_dbg_launch_count", "opta_dbg_profile_enable", "opta_dbg_scan1_wait",
    "opta_dbg_profile_read", "optA_debug_scan1", "Handle", "lib", "OptaResult", "SearchContext", "SearchGraph", "Server",
]

lib = _lib.lib


class OptaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        name = STATUS.get(self.code, str(code))
        super().__init__(f"{what}: {name}" if what else name)


def _check(code: int, what: str):
    if code != 0:
        raise OptaError(code, what)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return c_void_p(0)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _array_desc(a, kind):
    """(rows, cols, stride_elems, dtype_code, on_device, ptr, keepalive)."""
    if _is_torch(a):
        import torch
        if a.dim() != 2 or a.stride(1) != 1:
            raise ValueError(f"{kind} must be a 2-D tensor with unit column stride")
        if a.dtype == torch.uint8:
            code = _lib.OPTA_U8
        elif a.dtype == torch.float32:
            code = _lib.OPTA_F32
        else:
            raise TypeError(f"{kind} dtype must be uint8 or float32")
        return a.shape[0], a.shape[1], a.stride(0), code, int(a.is_cuda), a.data_ptr(), a
    import numpy as np
    a = np.asarray(a)
    if a.ndim != 2:
        raise ValueError(f"{kind} must be 2-D")
    if a.dtype not in (np.uint8, np.float32) or a.strides[1] != a.itemsize:
        a = np.ascontiguousarray(a, dtype=np.float32 if a.dtype != np.uint8 else np.uint8)
    code = _lib.OPTA_U8 if a.dtype == np.uint8 else _lib.OPTA_F32
    return a.shape[0], a.shape[1], a.strides[0] // a.itemsize, code, 0, a.ctypes.data, a


def _image(a):
    r, c, s, code, dev, ptr, keep = _array_desc(a, "image")
    return OptaImage(r, c, s, code, dev, ptr), keep


def _template(a):
    r, c, s, code, dev, ptr, keep = _array_desc(a, "template")
    if code != _lib.OPTA_F32:
        if _is_torch(keep):
            keep = keep.float()
            s = keep.stride(0); ptr = keep.data_ptr()
        else:
            import numpy as np
            keep = np.ascontiguousarray(keep, dtype=np.float32)
            s = keep.strides[0] // 4; ptr = keep.ctypes.data
    return OptaTemplate(r, c, s, dev, 0, ptr), keep


def opta_params_default(**overrides) -> OptaParams:
    """Section 7 defaults, with keyword overrides (sigma_levels as a sequence)."""
    p = OptaParams()
    lib().opta_params_default(byref(p))
    for k, v in overrides.items():
        if k == "sigma_levels":
            v = list(v)
            p.n_levels = len(v)
            for i in range(8):
                p.sigma_levels[i] = float(v[i]) if i < len(v) else 0.0
        else:
            setattr(p, k, v)
    return p


class Handle:
    """Owns an opta_handle*; released by close() or garbage collection."""

    def __init__(self, ptr: int, rows: int, cols: int):
        self._ptr = c_void_p(ptr)
        self.rows, self.cols = rows, cols

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("handle closed")
        return self._ptr

    def close(self):
        if self._ptr:
            lib().optA_destroy(self._ptr)
            self._ptr = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def optA_prepare(image, params: OptaParams | None = None, sizes=None, stream=None) -> Handle:
    img, keep = _image(image)
    sz = list(sizes or [])
    arr = (c_int32 * (2 * len(sz) or 1))()
    for i, s in enumerate(sz):
        m, n = (s, s) if isinstance(s, int) else s
        arr[2 * i], arr[2 * i + 1] = int(m), int(n)
    out = c_void_p(0)
    code = lib().optA_prepare(byref(img), byref(params) if params is not None else None,
                              arr if sz else None, len(sz), _stream(stream), byref(out))
    del keep
    _check(code, "optA_prepare")
    return Handle(out.value, img.rows, img.cols)


class SearchContext:
    """Owns an opta_search_ctx*: search scratch usable with any handle on the
    device of the handle it is created with (see optA_ctx_create)."""

    def __init__(self, handle: Handle):
        out = c_void_p(0)
        _check(lib().optA_ctx_create(handle.ptr, byref(out)), "optA_ctx_create")
        self._ptr = out

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("context closed")
        return self._ptr

    def memory_bytes(self) -> int:
        b = c_size_t(0)
        _check(lib().optA_ctx_memory_bytes(self.ptr, byref(b)), "optA_ctx_memory_bytes")
        return b.value

    def close(self):
        if self._ptr:
            _check(lib().optA_ctx_destroy(self._ptr), "optA_ctx_destroy")
            self._ptr = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def optA_search(handle: Handle, templates, stream=None, check: bool = True,
                ctx: SearchContext | None = None):
    """Best match per template: list of OptaResult (status per template).
    With `ctx`, the search runs through that context (optA_search_ctx)."""
    if not isinstance(templates, (list, tuple)):
        templates = [templates]
    n = len(templates)
    descs = (OptaTemplate * max(n, 1))()
    keep = []
    for i, t in enumerate(templates):
        d, k = _template(t)
        descs[i] = d
        keep.append(k)
    out = (OptaResult * max(n, 1))()
    if ctx is None:
        code = lib().optA_search(handle.ptr, descs, n, out, _stream(stream))
    else:
        code = lib().optA_search_ctx(handle.ptr, ctx.ptr, descs, n, out, _stream(stream))
    if check and code not in (0, 2):
        raise OptaError(code, "optA_search")
    return [out[i] for i in range(n)]


class SearchGraph:
    """optA_graph_*: the batched search of a fixed list of template sizes
    captured as one CUDA graph; set(i, t) replaces template i's data,
    launch() replays the graph and returns the results."""

    def __init__(self, handle: Handle, templates, stream=None):
        n = len(templates)
        descs = (OptaTemplate * n)()
        keep = []
        for i, t in enumerate(templates):
            d, k = _template(t)
            descs[i] = d
            keep.append(k)
        out = c_void_p(0)
        _check(lib().optA_graph_create(handle.ptr, descs, n, _stream(stream), byref(out)),
               "optA_graph_create")
        del keep
        self._ptr, self.n, self._handle = out, n, handle

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("graph closed")
        return self._ptr

    def set(self, i: int, template, stream=None):
        """Replace template i's data (same size).  A host array is copied
        before the call returns; a device tensor is copied on `stream`, so
        launch on the same stream (and keep the tensor until then)."""
        d, keep = _template(template)
        _check(lib().optA_graph_set_template(self.ptr, i, byref(d), _stream(stream)),
               "optA_graph_set_template")
        return keep

    def launch(self, stream=None, check: bool = True):
        out = (OptaResult * self.n)()
        code = lib().optA_graph_launch(self.ptr, out, _stream(stream))
        if check and code not in (0, 2):
            raise OptaError(code, "optA_graph_launch")
        return [out[i] for i in range(self.n)]

    def nodes(self) -> int:
        n = c_int64(0)
        _check(lib().optA_graph_info(self.ptr, byref(n)), "optA_graph_info")
        return n.value

    def close(self):
        if self._ptr:
            lib().optA_graph_destroy(self._ptr)
            self._ptr = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop of include/opta_serve.h: resident prepared images,
    template queries batched by worker threads as they arrive, admission by
    a device-memory budget.  Templates are host arrays (copied on submit)."""

    def __init__(self, n_workers: int = 4, max_batch: int = 64, memory_budget: int = 0):
        from ._lib import OptaServerConfig
        cfg = OptaServerConfig()
        lib().opta_server_config_default(byref(cfg))
        cfg.n_workers, cfg.max_batch, cfg.memory_budget = n_workers, max_batch, memory_budget
        out = c_void_p(0)
        _check(lib().opta_server_create(byref(cfg), byref(out)), "opta_server_create")
        self._ptr = out

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("server closed")
        return self._ptr

    def add_image(self, image, params: OptaParams | None = None, sizes=None) -> int:
        img, keep = _image(image)
        sz = list(sizes or [])
        arr = (c_int32 * (2 * len(sz) or 1))()
        for i, sm in enumerate(sz):
            m, n = (sm, sm) if isinstance(sm, int) else sm
            arr[2 * i], arr[2 * i + 1] = int(m), int(n)
        iid = c_int32(0)
        code = lib().opta_server_add_image(self.ptr, byref(img),
                                           byref(params) if params is not None else None,
                                           arr if sz else None, len(sz), byref(iid))
        del keep
        _check(code, "opta_server_add_image")
        return iid.value

    def submit(self, image_id: int, template) -> int:
        import numpy as np
        t = np.ascontiguousarray(template, dtype=np.float32)
        d = OptaTemplate(t.shape[0], t.shape[1], t.shape[1], 0, 0, t.ctypes.data)
        rid = ctypes.c_uint64(0)
        _check(lib().opta_server_submit(self.ptr, image_id, byref(d), byref(rid)), "opta_server_submit")
        return rid.value

    def wait(self, min_count: int = 1, capacity: int = 1024, timeout_ms: int = -1):
        """Finished requests (OptaCompletion list, oldest first)."""
        from ._lib import OptaCompletion
        buf = (OptaCompletion * max(capacity, 1))()
        n = c_int32(0)
        _check(lib().opta_server_wait(self.ptr, buf, capacity, min_count, timeout_ms, byref(n)),
               "opta_server_wait")
        return [buf[i] for i in range(n.value)]

    def memory(self, image_id: int):
        """(device bytes of the resident image, bytes of the workers' scratch)."""
        a, b = c_int64(0), c_int64(0)
        _check(lib().opta_server_memory(self.ptr, image_id, byref(a), byref(b)), "opta_server_memory")
        return a.value, b.value

    def pending(self) -> int:
        n = c_int64(0)
        _check(lib().opta_server_pending(self.ptr, byref(n)), "opta_server_pending")
        return n.value

    def close(self):
        if self._ptr:
            lib().opta_server_destroy(self._ptr)
            self._ptr = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def zncc_full(image, template, rho_map=None, stream=None, check: bool = True) -> OptaResult:
    """Exhaustive search; rho_map (optional) is a CUDA float32 tensor of L elements."""
    img, k1 = _image(image)
    t, k2 = _template(template)
    res = OptaResult()
    ptr = c_void_p(rho_map.data_ptr()) if rho_map is not None else c_void_p(0)
    code = lib().zncc_full(byref(img), byref(t), ptr, byref(res), _stream(stream))
    del k1, k2
    if check and code not in (0, 2):
        raise OptaError(code, "zncc_full")
    return res


def zncc_full_noalloc(image, template, rho_map=None, stream=None, check: bool = True) -> OptaResult:
    """zncc_full on the library's fixed device scratch: no device allocation.

    For callers that must not allocate device memory during a search (see
    include/opta.h for the limits and the one-time set-up per device)."""
    img, k1 = _image(image)
    t, k2 = _template(template)
    res = OptaResult()
    ptr = c_void_p(rho_map.data_ptr()) if rho_map is not None else c_void_p(0)
    code = lib().zncc_full_noalloc(byref(img), byref(t), ptr, byref(res), _stream(stream))
    del k1, k2
    if check and code not in (0, 2):
        raise OptaError(code, "zncc_full_noalloc")
    return res


def optA_debug_bounds(handle: Handle, template, ub_map=None, survived=None, stream=None) -> int:
    t, k = _template(template)
    code = lib().optA_debug_bounds(handle.ptr, byref(t),
                                   c_void_p(ub_map.data_ptr() if ub_map is not None else 0),
                                   c_void_p(survived.data_ptr() if survived is not None else 0),
                                   _stream(stream))
    del k
    if code not in (0, 2):
        raise OptaError(code, "optA_debug_bounds")
    return code


def opta_dbg_survivors(handle: Handle, template, idx_dev, rho_dev, eps_dev, form: int = -1,
                       stream=None) -> int:
    """rho and its error bound at the locations idx_dev (int32 device tensor of
    linear indices) by survivor form `form` (0 lane, 1 warp, -1 the search's);
    returns the status (0, or 2 for a flat template)."""
    t, k = _template(template)
    n = idx_dev.numel()
    code = lib().opta_dbg_survivors(handle.ptr, byref(t), c_void_p(idx_dev.data_ptr() if n else 0), n,
                                    int(form), c_void_p(rho_dev.data_ptr() if n else 0),
                                    c_void_p(eps_dev.data_ptr() if n else 0), _stream(stream))
    del k
    if code not in (0, 2):
        raise OptaError(code, "opta_dbg_survivors")
    return code


def opta_dbg_survivor_lane_min(m: int, n: int, u8: bool) -> tuple:
    """(lane_min, tuned) of an m x n size on the current device: sweeps with at
    least lane_min entries take the lane form; tuned: measured by the tuner."""
    lm, tu = c_int32(0), c_int32(0)
    _check(lib().opta_dbg_survivor_lane_min(m, n, 1 if u8 else 0, byref(lm), byref(tu)),
           "opta_dbg_survivor_lane_min")
    return int(lm.value), bool(tu.value)


def optA_size_info(handle: Handle, m: int, n: int) -> dict:
    info = OptaSizeInfo()
    _check(lib().optA_size_info(handle.ptr, m, n, byref(info)), "optA_size_info")
    return info.as_dict()


def optA_memory_bytes(handle: Handle) -> int:
    b = c_size_t(0)
    _check(lib().optA_memory_bytes(handle.ptr, byref(b)), "optA_memory_bytes")
    return int(b.value)


def optA_destroy(handle: Handle) -> None:
    handle.close()


def optA_debug_maps(handle: Handle, m: int, n: int, pivot=None, rho_co=None, stream=None):
    """Copies the prepared pivot image / rho_co map into CUDA tensors; returns the sigma map."""
    import numpy as np
    by = (handle.rows + 63) // 64
    info = optA_size_info(handle, m, n)
    smap = np.zeros((info["blocks_y"], info["blocks_x"]), dtype=np.float32)
    _check(lib().optA_debug_maps(handle.ptr, m, n,
                                 c_void_p(pivot.data_ptr() if pivot is not None else 0),
                                 c_void_p(rho_co.data_ptr() if rho_co is not None else 0),
                                 smap.ctypes.data_as(ctypes.POINTER(c_float)), _stream(stream)),
           "optA_debug_maps")
    del by
    return smap


def opta_dbg_window_stats(I_dev, m: int, n: int, inv_sigma_dev, stream=None):
    p, q = I_dev.shape
    _check(lib().opta_dbg_window_stats(c_void_p(I_dev.data_ptr()), p, q, m, n,
                                       c_void_p(inv_sigma_dev.data_ptr()), _stream(stream)),
           "opta_dbg_window_stats")


def opta_dbg_blur(I_dev, sigma_map, block: int, P_dev, stream=None):
    import numpy as np
    p, q = I_dev.shape
    sm = np.ascontiguousarray(sigma_map, dtype=np.float32)
    _check(lib().opta_dbg_blur(c_void_p(I_dev.data_ptr()), p, q,
                               sm.ctypes.data_as(ctypes.POINTER(c_float)), block,
                               c_void_p(P_dev.data_ptr()), _stream(stream)), "opta_dbg_blur")


def opta_dbg_i64_to_f32(v_dev, out_dev, stream=None):
    _check(lib().opta_dbg_i64_to_f32(c_void_p(v_dev.data_ptr()), c_void_p(out_dev.data_ptr()),
                                     v_dev.numel(), _stream(stream)), "opta_dbg_i64_to_f32")


def opta_dbg_blur_corr(P_dev, I_dev, m: int, n: int, R_dev, lam: float = 0.0, block: int = 64,
                       fail_dev=None, stream=None):
    p, q = I_dev.shape
    _check(lib().opta_dbg_blur_corr(c_void_p(P_dev.data_ptr()), c_void_p(I_dev.data_ptr()),
                                    p, q, m, n, c_void_p(R_dev.data_ptr() if R_dev is not None else 0),
                                    c_float(lam), block,
                                    c_void_p(fail_dev.data_ptr() if fail_dev is not None else 0),
                                    _stream(stream)),
           "opta_dbg_blur_corr")


def opta_dbg_rho_co(P_dev, I_dev, m: int, n: int, h: int, rco_dev=None, rho_cut: float = 0.6,
                    stream=None) -> int:
    p, q = I_dev.shape
    cnt = c_int64(0)
    _check(lib().opta_dbg_rho_co(c_void_p(P_dev.data_ptr()), c_void_p(I_dev.data_ptr()), p, q,
                                 m, n, h, c_void_p(rco_dev.data_ptr() if rco_dev is not None else 0),
                                 c_double(rho_cut), byref(cnt), _stream(stream)), "opta_dbg_rho_co")
    return int(cnt.value)


def opta_dbg_scan1_wait(wait_ns: int = 0, stall: bool = False) -> None:
    """Budget of scan 1's waits for progress (0: the default) and its stall
    switch (include/opta_debug.h); for the failure-detection test."""
    lib().opta_dbg_scan1_wait(int(wait_ns), 1 if stall else 0)


def opta_dbg_launch_count() -> int:
    """Kernel launches issued by the library so far in this process."""
    return int(lib().opta_dbg_launch_count())


def opta_dbg_profile_enable(on: bool = True) -> None:
    lib().opta_dbg_profile_enable(1 if on else 0)


def opta_dbg_profile_read(capacity: int = 64) -> dict:
    """{kernel_name: (total_ms, launches)} recorded since the last read."""
    stride = 64
    names = ctypes.create_string_buffer(stride * capacity)
    tot = (c_double * capacity)()
    cnt = (c_int64 * capacity)()
    n = lib().opta_dbg_profile_read(names, stride, tot, cnt, capacity)
    out = {}
    for i in range(min(n, capacity)):
        nm = names.raw[i * stride:(i + 1) * stride].split(b"\0", 1)[0].decode()
        out[nm] = (float(tot[i]), int(cnt[i]))
    return out


def optA_debug_scan1(handle: Handle, templates, rho_out, theta_out=None, stream=None) -> None:
    """Scan 1 of same-size templates: rho(t, pivot) per centre into CUDA tensors."""
    n = len(templates)
    descs = (OptaTemplate * n)()
    keep = []
    for i, t in enumerate(templates):
        d, k = _template(t)
        descs[i] = d
        keep.append(k)
    _check(lib().optA_debug_scan1(handle.ptr, descs, n, c_void_p(rho_out.data_ptr()),
                                  c_void_p(theta_out.data_ptr() if theta_out is not None else 0),
                                  _stream(stream)), "optA_debug_scan1")
