"""Thin Python binding of ``libhpdr.so`` (the C ABI in ``include/hpdr.h``).

Argument marshalling only: every step of the reduction runs in the library's
CUDA kernels.  Tensors are PyTorch CUDA tensors (PyTorch supplies device memory
and the current stream); the library must have been built
(``__graft_entry__.build()``) -- a missing library is an error, there is no
fallback.

Function names follow the C ABI:
  hpdr_compress, hpdr_decompress, hpdr_inspect, hpdr_compress_bound,
  hpdr_decompose, hpdr_recompose, hpdr_recompose_adjoint,
  hpdr_decompose_adjoint, hpdr_huffman_encode, hpdr_huffman_decode,
  hpdr_decompose_noalloc, hpdr_debug_set_wait_limit.
"""
import ctypes as C
import math
import os
import numpy as np

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpdr.so")

F32, F64 = 0, 1
LINF, L2, L2_STAT = 0, 1, 2
ABS, REL = 0, 1
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "output buffer too small",
          -4: "malformed container", -5: "device wait timed out", -6: "device allocation failed"}


class HpdrError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s: %s (status %d)" % (what, STATUS.get(status, "?"), status))
        self.status = status


class Config(C.Structure):
    _fields_ = [("dict_size", C.c_uint32), ("chunk", C.c_uint32)]


class PipelineModel(C.Structure):
    """Adaptive pipeline model (Sec. V-C): Phi(C) = alpha*C + beta below
    c_threshold bytes, gamma above (bytes/s); Theta(t) = t * h2d bytes."""
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("c_threshold", C.c_double), ("h2d", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Field(C.Structure):
    _fields_ = [("d_in", C.c_void_p), ("dtype", C.c_int), ("ndim", C.c_int), ("dims", C.c_size_t * 3),
                ("tol", C.c_double), ("tol_kind", C.c_int), ("mode", C.c_int)]


_lib = None
_ctx = {}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhpdr.so is not built: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.POINTER(C.c_size_t)
        sigs = {
            "hpdr_ctx_create": [C.POINTER(vp), C.c_int],
            "hpdr_ctx_destroy": [vp],
            "hpdr_compress": [vp, vp, C.c_int, C.c_int, sz, C.c_double, C.c_int, C.c_int,
                              C.POINTER(Config), vp, C.c_size_t, sz, vp],
            "hpdr_decompress": [vp, vp, C.c_size_t, vp, C.c_size_t, vp],
            "hpdr_inspect": [vp, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int), sz],
            "hpdr_decompose": [vp, vp, vp, C.c_int, C.c_int, sz, vp],
            "hpdr_recompose": [vp, vp, vp, C.c_int, C.c_int, sz, vp],
            "hpdr_compress_coords": [vp, vp, C.c_int, C.c_int, sz, C.POINTER(C.c_double), C.c_double, C.c_int,
                                     C.c_int, C.POINTER(Config), vp, C.c_size_t, sz, vp],
            "hpdr_decompose_coords": [vp, vp, vp, C.c_int, C.c_int, sz, C.POINTER(C.c_double), vp],
            "hpdr_recompose_coords": [vp, vp, vp, C.c_int, C.c_int, sz, C.POINTER(C.c_double), vp],
            "hpdr_recompose_adjoint_coords": [vp, vp, vp, C.c_int, C.c_int, sz, C.POINTER(C.c_double), vp],
            "hpdr_decompose_adjoint_coords": [vp, vp, vp, C.c_int, C.c_int, sz, C.POINTER(C.c_double), vp],
            "hpdr_recompose_adjoint": [vp, vp, vp, C.c_int, C.c_int, sz, vp],
            "hpdr_decompose_adjoint": [vp, vp, vp, C.c_int, C.c_int, sz, vp],
            "hpdr_huffman_encode": [vp, vp, C.c_uint64, C.c_uint32, C.c_uint32, vp, vp, vp,
                                    C.c_uint64, C.POINTER(C.c_uint64), vp],
            "hpdr_huffman_decode": [vp, vp, C.c_uint64, vp, C.c_uint64, C.c_uint32, C.c_uint32,
                                    vp, vp, vp],
            "hpdr_decompose_noalloc": [vp, vp, C.c_int, C.c_int, sz, vp],
            "hpdr_compress_async": [vp, vp, C.c_int, C.c_int, sz, C.c_double, C.c_int, C.c_int,
                                    C.POINTER(Config), vp, C.c_size_t, vp, vp],
            "hpdr_decompress_async": [vp, vp, C.c_size_t, C.c_int, C.c_int, sz, C.POINTER(Config), vp,
                                      C.c_size_t, vp, vp],
            "hpdr_device_status": [C.c_uint64],
            "hpdr_compress_host_streamed": [vp, vp, C.c_int, C.c_int, sz, C.c_double, C.c_int, C.c_int,
                                            C.POINTER(Config), C.c_size_t, vp, C.c_size_t, sz],
            "hpdr_decompress_host_streamed": [vp, vp, C.c_size_t, vp, C.c_size_t],
            "hpdr_compress_batched": [vp, C.c_int, C.POINTER(Field), C.POINTER(Config), vp, C.c_size_t,
                                      sz, sz, vp],
            "hpdr_batched_streams": [vp],
            "hpdr_batched_cached": [vp],
            "hpdr_lossless_compress": [vp, vp, C.c_uint64, C.c_int, C.c_uint32, vp, C.c_size_t, sz, vp],
            "hpdr_lossless_decompress": [vp, vp, C.c_size_t, vp, C.c_size_t, vp],
            "hpdr_lossless_inspect": [vp, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_uint64)],
            "hpdr_zfp_compress": [vp, vp, C.c_int, C.c_int, sz, C.c_uint32, vp, C.c_size_t, sz, vp],
            "hpdr_zfp_decompress": [vp, vp, C.c_size_t, vp, C.c_size_t, vp],
            "hpdr_zfp_inspect": [vp, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int), sz,
                                 C.POINTER(C.c_uint32)],
            "hpdr_pipeline_fit": [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_double,
                                  C.c_double, C.POINTER(PipelineModel)],
            "hpdr_pipeline_profile": [vp, vp, C.c_int, C.c_int, sz, C.c_double, C.c_int, C.c_int,
                                      C.POINTER(Config), sz, C.c_int, C.c_int, C.c_double,
                                      C.POINTER(PipelineModel)],
            "hpdr_compress_host_adaptive": [vp, vp, C.c_int, C.c_int, sz, C.c_double, C.c_int, C.c_int,
                                            C.POINTER(Config), C.POINTER(PipelineModel), C.c_size_t,
                                            C.c_size_t, vp, C.c_size_t, sz],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.hpdr_compress_bound.argtypes = [C.c_int, sz, C.c_int, C.POINTER(Config)]
        L.hpdr_compress_bound.restype = C.c_size_t
        L.hpdr_lossless_bound.argtypes = [C.c_uint64, C.c_int, C.c_uint32]
        L.hpdr_lossless_bound.restype = C.c_size_t
        L.hpdr_pipeline_plan.argtypes = [C.POINTER(PipelineModel), C.c_size_t, C.c_size_t, C.c_size_t,
                                          C.c_size_t, sz, C.c_size_t]
        L.hpdr_pipeline_plan.restype = C.c_size_t
        L.hpdr_streamed_bound.argtypes = [C.c_int, sz, C.c_int, C.POINTER(Config), sz, C.c_size_t]
        L.hpdr_streamed_bound.restype = C.c_size_t
        L.hpdr_status_string.argtypes = [C.c_int]
        L.hpdr_debug_set_wait_limit.argtypes = [C.c_int]
        L.hpdr_debug_set_wait_limit.restype = C.c_int
        L.hpdr_zfp_bound.restype = C.c_size_t
        L.hpdr_zfp_bound.argtypes = [C.c_int, sz, C.c_int, C.c_uint32]
        L.hpdr_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st, what):
    if st != 0:
        raise HpdrError(st, what)


def context(device=None):
    """Per-device library context (plans and workspaces are cached in it)."""
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _ctx:
        h = C.c_void_p()
        _check(lib().hpdr_ctx_create(C.byref(h), dev), "hpdr_ctx_create")
        _ctx[dev] = h
    return _ctx[dev]


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dims(shape):
    shape = tuple(int(s) for s in shape)
    return len(shape), (C.c_size_t * 3)(*(list(shape) + [1] * (3 - len(shape))))


def _dtype_code(t):
    if t == torch.float32:
        return F32
    if t == torch.float64:
        return F64
    raise TypeError("only float32 and float64 fields are supported, got %s" % t)


def _cfg(dict_size, chunk):
    return Config(int(dict_size), int(chunk))


def _dev_tensor(t, what):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA tensor" % what)
    return t


def _dev_buf(t, what, device, dtype=None, numel=0):
    """A tensor the library reads or writes whole: contiguous, on `device`, of
    `dtype` (element size checked when dtype is an int) and at least `numel`
    elements.  Several C entries are given no size for it (the element count
    follows from the shape), so a smaller tensor would be read or written
    past its end by the kernels: the check is made here, before the call."""
    _dev_tensor(t, what)
    if t.device != device:
        raise ValueError("%s is on %s, the call runs on %s" % (what, t.device, device))
    if isinstance(dtype, int):
        if t.element_size() != dtype:
            raise TypeError("%s must have %d-byte elements, got %s" % (what, dtype, t.dtype))
    elif dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if t.numel() < numel:
        raise ValueError("%s holds %d elements, %d are needed" % (what, t.numel(), numel))
    return t


def _host_buf(t, what):
    """A host tensor the library copies from or into (pinned memory lets the
    copies overlap the kernels; pageable memory works, with staged copies)."""
    if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CPU tensor" % what)
    return t


def _numel(shape):
    return math.prod(int(x) for x in shape)


def hpdr_compress_bound(shape, dtype=torch.float32, dict_size=8192, chunk=0):
    nd, dims = _dims(shape)
    cfg = _cfg(dict_size, chunk)
    return int(lib().hpdr_compress_bound(nd, dims, _dtype_code(dtype), C.byref(cfg)))


def _coords(coords, shape):
    """Node coordinates as one host double array (dimension 0's, then 1's,
    ...), or None for unit spacing.  `coords` is one 1-D sequence per
    dimension, of that dimension's length."""
    if coords is None:
        return None
    if len(coords) != len(shape):
        raise ValueError("coords needs one array per dimension")
    parts = []
    for k, c in enumerate(coords):
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
        if c.size != shape[k]:
            raise ValueError("coords[%d] has %d entries for a dimension of %d" % (k, c.size, shape[k]))
        parts.append(c)
    flat = np.ascontiguousarray(np.concatenate(parts))
    return flat, flat.ctypes.data_as(C.POINTER(C.c_double))


def hpdr_compress(u, tol, tol_kind=REL, mode=LINF, dict_size=8192, chunk=0, out=None,
                  stream=None, coords=None):
    """Compress a CUDA field; returns a uint8 CUDA tensor holding the
    container.  coords: optional node coordinates, one array per dimension
    (non-uniform grid); the container then carries them."""
    _dev_tensor(u, "u")
    nd, dims = _dims(u.shape)
    cfg = _cfg(dict_size, chunk)
    if out is None:
        out = torch.empty(hpdr_compress_bound(u.shape, u.dtype, dict_size, chunk), dtype=torch.uint8,
                          device=u.device)
    _dev_buf(out, "out", u.device, torch.uint8)
    nb = C.c_size_t()
    co = _coords(coords, tuple(u.shape))
    _check(lib().hpdr_compress_coords(context(u.device.index), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype),
                                      nd, dims, co[1] if co else None, float(tol), int(tol_kind), int(mode),
                                      C.byref(cfg), C.c_void_p(out.data_ptr()), out.numel(), C.byref(nb),
                                      _stream(stream)), "hpdr_compress")
    return out[:nb.value]


def hpdr_compress_async(u, tol, out, result, tol_kind=REL, mode=LINF, dict_size=8192, chunk=0, stream=None):
    """Queue a compression without any host wait: `out` (uint8 CUDA tensor of
    at least hpdr_compress_bound bytes) receives the container, `result` (int64
    CUDA tensor of 2) receives {container bytes, device status} when the stream
    gets there."""
    _dev_tensor(u, "u")
    _dev_buf(out, "out", u.device, torch.uint8)
    _dev_buf(result, "result", u.device, 8, 2)
    nd, dims = _dims(u.shape)
    cfg = _cfg(dict_size, chunk)
    _check(lib().hpdr_compress_async(context(u.device.index), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype), nd, dims,
                                     float(tol), int(tol_kind), int(mode), C.byref(cfg), C.c_void_p(out.data_ptr()),
                                     out.numel(), C.c_void_p(result.data_ptr()), _stream(stream)),
           "hpdr_compress_async")


def hpdr_decompress_async(buf, out, result, dict_size=8192, chunk=0, stream=None):
    """Queue a decompression whose header is parsed on the device: `out` has
    the field's shape and type (they must match the container), `result`
    (int64 CUDA tensor of 1) receives the device status."""
    _dev_tensor(buf, "buf")
    _dev_buf(out, "out", buf.device)
    _dev_buf(result, "result", buf.device, 8, 1)
    nd, dims = _dims(out.shape)
    cfg = _cfg(dict_size, chunk)
    _check(lib().hpdr_decompress_async(context(buf.device.index), C.c_void_p(buf.data_ptr()), buf.numel(),
                                       _dtype_code(out.dtype), nd, dims, C.byref(cfg), C.c_void_p(out.data_ptr()),
                                       out.numel() * out.element_size(), C.c_void_p(result.data_ptr()),
                                       _stream(stream)), "hpdr_decompress_async")


def device_status(code):
    """hpdr_status of a device status code (0: ok)."""
    return lib().hpdr_device_status(int(code))


def hpdr_inspect(buf):
    """(torch dtype, shape) of a container held in a CUDA or CPU uint8 tensor."""
    dt, nd = C.c_int(), C.c_int()
    dims = (C.c_size_t * 3)()
    _check(lib().hpdr_inspect(C.c_void_p(buf.data_ptr()), buf.numel(), C.byref(dt), C.byref(nd),
                              dims), "hpdr_inspect")
    return (torch.float32 if dt.value == F32 else torch.float64), tuple(dims[:nd.value])


def hpdr_decompress(buf, out=None, stream=None):
    _dev_tensor(buf, "buf")
    dt, shape = hpdr_inspect(buf)
    if out is None:
        out = torch.empty(shape, dtype=dt, device=buf.device)
    _dev_buf(out, "out", buf.device, dt, _numel(shape))
    _check(lib().hpdr_decompress(context(buf.device.index), C.c_void_p(buf.data_ptr()), buf.numel(),
                                 C.c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                                 _stream(stream)), "hpdr_decompress")
    return out


def _field_call(name, src, out, shape, stream):
    nd, dims = _dims(shape)
    _check(getattr(lib(), name)(context(src.device.index), C.c_void_p(src.data_ptr()),
                                C.c_void_p(out.data_ptr()), _dtype_code(src.dtype), nd, dims,
                                _stream(stream)), name)
    return out


def _coords_call(name, src, out, shape, coords, stream):
    nd, dims = _dims(shape)
    co = _coords(coords, tuple(shape))
    _check(getattr(lib(), name)(context(src.device.index), C.c_void_p(src.data_ptr()),
                                C.c_void_p(out.data_ptr()), _dtype_code(src.dtype), nd, dims,
                                co[1] if co else None, _stream(stream)), name)
    return out


def hpdr_decompose(u, out=None, stream=None, coords=None):
    """Level-major coefficient stream (1-D tensor) of the field u (coords:
    optional node coordinates, one array per dimension)."""
    _dev_tensor(u, "u")
    if out is None:
        out = torch.empty(u.numel(), dtype=u.dtype, device=u.device)
    _dev_buf(out, "out", u.device, u.dtype, u.numel())
    if coords is not None:
        return _coords_call("hpdr_decompose_coords", u, out, u.shape, coords, stream)
    return _field_call("hpdr_decompose", u, out, u.shape, stream)


def hpdr_decompose_noalloc(u, out=None, stream=None):
    """hpdr_decompose without device allocation inside the library: the
    scratch lives in a fixed device array of the library (see include/hpdr.h)."""
    _dev_tensor(u, "u")
    if out is None:
        out = torch.empty(u.numel(), dtype=u.dtype, device=u.device)
    _dev_buf(out, "out", u.device, u.dtype, u.numel())
    nd, dims = _dims(u.shape)
    with torch.cuda.device(u.device):
        _check(lib().hpdr_decompose_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()),
                                            _dtype_code(u.dtype), nd, dims, _stream(stream)),
               "hpdr_decompose_noalloc")
    return out


def streamed_bound(shape, dtype=torch.float32, slab_bytes=256 << 20, dict_size=8192, chunk=0):
    """Capacity that always holds the streamed container of a field."""
    esz = 4 if dtype == torch.float32 else 8
    plane = esz
    for s in shape[1:]:
        plane *= int(s)
    per = max(2, slab_bytes // plane) if len(shape) > 1 else int(shape[0])
    nslab = max(1, -(-int(shape[0]) // per))
    slab = (min(-(-int(shape[0]) // nslab), int(shape[0])),) + tuple(shape[1:])
    return 64 + 32 * nslab + 16 + nslab * (hpdr_compress_bound(slab, dtype, dict_size, chunk) + 16)


def hpdr_compress_host_streamed(u, tol, tol_kind=REL, mode=LINF, slab_bytes=256 << 20, dict_size=8192,
                                chunk=0, out=None, device=None):
    """Compress a CPU tensor (pinned for overlapped copies) in slabs; returns a
    CPU uint8 tensor holding the streamed container."""
    if u.is_cuda or not u.is_contiguous():
        raise TypeError("u must be a contiguous CPU tensor")
    nd, dims = _dims(u.shape)
    cfg = _cfg(dict_size, chunk)
    if out is None:
        out = torch.empty(streamed_bound(u.shape, u.dtype, slab_bytes, dict_size, chunk), dtype=torch.uint8,
                          pin_memory=True)
    _host_buf(out, "out")
    nb = C.c_size_t()
    _check(lib().hpdr_compress_host_streamed(context(device), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype),
                                             nd, dims, float(tol), int(tol_kind), int(mode), C.byref(cfg),
                                             int(slab_bytes), C.c_void_p(out.data_ptr()), out.numel(),
                                             C.byref(nb)), "hpdr_compress_host_streamed")
    return out[:nb.value]


def _key_bytes(dtype):
    if dtype == torch.uint8:
        return 1
    if dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return 2
    raise TypeError("keys must be uint8 (byte keys) or int16/uint16 (16-bit keys)")


def lossless_bound(n, key_bytes, K=0):
    """Container capacity for n keys of key_bytes bytes; host only."""
    b = lib().hpdr_lossless_bound(int(n), int(key_bytes), int(K))
    if b == 0:
        raise HpdrError(-1, "hpdr_lossless_bound")
    return b


def hpdr_lossless_compress(keys, K=0, out=None, stream=None):
    """Huffman-compress a CUDA tensor of byte keys (uint8) or 16-bit keys
    (int16/uint16 bit patterns); returns the HPDL container (uint8, CUDA)."""
    _dev_tensor(keys, "keys")
    kb = _key_bytes(keys.dtype)
    n = keys.numel()
    if out is None:
        out = torch.empty(lossless_bound(n, kb, K), dtype=torch.uint8, device=keys.device)
    _dev_buf(out, "out", keys.device, torch.uint8)
    nb = C.c_size_t()
    with torch.cuda.device(keys.device):
        _check(lib().hpdr_lossless_compress(context(keys.device.index), C.c_void_p(keys.data_ptr()), n, kb, int(K),
                                            C.c_void_p(out.data_ptr()), out.numel(), C.byref(nb), _stream(stream)),
               "hpdr_lossless_compress")
    return out[:nb.value]


def hpdr_lossless_decompress(buf, out=None, stream=None):
    """Inverse of hpdr_lossless_compress (CUDA tensors in and out): uint8 keys
    or int16 bit patterns of 16-bit keys."""
    _dev_tensor(buf, "buf")
    kb, n = C.c_int(), C.c_uint64()
    _check(lib().hpdr_lossless_inspect(C.c_void_p(buf.data_ptr()), buf.numel(), C.byref(kb), C.byref(n)),
           "hpdr_lossless_inspect")
    if out is None:
        out = torch.empty(n.value, dtype=torch.uint8 if kb.value == 1 else torch.int16, device=buf.device)
    _dev_buf(out, "out", buf.device)
    with torch.cuda.device(buf.device):
        _check(lib().hpdr_lossless_decompress(context(buf.device.index), C.c_void_p(buf.data_ptr()), buf.numel(),
                                              C.c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                                              _stream(stream)), "hpdr_lossless_decompress")
    return out


def pipeline_fit(chunk_bytes, throughput, h2d, f=0.1):
    """Fit of the throughput model Phi from profiled (chunk bytes, bytes/s)
    pairs (Sec. V-C); host only."""
    n = len(chunk_bytes)
    cb = (C.c_double * n)(*[float(x) for x in chunk_bytes])
    tp = (C.c_double * n)(*[float(x) for x in throughput])
    m = PipelineModel()
    _check(lib().hpdr_pipeline_fit(cb, tp, n, float(f), float(h2d), C.byref(m)), "hpdr_pipeline_fit")
    return m


def pipeline_plan(model, n0, plane_bytes, c_init, c_limit=0):
    """Plane counts of the chunks of Alg. 4 for n0 planes; host only."""
    L = lib()
    n = L.hpdr_pipeline_plan(C.byref(model), int(n0), int(plane_bytes), int(c_init), int(c_limit), None, 0)
    if n == 0:
        raise HpdrError(-1, "hpdr_pipeline_plan")
    buf = (C.c_size_t * n)()
    L.hpdr_pipeline_plan(C.byref(model), int(n0), int(plane_bytes), int(c_init), int(c_limit), buf, n)
    return list(buf)


def streamed_bound_plan(shape, dtype, planes, dict_size=8192, chunk=0):
    """Capacity that always holds the streamed container of a field cut into
    chunks of planes[i] planes along dimension 0; host only."""
    nd, dims = _dims(shape)
    cfg = _cfg(dict_size, chunk)
    pl = (C.c_size_t * len(planes))(*[int(p) for p in planes])
    b = lib().hpdr_streamed_bound(nd, dims, _dtype_code(dtype), C.byref(cfg), pl, len(planes))
    if b == 0:
        raise HpdrError(-1, "hpdr_streamed_bound")
    return b


def pipeline_profile(u, tol, chunk_bytes, tol_kind=REL, mode=LINF, reps=3, f=0.1, dict_size=8192, chunk=0,
                     device=None):
    """Model of the adaptive pipeline profiled on the CPU field u itself:
    timed host-to-device copy and device compressions of its first planes."""
    if u.is_cuda or not u.is_contiguous():
        raise TypeError("u must be a contiguous CPU tensor")
    nd, dims = _dims(u.shape)
    cfg = _cfg(dict_size, chunk)
    cb = (C.c_size_t * len(chunk_bytes))(*[int(x) for x in chunk_bytes])
    m = PipelineModel()
    _check(lib().hpdr_pipeline_profile(context(device), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype), nd, dims,
                                       float(tol), int(tol_kind), int(mode), C.byref(cfg), cb, len(chunk_bytes),
                                       int(reps), float(f), C.byref(m)), "hpdr_pipeline_profile")
    return m


def hpdr_compress_host_adaptive(u, tol, model, c_init=64 << 20, c_limit=1 << 30, tol_kind=REL, mode=LINF,
                                dict_size=8192, chunk=0, out=None, device=None):
    """Compress a CPU tensor with the adaptive chunk sizes of Alg. 4; returns a
    CPU uint8 tensor holding the streamed container."""
    if u.is_cuda or not u.is_contiguous():
        raise TypeError("u must be a contiguous CPU tensor")
    nd, dims = _dims(u.shape)
    cfg = _cfg(dict_size, chunk)
    if out is None:
        plane = u.element_size() * (math.prod(int(s) for s in u.shape[1:]) if u.dim() > 1 else 1)
        planes = pipeline_plan(model, u.shape[0], plane, c_init, c_limit)
        out = torch.empty(streamed_bound_plan(u.shape, u.dtype, planes, dict_size, chunk), dtype=torch.uint8,
                          pin_memory=True)
    _host_buf(out, "out")
    nb = C.c_size_t()
    _check(lib().hpdr_compress_host_adaptive(context(device), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype),
                                             nd, dims, float(tol), int(tol_kind), int(mode), C.byref(cfg),
                                             C.byref(model), int(c_init), int(c_limit),
                                             C.c_void_p(out.data_ptr()), out.numel(), C.byref(nb)),
           "hpdr_compress_host_adaptive")
    return out[:nb.value]


def hpdr_decompress_host_streamed(buf, out=None, device=None):
    """Inverse of hpdr_compress_host_streamed (CPU tensors in and out)."""
    _host_buf(buf, "buf")
    if buf.numel() < 64:
        raise HpdrError(-4, "hpdr_decompress_host_streamed")
    b = bytes(buf[:64].numpy().tobytes())
    ns = int.from_bytes(b[8:12], "little")
    dt = torch.float32 if int.from_bytes(b[12:16], "little") == 0 else torch.float64
    nd = int.from_bytes(b[40:44], "little")
    shape = tuple(int.from_bytes(b[16 + 8 * k:24 + 8 * k], "little") for k in range(nd))
    if out is None:
        out = torch.empty(shape, dtype=dt, pin_memory=True)
    _host_buf(out, "out")
    _check(lib().hpdr_decompress_host_streamed(context(device), C.c_void_p(buf.data_ptr()), buf.numel(),
                                               C.c_void_p(out.data_ptr()), out.numel() * out.element_size()),
           "hpdr_decompress_host_streamed")
    del ns
    return out


def batched_capacity(shapes_dtypes, dict_size=8192, chunk=0):
    """Output bytes hpdr_compress_batched needs for these (shape, dtype) fields."""
    total = 0
    for shape, dt in shapes_dtypes:
        total = (total + hpdr_compress_bound(shape, dt, dict_size, chunk) + 255) & ~255
    return total


def hpdr_compress_batched(fields, tols, tol_kind=REL, mode=LINF, dict_size=8192, chunk=0, out=None,
                          stream=None):
    """Compress a list of CUDA fields (one graph replay; see include/hpdr.h).
    Returns (out uint8 tensor, offsets list, sizes list)."""
    n = len(fields)
    arr = (Field * n)()
    for i, (u, tol) in enumerate(zip(fields, tols)):
        _dev_tensor(u, "field")
        nd, dims = _dims(u.shape)
        arr[i] = Field(C.c_void_p(u.data_ptr()), _dtype_code(u.dtype), nd, dims, float(tol), int(tol_kind),
                       int(mode))
    if n == 0:
        raise ValueError("hpdr_compress_batched needs at least one field")
    for u in fields:
        if u.device != fields[0].device:
            raise ValueError("every field of a batch must be on one device")
    if out is None:
        out = torch.empty(batched_capacity([(u.shape, u.dtype) for u in fields], dict_size, chunk),
                          dtype=torch.uint8, device=fields[0].device)
    _dev_buf(out, "out", fields[0].device, torch.uint8)
    cfg = _cfg(dict_size, chunk)
    offs = (C.c_size_t * (n + 1))()
    sizes = (C.c_size_t * n)()
    _check(lib().hpdr_compress_batched(context(fields[0].device.index), n, arr, C.byref(cfg),
                                       C.c_void_p(out.data_ptr()), out.numel(), offs, sizes, _stream(stream)),
           "hpdr_compress_batched")
    return out, list(offs), list(sizes)


def hpdr_recompose(coef, shape, out=None, stream=None, coords=None):
    _dev_tensor(coef, "coef")
    if coef.numel() != _numel(shape):
        raise ValueError("coef holds %d coefficients, the shape %s has %d nodes" % (coef.numel(), tuple(shape),
                                                                                   _numel(shape)))
    if out is None:
        out = torch.empty(tuple(shape), dtype=coef.dtype, device=coef.device)
    _dev_buf(out, "out", coef.device, coef.dtype, coef.numel())
    if coords is not None:
        return _coords_call("hpdr_recompose_coords", coef, out, shape, coords, stream)
    return _field_call("hpdr_recompose", coef, out, shape, stream)


def hpdr_recompose_adjoint(grad_u, out=None, stream=None, coords=None):
    _dev_tensor(grad_u, "grad_u")
    if out is None:
        out = torch.empty(grad_u.numel(), dtype=grad_u.dtype, device=grad_u.device)
    _dev_buf(out, "out", grad_u.device, grad_u.dtype, grad_u.numel())
    if coords is not None:
        return _coords_call("hpdr_recompose_adjoint_coords", grad_u, out, grad_u.shape, coords, stream)
    return _field_call("hpdr_recompose_adjoint", grad_u, out, grad_u.shape, stream)


def hpdr_decompose_adjoint(grad_coef, shape, out=None, stream=None, coords=None):
    _dev_tensor(grad_coef, "grad_coef")
    if grad_coef.numel() != _numel(shape):
        raise ValueError("grad_coef holds %d values, the shape %s has %d nodes" % (grad_coef.numel(), tuple(shape),
                                                                                  _numel(shape)))
    if out is None:
        out = torch.empty(tuple(shape), dtype=grad_coef.dtype, device=grad_coef.device)
    _dev_buf(out, "out", grad_coef.device, grad_coef.dtype, grad_coef.numel())
    if coords is not None:
        return _coords_call("hpdr_decompose_adjoint_coords", grad_coef, out, shape, coords, stream)
    return _field_call("hpdr_decompose_adjoint", grad_coef, out, shape, stream)


def hpdr_huffman_encode(symbols, D=8192, K=1024, stream=None):
    """Huffman-encode a CUDA int16 tensor holding uint16 symbols < D.

    Returns (lengths uint8[D], chunk table int64[ceil(N/K)], words int32[...],
    total_bits)."""
    _dev_tensor(symbols, "symbols")
    _dev_buf(symbols, "symbols", symbols.device, 2)
    N = symbols.numel()
    dev = symbols.device
    lengths = torch.empty(D, dtype=torch.uint8, device=dev)
    chunk = torch.empty((N + K - 1) // K, dtype=torch.int64, device=dev)
    cap = (63 * N + 31) // 32 + 4
    words = torch.empty(cap, dtype=torch.int32, device=dev)
    tb = C.c_uint64()
    _check(lib().hpdr_huffman_encode(context(dev.index), C.c_void_p(symbols.data_ptr()), N, D, K,
                                     C.c_void_p(lengths.data_ptr()), C.c_void_p(chunk.data_ptr()),
                                     C.c_void_p(words.data_ptr()), cap, C.byref(tb),
                                     _stream(stream)), "hpdr_huffman_encode")
    return lengths, chunk, words[:(tb.value + 31) // 32], tb.value


def hpdr_huffman_decode(words, total_bits, chunk, N, lengths, D=8192, K=1024, out=None,
                        stream=None):
    _dev_tensor(words, "words")
    dev = words.device
    N, K, D = int(N), int(K), int(D)
    _dev_buf(words, "words", dev, 4, (int(total_bits) + 31) // 32)
    _dev_buf(chunk, "chunk", dev, 8, (N + K - 1) // K)
    _dev_buf(lengths, "lengths", dev, torch.uint8, D)
    if out is None:
        out = torch.empty(N, dtype=torch.int16, device=dev)
    _dev_buf(out, "out", dev, 2, N)
    _check(lib().hpdr_huffman_decode(context(dev.index), C.c_void_p(words.data_ptr()),
                                     int(total_bits), C.c_void_p(chunk.data_ptr()), N, D, K,
                                     C.c_void_p(lengths.data_ptr()), C.c_void_p(out.data_ptr()),
                                     _stream(stream)), "hpdr_huffman_decode")
    return out


# ---- fixed-rate ZFP (Alg. 3) ------------------------------------------------

def zfp_bound(shape, rate, dtype=torch.float32):
    nd, dims = _dims(shape)
    return int(lib().hpdr_zfp_bound(nd, dims, _dtype_code(dtype), int(rate)))


def hpdr_zfp_compress(u, rate, out=None, stream=None):
    """Fixed-rate ZFP container (uint8 CUDA tensor) of a CUDA field; rate =
    bits per value (rate * 4^ndim a multiple of 32)."""
    _dev_tensor(u, "u")
    nd, dims = _dims(u.shape)
    cap = zfp_bound(u.shape, rate, u.dtype)
    if cap == 0:
        raise ValueError("invalid ZFP rate %r for %d dimensions" % (rate, nd))
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=u.device)
    _dev_buf(out, "out", u.device, torch.uint8)
    nb = C.c_size_t()
    _check(lib().hpdr_zfp_compress(context(u.device.index), C.c_void_p(u.data_ptr()), _dtype_code(u.dtype), nd,
                                   dims, int(rate), C.c_void_p(out.data_ptr()), out.numel(), C.byref(nb),
                                   _stream(stream)), "hpdr_zfp_compress")
    return out[:nb.value]


def hpdr_zfp_inspect(buf):
    dt, nd, r = C.c_int(), C.c_int(), C.c_uint32()
    dims = (C.c_size_t * 3)()
    _check(lib().hpdr_zfp_inspect(C.c_void_p(buf.data_ptr()), buf.numel(), C.byref(dt), C.byref(nd), dims,
                                  C.byref(r)), "hpdr_zfp_inspect")
    return (torch.float32 if dt.value == F32 else torch.float64), tuple(dims[:nd.value]), r.value


def hpdr_zfp_decompress(buf, out=None, stream=None):
    _dev_tensor(buf, "buf")
    dt, shape, _ = hpdr_zfp_inspect(buf)
    if out is None:
        out = torch.empty(shape, dtype=dt, device=buf.device)
    _dev_buf(out, "out", buf.device, dt)
    _check(lib().hpdr_zfp_decompress(context(buf.device.index), C.c_void_p(buf.data_ptr()), buf.numel(),
                                     C.c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                                     _stream(stream)), "hpdr_zfp_decompress")
    return out
