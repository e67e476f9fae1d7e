"""GB300-native LSB substitution steganography.

A thin Python binding over ``libstego.so`` (declared in ``include/stego.h``).
Every function here only marshals torch tensors into device pointers and
calls the C entry point of the same name; all steganography arithmetic runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.

There is no CPU fallback: if the library has not been built (see
``paper_0912_0947_gb300.build.build()``) or a tensor is not a contiguous
CUDA uint8 tensor, the call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

# -- flags / status (values of include/stego.h) ------------------------------
LAYOUT_STREAM1 = 0x0
LAYOUT_PAPER2 = 0x1
HEADER_BE32 = 0x10
FUSE_STATS = 0x20
PLANE_ONLY = 0x40   # stream layout: carry only in channel geom.plane, pixel order


def BITS(k: int) -> int:
    """Stream-layout flag for k = 1..4 bits per carrying byte."""
    if not 1 <= k <= 4:
        raise ValueError("k must be 1..4")
    return (k - 1) << 8

OK = 0
E_INVAL = -1
E_CAPACITY = -2
E_BAD_HEADER = -3
E_MSG_TOO_SMALL = -4
E_CUDA = -5
E_NOMEM = -6
E_TIMEOUT = -7

OP_EMBED, OP_EXTRACT, OP_CHANGED, OP_EMBED_BATCHED, OP_EXTRACT_BATCHED = range(5)

RESULT_WORDS = 4  # stego_result: changed, sse, msg_bytes, status|reserved (int64 view)

# stego_desc as laid out in device memory (72 bytes)
DESC_DTYPE = np.dtype([
    ("cover", "<u8"), ("stego", "<u8"), ("msg", "<u8"),
    ("cover_bytes", "<u8"), ("msg_bytes", "<u8"), ("msg_len", "<u8"),
    ("flags", "<u4"), ("reserved", "<u4"),
    ("width", "<u4"), ("height", "<u4"), ("channels", "<u4"), ("plane", "<u4"),
])
assert DESC_DTYPE.itemsize == 72


class StegoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, strerror(status), status))


class Geom(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("channels", ctypes.c_uint32), ("plane", ctypes.c_uint32)]


class Tune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("vec_per_thread", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("tile_bytes", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("budget_bytes", ctypes.c_uint64), ("tune_embed", Tune),
                ("tune_extract", Tune)]


PIPE_AUTO, PIPE_STAGED = 0, 1


class PipelineConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_descs", ctypes.c_uint32),
                ("slot_bytes", ctypes.c_uint64), ("mode", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("tune_embed", Tune),
                ("tune_extract", Tune)]


# stego_host_job as laid out in host memory (80 bytes)
HOST_JOB_DTYPE = np.dtype([
    ("cover", "<u8"), ("stego", "<u8"), ("msg", "<u8"), ("readback", "<u8"),
    ("cover_bytes", "<u8"), ("msg_bytes", "<u8"), ("msg_len", "<u8"),
    ("flags", "<u4"), ("reserved", "<u4"),
    ("width", "<u4"), ("height", "<u4"), ("channels", "<u4"), ("plane", "<u4"),
])
assert HOST_JOB_DTYPE.itemsize == 80

# stego_request (80 bytes) / stego_completion (64 bytes) as laid out in host memory
REQUEST_DTYPE = np.dtype([
    ("op", "<u4"), ("flags", "<u4"), ("cover", "<u8"), ("stego", "<u8"), ("msg", "<u8"),
    ("cover_bytes", "<u8"), ("msg_bytes", "<u8"), ("msg_len", "<u8"), ("tag", "<u8"),
    ("width", "<u4"), ("height", "<u4"), ("channels", "<u4"), ("plane", "<u4"),
])
COMPLETION_DTYPE = np.dtype([
    ("tag", "<u8"), ("changed", "<u8"), ("sse", "<u8"), ("msg_bytes", "<u8"),
    ("status", "<i4"), ("batch_size", "<i4"),
    ("t_submit", "<f8"), ("t_dispatch", "<f8"), ("t_done", "<f8"),
])
assert REQUEST_DTYPE.itemsize == 80 and COMPLETION_DTYPE.itemsize == 64

_LIB = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_int = ctypes.c_int


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded ``libstego.so``; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libstego.so is not built (%s); run "
                               "paper_0912_0947_gb300.build.build() first" % path)
        L = ctypes.CDLL(path)
        L.stego_version.restype = _int
        L.stego_strerror.argtypes = [_int]
        L.stego_strerror.restype = ctypes.c_char_p
        L.stego_capacity.argtypes = [_u64, ctypes.POINTER(Geom), _u32, ctypes.POINTER(_u64)]
        L.stego_capacity.restype = _int
        L.stego_embed.argtypes = [_vp, _vp, _u64, _vp, _u64, ctypes.POINTER(Geom), _u32, _vp, _vp]
        L.stego_embed.restype = _int
        L.stego_extract.argtypes = [_vp, _u64, _vp, _u64, _u64, ctypes.POINTER(Geom), _u32, _vp, _vp]
        L.stego_extract.restype = _int
        L.stego_extract_ballot.argtypes = [_vp, _u64, _vp, _u64, _u64, ctypes.POINTER(Geom), _u32, _vp, _vp]
        L.stego_extract_ballot.restype = _int
        L.stego_changed_bytes.argtypes = [_vp, _vp, _u64, _vp, _vp]
        L.stego_changed_bytes.restype = _int
        L.stego_batched_workspace_bytes.argtypes = [_u32]
        L.stego_batched_workspace_bytes.restype = _u64
        for name in ("stego_embed_batched", "stego_extract_batched"):
            f = getattr(L, name)
            f.argtypes = [_vp, _u32, _vp, _u32, ctypes.POINTER(Tune), _vp, _u64, _vp]
            f.restype = _int
        L.stego_embed_batched_noalloc.argtypes = [_vp, _u32, _vp, _u32, ctypes.POINTER(Tune), _vp]
        L.stego_embed_batched_noalloc.restype = _int
        L.stego_pointer_kind.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]
        L.stego_pointer_kind.restype = _int
        L.stego_server_arena_bytes.argtypes = [ctypes.POINTER(ServerConfig)]
        L.stego_server_arena_bytes.restype = _u64
        L.stego_server_create.argtypes = [ctypes.POINTER(ServerConfig), _vp, _u64,
                                          ctypes.POINTER(_vp)]
        L.stego_server_create.restype = _int
        L.stego_server_submit.argtypes = [_vp, _vp, _u32]
        L.stego_server_submit.restype = _int
        L.stego_server_poll.argtypes = [_vp, _vp, _u32, ctypes.POINTER(_u32)]
        L.stego_server_poll.restype = _int
        L.stego_server_drain.argtypes = [_vp, ctypes.c_double]
        L.stego_server_drain.restype = _int
        L.stego_server_run_open_loop.argtypes = [_vp, _vp, _vp, _u32, _vp, ctypes.c_double]
        L.stego_server_run_open_loop.restype = _int
        L.stego_server_clock.argtypes = [_vp]
        L.stego_server_clock.restype = ctypes.c_double
        L.stego_server_stats.argtypes = [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                         ctypes.POINTER(_u64)]
        L.stego_server_stats.restype = _int
        L.stego_server_destroy.argtypes = [_vp]
        L.stego_server_destroy.restype = _int
        L.stego_pipeline_arena_bytes.argtypes = [ctypes.POINTER(PipelineConfig)]
        L.stego_pipeline_arena_bytes.restype = _u64
        L.stego_pipeline_create.argtypes = [ctypes.POINTER(PipelineConfig), _vp, _u64,
                                            ctypes.POINTER(_vp)]
        L.stego_pipeline_create.restype = _int
        L.stego_pipeline_embed.argtypes = [_vp, _vp, _u32, _vp, _vp, _u32]
        L.stego_pipeline_embed.restype = _int
        L.stego_pipeline_extract.argtypes = [_vp, _vp, _u32, _vp]
        L.stego_pipeline_extract.restype = _int
        L.stego_pipeline_destroy.argtypes = [_vp]
        L.stego_pipeline_destroy.restype = _int
        L.stego_partition.argtypes = [_vp, _u32, _u32, _vp, _vp]
        L.stego_partition.restype = _int
        L.stego_test_bounded_wait.argtypes = [_u64, _u32]
        L.stego_test_bounded_wait.restype = _int
        L.stego_set_tune.argtypes = [_int, ctypes.POINTER(Tune)]
        L.stego_set_tune.restype = _int
        L.stego_get_tune.argtypes = [_int, ctypes.POINTER(Tune)]
        L.stego_get_tune.restype = _int
        L.stego_graph_capture_batched.argtypes = [_int, _vp, _u32, _vp, _u32, ctypes.POINTER(Tune),
                                                  _vp, _u64, ctypes.POINTER(_vp)]
        L.stego_graph_capture_batched.restype = _int
        L.stego_graph_launch.argtypes = [_vp, _vp]
        L.stego_graph_launch.restype = _int
        L.stego_graph_destroy.argtypes = [_vp]
        L.stego_graph_destroy.restype = _int
        _LIB = L
    return _LIB


def strerror(status: int) -> str:
    try:
        return lib().stego_strerror(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _check(st: int, where: str) -> int:
    if st != OK:
        raise StegoError(st, where)
    return st


# -- marshalling helpers -------------------------------------------------------

def _dev_ptr(t, what: str, dtype=torch.uint8):
    """Address of a contiguous tensor the kernels can dereference (or None):
    CUDA memory, or pinned host memory mapped into the device's address space
    (the kernels then read and write it over the CPU-GPU link; no copy).
    Pageable CPU tensors are refused: there is no CPU fallback."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % what)
    if not t.is_cuda:  # (a bool property: cheaper than building t.device)
        if not (t.device.type == "cpu" and t.is_pinned()):
            raise ValueError("%s must live on a CUDA device or in pinned host memory "
                             "(no CPU fallback)" % what)
        if t.numel() > 0 and not stego_pointer_kind(t.data_ptr())[1]:
            raise ValueError("%s: pinned host memory not mapped for the device" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return t.data_ptr() if t.numel() > 0 else None


def _stream_ptr(stream, device=None):
    if stream is None:
        if device is not None and torch.device(device).type != "cuda":
            device = None  # host (zero-copy) buffers: the current CUDA device
        stream = torch.cuda.current_stream(device)
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _geom(geom):
    if geom is None:
        return None
    if isinstance(geom, Geom):
        return ctypes.byref(geom)
    w, h, c, p = geom
    return ctypes.byref(Geom(int(w), int(h), int(c), int(p)))


def _tune(tune):
    if tune is None:
        return None
    if isinstance(tune, Tune):
        return ctypes.byref(tune)
    return ctypes.byref(Tune(*[int(x) for x in tune]))


def new_result(device="cuda", n: int | None = None) -> torch.Tensor:
    """Device storage for one stego_result (n=None) or n of them (int64 view)."""
    shape = (RESULT_WORDS,) if n is None else (n, RESULT_WORDS)
    return torch.zeros(shape, dtype=torch.int64, device=device)


def read_result(res) -> dict | list[dict]:
    """Host view of stego_result(s) (a tensor or an int64 numpy array):
    changed, sse, msg_bytes, status."""
    a = res.detach().cpu().numpy() if isinstance(res, torch.Tensor) else np.asarray(res)
    one = a.ndim == 1
    a = a.reshape(-1, RESULT_WORDS)
    out = []
    for row in a:
        st = int(np.int64(row[3]).astype(np.uint64) & np.uint64(0xFFFFFFFF))
        st = st - (1 << 32) if st >= (1 << 31) else st
        out.append({"changed": int(row[0]), "sse": int(row[1]),
                    "msg_bytes": int(row[2]), "status": st})
    return out[0] if one else out


# -- entry points (same names as the C ABI) ------------------------------------

def stego_version() -> int:
    return lib().stego_version()


def stego_capacity(cover_bytes: int, flags: int, geom=None) -> int:
    out = _u64(0)
    _check(lib().stego_capacity(int(cover_bytes), _geom(geom), int(flags), ctypes.byref(out)),
           "stego_capacity")
    return int(out.value)


def stego_embed(cover, stego, msg, flags: int, result=None, geom=None, stream=None) -> None:
    """stego <- embed(cover, msg).  ``stego`` may be ``cover`` (in place)."""
    c = _dev_ptr(cover, "cover")
    s = _dev_ptr(stego, "stego")
    m = _dev_ptr(msg, "msg") if msg is not None else None
    r = _dev_ptr(result, "result", torch.int64)
    if stego.numel() != cover.numel():
        raise ValueError("cover and stego sizes differ")
    st = lib().stego_embed(c, s, cover.numel(), m, 0 if msg is None else msg.numel(),
                           _geom(geom), int(flags), r, _stream_ptr(stream, cover.device))
    _check(st, "stego_embed")


def stego_extract(stego, msg, msg_len: int, flags: int, result=None, geom=None,
                  stream=None) -> None:
    """msg <- extract(stego).  With HEADER_BE32 the length (and status) go to
    ``result``; otherwise ``msg_len`` bytes are extracted."""
    s = _dev_ptr(stego, "stego")
    m = _dev_ptr(msg, "msg") if msg is not None else None
    r = _dev_ptr(result, "result", torch.int64)
    st = lib().stego_extract(s, stego.numel(), m, 0 if msg is None else msg.numel(),
                             int(msg_len), _geom(geom), int(flags), r,
                             _stream_ptr(stream, stego.device))
    _check(st, "stego_extract")


def stego_extract_ballot(stego, msg, msg_len: int, flags: int, result=None, geom=None,
                         stream=None) -> None:
    """stego_extract computed by the ballot-gather kernel (one-bit stream
    layout only)."""
    s = _dev_ptr(stego, "stego")
    m = _dev_ptr(msg, "msg") if msg is not None else None
    r = _dev_ptr(result, "result", torch.int64)
    st = lib().stego_extract_ballot(s, stego.numel(), m, 0 if msg is None else msg.numel(),
                                    int(msg_len), _geom(geom), int(flags), r,
                                    _stream_ptr(stream, stego.device))
    _check(st, "stego_extract_ballot")


def stego_changed_bytes(a, b, out2, stream=None) -> None:
    """out2 (int64[2], device) <- [changed bytes, sum of squared differences]."""
    if a.numel() != b.numel():
        raise ValueError("sizes differ")
    st = lib().stego_changed_bytes(_dev_ptr(a, "a"), _dev_ptr(b, "b"), a.numel(),
                                   _dev_ptr(out2, "out2", torch.int64),
                                   _stream_ptr(stream, a.device))
    _check(st, "stego_changed_bytes")


def stego_batched_workspace_bytes(n: int) -> int:
    return int(lib().stego_batched_workspace_bytes(int(n)))


def stego_embed_batched(descs, n: int, results, flags: int, ws, tune=None, stream=None) -> None:
    st = lib().stego_embed_batched(_dev_ptr(descs, "descs", None), int(n),
                                   _dev_ptr(results, "results", torch.int64), int(flags),
                                   _tune(tune), _dev_ptr(ws, "ws", None),
                                   ws.numel() * ws.element_size(),
                                   _stream_ptr(stream, descs.device))
    _check(st, "stego_embed_batched")


def stego_extract_batched(descs, n: int, results, flags: int, ws, tune=None, stream=None) -> None:
    st = lib().stego_extract_batched(_dev_ptr(descs, "descs", None), int(n),
                                     _dev_ptr(results, "results", torch.int64), int(flags),
                                     _tune(tune), _dev_ptr(ws, "ws", None),
                                     ws.numel() * ws.element_size(),
                                     _stream_ptr(stream, descs.device))
    _check(st, "stego_extract_batched")


# largest batch stego_embed_batched_noalloc accepts (STEGO_NOALLOC_MAX_DESCS)
NOALLOC_MAX_DESCS = 8192


def stego_embed_batched_noalloc(descs, n: int, results, flags: int, tune=None,
                                stream=None) -> None:
    """Batched embed with no workspace argument, for callers that cannot
    allocate device memory: the library's own per-GPU scratch array stands in
    for it.  At most NOALLOC_MAX_DESCS covers; calls that overlap on the GPU
    race on the shared scratch, so issue them on one stream."""
    st = lib().stego_embed_batched_noalloc(_dev_ptr(descs, "descs", None), int(n),
                                           _dev_ptr(results, "results", torch.int64), int(flags),
                                           _tune(tune), _stream_ptr(stream, descs.device))
    _check(st, "stego_embed_batched_noalloc")


MEM_PAGEABLE, MEM_PINNED, MEM_DEVICE, MEM_MANAGED = range(4)


def stego_pointer_kind(ptr: int):
    """(kind, device_accessible) of an address (see include/stego.h)."""
    k, a = _int(0), _int(0)
    _check(lib().stego_pointer_kind(_vp(ptr), ctypes.byref(k), ctypes.byref(a)),
           "stego_pointer_kind")
    return k.value, bool(a.value)


def stego_partition(sizes, world: int):
    """(rank of each cover, bytes of each rank): covers split among `world`
    GPUs by byte volume (stego_partition)."""
    b = np.ascontiguousarray(np.asarray(sizes, dtype=np.uint64))
    rank_of = np.zeros(max(len(b), 1), dtype=np.uint32)
    rank_bytes = np.zeros(max(int(world), 1), dtype=np.uint64)
    _check(lib().stego_partition(b.ctypes.data if len(b) else None, len(b), int(world),
                                 rank_of.ctypes.data, rank_bytes.ctypes.data),
           "stego_partition")
    return rank_of[: len(b)], rank_bytes[: int(world)]


def stego_test_bounded_wait(limit_ns: int, withhold_arrival: int) -> None:
    """Bound of the staged kernels' waits and the withheld-arrival switch
    that makes them run out (a test hook; see include/stego.h)."""
    _check(lib().stego_test_bounded_wait(int(limit_ns), int(withhold_arrival)),
           "stego_test_bounded_wait")


def stego_set_tune(op: int, tune) -> None:
    t = tune if isinstance(tune, Tune) else Tune(*[int(x) for x in tune])
    _check(lib().stego_set_tune(int(op), ctypes.byref(t)), "stego_set_tune")


def stego_get_tune(op: int) -> Tune:
    t = Tune()
    _check(lib().stego_get_tune(int(op), ctypes.byref(t)), "stego_get_tune")
    return t


class BatchedGraph:
    """A captured batched call (stego_graph_capture_batched); replay with
    ``launch(stream)``."""

    def __init__(self, op: int, descs, n: int, results, flags: int, ws, tune=None):
        h = _vp(0)
        st = lib().stego_graph_capture_batched(int(op), _dev_ptr(descs, "descs", None), int(n),
                                               _dev_ptr(results, "results", torch.int64),
                                               int(flags), _tune(tune), _dev_ptr(ws, "ws", None),
                                               ws.numel() * ws.element_size(), ctypes.byref(h))
        _check(st, "stego_graph_capture_batched")
        self._h = h
        # keep the captured buffers alive as long as the graph
        self._keep = (descs, results, ws)

    def launch(self, stream=None) -> None:
        _check(lib().stego_graph_launch(self._h, _stream_ptr(stream)), "stego_graph_launch")

    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().stego_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -- descriptor packing (host side) ---------------------------------------------

def pack_descs(items) -> np.ndarray:
    """Pack a list of dicts (keys of DESC_DTYPE; tensors allowed for cover,
    stego, msg) into a host array of stego_desc records."""
    a = np.zeros(len(items), dtype=DESC_DTYPE)
    for i, it in enumerate(items):
        for k, v in it.items():
            if isinstance(v, torch.Tensor):
                v = _dev_ptr(v, k) or 0
            a[i][k] = v
    return a


def descs_to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    t = torch.from_numpy(a.view(np.uint8).copy())
    return t.to(device)


# -- serving ---------------------------------------------------------------------

class Server:
    """A stego_server: continuous batching of embed / extract requests
    (include/stego.h).  The device arena is a torch tensor owned here."""

    def __init__(self, slots: int = 4, max_batch: int = 256, budget_bytes: int = 40 << 30,
                 tune_embed=(0, 0, 0, 0), tune_extract=(0, 0, 0, 0), device="cuda"):
        cfg = ServerConfig(int(slots), int(max_batch), int(budget_bytes),
                           Tune(*tune_embed), Tune(*tune_extract))
        n = int(lib().stego_server_arena_bytes(ctypes.byref(cfg)))
        if n == 0:
            raise StegoError(E_INVAL, "stego_server_arena_bytes")
        self.arena = torch.empty(n, dtype=torch.uint8, device=device)
        h = _vp(0)
        _check(lib().stego_server_create(ctypes.byref(cfg), self.arena.data_ptr(), n,
                                         ctypes.byref(h)), "stego_server_create")
        self._h = h
        self.cfg = cfg

    @staticmethod
    def requests(items) -> np.ndarray:
        """Pack dicts (keys of REQUEST_DTYPE; tensors allowed for cover,
        stego, msg) into a host array of stego_request records."""
        a = np.zeros(len(items), dtype=REQUEST_DTYPE)
        for i, it in enumerate(items):
            for k, v in it.items():
                if isinstance(v, torch.Tensor):
                    v = _dev_ptr(v, k) or 0
                a[i][k] = v
        return a

    def submit(self, reqs: np.ndarray) -> None:
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
        _check(lib().stego_server_submit(self._h, reqs.ctypes.data, len(reqs)),
               "stego_server_submit")

    def poll(self, max_n: int = 4096) -> np.ndarray:
        out = np.zeros(max_n, dtype=COMPLETION_DTYPE)
        k = _u32(0)
        _check(lib().stego_server_poll(self._h, out.ctypes.data, max_n, ctypes.byref(k)),
               "stego_server_poll")
        return out[: k.value]

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(lib().stego_server_drain(self._h, float(timeout_s)), "stego_server_drain")

    def run_open_loop(self, reqs: np.ndarray, arrival_s: np.ndarray,
                      timeout_s: float = 120.0) -> np.ndarray:
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        out = np.zeros(len(reqs), dtype=COMPLETION_DTYPE)
        _check(lib().stego_server_run_open_loop(self._h, reqs.ctypes.data, arr.ctypes.data,
                                                len(reqs), out.ctypes.data, float(timeout_s)),
               "stego_server_run_open_loop")
        return out

    def clock(self) -> float:
        return float(lib().stego_server_clock(self._h))

    def stats(self) -> dict:
        b, o, p = _u64(0), _u64(0), _u64(0)
        _check(lib().stego_server_stats(self._h, ctypes.byref(b), ctypes.byref(o),
                                        ctypes.byref(p)), "stego_server_stats")
        return {"batches": b.value, "outstanding": o.value, "peak_in_flight_bytes": p.value}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().stego_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -- host-resident covers: the overlapped copy pipeline ----------------------------

def _host_ptr(t, what: str):
    """Address of a contiguous uint8 CPU tensor (pinned for the copies to
    overlap) or None."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError("%s must be a CPU tensor (host memory)" % what)
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous uint8 tensor" % what)
    return t.data_ptr() if t.numel() > 0 else None


class Pipeline:
    """A stego_pipeline: embed / extract batches of covers held in host
    memory, with host->device copies, kernels and device->host copies of
    neighbouring chunks overlapped (include/stego.h).  The device arena is
    a torch tensor owned here."""

    def __init__(self, slots: int = 2, max_descs: int = 1024, slot_bytes: int = 256 << 20,
                 mode: int = PIPE_AUTO, tune_embed=(0, 0, 0, 0), tune_extract=(0, 0, 0, 0),
                 device="cuda"):
        cfg = PipelineConfig(int(slots), int(max_descs), int(slot_bytes), int(mode), 0,
                             Tune(*tune_embed), Tune(*tune_extract))
        n = int(lib().stego_pipeline_arena_bytes(ctypes.byref(cfg)))
        if n == 0:
            raise StegoError(E_INVAL, "stego_pipeline_arena_bytes")
        self.arena = torch.empty(n, dtype=torch.uint8, device=device)
        h = _vp(0)
        _check(lib().stego_pipeline_create(ctypes.byref(cfg), self.arena.data_ptr(), n,
                                           ctypes.byref(h)), "stego_pipeline_create")
        self._h = h
        self.cfg = cfg

    @staticmethod
    def jobs(items) -> np.ndarray:
        """Pack dicts (keys of HOST_JOB_DTYPE; CPU tensors allowed for cover,
        stego, msg, readback) into a host array of stego_host_job records."""
        a = np.zeros(len(items), dtype=HOST_JOB_DTYPE)
        for i, it in enumerate(items):
            for k, v in it.items():
                if isinstance(v, torch.Tensor):
                    v = _host_ptr(v, k)
                a[i][k] = 0 if v is None else v
        return a

    def embed(self, jobs: np.ndarray, flags: int = FUSE_STATS, readback_results: bool = False,
              raw: bool = False):
        """Results (list of dicts; with raw, the int64 [n, 4] array of
        stego_result records) and, with readback_results, the read-back
        extractions' results too."""
        jobs = np.ascontiguousarray(jobs, dtype=HOST_JOB_DTYPE)
        n = len(jobs)
        res = np.zeros((max(n, 1), RESULT_WORDS), dtype=np.int64)
        rb = np.zeros((max(n, 1), RESULT_WORDS), dtype=np.int64) if readback_results else None
        _check(lib().stego_pipeline_embed(self._h, jobs.ctypes.data, n, res.ctypes.data,
                                          rb.ctypes.data if rb is not None else None,
                                          int(flags)), "stego_pipeline_embed")
        conv = (lambda a: a[:n]) if raw else (lambda a: read_result(a[:n]) if n else [])
        if readback_results:
            return conv(res), conv(rb)
        return conv(res)

    def extract(self, jobs: np.ndarray, raw: bool = False):
        jobs = np.ascontiguousarray(jobs, dtype=HOST_JOB_DTYPE)
        n = len(jobs)
        res = np.zeros((max(n, 1), RESULT_WORDS), dtype=np.int64)
        _check(lib().stego_pipeline_extract(self._h, jobs.ctypes.data, n, res.ctypes.data),
               "stego_pipeline_extract")
        if raw:
            return res[:n]
        return read_result(res[:n]) if n else []

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().stego_pipeline_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
