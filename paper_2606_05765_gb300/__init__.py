"""PivCo-Huffman for GB300 (sm_103a): Python binding of the C ABI in include/pivco.h.

Every function here only marshals arguments: torch tensors supply device
memory and the current CUDA stream; all codec work runs in the CUDA kernels of
``libpivco.so``.  If the library has not been built the import succeeds but the
first call raises -- there is no CPU fallback.

Low-level calls mirror the C ABI one to one (``histogram``, ``code_lengths``,
``build_layout``, ``exclusive_scan``, ``encode_blocks``, ``ans_encode_blocks``,
``decode_workspace_size``, ``decode_blocks``, ``ans_encode``, ``ans_decode``).
``encode`` / ``decode`` chain them for a batch of blocks.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpivco.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_TIMEOUT, ERR_CUDA = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "CORRUPT", 4: "TIMEOUT", 5: "CUDA"}

# name -> argument types; every function returns int32 status unless noted
_P, _I32, _SZ = C.c_void_p, C.c_int32, C.c_size_t
_SIGS = {
    "pivco_histogram": [_P, _P, _I32, _P, _P],
    "pivco_code_lengths": [_P, _I32, _I32, _P, _P, _P],
    "pivco_build_layout": [_P, _P, _I32, _P, _P, _P, _P, _P],
    "pivco_exclusive_scan": [_P, _I32, _P, _P, _SZ, _P, _P],
    "pivco_encode_blocks": [_P, _P, _I32, _P, _P, _P, _P, _P, _P],
    "pivco_histogram_chunks": [_P, _P, _I32, _P, _P, _P],
    "pivco_plan_blocks": [_P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P],
    "pivco_host_codec_create": [_P, _I32, _P, _I32, _P],
    "pivco_host_codec_destroy": [_P],
    "pivco_host_compress": [_P, _P, _P, C.c_uint64, _P, _P],
    "pivco_host_decompress": [_P, _P, _P, _P, _P],
    "pivco_encode_blocks_chunked": [_P, _P, _I32, _P, _P, _P, _P, _P, _P, _P],
    "pivco_ans_encode_blocks": [_P, _I32, _P, _P, _P, _P, _SZ, _P, _P],
    "pivco_decode_workspace_size": [_P, _P, _I32, _P, _SZ, _P, C.POINTER(C.c_size_t), _P],
    "pivco_decode_blocks": [_P, _P, _I32, _P, _P, _P, _SZ, _P, _P],
    "pivco_decode_blocks_static": [_P, _P, _I32, _P, _P, _P, _P],
    "pivco_decode_plan": [_P, _P, _I32, _P, _SZ, _P, _P],
    "pivco_decode_ans": [_P, _P, _I32, _P, _SZ, _P, _P],
    "pivco_decode_merge": [_P, _P, _I32, _P, _P, _P, _SZ, _P, _P],
    "pivco_ans_tables": [_P, _P],
    "pivco_ans_encode": [_P, _P, _P, _I32, _P, _P, _P, _P, _P],
    "pivco_ans_decode": [_P, _P, _P, _I32, _P, _P, _P, _P],
    "pivco_decode_batched": [_P, _P, _I32, _P, _P, _P, _SZ, _P, _P],
    "pivco_get_tuning": [_P],
    "pivco_set_tuning": [_P],
    "pivco_autotune_decode": [_P, _P, _I32, _P, _P, _P, _SZ, _P, _I32, _P, _P, _P],
    "pivco_graph_begin": [_P],
    "pivco_graph_end": [_P, _P],
    "pivco_graph_launch": [_P, _P],
    "pivco_graph_destroy": [_P],
    "pivco_server_create": [_P, _SZ, _P, _P],
    "pivco_server_submit": [_P, _P, _P, _I32, _P, _P, C.POINTER(C.c_uint64)],
    "pivco_server_poll": [_P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)],
    "pivco_server_drain": [_P, _I32],
    "pivco_server_forget": [_P, C.c_uint64],
    "pivco_server_destroy": [_P],
    "pivco_set_wait_limit": [C.c_uint64],
    "pivco_access_workspace_size": [_P, _P, _I32, _P, _SZ, _P, C.POINTER(C.c_size_t), _P],
    "pivco_access_prepare": [_P, _P, _I32, _P, _SZ, _P, _P],
    "pivco_access": [_P, _P, _I32, _P, _P, _I32, _P, _P, _P, _SZ, _P, _P],
    "pivco_golomb_plan": [_P, _P, _I32, _P, _P, _P],
    "pivco_golomb_encode": [_P, _P, _I32, _P, _P, _P, _P, _P],
    "pivco_golomb_decode": [_P, _P, _I32, _P, _P, _P, _P],
}
_OTHER = {
    "pivco_version": ([], C.c_char_p),
    "pivco_layout_bytes": ([], _I32),
    "pivco_scan_workspace_size": ([_I32], _SZ),
    "pivco_decode_plan_bytes": ([_I32], _SZ),
    "pivco_launch_count": ([], C.c_uint64),
    "pivco_host_codec_comp_capacity": ([_P], C.c_uint64),
    "pivco_get_wait_limit": ([], C.c_uint64),
}


class Params(C.Structure):
    """Encoder parameters (struct pivco_params): L = 11 (App. D), the
    Sec. 5.2 ANS knobs (32 bytes, skew > 5/8, ratio < 95 %) and the
    regrouped tree with flat subtrees (Sec. 2.2.3-2.2.4, records "PVC2")."""
    _fields_ = [("max_len", C.c_int32), ("ans_enable", C.c_int32), ("ans_min_bytes", C.c_int32),
                ("ans_skew_num", C.c_int32), ("ans_skew_den", C.c_int32), ("ans_ratio_pct", C.c_int32),
                ("flat", C.c_int32)]


def params(max_len=11, ans=False, flat=False):
    return Params(max_len, 1 if ans else 0, 32, 5, 8, 95, 1 if flat else 0)


class PivcoError(RuntimeError):
    pass


def lib():
    """Load libpivco.so; fail loudly when it is missing (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PivcoError("libpivco.so is not built (run paper_2606_05765_gb300/build.py); "
                             "the PivCo-Huffman path has no CPU fallback")
        l = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = C.c_int32
        for name, (args, res) in _OTHER.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = res
        _lib = l
    return _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(rc, what):
    if rc != OK:
        raise PivcoError("%s failed: %s" % (what, STATUS_NAMES.get(rc, rc)))


def version():
    return lib().pivco_version().decode()


def layout_bytes():
    return lib().pivco_layout_bytes()


# ----------------------------------------------------------------- C ABI ----
def histogram(data, blk_off, hist, stream=None):
    nblk = blk_off.numel() - 1
    _check(lib().pivco_histogram(_ptr(data), _ptr(blk_off), nblk, _ptr(hist), _stream(stream)), "pivco_histogram")


def code_lengths(hist, nblk, max_len, lens, status, stream=None):
    _check(lib().pivco_code_lengths(_ptr(hist), nblk, max_len, _ptr(lens), _ptr(status), _stream(stream)),
           "pivco_code_lengths")


def build_layout(hist, lens, nblk, prm, layout, rec_bound, status, stream=None):
    _check(lib().pivco_build_layout(_ptr(hist), _ptr(lens), nblk, C.byref(prm), _ptr(layout), _ptr(rec_bound),
                                    _ptr(status), _stream(stream)), "pivco_build_layout")


def scan_workspace_size(n):
    return lib().pivco_scan_workspace_size(n)


def exclusive_scan(values, n, out, ws, status=None, stream=None):
    _check(lib().pivco_exclusive_scan(_ptr(values), n, _ptr(out), _ptr(ws), ws.numel(), _ptr(status),
                                      _stream(stream)), "pivco_exclusive_scan")


def encode_blocks(data, blk_off, nblk, layout, out, out_off, rec_bytes, status, stream=None):
    _check(lib().pivco_encode_blocks(_ptr(data), _ptr(blk_off), nblk, _ptr(layout), _ptr(out), _ptr(out_off),
                                     _ptr(rec_bytes), _ptr(status), _stream(stream)), "pivco_encode_blocks")


CHUNKS = 8


def histogram_chunks(data, blk_off, hist, chunk_hist, stream=None):
    """Block histograms plus the encoder's warp-chunk histograms ([nblk][8][256])."""
    _check(lib().pivco_histogram_chunks(_ptr(data), _ptr(blk_off), blk_off.numel() - 1, _ptr(hist), _ptr(chunk_hist),
                                        _stream(stream)), "pivco_histogram_chunks")


def plan_blocks(data, blk_off, prm, hist, chunk_hist, lens, layout, rec_bound, status, stream=None):
    """Chunk histograms, code lengths and layout of every block in one launch."""
    _check(lib().pivco_plan_blocks(_ptr(data), _ptr(blk_off), blk_off.numel() - 1, C.byref(prm), _ptr(hist),
                                   _ptr(chunk_hist), _ptr(lens), _ptr(layout), _ptr(rec_bound), _ptr(status),
                                   _stream(stream)), "pivco_plan_blocks")


def encode_blocks_chunked(data, blk_off, nblk, layout, chunk_hist, out, out_off, rec_bytes, status, stream=None):
    _check(lib().pivco_encode_blocks_chunked(_ptr(data), _ptr(blk_off), nblk, _ptr(layout), _ptr(chunk_hist),
                                             _ptr(out), _ptr(out_off), _ptr(rec_bytes), _ptr(status),
                                             _stream(stream)), "pivco_encode_blocks_chunked")


def ans_encode_blocks(layout, nblk, out, out_off, rec_bytes, ws, status, stream=None):
    _check(lib().pivco_ans_encode_blocks(_ptr(layout), nblk, _ptr(out), _ptr(out_off), _ptr(rec_bytes), _ptr(ws),
                                         ws.numel(), _ptr(status), _stream(stream)), "pivco_ans_encode_blocks")


def decode_plan_bytes(nblk):
    return lib().pivco_decode_plan_bytes(nblk)


def decode_workspace_size(comp, comp_off, nblk, ws, status, stream=None):
    need = C.c_size_t(0)
    _check(lib().pivco_decode_workspace_size(_ptr(comp), _ptr(comp_off), nblk, _ptr(ws), ws.numel(), _ptr(status),
                                             C.byref(need), _stream(stream)), "pivco_decode_workspace_size")
    return need.value


def decode_blocks(comp, comp_off, nblk, out, out_off, ws, status, stream=None, ws_bytes=None):
    _check(lib().pivco_decode_blocks(_ptr(comp), _ptr(comp_off), nblk, _ptr(out), _ptr(out_off), _ptr(ws),
                                     ws.numel() if ws_bytes is None else ws_bytes, _ptr(status), _stream(stream)),
           "pivco_decode_blocks")


DECODE_STATIC_WS_BYTES = 16 << 20


def decode_blocks_static(comp, comp_off, nblk, out, out_off, status, stream=None):
    """pivco_decode_blocks with the library's own 16 MiB device workspace,
    for callers that cannot allocate one.  Calls whose GPU work overlaps race
    on that workspace; the first call on a device should precede any stream
    capture."""
    _check(lib().pivco_decode_blocks_static(_ptr(comp), _ptr(comp_off), nblk, _ptr(out), _ptr(out_off),
                                            _ptr(status), _stream(stream)), "pivco_decode_blocks_static")


def decode_plan(comp, comp_off, nblk, ws, status, stream=None):
    _check(lib().pivco_decode_plan(_ptr(comp), _ptr(comp_off), nblk, _ptr(ws), ws.numel(), _ptr(status),
                                   _stream(stream)), "pivco_decode_plan")


def decode_ans(comp, comp_off, nblk, ws, status, stream=None):
    _check(lib().pivco_decode_ans(_ptr(comp), _ptr(comp_off), nblk, _ptr(ws), ws.numel(), _ptr(status),
                                  _stream(stream)), "pivco_decode_ans")


def decode_merge(comp, comp_off, nblk, out, out_off, ws, status, stream=None):
    _check(lib().pivco_decode_merge(_ptr(comp), _ptr(comp_off), nblk, _ptr(out), _ptr(out_off), _ptr(ws),
                                    ws.numel(), _ptr(status), _stream(stream)), "pivco_decode_merge")


class Access:
    """Random access to the symbols of a batch of records (pivco_access_*):
    prepare once (plans, ANS bitmaps, a rank directory per block), then
    query (block, position) pairs any number of times."""

    def __init__(self, comp, comp_off, nblk, stream=None):
        import torch
        dev = comp.device
        self.comp, self.comp_off, self.nblk = comp, comp_off, nblk
        self.status = torch.empty(max(nblk, 1), dtype=torch.int32, device=dev)
        self.ws = torch.empty(decode_plan_bytes(nblk), dtype=torch.uint8, device=dev)
        need = C.c_size_t(0)
        _check(lib().pivco_access_workspace_size(_ptr(comp), _ptr(comp_off), nblk, _ptr(self.ws), self.ws.numel(),
                                                 _ptr(self.status), C.byref(need), _stream(stream)),
               "pivco_access_workspace_size")
        if need.value > self.ws.numel():
            self.ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
        _check(lib().pivco_access_prepare(_ptr(comp), _ptr(comp_off), nblk, _ptr(self.ws), self.ws.numel(),
                                          _ptr(self.status), _stream(stream)), "pivco_access_prepare")

    def __call__(self, qblk, qpos, sym=None, qstatus=None, stream=None):
        """qblk, qpos: int32/uint32 CUDA tensors of equal length; returns (sym, qstatus)."""
        import torch
        nq = qblk.numel()
        sym = torch.empty(max(nq, 1), dtype=torch.uint8, device=qblk.device) if sym is None else sym
        qstatus = torch.empty(max(nq, 1), dtype=torch.int32, device=qblk.device) if qstatus is None else qstatus
        _check(lib().pivco_access(_ptr(self.comp), _ptr(self.comp_off), self.nblk, _ptr(qblk), _ptr(qpos), nq,
                                  _ptr(sym), _ptr(qstatus), _ptr(self.ws), self.ws.numel(), _ptr(self.status),
                                  _stream(stream)), "pivco_access")
        return sym[:nq], qstatus[:nq]


GOLOMB_MAX_BLOCK = 32768


def golomb_encode(data, blk_off, stream=None):
    """PivCo-Golomb records of the blocks of `data` (uint8 values): plan,
    place by an exclusive scan, encode.  Returns Encoded(comp, off, rec_bytes, status)."""
    import torch
    nblk = blk_off.numel() - 1
    dev = data.device
    size = torch.empty(max(nblk, 1), dtype=torch.int64, device=dev)
    status = torch.empty(max(nblk, 1), dtype=torch.int32, device=dev)
    _check(lib().pivco_golomb_plan(_ptr(data), _ptr(blk_off), nblk, _ptr(size), _ptr(status), _stream(stream)),
           "pivco_golomb_plan")
    off = torch.empty(nblk + 1, dtype=torch.int64, device=dev)
    ws = torch.empty(scan_workspace_size(nblk), dtype=torch.uint8, device=dev)
    exclusive_scan(size, nblk, off, ws, None, stream)
    total = int(off[-1].item()) if nblk else 0
    comp = torch.empty(max(total, 16), dtype=torch.uint8, device=dev)
    rec_bytes = torch.empty(max(nblk, 1), dtype=torch.int64, device=dev)
    _check(lib().pivco_golomb_encode(_ptr(data), _ptr(blk_off), nblk, _ptr(comp), _ptr(off), _ptr(rec_bytes),
                                     _ptr(status), _stream(stream)), "pivco_golomb_encode")
    return Encoded(comp, off, rec_bytes[:nblk], status[:nblk])


def golomb_decode(comp, comp_off, out, out_off, status, stream=None):
    _check(lib().pivco_golomb_decode(_ptr(comp), _ptr(comp_off), comp_off.numel() - 1, _ptr(out), _ptr(out_off),
                                     _ptr(status), _stream(stream)), "pivco_golomb_decode")


def launch_count():
    return int(lib().pivco_launch_count())


def set_wait_limit(ns=10 ** 9):
    """Bound (ns) of the library's device-side waits; expired waits report TIMEOUT."""
    _check(lib().pivco_set_wait_limit(int(ns)), "pivco_set_wait_limit")


def get_wait_limit():
    return int(lib().pivco_get_wait_limit())


# ------------------------------------------------------------- batching ----
class Tuning(C.Structure):
    """struct pivco_tuning: longest root tile, rank-directory granularity,
    persistent CTAs per SM.  Never changes any output."""
    _fields_ = [("tile_max", C.c_int32), ("dir_bits", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {"tile_max": self.tile_max, "dir_bits": self.dir_bits, "ctas_per_sm": self.ctas_per_sm}


def decode_batched(comp, comp_off, nblk, out, out_off, ws, status, stream=None):
    _check(lib().pivco_decode_batched(_ptr(comp), _ptr(comp_off), nblk, _ptr(out), _ptr(out_off), _ptr(ws),
                                      ws.numel(), _ptr(status), _stream(stream)), "pivco_decode_batched")


def get_tuning():
    t = Tuning()
    _check(lib().pivco_get_tuning(C.byref(t)), "pivco_get_tuning")
    return t


def set_tuning(tile_max=1 << 20, dir_bits=128, ctas_per_sm=0):
    t = Tuning(tile_max, dir_bits, ctas_per_sm, 0)
    _check(lib().pivco_set_tuning(C.byref(t)), "pivco_set_tuning")


def autotune_decode(comp, comp_off, nblk, out, out_off, ws, status, reps=3, stream=None):
    """Picks the fastest tuning for these records (synchronous); returns (Tuning, ms)."""
    best = Tuning()
    ms = C.c_float(0)
    _check(lib().pivco_autotune_decode(_ptr(comp), _ptr(comp_off), nblk, _ptr(out), _ptr(out_off), _ptr(ws),
                                       ws.numel(), _ptr(status), reps, _stream(stream), C.byref(best), C.byref(ms)),
           "pivco_autotune_decode")
    return best, ms.value


class Graph:
    """A captured sequence of library calls (CUDA graph), replayed with launch()."""

    def __init__(self, stream):
        self.stream = stream
        self.handle = C.c_void_p()

    def __enter__(self):
        _check(lib().pivco_graph_begin(_stream(self.stream)), "pivco_graph_begin")
        return self

    def __exit__(self, exc_type, exc, tb):
        rc = lib().pivco_graph_end(_stream(self.stream), C.byref(self.handle))
        if exc_type is None:
            _check(rc, "pivco_graph_end")
        return False

    def launch(self, stream=None):
        _check(lib().pivco_graph_launch(self.handle, _stream(stream or self.stream)), "pivco_graph_launch")

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.pivco_graph_destroy(self.handle)
            self.handle = C.c_void_p()


# --------------------------------------------------------- host buffers ----
class HostCodec:
    """pivco_host_codec: compress / decompress batches held in host memory,
    copies overlapped with the kernels piece by piece.  blk_off: the blocks'
    offsets (nblk + 1 integers, host).  Host buffers should be pinned CPU
    tensors (or numpy arrays)."""

    def __init__(self, blk_off, prm=None, segments=4):
        self.blk_off = np.ascontiguousarray(np.asarray(blk_off), np.uint64)
        self.nblk = self.blk_off.size - 1
        self.prm = prm or params()
        self.handle = C.c_void_p()
        _check(lib().pivco_host_codec_create(C.c_void_p(self.blk_off.ctypes.data), self.nblk, C.byref(self.prm),
                                             segments, C.byref(self.handle)), "pivco_host_codec_create")
        self.capacity = int(lib().pivco_host_codec_comp_capacity(self.handle))
        self.comp_off = np.zeros(self.nblk + 1, np.uint64)
        self.status = np.zeros(max(self.nblk, 1), np.int32)

    def compress(self, data, comp):
        """Records of `data` into `comp` (capacity >= self.capacity is always
        enough); returns (comp_off, status) as numpy arrays (views, valid
        until the next call)."""
        n = comp.numel() if hasattr(comp, "numel") else comp.size
        _check(lib().pivco_host_compress(self.handle, _host_ptr(data), _host_ptr(comp), n,
                                         C.c_void_p(self.comp_off.ctypes.data), C.c_void_p(self.status.ctypes.data)),
               "pivco_host_compress")
        return self.comp_off, self.status[: self.nblk]

    def decompress(self, comp, comp_off, out):
        """Blocks of `comp` (records at comp_off) into `out`; returns status."""
        co = np.ascontiguousarray(comp_off, np.uint64)
        _check(lib().pivco_host_decompress(self.handle, _host_ptr(comp), C.c_void_p(co.ctypes.data), _host_ptr(out),
                                           C.c_void_p(self.status.ctypes.data)), "pivco_host_decompress")
        return self.status[: self.nblk]

    def close(self):
        if self.handle:
            _check(lib().pivco_host_codec_destroy(self.handle), "pivco_host_codec_destroy")
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- serving ----
class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("idle_us", C.c_int32), ("epoch_us", C.c_int32)]


PENDING, ADMITTED, DONE = 1, 2, 3


def _host_ptr(a):
    """Address of a host buffer: a CPU torch tensor (pinned or not) or a numpy array."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise PivcoError("these buffers are host memory")
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


class Server:
    """Decompression server (pivco_server_*): a device-resident request loop
    with admission by a device-memory budget.  `arena` is a uint8 CUDA tensor
    the server lives in; it must outlive the server."""

    def __init__(self, arena, budget_bytes=0, idle_us=200, epoch_us=4000):
        self.arena = arena
        self.handle = C.c_void_p()
        cfg = ServerConfig(budget_bytes, idle_us, epoch_us)
        _check(lib().pivco_server_create(_ptr(arena), arena.numel(), C.byref(cfg), C.byref(self.handle)),
               "pivco_server_create")
        self._keep = {}

    def submit(self, comp, comp_off, out_off, out):
        """comp / out: host buffers (pinned recommended), kept alive until the
        request is done; comp_off / out_off: uint64 numpy arrays (nblk + 1)."""
        co = np.ascontiguousarray(comp_off, np.uint64)
        oo = np.ascontiguousarray(out_off, np.uint64)
        rid = C.c_uint64()
        _check(lib().pivco_server_submit(self.handle, _host_ptr(comp), C.c_void_p(co.ctypes.data), co.size - 1,
                                         C.c_void_p(oo.ctypes.data), _host_ptr(out), C.byref(rid)),
               "pivco_server_submit")
        self._keep[rid.value] = (comp, out)
        return rid.value

    def poll(self, rid):
        st, status, lat = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().pivco_server_poll(self.handle, rid, C.byref(st), C.byref(status), C.byref(lat)),
               "pivco_server_poll")
        if st.value == DONE:
            self._keep.pop(rid, None)
        return st.value, status.value, lat.value

    def drain(self, timeout_ms=60000):
        _check(lib().pivco_server_drain(self.handle, timeout_ms), "pivco_server_drain")

    def forget(self, rid):
        _check(lib().pivco_server_forget(self.handle, rid), "pivco_server_forget")

    def close(self):
        if self.handle and self.handle.value:
            rc = lib().pivco_server_destroy(self.handle)
            self.handle = C.c_void_p()
            self._keep.clear()
            _check(rc, "pivco_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
        return False

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.pivco_server_destroy(self.handle)
            self.handle = C.c_void_p()


def ans_tables():
    fq = np.zeros(50, np.int32)
    cf = np.zeros(450, np.uint32)
    _check(lib().pivco_ans_tables(C.c_void_p(fq.ctypes.data), C.c_void_p(cf.ctypes.data)), "pivco_ans_tables")
    return fq, cf.reshape(50, 9)


def ans_encode(bitmaps, bm_off, table, nbm, bodies, body_off, body_bytes, status, stream=None):
    _check(lib().pivco_ans_encode(_ptr(bitmaps), _ptr(bm_off), _ptr(table), nbm, _ptr(bodies), _ptr(body_off),
                                  _ptr(body_bytes), _ptr(status), _stream(stream)), "pivco_ans_encode")


def ans_decode(bodies, body_off, table, nbm, bitmaps, bm_off, status, stream=None):
    _check(lib().pivco_ans_decode(_ptr(bodies), _ptr(body_off), _ptr(table), nbm, _ptr(bitmaps), _ptr(bm_off),
                                  _ptr(status), _stream(stream)), "pivco_ans_decode")


# ------------------------------------------------------ batch pipelines ----
class Encoded:
    """Records of a batch: block b's record is comp[off[b] : off[b] + rec_bytes[b]]."""

    def __init__(self, comp, off, rec_bytes, status):
        self.comp, self.off, self.rec_bytes, self.status = comp, off, rec_bytes, status


class Encoder:
    """Plain (per-step launches) encoder with buffers reused across calls."""

    def __init__(self, nblk, prm=None, device="cuda"):
        import torch
        self.nblk, self.prm, self.dev = nblk, prm or params(), device
        self.hist = torch.empty(nblk * 256, dtype=torch.int32, device=device)
        self.chunk_hist = torch.empty(nblk * CHUNKS * 256, dtype=torch.int32, device=device)
        self.lens = torch.empty(nblk * 256, dtype=torch.uint8, device=device)
        self.layout = torch.empty(nblk * layout_bytes(), dtype=torch.uint8, device=device)
        self.bound = torch.empty(nblk, dtype=torch.int64, device=device)
        self.off = torch.empty(nblk + 1, dtype=torch.int64, device=device)
        self.rec_bytes = torch.empty(nblk, dtype=torch.int64, device=device)
        self.status = torch.empty(nblk, dtype=torch.int32, device=device)
        self.scan_ws = torch.empty(scan_workspace_size(nblk), dtype=torch.uint8, device=device)
        self.comp = None
        self.ans_ws = None

    def plan(self, data, blk_off, stream=None):
        """Statistics, code and layout; returns the total output bytes (synchronises)."""
        n = self.nblk
        plan_blocks(data, blk_off, self.prm, self.hist, self.chunk_hist, self.lens, self.layout, self.bound,
                    self.status, stream)
        exclusive_scan(self.bound, n, self.off, self.scan_ws, self.status, stream)
        return int(self.off[-1].item())

    def ensure(self, total):
        import torch
        if self.comp is None or self.comp.numel() < max(total, 1):
            self.comp = torch.empty(max(total, 1), dtype=torch.uint8, device=self.dev)
            if self.prm.ans_enable:
                self.ans_ws = torch.empty(max(total, 1) + 256 * self.nblk, dtype=torch.uint8, device=self.dev)

    def run(self, data, blk_off, stream=None, replan=True):
        """Full encode without host synchronisation (buffers must be sized)."""
        n = self.nblk
        if replan:
            plan_blocks(data, blk_off, self.prm, self.hist, self.chunk_hist, self.lens, self.layout, self.bound,
                        self.status, stream)
            exclusive_scan(self.bound, n, self.off, self.scan_ws, self.status, stream)
        encode_blocks_chunked(data, blk_off, n, self.layout, self.chunk_hist, self.comp, self.off, self.rec_bytes,
                              self.status, stream)
        if self.prm.ans_enable:
            ans_encode_blocks(self.layout, n, self.comp, self.off, self.rec_bytes, self.ans_ws, self.status, stream)
        return Encoded(self.comp, self.off, self.rec_bytes, self.status)

    def __call__(self, data, blk_off, stream=None):
        self.ensure(self.plan(data, blk_off, stream))
        return self.run(data, blk_off, stream, replan=False)


class Decoder:
    """Decoder.  batched=False: plan, ANS pass, rank directories and merge as
    separate launches; batched=True: one persistent work-queue launch."""

    def __init__(self, nblk, device="cuda", batched=False):
        import torch
        self.nblk, self.dev, self.batched = nblk, device, batched
        self.status = torch.empty(nblk, dtype=torch.int32, device=device)
        self.ws = torch.empty(decode_plan_bytes(nblk), dtype=torch.uint8, device=device)

    def prepare(self, comp, comp_off, stream=None):
        import torch
        need = decode_workspace_size(comp, comp_off, self.nblk, self.ws, self.status, stream)
        if need > self.ws.numel():
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.dev)
        return need

    def run(self, comp, comp_off, out, out_off, stream=None):
        if self.batched:
            decode_batched(comp, comp_off, self.nblk, out, out_off, self.ws, self.status, stream)
        else:
            decode_blocks(comp, comp_off, self.nblk, out, out_off, self.ws, self.status, stream)
        return out

    def __call__(self, comp, comp_off, out_off, stream=None):
        import torch
        self.prepare(comp, comp_off, stream)
        out = torch.empty(max(int(out_off[-1].item()), 1), dtype=torch.uint8, device=self.dev)
        return self.run(comp, comp_off, out, out_off, stream)


def encode(data, blk_off, prm=None, stream=None):
    return Encoder(blk_off.numel() - 1, prm, data.device)(data, blk_off, stream)


def decode(comp, comp_off, out_off, stream=None, batched=False):
    d = Decoder(out_off.numel() - 1, comp.device, batched=batched)
    out = d(comp, comp_off, out_off, stream)
    return out, d.status
