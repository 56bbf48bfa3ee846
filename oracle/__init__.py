"""PivCo-Huffman CPU oracle (ctypes wrapper around ``pivco_ref.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The GPU
library never imports, links or calls it, and the two share no code.

The C source restates the method of the paper (Sec. 1-5, App. D) plainly; see
its header for the step list and for the readings taken where the paper is
silent.  ``build()`` compiles it with gcc into ``oracle/liboracle.so``.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pivco_ref.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT = 0, 1, 2, 3
MARK_RAW_SELECTED = 0xFF


class Params(C.Structure):
    """Encoder parameters (App. D: L = 11; Sec. 5.2: the three ANS knobs;
    Sec. 2.2.3-2.2.4: the regrouped tree with flat subtrees)."""
    _fields_ = [("max_len", C.c_int32), ("ans_enable", C.c_int32),
                ("ans_min_bytes", C.c_int32), ("ans_skew_num", C.c_int32),
                ("ans_skew_den", C.c_int32), ("ans_ratio_pct", C.c_int32),
                ("flat", C.c_int32)]


def params(max_len=11, ans=False, flat=False):
    return Params(max_len, 1 if ans else 0, 32, 5, 8, 95, 1 if flat else 0)


def build(force=False):
    """Compile the oracle with gcc (plain C, -O2; no vector intrinsics)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        u64, i32, u32 = C.c_uint64, C.c_int32, C.c_uint32
        sig = {
            "ref_histogram": [P, u64, P],
            "ref_code_lengths": [P, C.c_int, P],
            "ref_canonical_codes": [P, P],
            "ref_tree_info": [P, P, P, P, P],
            "ref_tree_info_ex": [P, C.c_int, P, P, P, P, P, P],
            "ref_flat_codes": [P, P, P],
            "ref_ans_class_freqs": [C.c_int, P],
            "ref_fse_h_q16": [C.c_int],
            "ref_rans_encode": [P, u32, C.c_int, P, u64, P],
            "ref_rans_decode": [P, u64, C.c_int, P, u32],
            "ref_ans_select": [u64, u64, C.c_int, P],
            "ref_record_bound": [P, P, P],
            "ref_encode_block": [P, u64, P, P, u64, P],
            "ref_decode_block": [P, u64, P, u64, P],
            "ref_encode_batch": [P, P, C.c_int, P, P, P, P, P],
            "ref_decode_batch": [P, P, P, C.c_int, P, P, P],
            "ref_golomb_bound": [P, u64, P],
            "ref_golomb_encode": [P, u64, P, u64, P],
            "ref_golomb_decode": [P, u64, P, u64, P],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _lib.ref_binary_entropy.argtypes = [C.c_double]
        _lib.ref_binary_entropy.restype = C.c_double
        _lib.ref_node_benefit.argtypes = [u64, u64, u64]
        _lib.ref_node_benefit.restype = C.c_double
        _lib.ref_fse_h.argtypes = [C.c_int]
        _lib.ref_fse_h.restype = C.c_double
        del i32
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data)


def _check(rc, what):
    if rc != OK:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def histogram(x):
    x = np.ascontiguousarray(x, dtype=np.uint8)
    h = np.zeros(256, np.uint32)
    _check(lib().ref_histogram(_p(x), x.size, _p(h)), "histogram")
    return h


def code_lengths(hist, max_len=11):
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    lens = np.zeros(256, np.uint8)
    _check(lib().ref_code_lengths(_p(h), max_len, _p(lens)), "code_lengths")
    return lens


def canonical_codes(lens):
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    codes = np.zeros(256, np.uint32)
    _check(lib().ref_canonical_codes(_p(lens), _p(codes)), "canonical_codes")
    return codes


def tree_info(lens):
    """(depth[V], prefix[V], child[V,2]); child >= 0 internal id, < 0 leaf -(sym+1)."""
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    nv = np.zeros(1, np.int32)
    depth = np.zeros(256, np.int32)
    prefix = np.zeros(256, np.uint32)
    child = np.zeros(512, np.int32)
    _check(lib().ref_tree_info(_p(lens), _p(nv), _p(depth), _p(prefix), _p(child)), "tree_info")
    V = int(nv[0])
    return depth[:V].copy(), prefix[:V].copy(), child[:2 * V].reshape(V, 2).copy()


def flat_codes(lens):
    """Regrouped codes (Sec. 2.2.4): (codes[256], fd[256]); fd[s] is the
    depth D of the flat node symbol s belongs to, 0 if none."""
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    codes = np.zeros(256, np.uint32)
    fd = np.zeros(256, np.int32)
    _check(lib().ref_flat_codes(_p(lens), _p(codes), _p(fd)), "flat_codes")
    return codes, fd


def tree_info_ex(lens, flat=True):
    """(depth[V], prefix[V], child[V,2], D[V], ftab[V,256]) of the canonical
    (flat=False) or regrouped (flat=True) tree; D = 0 for ordinary nodes,
    ftab[v, x] = symbol of index x of flat node v (-1 past 2^D)."""
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    nv = np.zeros(1, np.int32)
    depth = np.zeros(256, np.int32)
    prefix = np.zeros(256, np.uint32)
    child = np.zeros(512, np.int32)
    fdep = np.zeros(256, np.int32)
    ftab = np.zeros(256 * 256, np.int32)
    _check(lib().ref_tree_info_ex(_p(lens), 1 if flat else 0, _p(nv), _p(depth), _p(prefix), _p(child), _p(fdep),
                                  _p(ftab)), "tree_info_ex")
    V = int(nv[0])
    return (depth[:V].copy(), prefix[:V].copy(), child[:2 * V].reshape(V, 2).copy(), fdep[:V].copy(),
            ftab[:256 * V].reshape(V, 256).copy())


def ans_class_freqs(t):
    q = np.zeros(9, np.uint32)
    _check(lib().ref_ans_class_freqs(t, _p(q)), "ans_class_freqs")
    return q


def fse_h(t):
    return lib().ref_fse_h(t)


def binary_entropy(p):
    return lib().ref_binary_entropy(p)


def node_benefit(n_v, n1, n_total):
    """Sec. 5.1: (n_v / n_total) * (1 - H_b(max(n0, n1) / n_v))."""
    return lib().ref_node_benefit(n_v, n1, n_total)


def fse_h_q16(t):
    return lib().ref_fse_h_q16(t)


def rans_encode(data, t):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    cap = 4 * ((data.size + 16383) // 16384) * 34 + 2 * data.size + 64
    body = np.zeros(cap, np.uint8)
    nb = np.zeros(1, np.uint64)
    _check(lib().ref_rans_encode(_p(data), data.size, t, _p(body), cap, _p(nb)), "rans_encode")
    return body[: int(nb[0])].copy()


def rans_decode(body, nbytes, t):
    body = np.ascontiguousarray(body, dtype=np.uint8)
    out = np.zeros(nbytes, np.uint8)
    rc = lib().ref_rans_decode(_p(body), body.size, t, _p(out), nbytes)
    if rc != OK:
        raise ValueError("corrupt ANS body (status %d)" % rc)
    return out


def ans_select(n_v, n1, depth, prm=None):
    prm = prm or params(ans=True)
    return lib().ref_ans_select(n_v, n1, depth, C.byref(prm))


def record_bound(hist, prm=None):
    prm = prm or params()
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    b = np.zeros(1, np.uint64)
    _check(lib().ref_record_bound(_p(h), C.byref(prm), _p(b)), "record_bound")
    return int(b[0])


def encode_block(x, prm=None):
    prm = prm or params()
    x = np.ascontiguousarray(x, dtype=np.uint8)
    cap = record_bound(histogram(x), prm)
    rec = np.zeros(cap, np.uint8)
    nb = np.zeros(1, np.uint64)
    _check(lib().ref_encode_block(_p(x), x.size, C.byref(prm), _p(rec), cap, _p(nb)), "encode_block")
    return rec[: int(nb[0])].copy()


def decode_block(rec, cap=None):
    """Returns (status, symbols)."""
    rec = np.ascontiguousarray(rec, dtype=np.uint8)
    if cap is None:
        cap = int(np.frombuffer(rec[4:8].tobytes(), np.uint32)[0]) if rec.size >= 8 else 0
    out = np.zeros(max(cap, 1), np.uint8)
    n = np.zeros(1, np.uint64)
    rc = lib().ref_decode_block(_p(rec), rec.size, _p(out), cap, _p(n))
    return rc, out[: int(n[0])].copy() if rc == OK else None


def encode_batch(x, blk_off, prm=None):
    """Encode every block; records are laid out densely.  Returns (buf, rec_off, rec_bytes)."""
    prm = prm or params()
    x = np.ascontiguousarray(x, dtype=np.uint8)
    blk_off = np.ascontiguousarray(blk_off, dtype=np.uint64)
    nblk = blk_off.size - 1
    recs = [encode_block(x[int(blk_off[b]):int(blk_off[b + 1])], prm) for b in range(nblk)]
    sizes = np.array([r.size for r in recs], np.uint64)
    rec_off = np.zeros(nblk + 1, np.uint64)
    rec_off[1:] = np.cumsum(sizes)
    buf = np.concatenate(recs) if recs else np.zeros(0, np.uint8)
    return buf, rec_off, sizes


def encode_batch_native(x, blk_off, rec_off, rec_cap, prm=None):
    """One C call over all blocks (used for timing): records at rec_off."""
    prm = prm or params()
    nblk = blk_off.size - 1
    buf = np.zeros(int(rec_off[-1]), np.uint8)
    nb = np.zeros(nblk, np.uint64)
    _check(lib().ref_encode_batch(_p(x), _p(blk_off), nblk, C.byref(prm), _p(buf), _p(rec_off), _p(rec_cap), _p(nb)),
           "encode_batch")
    return buf, nb


def decode_batch(buf, rec_off, rec_avail, out_off):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    nblk = rec_off.size - 1 if rec_off.size == rec_avail.size + 1 else rec_off.size
    out = np.zeros(max(int(out_off[-1]), 1), np.uint8)
    st = np.zeros(nblk, np.int32)
    lib().ref_decode_batch(_p(buf), _p(np.ascontiguousarray(rec_off, np.uint64)),
                           _p(np.ascontiguousarray(rec_avail, np.uint64)), nblk, _p(out),
                           _p(np.ascontiguousarray(out_off, np.uint64)), _p(st))
    return st, out[: int(out_off[-1])]


# ---------------------------------------------------------------- PivCo-Golomb
def golomb_encode(x):
    """PivCo-Golomb record of the values x (App. G; see the C header)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    bound = np.zeros(1, np.uint64)
    _check(lib().ref_golomb_bound(_p(x), x.size, _p(bound)), "golomb_bound")
    rec = np.zeros(int(bound[0]), np.uint8)
    nb = np.zeros(1, np.uint64)
    _check(lib().ref_golomb_encode(_p(x), x.size, _p(rec), rec.size, _p(nb)), "golomb_encode")
    return rec[: int(nb[0])]


def golomb_decode(rec, cap=None):
    """(status, values) of a PivCo-Golomb record."""
    rec = np.ascontiguousarray(rec, dtype=np.uint8)
    cap = (1 << 32) - 1 if cap is None else cap
    n = np.zeros(1, np.uint64)
    rc = lib().ref_golomb_decode(_p(rec), rec.size, None, 0, _p(n))
    if rc not in (OK, ERR_CAPACITY):
        return rc, None
    out = np.zeros(max(int(n[0]), 1), np.uint8)
    rc = lib().ref_golomb_decode(_p(rec), rec.size, _p(out), min(cap, out.size), _p(n))
    return rc, out[: int(n[0])] if rc == OK else None
