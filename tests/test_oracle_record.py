"""Oracle pins for the block record: layout invariants, degenerate blocks,
round trips on every workload shape, corruption detection."""
import numpy as np
import pytest

import workloads


def parse(rec):
    hdr = np.frombuffer(rec[:8].tobytes(), np.uint32)
    V = int(rec[8]) | int(rec[9]) << 8
    out = {"rec_bytes": int(hdr[0]), "n": int(hdr[1]), "V": V, "kind": int(rec[10]), "aux": int(rec[11])}
    if out["kind"] == 2:
        lens = np.zeros(256, np.uint8)
        lens[0::2] = rec[16:144] & 15
        lens[1::2] = rec[16:144] >> 4
        out["lens"] = lens
        out["nv"] = np.frombuffer(rec[144:144 + 4 * V].tobytes(), np.uint32).astype(np.int64)
        out["marker"] = rec[144 + 4 * V:144 + 5 * V].copy()
        off = (144 + 5 * V + 3) & ~3
        nsel = int(np.count_nonzero(out["marker"]))
        out["alen"] = np.frombuffer(rec[off:off + 4 * nsel].tobytes(), np.uint32).astype(np.int64)
        off += 4 * nsel
        bodies = {}
        for v in range(V):
            if out["marker"][v] == 0:
                b = (out["nv"][v] + 7) // 8
                bodies[v] = rec[off:off + b]
                off += b
        k = 0
        for v in range(V):
            if out["marker"][v]:
                bodies[v] = rec[off:off + out["alen"][k]]
                off += out["alen"][k]
                k += 1
        out["bodies"] = bodies
        out["end"] = off
    return out


def test_degenerate_blocks(oracle):
    for x, kind in [(b"", 0), (b"a", 1), (b"zzzz", 1)]:
        rec = oracle.encode_block(np.frombuffer(x, np.uint8))
        p = parse(rec)
        assert rec.size == 16 and p["kind"] == kind and p["n"] == len(x)
        assert bytes(rec[12:16]) == b"PVC1"
        st, y = oracle.decode_block(rec)
        assert st == 0 and y.tobytes() == x
    rec = oracle.encode_block(np.frombuffer(b"ab", np.uint8))
    p = parse(rec)
    assert p["kind"] == 2 and p["V"] == 1 and list(p["nv"]) == [2]
    assert oracle.decode_block(rec)[1].tobytes() == b"ab"


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 65535])
@pytest.mark.parametrize("K", [2, 3, 17, 256])
def test_round_trip_sizes(oracle, n, K):
    rng = np.random.default_rng(n * 1000 + K)
    x = rng.integers(0, K, n).astype(np.uint8)
    for ans in (False, True):
        rec = oracle.encode_block(x, oracle.params(ans=ans))
        st, y = oracle.decode_block(rec)
        assert st == 0 and np.array_equal(x, y)


def _bitmaps_raw(p):
    return {v: np.unpackbits(np.asarray(b, np.uint8), bitorder="little")[:p["nv"][v]]
            for v, b in p["bodies"].items() if p["marker"][v] in (0, 0xFF)}


def test_layout_invariants(oracle):
    """n_root = n; popcount(B_v) = n_right (App. D); sum n_v = sum f l; pad bits 0."""
    rng = np.random.default_rng(21)
    for trial in range(25):
        K = int(rng.integers(2, 257))
        x = rng.choice(K, int(rng.integers(2, 30000)), p=rng.dirichlet(np.ones(K) * 0.3)).astype(np.uint8)
        if np.unique(x).size < 2:
            continue
        h = oracle.histogram(x)
        lens = oracle.code_lengths(h)
        rec = oracle.encode_block(x)
        p = parse(rec)
        assert p["rec_bytes"] == rec.size and rec.size % 16 == 0
        assert p["nv"][0] == x.size
        assert int(p["nv"].sum()) == int((h.astype(np.int64) * lens).sum())
        assert np.all(rec[p["end"]:] == 0)
        depth, prefix, child = oracle.tree_info(lens)
        bm = _bitmaps_raw(p)
        for v in range(p["V"]):
            ones = int(bm[v].sum())
            r = child[v, 1]
            n_right = p["nv"][r] if r >= 0 else int(h[-r - 1])
            assert ones == n_right
            nbytes = (p["nv"][v] + 7) // 8
            tail = np.unpackbits(np.asarray(p["bodies"][v], np.uint8), bitorder="little")[p["nv"][v]:8 * nbytes]
            assert not tail.any()
        assert rec.size == oracle.record_bound(h)


def test_definition_of_node_bitmaps(oracle):
    """B_v lists bit d of the code of each symbol under prefix v, in block order."""
    rng = np.random.default_rng(4)
    x = rng.choice(40, 5000, p=rng.dirichlet(np.ones(40))).astype(np.uint8)
    h = oracle.histogram(x)
    lens = oracle.code_lengths(h)
    codes = oracle.canonical_codes(lens)
    p = parse(oracle.encode_block(x))
    bm = _bitmaps_raw(p)
    depth, prefix, child = oracle.tree_info(lens)
    strs = {s: format(int(codes[s]), "0%db" % lens[s]) for s in range(256) if lens[s]}
    for v in range(p["V"]):
        pre = format(int(prefix[v]), "0%db" % depth[v]) if depth[v] else ""
        want = [int(strs[s][depth[v]]) for s in x if strs[s].startswith(pre) and len(strs[s]) > depth[v]]
        assert list(bm[v]) == want


@pytest.mark.parametrize("name,kw", [
    ("zipf1", dict(n=1 << 16)),
    ("skew80", dict(nblk=6, bs=65536)),
    ("skew95", dict(nblk=3, bs=131072)),
    ("mixed", dict(nblk=12, hi=1 << 17)),
])
def test_round_trip_workloads(oracle, name, kw):
    w = workloads.by_name(name, **kw)
    buf, rec_off, sizes = oracle.encode_batch(w.data, w.blk_off, oracle.params(ans=w.ans))
    st, out = oracle.decode_batch(buf, rec_off[:-1], sizes, w.blk_off)
    assert not st.any()
    assert np.array_equal(out, w.data)


def test_skew95_selects_root_ans(oracle):
    """The 0.95-skew configuration ANS-codes its root (Sec. 5.2 rule) and shrinks."""
    w = workloads.skew95(nblk=1, bs=131072)
    rec_ans = oracle.encode_block(w.data, oracle.params(ans=True))
    rec_raw = oracle.encode_block(w.data, oracle.params(ans=False))
    p = parse(rec_ans)
    assert p["marker"][0] not in (0, 0xFF) and p["marker"][0] & 0x7F == 95 - 49
    assert rec_ans.size < 0.6 * rec_raw.size
    assert oracle.decode_block(rec_ans)[1].tobytes() == w.data.tobytes()


def test_permuted_byte_values_same_cost(oracle):
    """Nothing depends on which byte value carries which rank."""
    a = workloads.skew80(nblk=1, bs=65536)
    b = workloads.skew80(nblk=1, bs=65536, permute=True)
    ha, hb = oracle.histogram(a.data), oracle.histogram(b.data)
    ca = int((ha.astype(np.int64) * oracle.code_lengths(ha)).sum())
    cb = int((hb.astype(np.int64) * oracle.code_lengths(hb)).sum())
    assert ca == cb


def test_corruption_detected(oracle):
    rng = np.random.default_rng(8)
    x = rng.choice(30, 20000, p=rng.dirichlet(np.ones(30))).astype(np.uint8)
    rec = oracle.encode_block(x)
    cases = []
    bad = rec.copy(); bad[12] = ord("X"); cases.append(bad)              # magic
    bad = rec.copy(); bad[0] = (bad[0] + 16) & 0xFF; cases.append(bad)   # size
    bad = rec.copy(); bad[144] ^= 1; cases.append(bad)                   # n_root
    V = int(rec[8])
    bad = rec.copy(); bad[144 + 4 * V] = 77; cases.append(bad)           # marker id 77
    bad = rec.copy(); bad[16] = 0xFF; cases.append(bad)                  # lengths break Kraft
    for bad in cases:
        st, _ = oracle.decode_block(bad, cap=x.size)
        assert st != 0
    st, _ = oracle.decode_block(rec[:-16], cap=x.size)
    assert st != 0
    st, _ = oracle.decode_block(rec, cap=x.size - 1)
    assert st != 0
