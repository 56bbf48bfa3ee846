"""Oracle pins for flat subtrees and the regrouped tree (Sec. 2.2.3-2.2.4,
App. D), checked against things other than the oracle's own code: a record
derived by hand for the Sec. 2.2 example, Table 7's node count, special cases
that reduce to plain bit packing, properties the regrouping must keep
(lengths, prefix-freeness, Kraft equality, total bits) and a bottom-up decode
restated from the merge primitives of Sec. 3.2 (a different algorithm from the
oracle's top-down cursor walk)."""
import json
import os

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
PINS = json.load(open(os.path.join(HERE, "golden", "paper_pins.json")))


def _header(rec):
    n = int(rec[4:8].view(np.uint32)[0])
    V = int(rec[8:10].view(np.uint16)[0])
    return n, V


def _bodies(rec, D):
    """Raw bodies of every node (records without ANS nodes); a flat node's
    marker byte is 0xF0 + D, an ordinary raw node's 0."""
    n, V = _header(rec)
    nv = rec[144:144 + 4 * V].view(np.uint32).astype(np.int64)
    marker = rec[144 + 4 * V:144 + 5 * V]
    assert list(marker) == [0xF0 + int(d) if d else 0 for d in D]
    off = (144 + 5 * V + 3) & ~3
    out = []
    for v in range(V):
        nb = (int(nv[v]) * max(int(D[v]), 1) + 7) // 8
        out.append(rec[off:off + nb])
        off += nb
    return nv, out, off


def test_hand_derived_record(oracle):
    g = PINS["coconut_papaya_flat_hand_derived"]
    x = np.frombuffer(g["word"].encode(), np.uint8)
    lens = oracle.code_lengths(oracle.histogram(x))
    assert {chr(s): int(lens[s]) for s in np.nonzero(lens)[0]} == g["lens"]
    rec = oracle.encode_block(x, oracle.params(flat=True))
    assert rec.size == g["record_bytes"] and bytes(rec[12:16]) == b"PVC2"
    depth, prefix, child, D, ftab = oracle.tree_info_ex(lens, flat=True)
    assert list(D) == g["flat_depth"]
    for v, syms in g["flat_symbols"].items():
        assert "".join(chr(c) for c in ftab[int(v)][: 1 << D[int(v)]]) == syms
    nv, bodies, end = _bodies(rec, D)
    assert list(nv) == g["n_v"]
    assert list(rec[144 + 16:144 + 20]) == g["markers"]
    assert [list(b) for b in bodies] == g["bodies"]
    assert not rec[end:].any()
    st, y = oracle.decode_block(rec)
    assert st == 0 and bytes(y) == g["word"].encode()


def test_table7_proba80_node_count(oracle):
    """Table 7: no length class of proba80 has four symbols, so the
    flat-opt tree has the naive tree's 5 nodes (a pair stays a node)."""
    g = PINS["table7_flat_nodes"]
    lens = np.zeros(256, np.uint8)
    lens[: g["proba80_symbols"]] = g["proba80_lens"]
    assert len(oracle.tree_info(lens)[0]) == g["naive_nodes"]
    depth, prefix, child, D, ftab = oracle.tree_info_ex(lens, flat=True)
    assert len(depth) == g["flat_opt_nodes"] and not D.any()


def test_uniform_256_is_the_input(oracle):
    """256 equally frequent bytes: all codes have 8 bits, the whole alphabet
    is one group of 2^8 under the root, and index x of the group is byte x.
    The record holds one flat node whose body is the block itself."""
    rng = np.random.default_rng(7)
    x = np.repeat(np.arange(256, dtype=np.uint8), 40)
    rng.shuffle(x)
    rec = oracle.encode_block(x, oracle.params(flat=True))
    n, V = _header(rec)
    assert V == 1 and n == x.size
    D = oracle.tree_info_ex(oracle.code_lengths(oracle.histogram(x)), flat=True)[3]
    assert list(D) == [8]
    nv, bodies, _ = _bodies(rec, D)
    assert np.array_equal(bodies[0], x)


def test_four_symbols_pack_two_bits(oracle):
    """Four equally frequent bytes: one flat node of depth 2 at the root,
    its body the 2-bit ranks of the symbols packed LSB first (App. D)."""
    rng = np.random.default_rng(8)
    alpha = np.array([10, 20, 200, 201], np.uint8)
    x = np.repeat(alpha, 25)
    rng.shuffle(x)
    rec = oracle.encode_block(x, oracle.params(flat=True))
    D = oracle.tree_info_ex(oracle.code_lengths(oracle.histogram(x)), flat=True)[3]
    assert list(D) == [2]
    _, bodies, _ = _bodies(rec, D)
    rank = np.searchsorted(alpha, x)
    packed = np.zeros(x.size * 2, np.uint8)
    packed[0::2] = rank & 1
    packed[1::2] = rank >> 1
    assert np.array_equal(bodies[0], np.packbits(packed, bitorder="little"))


def _lens_cases():
    rng = np.random.default_rng(11)
    cases = []
    for k in (2, 3, 5, 17, 64, 130, 255, 256):
        for s in (0.0, 0.7, 1.3):
            f = np.zeros(256, np.uint32)
            f[rng.permutation(256)[:k]] = np.maximum(1, (5000 / np.arange(1, k + 1) ** s).astype(np.int64))
            cases.append(f)
    return cases


@pytest.mark.parametrize("case", range(24))
def test_regrouping_keeps_lengths_and_is_prefix_free(oracle, case):
    """Sec. 2.2.4: the regrouped tree has exactly the same code lengths; its
    codes are still a complete prefix code (Kraft equality, no code a prefix
    of another), so every symbol still has a leaf."""
    hist = _lens_cases()[case]
    for L in (11, 9):
        lens = oracle.code_lengths(hist, L)
        codes, fd = oracle.flat_codes(lens)
        syms = [s for s in range(256) if lens[s]]
        words = sorted(format(int(codes[s]), "0%db" % lens[s]) for s in syms)
        assert all(len(format(int(codes[s]), "b")) <= lens[s] for s in syms)
        for a, b in zip(words, words[1:]):      # sorted: a prefix sits just before its extensions
            assert not b.startswith(a)
        assert sum(2.0 ** -int(lens[s]) for s in syms) == 1.0
        # a flat group is 2^D symbols of one length, ascending in index order
        for D in set(fd[fd > 0].tolist()):
            members = [s for s in syms if fd[s] == D]
            assert len(members) % (1 << D) == 0


@pytest.mark.parametrize("case", range(24))
def test_groups_are_the_binary_digits_of_each_class(oracle, case):
    """Sec. 2.2.4 combines the largest power of two of each length class
    and repeats: the group sizes of a class are the powers of two of its
    size's binary digits; the flat nodes are those of 4 or more."""
    hist = _lens_cases()[case]
    lens = oracle.code_lengths(hist)
    depth, prefix, child, D, ftab = oracle.tree_info_ex(lens, flat=True)
    for l in range(1, 12):
        size = int((lens == l).sum())
        want = sorted(1 << b for b in range(9) if size >> b & 1 and b >= 2)
        got = sorted(1 << int(D[v]) for v in range(len(D)) if D[v] and int(depth[v]) + int(D[v]) == l)
        assert got == want, (l, size)
    # nodes: one per item except the leaves' parents' count; a flat node
    # replaces 2^D - 1 ordinary nodes with one
    K = int((lens > 0).sum())
    assert len(D) == K - 1 - sum((1 << int(d)) - 2 for d in D if d)


@pytest.mark.parametrize("wl", ["zipf1", "skew80", "skew95", "mixed"])
def test_total_bits_unchanged(oracle, wl):
    """Sum over nodes of n_v * D_v (D = 1 for ordinary nodes) equals
    sum f_s l_s: regrouping keeps the average code length (Sec. 2.2.4)."""
    w = workloads.by_name(wl, nblk=6) if wl != "zipf1" else workloads.zipf1(n=1 << 16)
    for b in range(min(w.nblk, 6)):
        x = w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])]
        h = oracle.histogram(x)
        lens = oracle.code_lengths(h)
        if (lens > 0).sum() < 2:
            continue
        rec = oracle.encode_block(x, oracle.params(flat=True))
        D = oracle.tree_info_ex(lens, flat=True)[3]
        nv, _, _ = _bodies(rec, D)
        assert int((nv * np.maximum(D, 1)).sum()) == int((h.astype(np.int64) * lens).sum())


def _bottom_up(rec, lens, oracle):
    """Sec. 3.2 bottom-up: children before parents; an ordinary node merges
    its children's outputs by its bitmap (MVV/MCV/MVC/MCC), a flat node maps
    each D-bit index through its symbol table (merge_flat_D)."""
    depth, prefix, child, D, ftab = oracle.tree_info_ex(lens, flat=True)
    nv, bodies, _ = _bodies(rec, D)
    out = [None] * len(D)
    for v in sorted(range(len(D)), key=lambda v: -int(depth[v])):
        if D[v]:
            bits = np.unpackbits(bodies[v], bitorder="little")[: int(nv[v]) * int(D[v])].reshape(-1, int(D[v]))
            idx = (bits.astype(np.int64) << np.arange(int(D[v]))).sum(axis=1)
            out[v] = ftab[v][idx].astype(np.uint8)
            continue
        bits = np.unpackbits(bodies[v], bitorder="little")[: int(nv[v])].astype(bool)
        res = np.zeros(int(nv[v]), np.uint8)
        for b, sel in ((0, ~bits), (1, bits)):
            c = int(child[v][b])
            res[sel] = out[c] if c >= 0 else np.uint8(-c - 1)
        out[v] = res
    return out[0]


@pytest.mark.parametrize("wl", ["zipf1", "skew80", "mixed"])
def test_bottom_up_merge_decodes(oracle, wl):
    w = workloads.by_name(wl, nblk=5) if wl != "zipf1" else workloads.zipf1(n=1 << 15)
    for b in range(min(w.nblk, 5)):
        x = w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])][: 1 << 15]
        lens = oracle.code_lengths(oracle.histogram(x))
        if (lens > 0).sum() < 2:
            continue
        rec = oracle.encode_block(x, oracle.params(flat=True))
        assert np.array_equal(_bottom_up(rec, lens, oracle), x)


@pytest.mark.parametrize("ans", [False, True])
@pytest.mark.parametrize("wl", ["skew95", "mixed"])
def test_round_trip_and_no_ans_on_flat_nodes(oracle, wl, ans):
    w = workloads.by_name(wl, nblk=6)
    for b in range(6):
        x = w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])]
        rec = oracle.encode_block(x, oracle.params(ans=ans, flat=True))
        st, y = oracle.decode_block(rec)
        assert st == 0 and np.array_equal(y, x)
        n, V = _header(rec)
        lens = oracle.code_lengths(oracle.histogram(x))
        if V:
            D = oracle.tree_info_ex(lens, flat=True)[3]
            marker = rec[144 + 4 * V:144 + 5 * V]
            assert list(marker[D > 0]) == [0xF0 + int(d) for d in D[D > 0]]
            # the canonical record of the same block decodes to the same bytes
            rec1 = oracle.encode_block(x, oracle.params(ans=ans))
            assert oracle.decode_block(rec1)[1].tobytes() == x.tobytes()


@pytest.mark.parametrize("x", [np.zeros(0, np.uint8), np.full(9, 7, np.uint8), np.array([1, 2], np.uint8),
                               np.array([3, 3, 3, 4], np.uint8), np.arange(256, dtype=np.uint8),
                               np.arange(255, dtype=np.uint8), np.arange(4, dtype=np.uint8)])
def test_degenerate_blocks(oracle, x):
    rec = oracle.encode_block(x, oracle.params(flat=True))
    assert bytes(rec[12:16]) == b"PVC2"
    st, y = oracle.decode_block(rec)
    assert st == 0 and np.array_equal(y, x)


def test_corrupt_flat_records_are_refused(oracle):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 8, 1001).astype(np.uint8)          # 8 symbols: one flat node of 8
    rec = oracle.encode_block(x, oracle.params(flat=True))
    lens = oracle.code_lengths(oracle.histogram(x))
    D = oracle.tree_info_ex(lens, flat=True)[3]
    assert list(D) == [3]
    # the same record read as a canonical tree: wrong node count
    bad = rec.copy(); bad[15] = ord("1")
    assert oracle.decode_block(bad)[0] == 3
    # a pad bit past n * D set
    nv, bodies, end = _bodies(rec, D)
    assert int(nv[0]) * 3 % 8 == 3
    bad = rec.copy(); bad[end - 1] |= 0x80
    assert oracle.decode_block(bad)[0] == 3
    # a flat node marked as ANS coded, raw, or flat of another depth
    for m in (5, 0, 0xF2, 0xF4):
        bad = rec.copy(); bad[144 + 4] = m
        assert oracle.decode_block(bad)[0] == 3
