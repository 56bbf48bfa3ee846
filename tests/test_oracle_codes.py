"""Oracle pins for code construction: lengths, canonical codes, tree, bitmaps.

Every test here checks the oracle against something other than itself: values
the paper prints for its worked examples (tests/golden/paper_pins.json),
brute-force optimality, Kraft's equality, a textbook heap Huffman, and the
closed form of the proba80 distribution.
"""
import heapq
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))


def word_hist(word):
    h = np.zeros(256, np.uint32)
    for ch in word.encode():
        h[ch] += 1
    return h


def code_str(codes, lens, s):
    return format(int(codes[s]), "0%db" % int(lens[s]))


def test_huffman_h_is_101(oracle):
    """Sec. 1.1 / Listing 1: 'h' decodes with the bits 1 0 1."""
    g = GOLD["huffman_word"]
    lens = oracle.code_lengths(word_hist(g["value"]))
    codes = oracle.canonical_codes(lens)
    assert code_str(codes, lens, ord("h")) == g["h_code"]


def test_huffman_bitmaps_hand_derived(oracle):
    """The pivoted bitmaps of 'huffman', derived by hand (Sec. 2 layout)."""
    g = GOLD["huffman_bitmaps_hand_derived"]
    rec = oracle.encode_block(np.frombuffer(b"huffman", np.uint8))
    V = int(rec[8])
    assert V == len(g["nodes"])
    nv = np.frombuffer(rec[144:144 + 4 * V].tobytes(), np.uint32)
    off = (144 + 5 * V + 3) & ~3            # no ANS: no alen table
    depth, prefix, child = oracle.tree_info(oracle.code_lengths(word_hist("huffman")))
    for v, node in enumerate(g["nodes"]):
        d = len(node["prefix"])
        assert depth[v] == d and (d == 0 or prefix[v] == int(node["prefix"], 2))
        assert nv[v] == node["n"]
        nbytes = (node["n"] + 7) // 8
        assert list(rec[off:off + nbytes]) == [node["byte"]]
        bits = "".join(str((node["byte"] >> j) & 1) for j in range(node["n"]))
        assert bits == node["bits"]
        off += nbytes


def test_coconut_papaya_ops_and_subtrees(oracle):
    """Sec. 2.2: 4.071 ops/B naive, 3.286 with merged leaves; Sec. 2.2.3/2.2.4 shapes."""
    g = GOLD["coconut_papaya"]
    w = g["word"]
    h = word_hist(w)
    lens = oracle.code_lengths(h)
    codes = oracle.canonical_codes(lens)
    n = len(w)
    # naive top-down: len(code) partitions + 1 scatter per symbol (Sec. 2.1)
    naive = sum(int(h[s]) * (int(lens[s]) + 1) for s in range(256))
    assert round(naive / n, 3) == g["ops_per_byte_naive"]
    # merged leaves: a symbol whose sibling is also a leaf needs len(code) ops
    depth, prefix, child = oracle.tree_info(lens)
    paired = set()
    for v in range(len(depth)):
        if child[v, 0] < 0 and child[v, 1] < 0:
            paired.update([-child[v, 0] - 1, -child[v, 1] - 1])
    merged = sum(int(h[s]) * (int(lens[s]) + (0 if s in paired else 1)) for s in range(256))
    assert round(merged / n, 3) == g["ops_per_byte_merged_leaves"]
    # '- n t u': all four leaves of one internal node's subtree, same length
    flat = [ord(c) for c in g["flat_subtree"]]
    L = {int(lens[s]) for s in flat}
    assert len(L) == 1
    top = {code_str(codes, lens, s)[:-2] for s in flat}
    assert len(top) == 1                          # one depth-(L-2) subtree holds exactly these 4
    root4 = next(iter(top))
    under = [s for s in range(256) if lens[s] and code_str(codes, lens, s).startswith(root4)]
    assert sorted(under) == sorted(flat)
    # 'c o p y': same length, but no single subtree holds exactly those four
    cop = [ord(c) for c in g["same_length_not_one_subtree"]]
    assert len({int(lens[s]) for s in cop}) == 1
    strs = [code_str(codes, lens, s) for s in cop]
    assert len({s[:-2] for s in strs}) == 2


def _cost(h, lens):
    return int(sum(int(h[s]) * int(lens[s]) for s in range(256)))


def _brute_min(freqs, L):
    K = len(freqs)
    best = None
    for ls in itertools.product(range(1, L + 1), repeat=K):
        if sum(2.0 ** -l for l in ls) <= 1.0 + 1e-12:
            c = sum(f * l for f, l in zip(freqs, ls))
            best = c if best is None or c < best else best
    return best


@pytest.mark.parametrize("K", [2, 3, 4, 5, 6, 7, 8])
def test_lengths_bruteforce_optimal(oracle, K):
    """Optimal under the length limit: equals exhaustive search (K <= 8)."""
    rng = np.random.default_rng(100 + K)
    for trial in range(6):
        syms = rng.choice(256, K, replace=False)
        f = rng.integers(1, 1000, K)
        if trial % 2:
            f = (rng.pareto(1.0, K) * 50).astype(int) + 1     # skewed: the limit binds
        Lmin = max(1, math.ceil(math.log2(K)))
        for L in sorted({Lmin, min(Lmin + 1, 15), 4, 5} - set(range(0, Lmin))):
            if K == 8 and L > 4:
                continue
            h = np.zeros(256, np.uint32)
            h[syms] = f
            lens = oracle.code_lengths(h, L)
            assert lens.max() <= L
            assert _cost(h, lens) == _brute_min(list(f), L), (K, L, f)


def _kraft(lens):
    return sum(2.0 ** -int(l) for l in lens if l)


def test_kraft_equality_and_limit(oracle):
    rng = np.random.default_rng(7)
    for trial in range(60):
        K = int(rng.integers(2, 257))
        h = np.zeros(256, np.uint32)
        syms = rng.choice(256, K, replace=False)
        h[syms] = (rng.pareto(0.6 + trial % 5 * 0.3, K) * 10).astype(np.uint32) + 1
        lens = oracle.code_lengths(h, 11)
        assert lens.max() <= 11
        assert abs(_kraft(lens) - 1.0) < 1e-12
        assert np.count_nonzero(lens) == K


def _heap_huffman_cost(freqs):
    heap = list(freqs)
    heapq.heapify(heap)
    cost = 0
    while len(heap) > 1:
        a, b = heapq.heappop(heap), heapq.heappop(heap)
        cost += a + b
        heapq.heappush(heap, a + b)
    return cost


def test_unbounded_limit_matches_textbook_huffman(oracle):
    """With a non-binding limit the cost equals a textbook heap Huffman's."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        K = int(rng.integers(2, 120))
        h = np.zeros(256, np.uint32)
        h[rng.choice(256, K, replace=False)] = rng.integers(1, 5000, K)
        lens = oracle.code_lengths(h, 15)
        if lens.max() >= 15:
            continue
        assert _cost(h, lens) == _heap_huffman_cost([int(x) for x in h if x])


def test_limit_binds_on_steep_distribution(oracle):
    """A Fibonacci-like histogram needs > 11 bits unbounded; L = 11 must cap it optimally."""
    fib = [1, 1]
    while len(fib) < 20:
        fib.append(fib[-1] + fib[-2])
    h = np.zeros(256, np.uint32)
    h[:20] = fib
    lens15 = oracle.code_lengths(h, 15)
    lens11 = oracle.code_lengths(h, 11)
    assert lens15.max() > 11 and lens11.max() == 11
    assert _cost(h, lens11) >= _cost(h, lens15)
    assert abs(_kraft(lens11) - 1.0) < 1e-12


def test_canonical_code_properties(oracle):
    rng = np.random.default_rng(5)
    for trial in range(20):
        h = np.zeros(256, np.uint32)
        K = int(rng.integers(2, 257))
        h[rng.choice(256, K, replace=False)] = rng.integers(1, 10000, K)
        lens = oracle.code_lengths(h)
        codes = oracle.canonical_codes(lens)
        syms = sorted([s for s in range(256) if lens[s]], key=lambda s: (lens[s], s))
        strs = [code_str(codes, lens, s) for s in syms]
        # left-aligned values strictly increase in (length, symbol) order
        la = [int(c, 2) << (16 - len(c)) for c in strs]
        assert all(a < b for a, b in zip(la, la[1:]))
        # prefix-free
        for a, b in zip(strs, strs[1:]):
            assert not b.startswith(a)
        assert int(strs[0], 2) == 0


def test_tree_shape(oracle):
    """One internal node per proper code prefix; 1 = right child (Listing 1)."""
    rng = np.random.default_rng(9)
    for trial in range(20):
        h = np.zeros(256, np.uint32)
        K = int(rng.integers(2, 257))
        h[rng.choice(256, K, replace=False)] = rng.integers(1, 1000, K)
        lens = oracle.code_lengths(h)
        codes = oracle.canonical_codes(lens)
        depth, prefix, child = oracle.tree_info(lens)
        assert len(depth) == K - 1
        pre = {(d, code_str(codes, lens, s)[:d]) for s in range(256) if lens[s] for d in range(int(lens[s]))}
        got = {(int(d), format(int(p), "0%db" % d) if d else "") for d, p in zip(depth, prefix)}
        assert pre == got
        # breadth-first order
        keys = list(zip(depth, prefix))
        assert keys == sorted(keys)
        for v in range(len(depth)):
            for b in (0, 1):
                c = child[v, b]
                ps = (format(int(prefix[v]), "0%db" % depth[v]) if depth[v] else "") + str(b)
                if c >= 0:
                    assert depth[c] == depth[v] + 1 and format(int(prefix[c]), "0%db" % depth[c]) == ps
                else:
                    assert code_str(codes, lens, -c - 1) == ps


def test_proba80_closed_form(oracle):
    """App. A Table 16 / Table 7: geometric with top p ~ 0.8 over 6 symbols."""
    g = GOLD["proba80"]
    p = 0.8 * 0.2 ** np.arange(6)
    p /= p.sum()
    n = 1 << 20
    h = np.zeros(256, np.uint32)
    h[:6] = np.round(p * n).astype(np.uint32)
    lens = oracle.code_lengths(h)
    nz = lens[h > 0]
    assert int(nz.min()) == g["min_len"] and int(nz.max()) == g["max_len"]
    avg = _cost(h, lens) / h.sum()
    H = float(-(p * np.log2(p)).sum())
    assert abs(avg - g["huffman_bits"]) < 0.01
    assert abs(H - g["H"]) < 0.01
    depth, prefix, child = oracle.tree_info(lens)
    assert len(depth) == g["table7_nodes"]
    # bottom-up ops per byte = one merge step per code bit = average length
    assert abs(avg - g["table7_ops_per_byte"]) < 0.01
