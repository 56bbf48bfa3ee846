"""Oracle pins for the selective-ANS part (Sec. 5): skew analysis, tables,
selection rule and the interleaved rANS coder."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
M = 1 << 15


def test_binary_entropy_and_benefit_table13(oracle):
    """Sec. 5.1 / Table 13 figures from the skew analysis."""
    p80 = GOLD["proba80"]
    assert round(oracle.node_benefit(1000000, 200000, 1000000), 3) == p80["max_node_benefit"]
    # the paper prints the skews rounded to 0.1 %, so its 3-digit H and
    # benefit figures carry about +-0.001 of rounding
    for case in GOLD["skew_benefits"]:
        assert abs(oracle.binary_entropy(case["skew"]) - case["H"]) < 0.0015
        n_total = 1000000
        n_v = int(round(case["frac"] * n_total))
        n1 = int(round((1 - case["skew"]) * n_v))
        assert abs(oracle.node_benefit(n_v, n1, n_total) - case["benefit"]) < 0.0015


def test_proba80_root_benefit_through_tree(oracle):
    """The root of the proba80-like tree carries the whole Table 13 benefit."""
    rng = np.random.default_rng(3)
    p = 0.8 * 0.2 ** np.arange(6)
    x = rng.choice(6, 1 << 18, p=p / p.sum()).astype(np.uint8)
    rec = oracle.encode_block(x)
    V = int(rec[8])
    nv = np.frombuffer(rec[144:144 + 4 * V].tobytes(), np.uint32)
    depth, prefix, child = oracle.tree_info(oracle.code_lengths(oracle.histogram(x)))
    n1 = nv[child[0, 1]] if child[0, 1] >= 0 else np.count_nonzero(x == -child[0, 1] - 1)
    assert abs(oracle.node_benefit(int(nv[0]), int(n1), x.size) - 0.278) < 0.005


def test_class_tables(oracle):
    """50 static tables (Sec. 5.2); frequencies sum to M; t = 50 is uniform."""
    for t in range(50, 100):
        q = oracle.ans_class_freqs(t)
        assert sum(math.comb(8, k) * int(q[k]) for k in range(9)) == M
        assert all(q >= 1)
        assert all(q[k] >= q[k + 1] for k in range(8))     # majority bit 0: fewer ones is likelier
    assert list(oracle.ans_class_freqs(50)) == [128] * 9
    with pytest.raises(RuntimeError):
        oracle.ans_class_freqs(49)
    with pytest.raises(RuntimeError):
        oracle.ans_class_freqs(100)


def test_fse_h_close_to_but_above_entropy(oracle):
    """Sec. 5.2: fse_H is close to H but usually a bit higher."""
    assert oracle.fse_h(50) == pytest.approx(1.0, abs=1e-12)
    for t in range(51, 100):
        hb = oracle.binary_entropy(t / 100)
        fh = oracle.fse_h(t)
        assert fh >= hb - 1e-12
        assert fh - hb < 0.005, (t, fh, hb)
        assert oracle.fse_h_q16(t) == int(math.floor(fh * 65536 + 0.5))


def _ideal_bits(data, t, oracle):
    q = oracle.ans_class_freqs(t)
    pc = np.array([bin(b).count("1") for b in range(256)])
    return float(np.log2(M / q[pc[data]].astype(np.float64)).sum())


@pytest.mark.parametrize("nbytes", [1, 2, 31, 32, 511, 512, 513, 1000, 16383, 16384, 16385, 40000])
def test_rans_round_trip_and_cost(oracle, nbytes):
    rng = np.random.default_rng(nbytes)
    for p1 in (0.03, 0.2, 0.45):
        bits = (rng.random(nbytes * 8) < p1).astype(np.uint8)
        data = np.packbits(bits, bitorder="little")
        t = max(50, min(99, int(round(100 * (1 - p1)))))
        body = oracle.rans_encode(data, t)
        assert np.array_equal(oracle.rans_decode(body, nbytes, t), data)
        # coded length vs the model's ideal code length: rANS adds only the
        # state words (32 bits per interleaved state, 16-bit flush granularity)
        S = (nbytes + 16383) // 16384
        W = sum(min(32, max(1, (min(16384, nbytes - k * 16384) + 511) // 512)) for k in range(S))
        payload_bits = 8 * (body.size - 4 * S - 4 * W)
        ideal = _ideal_bits(data, t, oracle)
        assert payload_bits <= ideal * 1.005 + 16 * W + 16
        assert payload_bits + 32 * W >= ideal * 0.995 - 16


def test_rans_lanes_layout(oracle):
    """Byte j is coded by state j mod W; W = min(32, ceil(bytes/512))."""
    for nbytes, W in [(1, 1), (512, 1), (513, 2), (16384, 32), (20000, 32 + 8)]:
        data = np.zeros(nbytes, np.uint8)
        body = oracle.rans_encode(data, 90)
        S = (nbytes + 16383) // 16384
        nw = np.frombuffer(body[:4 * S].tobytes(), np.uint32)
        assert body.size == 4 * S + 4 * W + 2 * int(nw.sum())


def test_rans_detects_corruption(oracle):
    rng = np.random.default_rng(1)
    data = np.packbits((rng.random(8 * 3000) < 0.1).astype(np.uint8), bitorder="little")
    body = oracle.rans_encode(data, 90)
    bad = body.copy()
    bad[4] ^= 0x40                       # a final state
    with pytest.raises(ValueError):
        oracle.rans_decode(bad, data.size, 90)
    with pytest.raises(ValueError):
        oracle.rans_decode(body[:-2], data.size, 90)


def test_selection_rule_boundaries(oracle):
    """Sec. 5.2 thresholds: >= 32 bytes, skew > 0.625, (d + fseH)/(d + 1) < 0.95."""
    g = GOLD["ans_rule"]
    # 32-byte minimum: 248 bits -> 31 bytes (no), 249..256 bits -> 32 bytes
    assert oracle.ans_select(248, 10, 0) == 0
    assert oracle.ans_select(256, 10, 0) != 0
    # skew strictly above 0.625
    assert oracle.ans_select(800, 300, 0) == 0              # 500/800 = 0.625 exactly
    assert oracle.ans_select(800, 299, 0) != 0 or oracle.fse_h(63) >= g["min_ratio"]
    # the root (depth 0) needs fseH < 0.95; depth d needs fseH < 0.95 - 0.05 d
    for t in (70, 80, 90, 95, 99):
        n = 100000
        n1 = n - (t * n) // 100
        fh = oracle.fse_h_q16(t) / 65536
        for d in range(0, 12):
            want = (d + fh) / (d + 1) < g["min_ratio"]
            m = oracle.ans_select(n, n1, d)
            assert (m != 0) == want, (t, d)
            if m:
                assert m & 0x7F == t - 49 and not m & 0x80
    # XOR flag when the ones are the majority
    m = oracle.ans_select(100000, 95000, 0)
    assert m & 0x80 and (m & 0x7F) == 95 - 49
    # table ids 1..50 <-> skew 50..99 %
    assert oracle.ans_select(100000, 1, 0) & 0x7F == 50
