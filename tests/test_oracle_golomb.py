"""Oracle pins for PivCo-Golomb (App. G), checked against things other than
the oracle's own code: a record derived by hand from the definition, the
plain (non-pivoted) unary code stream, closed forms of the counts, and a
bottom-up decode restated from App. G's merge rule (a different algorithm
from the oracle's top-down cursor walk)."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PINS = json.load(open(os.path.join(HERE, "golden", "paper_pins.json")))


def _parse(rec):
    n = int(rec[4:8].view(np.uint32)[0])
    m = int(rec[8:10].view(np.uint16)[0])
    nj = rec[16:16 + 4 * m].view(np.uint32).astype(np.int64)
    off = 16 + 4 * m
    maps = []
    for j in range(m):
        nb = (int(nj[j]) + 7) // 8
        bits = np.unpackbits(rec[off:off + nb], bitorder="little")[: nj[j]]
        maps.append(bits)
        off += nb
    return n, m, nj, maps, off


def test_hand_derived_record(oracle):
    g = PINS["golomb_hand_derived"]
    rec = oracle.golomb_encode(np.array(g["values"], np.uint8))
    assert rec.size == g["record_bytes"] and bytes(rec[12:16]) == b"PVG1" and rec[10] == 4
    n, m, nj, maps, off = _parse(rec)
    assert list(nj) == g["n_j"]
    body = rec[16 + 4 * m: off]
    assert list(body) == g["bitmap_bytes"]
    assert not rec[off:].any()


@pytest.mark.parametrize("seed", range(6))
def test_bits_are_the_unary_code(oracle, seed):
    """Reading each value's bits back bitmap by bitmap (its cursor in each)
    gives the plain unary code: v continue bits then a stop bit."""
    rng = np.random.default_rng(seed)
    x = rng.geometric(0.45, 300).astype(np.int64) - 1
    x = np.minimum(x, 40).astype(np.uint8)
    rec = oracle.golomb_encode(x)
    n, m, nj, maps, _ = _parse(rec)
    assert n == x.size and m == int(x.max()) + 1
    cur = [0] * m
    for v in x:
        code = []
        for j in range(int(v) + 1):
            code.append(int(maps[j][cur[j]]))
            cur[j] += 1
        assert code == [0] * int(v) + [1]
    assert cur == list(nj)


@pytest.mark.parametrize("seed", range(4))
def test_closed_forms(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    x = (rng.geometric(1 / (1.5 + seed), 5000) - 1).clip(0, 255).astype(np.uint8)
    n, m, nj, maps, _ = _parse(oracle.golomb_encode(x))
    # total bits = total code length = sum of (v + 1)
    assert nj.sum() == int(x.astype(np.int64).sum()) + x.size
    for j in range(m):
        assert nj[j] == int((x >= j).sum())
        assert int(maps[j].sum()) == int((x == j).sum())           # stop bits
        if j + 1 < m:
            assert nj[j + 1] == nj[j] - int(maps[j].sum())          # the rest continue
    assert maps[m - 1].all()                                        # the largest values all stop


def _bottom_up(maps):
    """App. G: from the last bitmap to the first, out_j = B_j ? 0 : out_{j+1}[rank0] + 1."""
    child = np.zeros(0, np.int64)
    for B in reversed(maps):
        out = np.zeros(B.size, np.int64)
        zeros = np.nonzero(B == 0)[0]
        out[zeros] = child[: zeros.size] + 1
        child = out
    return child


@pytest.mark.parametrize("seed", range(4))
def test_bottom_up_merge_gives_the_values(oracle, seed):
    rng = np.random.default_rng(200 + seed)
    x = (rng.geometric(0.3, 4000) - 1).clip(0, 255).astype(np.uint8)
    rec = oracle.golomb_encode(x)
    _, _, _, maps, _ = _parse(rec)
    assert np.array_equal(_bottom_up(maps), x.astype(np.int64))
    st, y = oracle.golomb_decode(rec)
    assert st == 0 and np.array_equal(y, x)


def test_edge_cases(oracle):
    for x in [np.zeros(0, np.uint8), np.zeros(1, np.uint8), np.full(1000, 255, np.uint8),
              np.arange(256, dtype=np.uint8), np.zeros(33, np.uint8)]:
        rec = oracle.golomb_encode(x)
        assert rec.size % 16 == 0
        st, y = oracle.golomb_decode(rec)
        assert st == 0 and np.array_equal(y, x)


def test_corrupt_records_rejected(oracle):
    x = (np.random.default_rng(9).geometric(0.5, 500) - 1).clip(0, 255).astype(np.uint8)
    rec = oracle.golomb_encode(x)
    n, m, nj, maps, off = _parse(rec)
    for mutate in [lambda r: r.__setitem__(12, 0),                   # magic
                   lambda r: r.__setitem__(16, r[16] ^ 1),           # n_0 != n
                   lambda r: r.__setitem__(16 + 4 * m, r[16 + 4 * m] ^ 0x10),   # a stop bit moved
                   lambda r: r.__setitem__(0, r[0] + 16)]:           # size past the record
        bad = rec.copy()
        mutate(bad)
        st, _ = oracle.golomb_decode(bad)
        assert st != 0
