"""GPU: PivCo-Golomb (App. G).  Records must be byte-identical to the
oracle's and decode to the input; the decoder must also read the oracle's
records, and reject corrupt ones and blocks over the size limit."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import dev, off64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_05765_gb300 as P
    return P


def _edge():
    rng = np.random.default_rng(12)
    blocks = [np.zeros(0, np.uint8), np.zeros(1, np.uint8), np.full(1, 255, np.uint8), np.full(1000, 255, np.uint8),
              np.arange(256, dtype=np.uint8), np.zeros(33, np.uint8), rng.integers(0, 3, 31).astype(np.uint8),
              (rng.geometric(0.2, 32768) - 1).clip(0, 255).astype(np.uint8),
              (rng.geometric(0.9, 32767) - 1).clip(0, 255).astype(np.uint8)]
    off = np.zeros(len(blocks) + 1, np.uint64)
    off[1:] = np.cumsum([b.size for b in blocks])
    return np.concatenate(blocks), off


def _check_against_oracle(P, oracle, data, off):
    import torch
    boff = off64(off)
    enc = P.golomb_encode(dev(data), boff)
    torch.cuda.synchronize()
    st = enc.status.cpu().numpy()
    assert not st.any(), st
    comp = enc.comp.cpu().numpy()
    coff = enc.off.cpu().numpy()
    rb = enc.rec_bytes.cpu().numpy()
    for b in range(off.size - 1):
        ref = oracle.golomb_encode(data[int(off[b]):int(off[b + 1])])
        assert rb[b] == ref.size and np.array_equal(comp[int(coff[b]):int(coff[b]) + ref.size], ref), b
    out = torch.empty(max(data.size, 1), dtype=torch.uint8, device="cuda")
    dst = torch.empty(off.size - 1, dtype=torch.int32, device="cuda")
    P.golomb_decode(enc.comp, enc.off, out, boff, dst)
    torch.cuda.synchronize()
    assert not dst.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: data.size], data)


@pytest.mark.parametrize("avg_len", [1.25, 2.0, 5.0])
def test_records_match_oracle(P, oracle, avg_len):
    w = workloads.golomb(nblk=24, bs=32768, avg_len=avg_len, seed=int(avg_len * 4))
    _check_against_oracle(P, oracle, w.data, w.blk_off)


def test_edge_blocks(P, oracle):
    data, off = _edge()
    _check_against_oracle(P, oracle, data, off)


def test_decodes_oracle_records_and_rejects_corrupt(P, oracle):
    import torch
    rng = np.random.default_rng(4)
    vals = [(rng.geometric(0.4, 5000 + 7 * i) - 1).clip(0, 255).astype(np.uint8) for i in range(4)]
    recs = [oracle.golomb_encode(v) for v in vals]
    bad = recs[2].copy()
    bad[16] ^= 1                    # n_0 != n
    recs[2] = bad
    roff = np.zeros(len(recs) + 1, np.uint64)
    roff[1:] = np.cumsum([r.size for r in recs])
    ooff = np.zeros(len(vals) + 1, np.uint64)
    ooff[1:] = np.cumsum([v.size for v in vals])
    out = torch.empty(int(ooff[-1]), dtype=torch.uint8, device="cuda")
    st = torch.empty(len(recs), dtype=torch.int32, device="cuda")
    P.golomb_decode(dev(np.concatenate(recs)), off64(roff), out, off64(ooff), st)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert list(s) == [0, 0, 3, 0]
    o = out.cpu().numpy()
    for i in (0, 1, 3):
        assert np.array_equal(o[int(ooff[i]):int(ooff[i + 1])], vals[i])


def test_oversized_block_refused(P):
    import torch
    data = np.zeros(32769, np.uint8)
    off = np.array([0, 32769], np.uint64)
    size = torch.empty(1, dtype=torch.int64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = P.lib().pivco_golomb_plan(P._ptr(dev(data)), P._ptr(off64(off)), 1, P._ptr(size), P._ptr(st), P._stream(None))
    torch.cuda.synchronize()
    assert rc == 0 and int(st.item()) == 1
