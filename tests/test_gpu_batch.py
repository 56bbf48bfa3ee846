"""GPU: batched (persistent work-queue) decode, tuning, graph capture, autotuner.

The batched path and every tuning must give exactly the bytes of the plain
path, which the oracle pins (test_gpu_parity).  Small tile lengths force the
rank-directory / tile-cursor path even on small blocks."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import WORKLOADS, dev, off64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_05765_gb300 as P
    P.set_tuning()
    yield P
    P.set_tuning()


@pytest.fixture(scope="module")
def encoded(P):
    """Every workload coded with ANS, canonical (PVC1) and regrouped with
    flat subtrees (PVC2)."""
    out = {}
    for name, make in WORKLOADS.items():
        w = make()
        for flat in (False, True):
            enc = P.encode(dev(w.data), off64(w.blk_off), P.params(ans=True, flat=flat))
            assert not enc.status.cpu().numpy().any()
            out[name, flat] = (w, enc)
    return out


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_batched_equals_input(P, encoded, name, flat):
    w, enc = encoded[name, flat]
    out, st = P.decode(enc.comp, enc.off, off64(w.blk_off), batched=True)
    assert not st.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("tuning", [(128, 32, 1), (4096, 256, 0), (16384, 96, 2), (65536, 160, 3), (1 << 20, 64, 0)])
def test_tunings_do_not_change_output(P, encoded, tuning, flat):
    P.set_tuning(*tuning)
    try:
        for name in ["zipf1_256k", "mixed_24", "skew95_4x128k", "edge", "shifting"]:
            w, enc = encoded[name, flat]
            for batched in (False, True):
                out, st = P.decode(enc.comp, enc.off, off64(w.blk_off), batched=batched)
                assert not st.cpu().numpy().any(), (name, batched)
                assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data), (name, batched, tuning)
    finally:
        P.set_tuning()


def test_graph_replay(P):
    import torch
    w = workloads.mixed(nblk=16, hi=1 << 17)
    data, boff = dev(w.data), off64(w.blk_off)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        enc = P.Encoder(w.nblk, P.params(ans=True))
        enc.ensure(enc.plan(data, boff, stream))
        r = enc.run(data, boff, stream, replan=False)
        d = P.Decoder(w.nblk, batched=True)
        d.prepare(r.comp, r.off, stream)
        out = torch.zeros(w.data.size, dtype=torch.uint8, device="cuda")
        stream.synchronize()
        g = P.Graph(stream)
        with g:
            enc.run(data, boff, stream)
            d.run(r.comp, r.off, out, boff, stream)
        for _ in range(2):
            out.zero_()
            enc.comp.zero_()
            g.launch()
            stream.synchronize()
            assert not enc.status.cpu().numpy().any() and not d.status.cpu().numpy().any()
            assert np.array_equal(out.cpu().numpy(), w.data)
    torch.cuda.synchronize()


def test_autotune_keeps_output(P, encoded):
    import torch
    w, enc = encoded["mixed_24", True]
    d = P.Decoder(w.nblk, batched=True)
    d.prepare(enc.comp, enc.off)
    out = torch.empty(w.data.size, dtype=torch.uint8, device="cuda")
    try:
        best, ms = P.autotune_decode(enc.comp, enc.off, w.nblk, out, off64(w.blk_off), d.ws, d.status, reps=1)
        assert best.tile_max in (16384, 65536, 1 << 20) and best.dir_bits in (64, 128, 256) and ms > 0
        t = P.get_tuning()
        assert (t.tile_max, t.dir_bits, t.ctas_per_sm) == (best.tile_max, best.dir_bits, best.ctas_per_sm)
        out.zero_()
        d.run(enc.comp, enc.off, out, off64(w.blk_off))
        assert not d.status.cpu().numpy().any()
        assert np.array_equal(out.cpu().numpy(), w.data)
    finally:
        P.set_tuning()


def test_batched_rejects_corrupt(P, oracle):
    rng = np.random.default_rng(11)
    good = [rng.choice(30, 20000, p=rng.dirichlet(np.ones(30))).astype(np.uint8) for _ in range(3)]
    recs = [oracle.encode_block(x) for x in good]
    bad = recs[1].copy()
    bad[144] ^= 2                       # n_v of the root
    recs[1] = bad
    buf = np.concatenate(recs)
    roff = np.zeros(4, np.int64); roff[1:] = np.cumsum([r.size for r in recs])
    ooff = np.zeros(4, np.int64); ooff[1:] = np.cumsum([x.size for x in good])
    out, st = P.decode(dev(buf), dev(roff), dev(ooff), batched=True)
    s = st.cpu().numpy()
    assert s[0] == 0 and s[2] == 0 and s[1] != 0
    o = out.cpu().numpy()
    assert np.array_equal(o[: good[0].size], good[0])
    assert np.array_equal(o[ooff[2]:ooff[3]], good[2])
