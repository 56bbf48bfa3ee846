"""GPU parity at the full sizes of the measured configurations, in the launch
configuration the benchmark times: the encode sequence and the persistent
decode each captured as a CUDA graph and replayed; regrouped trees with flat
subtrees (the benchmark's records) and canonical ones.

The oracle codes one block in milliseconds, so it checks a seeded sample of
blocks record by record (first, last and random ones); the whole batch is
checked through a property that holds at any size: the decode of the
records is the input, byte for byte."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

CONFIGS = {
    "zipf1_1x1MiB": lambda: workloads.zipf1(),                 # one block of 2^20 symbols
    "skew80_4096x64KiB": lambda: workloads.skew80(),           # 256 MiB, no ANS
    "skew95_2048x128KiB": lambda: workloads.skew95(),          # 256 MiB, selective ANS
    "mixed_4096": lambda: workloads.mixed(),                   # 4 KiB-1 MiB blocks, mixed ANS
}


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


@pytest.mark.parametrize("flat", [True, False])
@pytest.mark.parametrize("name", list(CONFIGS))
def test_full_size_graph_path(P, oracle, name, flat):
    import torch
    w = CONFIGS[name]()
    nblk = w.nblk
    stream = torch.cuda.Stream()
    data = torch.from_numpy(w.data).cuda()
    blk_off = torch.from_numpy(w.blk_off.astype(np.int64)).cuda()
    with torch.cuda.stream(stream):
        enc = P.Encoder(nblk, P.params(ans=w.ans, flat=flat))
        enc.ensure(enc.plan(data, blk_off, stream))
        dec = P.Decoder(nblk)
        res = enc.run(data, blk_off, stream)
        dec.prepare(res.comp, res.off, stream)
        out = torch.zeros(max(w.data.size, 1), dtype=torch.uint8, device="cuda")
        enc.comp.fill_(0xEE)                       # whatever the graph leaves must be its own output
        g_enc = P.Graph(stream)
        with g_enc:
            enc.run(data, blk_off, stream)
        g_dec = P.Graph(stream)
        with g_dec:
            P.decode_batched(res.comp, res.off, nblk, out, blk_off, dec.ws, dec.status, stream)
        g_enc.launch(stream)
        g_dec.launch(stream)
    stream.synchronize()
    assert not enc.status.cpu().numpy().any()
    assert not dec.status.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)
    comp, off, rb = enc.comp.cpu().numpy(), enc.off.cpu().numpy(), enc.rec_bytes.cpu().numpy()
    rng = np.random.default_rng(2026)
    sample = sorted({0, nblk - 1, *rng.choice(nblk, size=min(nblk, 10), replace=False).tolist()})
    prm = oracle.params(ans=w.ans, flat=flat)
    for b in sample:
        blk = w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])]
        ref = oracle.encode_block(blk, prm)
        got = comp[int(off[b]):int(off[b]) + int(rb[b])]
        assert got.size == ref.size and np.array_equal(got, ref), (name, b)
