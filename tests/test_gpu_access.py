"""GPU: random access by top-down rank walks (pivco_access_*).

The symbol at position p of block b must be byte p of the block's input,
i.e. what the bottom-up decode gives (which the parity tests pin to the
oracle): a walk from the root, each node's bit choosing the child and its
rank the child's position, is the same function of the record computed the
other way round.  Queries cover random positions of every workload (ANS-coded
nodes included), whole small blocks, several directory granularities, and
the error cases."""
import numpy as np
import pytest

from test_gpu_parity import WORKLOADS, dev, off64

pytestmark = pytest.mark.gpu

INVALID = 1


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


def _queries(w, n_rand, seed):
    rng = np.random.default_rng(seed)
    sizes = (w.blk_off[1:] - w.blk_off[:-1]).astype(np.int64)
    nz = np.nonzero(sizes)[0]
    b = rng.choice(nz, n_rand)
    p = (rng.random(n_rand) * sizes[b]).astype(np.int64)
    # every position of the small blocks too
    for bb in nz[sizes[nz] <= 4096]:
        b = np.concatenate([b, np.full(sizes[bb], bb)])
        p = np.concatenate([p, np.arange(sizes[bb])])
    return b.astype(np.uint32), p.astype(np.uint32)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_access_equals_input(P, name, flat):
    import torch
    w = WORKLOADS[name]()
    boff = off64(w.blk_off)
    enc = P.encode(dev(w.data), boff, P.params(ans=True, flat=flat))
    assert not enc.status.cpu().numpy().any()
    acc = P.Access(enc.comp, enc.off, w.nblk)
    assert not acc.status.cpu().numpy()[: w.nblk].any()
    qb, qp = _queries(w, 20000, 5)
    sym, st = acc(torch.from_numpy(qb).cuda(), torch.from_numpy(qp).cuda())
    torch.cuda.synchronize()
    assert not st.cpu().numpy().any()
    want = w.data[w.blk_off[qb].astype(np.int64) + qp.astype(np.int64)]
    assert np.array_equal(sym.cpu().numpy(), want)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("dir_bits", [32, 96, 256])
def test_access_any_granularity(P, dir_bits, flat):
    import torch
    w = WORKLOADS["mixed_24"]()
    enc = P.encode(dev(w.data), off64(w.blk_off), P.params(ans=True, flat=flat))
    P.set_tuning(16384, dir_bits, 0)
    try:
        acc = P.Access(enc.comp, enc.off, w.nblk)
        qb, qp = _queries(w, 5000, dir_bits)
        sym, st = acc(torch.from_numpy(qb).cuda(), torch.from_numpy(qp).cuda())
        torch.cuda.synchronize()
    finally:
        P.set_tuning()
    assert not st.cpu().numpy().any()
    assert np.array_equal(sym.cpu().numpy(), w.data[w.blk_off[qb].astype(np.int64) + qp.astype(np.int64)])


def test_access_rejects_bad_queries(P):
    import torch
    w = WORKLOADS["edge"]()
    enc = P.encode(dev(w.data), off64(w.blk_off), P.params(ans=True))
    acc = P.Access(enc.comp, enc.off, w.nblk)
    sizes = (w.blk_off[1:] - w.blk_off[:-1]).astype(np.int64)
    big = int(np.argmax(sizes))
    qb = np.array([w.nblk, w.nblk + 7, 0, big, big, 1], np.uint32)     # block 0 is empty
    qp = np.array([0, 0, 0, sizes[big], sizes[big] - 1, 0], np.uint32)
    sym, st = acc(torch.from_numpy(qb).cuda(), torch.from_numpy(qp).cuda())
    st = st.cpu().numpy()
    assert list(st[:4]) == [INVALID] * 4
    assert st[4] == 0 and sym.cpu().numpy()[4] == w.data[int(w.blk_off[big]) + sizes[big] - 1]
    assert st[5] == 0 and sym.cpu().numpy()[5] == 7          # the one-byte block
    # a decode workspace holds directories only for blocks split into tiles:
    # querying a single-tile block through it is refused, not guessed
    dec = P.Decoder(w.nblk, "cuda")
    dec.prepare(enc.comp, enc.off)
    P.decode_plan(enc.comp, enc.off, w.nblk, dec.ws, dec.status)
    qb2 = torch.tensor([big], dtype=torch.int32, device="cuda")
    qp2 = torch.tensor([0], dtype=torch.int32, device="cuda")
    sym2 = torch.empty(1, dtype=torch.uint8, device="cuda")
    st2 = torch.empty(1, dtype=torch.int32, device="cuda")
    import ctypes as C
    rc = P.lib().pivco_access(P._ptr(enc.comp), P._ptr(enc.off), w.nblk, P._ptr(qb2), P._ptr(qp2), 1, P._ptr(sym2),
                              P._ptr(st2), P._ptr(dec.ws), dec.ws.numel(), P._ptr(dec.status), P._stream(None))
    assert rc == 0
    assert int(st2.item()) == INVALID
