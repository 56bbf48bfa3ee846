"""GPU: bounded device waits that run out.

Every wait a kernel makes on another CTA's work (the decoupled look-backs,
the batched decode's waits on earlier queue items) gives up after the bound
set by pivco_set_wait_limit.  With the bound at 0 every wait that is not met
at once gives up: the kernels must return, the blocks concerned must report
PIVCO_ERR_TIMEOUT, no block whose work was abandoned may report OK, and the
blocks that do report OK must hold exactly their input.  Afterwards, with the
bound back at its default, the same batch decodes completely (the context is
still usable).  Nothing here faults or hangs the GPU: the waits end on a
device-clock bound and the kernels return."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import dev, off64

pytestmark = pytest.mark.gpu

TIMEOUT = 4


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_05765_gb300 as P
    P.set_wait_limit()
    yield P
    P.set_wait_limit()


@pytest.fixture(scope="module")
def batch(P):
    # many small blocks: the queue's plan items take several rounds of the
    # grid, so later items are taken while plans are still running
    w = workloads.mixed(nblk=6000, seed=31, lo=1024, hi=16 * 1024)
    boff = off64(w.blk_off)
    enc = P.encode(dev(w.data), boff, P.params(ans=True))
    assert not enc.status.cpu().numpy().any()
    return w, boff, enc


def _check_partial(w, out, st):
    out = out.cpu().numpy()
    for b in np.nonzero(st == 0)[0]:
        lo, hi = int(w.blk_off[b]), int(w.blk_off[b + 1])
        assert np.array_equal(out[lo:hi], w.data[lo:hi]), "block %d reports OK but is wrong" % b


def test_wait_limit_roundtrip(P):
    P.set_wait_limit(12345)
    assert P.get_wait_limit() == 12345
    P.set_wait_limit()
    assert P.get_wait_limit() == 10 ** 9


@pytest.mark.parametrize("batched", [True, False])
def test_expired_waits_report_timeout(P, batch, batched):
    import torch
    w, boff, enc = batch
    dec = P.Decoder(w.nblk, "cuda", batched=batched)
    dec.prepare(enc.comp, enc.off)
    out = torch.full((w.data.size,), 0x5A, dtype=torch.uint8, device="cuda")
    P.set_wait_limit(0)
    try:
        dec.run(enc.comp, enc.off, out, boff)
        torch.cuda.synchronize()
    finally:
        P.set_wait_limit()
    st = dec.status.cpu().numpy()
    assert set(np.unique(st)) <= {0, TIMEOUT}, np.unique(st)
    if batched:
        # the items after the plans are taken while plans still run
        assert (st == TIMEOUT).any()
    _check_partial(w, out, st)
    # the default bound: everything decodes, the device is fine
    out.fill_(0x5A)
    dec.run(enc.comp, enc.off, out, boff)
    torch.cuda.synchronize()
    assert not dec.status.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy(), w.data)


def test_scan_expired_waits(P):
    import torch
    n = 1 << 21
    vals = torch.from_numpy(np.random.default_rng(5).integers(0, 1000, n, dtype=np.int64)).cuda()
    ref = np.concatenate([[0], np.cumsum(vals.cpu().numpy())])
    out = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ws = torch.empty(P.scan_workspace_size(n), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.set_wait_limit(0)
    try:
        P.exclusive_scan(vals, n, out, ws, status)
        torch.cuda.synchronize()
    finally:
        P.set_wait_limit()
    s = int(status.item())
    assert s in (0, TIMEOUT)
    if s == 0:   # no wait ran out: the prefix is exact
        assert np.array_equal(out.cpu().numpy(), ref)
    P.exclusive_scan(vals, n, out, ws, status)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
