"""GPU: the host-buffer codec (pivco_host_*): batches in host memory, copies
overlapped with the kernels piece by piece.  Its records must be the device
encoder's, byte for byte and at the same offsets (which the oracle pins in
the parity tests), and its decode must give back the input."""
import numpy as np
import pytest

import workloads

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


def _pinned(a):
    import torch
    t = torch.empty(max(a.size, 1), dtype=torch.uint8, pin_memory=True)
    t[: a.size] = torch.from_numpy(a)
    return t


def _edge():
    rng = np.random.default_rng(11)
    blocks = [np.zeros(0, np.uint8), np.array([5], np.uint8), np.full(3000, 7, np.uint8),
              rng.integers(0, 256, 100000).astype(np.uint8), rng.integers(0, 3, 40000).astype(np.uint8),
              np.zeros(0, np.uint8), (rng.random(90000) < 0.9).astype(np.uint8)]
    off = np.zeros(len(blocks) + 1, np.uint64)
    off[1:] = np.cumsum([b.size for b in blocks])
    return workloads.Workload("edge", np.concatenate(blocks), off, True)


CASES = {
    "skew80_16x64k": lambda: workloads.skew80(nblk=16, bs=65536),
    "mixed_24": lambda: workloads.mixed(nblk=24, hi=1 << 18),
    "edge": _edge,
}


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("segments", [1, 3, 8])
@pytest.mark.parametrize("name", sorted(CASES))
def test_host_codec_matches_device(P, name, segments, flat):
    import torch
    w = CASES[name]()
    prm = P.params(ans=w.ans, flat=flat)
    boff = torch.from_numpy(w.blk_off.astype(np.int64)).cuda()
    ref = P.encode(torch.from_numpy(w.data).cuda(), boff, prm)
    assert not ref.status.cpu().numpy().any()
    r_comp, r_off, r_rb = ref.comp.cpu().numpy(), ref.off.cpu().numpy(), ref.rec_bytes.cpu().numpy()
    with P.HostCodec(w.blk_off, prm, segments) as hc:
        data = _pinned(w.data)
        comp = torch.empty(max(hc.capacity, 1), dtype=torch.uint8, pin_memory=True)
        comp_off, st = hc.compress(data, comp)
        assert not st.any(), st
        assert np.array_equal(comp_off.astype(np.int64), r_off)
        c = comp.numpy()
        for b in range(w.nblk):
            lo = int(r_off[b])
            assert np.array_equal(c[lo:lo + int(r_rb[b])], r_comp[lo:lo + int(r_rb[b])]), b
        out = torch.zeros(max(w.data.size, 1), dtype=torch.uint8, pin_memory=True)
        st = hc.decompress(comp, comp_off.copy(), out)
        assert not st.any(), st
        assert np.array_equal(out.numpy()[: w.data.size], w.data)


def test_host_codec_capacity_and_corrupt(P):
    import torch
    w = CASES["skew80_16x64k"]()
    with P.HostCodec(w.blk_off, P.params(), 4) as hc:
        data = _pinned(w.data)
        small = torch.empty(1024, dtype=torch.uint8, pin_memory=True)
        with pytest.raises(P.PivcoError, match="CAPACITY"):
            hc.compress(data, small)
        comp = torch.empty(hc.capacity, dtype=torch.uint8, pin_memory=True)
        comp_off, st = hc.compress(data, comp)
        assert not st.any()
        comp_off = comp_off.copy()
        bad = comp.clone()
        bad[int(comp_off[5]) + 144] ^= 2          # n_v of block 5's root
        out = torch.zeros(w.data.size, dtype=torch.uint8, pin_memory=True)
        st = hc.decompress(bad, comp_off, out)
        assert st[5] == P.ERR_CORRUPT
        assert not np.delete(st, 5).any()
        for b in range(w.nblk):
            if b != 5:
                lo, hi = int(w.blk_off[b]), int(w.blk_off[b + 1])
                assert np.array_equal(out.numpy()[lo:hi], w.data[lo:hi])
