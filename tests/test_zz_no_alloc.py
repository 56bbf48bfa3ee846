"""GPU: pivco_decode_blocks_static, the decode that uses the library's own
device workspace instead of one the caller allocates.

It must give exactly what pivco_decode_blocks gives (whose output the oracle
pins in the parity tests), on two calls in a row with different batches, so
that whatever the first call leaves in the library's array cannot leak into
the second.  The file sorts last so that it also runs after every other GPU
test in the same process; it needs nothing from them and passes alone."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batches():
    a = workloads.mixed(nblk=12, seed=21, hi=1 << 18)        # mixed sizes, alphabets, ANS nodes
    b = workloads.skew95(nblk=5, bs=96 * 1024 + 77, seed=22)  # ragged blocks, ANS on skewed nodes
    return [a, b]


@pytest.mark.parametrize("flat", [False, True])
def test_static_matches_workspace_decode_twice(P, flat):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for w in _batches():
            data = _dev(w.data)
            boff = _dev(w.blk_off.astype(np.int64))
            enc = P.encode(data, boff, P.params(ans=True, flat=flat), stream)
            assert not enc.status.cpu().numpy().any()
            # the existing entry point, with a workspace the caller sized
            ref_out, ref_st = P.decode(enc.comp, enc.off, boff, stream)
            # the library-owned workspace; the output starts as garbage on purpose
            out = torch.full((w.data.size,), 0xA5, dtype=torch.uint8, device="cuda")
            st = torch.full((w.nblk,), -7, dtype=torch.int32, device="cuda")
            P.decode_blocks_static(enc.comp, enc.off, w.nblk, out, boff, st, stream)
            stream.synchronize()
            assert np.array_equal(st.cpu().numpy(), ref_st.cpu().numpy())
            assert not st.cpu().numpy().any()
            assert torch.equal(out, ref_out[: w.data.size])
            assert np.array_equal(out.cpu().numpy(), w.data)


def test_static_rejects_oversized_batch(P):
    import torch
    # the plan part alone of 400k blocks (60 bytes each) exceeds 16 MiB: refused on the host
    n = 400_000
    comp = torch.zeros(16, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PivcoError, match="CAPACITY"):
        P.decode_blocks_static(comp, offs, n, comp, offs, st)
    assert P.decode_plan_bytes(n) > P.DECODE_STATIC_WS_BYTES


def test_static_reports_capacity_per_block(P):
    """Blocks whose ANS scratch or rank directories do not fit in what is left
    of the 16 MiB array report PIVCO_ERR_CAPACITY; the others decode exactly
    as pivco_decode_blocks decodes them."""
    import torch
    # 160 blocks of 1 MiB with an ANS-coded 128 KiB root bitmap each, split
    # into several tiles: about 180 KiB of workspace per block, 28 MiB in all
    w = workloads.skew95(nblk=160, bs=1 << 20, seed=23)
    data = _dev(w.data)
    boff = _dev(w.blk_off.astype(np.int64))
    enc = P.encode(data, boff, P.params(ans=True))
    assert not enc.status.cpu().numpy().any()
    ref_out, ref_st = P.decode(enc.comp, enc.off, boff)
    assert not ref_st.cpu().numpy().any()
    for _ in range(2):
        out = torch.full((w.data.size,), 0xA5, dtype=torch.uint8, device="cuda")
        st = torch.full((w.nblk,), -7, dtype=torch.int32, device="cuda")
        P.decode_blocks_static(enc.comp, enc.off, w.nblk, out, boff, st)
        torch.cuda.synchronize()
        s = st.cpu().numpy()
        assert set(np.unique(s)) <= {0, 2}, np.unique(s)       # OK or CAPACITY
        assert (s == 2).any() and (s == 0).any()
        o = out.cpu().numpy()
        for b in np.nonzero(s == 0)[0]:
            lo, hi = int(w.blk_off[b]), int(w.blk_off[b + 1])
            assert np.array_equal(o[lo:hi], w.data[lo:hi])
