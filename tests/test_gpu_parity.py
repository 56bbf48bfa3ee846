"""GPU parity: the sm_103a library against the CPU oracle, element by element.

Everything here is integer / byte work, so the bar is bit-exact: histograms,
code lengths, whole block records (bitmaps, directories, ANS states and words)
and decoded bytes.  All calls go through the C ABI (ctypes binding).
"""
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


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def off64(blk_off):
    return dev(np.asarray(blk_off, np.int64))


def edge_workload():
    """Degenerate and ragged blocks: empty, 1 byte, constant, two symbols,
    sizes around unit / chunk boundaries, a 256-symbol uniform block."""
    rng = np.random.default_rng(99)
    blocks = [np.zeros(0, np.uint8), np.array([7], np.uint8), np.full(1000, 3, np.uint8),
              np.array([1, 2], np.uint8), rng.integers(0, 2, 33).astype(np.uint8),
              rng.integers(0, 256, 127).astype(np.uint8), rng.integers(0, 256, 128).astype(np.uint8),
              rng.integers(0, 256, 129).astype(np.uint8), rng.integers(0, 5, 16383).astype(np.uint8),
              rng.integers(0, 5, 16384).astype(np.uint8), rng.integers(0, 5, 16385).astype(np.uint8),
              rng.integers(0, 256, 40000).astype(np.uint8),
              (rng.random(70000) < 0.97).astype(np.uint8) * 9]
    sizes = [b.size for b in blocks]
    off = np.zeros(len(blocks) + 1, np.uint64)
    off[1:] = np.cumsum(sizes)
    return workloads.Workload("edge", np.concatenate(blocks), off, True)


def shifting_workload():
    """Blocks whose statistics change mid-block: a skewed stretch followed by
    a uniform one, so chunks sized from the whole-block statistics overflow
    the level buffers and are shortened and redone."""
    rng = np.random.default_rng(7)
    blocks = []
    for n_skew, n_uni in [(60000, 20000), (100000, 60000), (5000, 120000), (200000, 1000)]:
        skew = np.where(rng.random(n_skew) < 0.97, 0, rng.integers(1, 256, n_skew)).astype(np.uint8)
        blocks.append(np.concatenate([skew, rng.integers(0, 256, n_uni).astype(np.uint8)]))
    off = np.zeros(len(blocks) + 1, np.uint64)
    off[1:] = np.cumsum([b.size for b in blocks])
    return workloads.Workload("shifting", np.concatenate(blocks), off, True)


WORKLOADS = {
    "shifting": shifting_workload,
    "zipf1_256k": lambda: workloads.zipf1(n=1 << 18),
    "skew80_8x64k": lambda: workloads.skew80(nblk=8, bs=65536),
    "skew95_4x128k": lambda: workloads.skew95(nblk=4, bs=131072),
    "mixed_24": lambda: workloads.mixed(nblk=24, hi=1 << 18),
    "edge": edge_workload,
}


def oracle_records(oracle, w, ans, flat=False):
    prm = oracle.params(ans=ans, flat=flat)
    return [oracle.encode_block(w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])], prm) for b in range(w.nblk)]


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_histogram(P, oracle, name):
    import torch
    w = WORKLOADS[name]()
    hist = torch.empty(w.nblk * 256, dtype=torch.int32, device="cuda")
    P.histogram(dev(w.data), off64(w.blk_off), hist)
    got = hist.cpu().numpy().view(np.uint32).reshape(w.nblk, 256)
    for b in range(w.nblk):
        assert np.array_equal(got[b], oracle.histogram(w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])])), b


def test_code_lengths(P, oracle):
    import torch
    rng = np.random.default_rng(5)
    hs = []
    for i in range(300):
        h = np.zeros(256, np.uint32)
        K = int(rng.integers(0, 257)) if i % 7 else int(rng.integers(0, 4))
        syms = rng.choice(256, K, replace=False)
        kind = i % 4
        if kind == 0:
            h[syms] = rng.integers(1, 1 << 16, K)
        elif kind == 1:
            h[syms] = (rng.pareto(0.7, K) * 30).astype(np.uint32) + 1
        elif kind == 2:
            h[syms] = 1 + (np.arange(K) % 3)                   # many ties
        else:
            h[syms[:min(K, 25)]] = [int(1.618 ** j) + 1 for j in range(min(K, 25))]   # limit binds
        hs.append(h)
    for i in range(24):
        # counts large enough for package weights past 32 bits (the 64-bit path)
        h = np.zeros(256, np.uint32)
        K = int(rng.integers(2, 257))
        h[rng.choice(256, K, replace=False)] = rng.integers(1 << 20, 1 << 31, K)
        hs.append(h)
    H = np.stack(hs)
    for L in (11, 8, 15):
        st = torch.empty(len(hs), dtype=torch.int32, device="cuda")
        lens = torch.empty(len(hs) * 256, dtype=torch.uint8, device="cuda")
        P.code_lengths(dev(H.reshape(-1).view(np.int32)), len(hs), L, lens, st)
        got = lens.cpu().numpy().reshape(len(hs), 256)
        stn = st.cpu().numpy()
        for i, h in enumerate(hs):
            if np.count_nonzero(h) > (1 << L):
                assert stn[i] == P.ERR_INVALID_ARG
                continue
            assert stn[i] == 0
            assert np.array_equal(got[i], oracle.code_lengths(h, L)), (L, i)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("ans", [False, True])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_encode_records(P, oracle, name, ans, flat):
    """Whole records, canonical (PVC1) and regrouped with flat subtrees
    (PVC2, Sec. 2.2.3-2.2.4), byte for byte."""
    w = WORKLOADS[name]()
    enc = P.encode(dev(w.data), off64(w.blk_off), P.params(ans=ans, flat=flat))
    st = enc.status.cpu().numpy()
    assert not st.any(), st
    comp, off, rb = enc.comp.cpu().numpy(), enc.off.cpu().numpy(), enc.rec_bytes.cpu().numpy()
    refs = oracle_records(oracle, w, ans, flat)
    for b, ref in enumerate(refs):
        got = comp[int(off[b]):int(off[b]) + int(rb[b])]
        assert got.size == ref.size, (b, got.size, ref.size)
        assert np.array_equal(got, ref), b


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("ans", [False, True])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_decode_oracle_records(P, oracle, name, ans, flat):
    """The GPU decodes the oracle's dense records to the original bytes."""
    w = WORKLOADS[name]()
    buf, rec_off, sizes = oracle.encode_batch(w.data, w.blk_off, oracle.params(ans=ans, flat=flat))
    out, st = P.decode(dev(buf if buf.size else np.zeros(16, np.uint8)), off64(rec_off), off64(w.blk_off))
    assert not st.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)


def test_round_trip_permuted_values(P):
    w = workloads.skew80(nblk=4, bs=65536, permute=True)
    enc = P.encode(dev(w.data), off64(w.blk_off))
    out, st = P.decode(enc.comp, enc.off, off64(w.blk_off))
    assert not st.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)


def test_decode_rejects_corrupt_records(P, oracle):
    rng = np.random.default_rng(3)
    x = rng.choice(40, 30000, p=rng.dirichlet(np.ones(40))).astype(np.uint8)
    y = (rng.random(200000) < 0.95).astype(np.uint8)
    z = rng.integers(0, 64, 20000).astype(np.uint8)
    recs = [oracle.encode_block(x), oracle.encode_block(y, oracle.params(ans=True)),
            oracle.encode_block(x, oracle.params(flat=True)), oracle.encode_block(z, oracle.params(flat=True))]
    cases = []
    for r in recs:
        V = int(r[8])
        c = r.copy(); c[12] = ord("Q"); cases.append((c, r))                       # magic
        c = r.copy(); c[144] ^= 4; cases.append((c, r))                            # n_v of the root
        c = r.copy(); c[144 + 4 * V] = 99; cases.append((c, r))                    # marker
        c = r.copy(); c[16] = 0xEE; cases.append((c, r))                           # code lengths
        c = r.copy(); c[-20] ^= 0x5A; cases.append((c, r))                         # body bytes
        c = r.copy(); c[15] ^= 3; cases.append((c, r))                             # tree kind: PVC1 <-> PVC2
        fm = [v for v in range(V) if r[144 + 4 * V + v] >= 0xF2]
        if fm:                                                                     # a flat node's marker
            c = r.copy(); c[144 + 4 * V + fm[0]] += 1; cases.append((c, r))
            c = r.copy(); c[144 + 4 * V + fm[0]] = 0; cases.append((c, r))
    for c, r in cases:
        n = int(np.frombuffer(r[4:8].tobytes(), np.uint32)[0])
        out, st = P.decode(dev(c), off64([0, c.size]), off64([0, n]))
        s = int(st.cpu().numpy()[0])
        ok_bytes = s == 0 and np.array_equal(out.cpu().numpy()[:n], oracle.decode_block(r)[1])
        # a flipped body bit may still be a valid stream; then the oracle must agree on it
        if s == 0 and not ok_bytes:
            rc, ref = oracle.decode_block(c)
            assert rc == 0 and np.array_equal(out.cpu().numpy()[:n], ref)
        if s != 0:
            assert oracle.decode_block(c)[0] != 0


def test_ans_primitives(P, oracle):
    import torch
    rng = np.random.default_rng(17)
    bms, tables = [], []
    for nbytes in [1, 32, 511, 512, 513, 4000, 16384, 16385, 50000]:
        p1 = float(rng.choice([0.02, 0.1, 0.3, 0.9]))
        bits = (rng.random(8 * nbytes) < p1).astype(np.uint8)
        bm = np.packbits(bits, bitorder="little")
        skew = max(p1, 1 - p1)
        t = max(50, min(99, int(round(100 * skew))))
        tables.append((t - 49) | (0x80 if p1 > 0.5 else 0))
        bms.append(bm)
    sizes = np.array([b.size for b in bms], np.int64)
    bm_off = np.zeros(len(bms) + 1, np.int64); bm_off[1:] = np.cumsum(sizes)
    cap = 4 * ((sizes + 16383) // 16384) * 34 + 2 * sizes + 64
    body_off = np.zeros(len(bms) + 1, np.int64); body_off[1:] = np.cumsum(cap)
    bodies = torch.zeros(int(body_off[-1]), dtype=torch.uint8, device="cuda")
    bb = torch.zeros(len(bms), dtype=torch.int64, device="cuda")
    st = torch.zeros(len(bms), dtype=torch.int32, device="cuda")
    tab = dev(np.array(tables, np.uint8))
    P.ans_encode(dev(np.concatenate(bms)), dev(bm_off), tab, len(bms), bodies, dev(body_off), bb, st)
    assert not st.cpu().numpy().any()
    got = bodies.cpu().numpy(); bbn = bb.cpu().numpy()
    for i, bm in enumerate(bms):
        t = (tables[i] & 0x7F) + 49
        src = bm ^ 0xFF if tables[i] & 0x80 else bm
        ref = oracle.rans_encode(src, t)
        assert np.array_equal(got[int(body_off[i]):int(body_off[i]) + int(bbn[i])], ref), i
    # decode the oracle's bodies on the GPU
    refs = [oracle.rans_encode(bm ^ 0xFF if tables[i] & 0x80 else bm, (tables[i] & 0x7F) + 49) for i, bm in enumerate(bms)]
    roff = np.zeros(len(refs) + 1, np.int64); roff[1:] = np.cumsum([r.size for r in refs])
    outb = torch.zeros(int(bm_off[-1]), dtype=torch.uint8, device="cuda")
    P.ans_decode(dev(np.concatenate(refs)), dev(roff), tab, len(refs), outb, dev(bm_off), st)
    assert not st.cpu().numpy().any()
    assert np.array_equal(outb.cpu().numpy(), np.concatenate(bms))


def test_exclusive_scan(P):
    import torch
    rng = np.random.default_rng(2)
    for n in [0, 1, 5, 1023, 1024, 1025, 100000]:
        v = rng.integers(0, 1 << 30, n).astype(np.int64)
        out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        ws = torch.empty(P.scan_workspace_size(n), dtype=torch.uint8, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        P.exclusive_scan(dev(v) if n else torch.zeros(1, dtype=torch.int64, device="cuda"), n, out, ws, st)
        ref = np.zeros(n + 1, np.int64); ref[1:] = np.cumsum(v)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert int(st.cpu().numpy()[0]) == 0


def _chunk_bounds(n):
    """The encoder's warp chunks of an n-symbol block: min(8, max(1, n // 4096))
    contiguous pieces, piece w starting at floor(n w / nw) rounded down to 32."""
    nw = min(8, max(1, n // 4096))
    starts = [(n * w // nw) & ~31 for w in range(nw)] + [n]
    return list(zip(starts[:-1], starts[1:]))


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_histogram_chunks(P, oracle, name):
    """Block histograms equal pivco_histogram's; each chunk's equals the
    oracle's histogram of that slice; absent chunks are zero."""
    import torch
    w = WORKLOADS[name]()
    hist = torch.empty(w.nblk * 256, dtype=torch.int32, device="cuda")
    ch = torch.full((w.nblk * P.CHUNKS * 256,), -1, dtype=torch.int32, device="cuda")
    P.histogram_chunks(dev(w.data), off64(w.blk_off), hist, ch)
    got = hist.cpu().numpy().view(np.uint32).reshape(w.nblk, 256)
    gch = ch.cpu().numpy().view(np.uint32).reshape(w.nblk, P.CHUNKS, 256)
    for b in range(w.nblk):
        blk = w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])]
        assert np.array_equal(got[b], oracle.histogram(blk)), b
        bounds = _chunk_bounds(blk.size)
        for c in range(P.CHUNKS):
            want = oracle.histogram(blk[bounds[c][0]:bounds[c][1]]) if c < len(bounds) else np.zeros(256, np.uint32)
            assert np.array_equal(gch[b, c], want), (b, c)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("name", ["shifting", "mixed_24", "edge"])
def test_encode_plain_equals_chunked(P, name, flat):
    """pivco_encode_blocks (chunks counted in the encoder) and
    pivco_encode_blocks_chunked write the same records."""
    import torch
    w = WORKLOADS[name]()
    data, boff = dev(w.data), off64(w.blk_off)
    enc = P.Encoder(w.nblk, P.params(flat=flat))
    total = enc.plan(data, boff)
    enc.ensure(total)
    P.encode_blocks_chunked(data, boff, w.nblk, enc.layout, enc.chunk_hist, enc.comp, enc.off, enc.rec_bytes,
                            enc.status)
    a = enc.comp[:total].clone()
    ra, sa = enc.rec_bytes.clone(), enc.status.clone()
    enc.comp.fill_(0x5A)
    P.encode_blocks(data, boff, w.nblk, enc.layout, enc.comp, enc.off, enc.rec_bytes, enc.status)
    assert not sa.cpu().numpy().any() and not enc.status.cpu().numpy().any()
    assert torch.equal(ra, enc.rec_bytes)
    off, rb = enc.off.cpu().numpy(), ra.cpu().numpy()
    ca, cb = a.cpu().numpy(), enc.comp[:total].cpu().numpy()
    for b in range(w.nblk):
        lo, hi = int(off[b]), int(off[b]) + int(rb[b])
        assert np.array_equal(ca[lo:hi], cb[lo:hi]), b


def _encode_with_chunks(P, enc, data, boff, ch, guard):
    import torch
    total = int(enc.off[-1].item())
    comp = torch.full((total + 2 * guard,), 0xA5, dtype=torch.uint8, device="cuda")
    P.encode_blocks_chunked(data, boff, enc.nblk, enc.layout, ch, comp, enc.off + guard, enc.rec_bytes, enc.status)
    return comp.cpu().numpy(), enc.status.cpu().numpy(), enc.rec_bytes.cpu().numpy()


def test_encode_chunked_stale_histograms(P):
    """Chunk histograms that do not describe the input never give a wrong
    record with an OK status, nor a write outside the blocks' records: chunk
    histograms of other data (block totals differ: an error status), and of
    the same blocks reversed (block totals agree, the chunks' do not; the
    shifting blocks also take the part-by-part path): each such block either
    reports PIVCO_ERR_INVALID_ARG or, where the encoder coded together the
    chunks whose summed counts are right, gives the exact record."""
    import torch
    w = shifting_workload()
    data, boff = dev(w.data), off64(w.blk_off)
    enc = P.Encoder(w.nblk)
    total = enc.plan(data, boff)
    good = enc.chunk_hist.clone()
    guard = 4096
    ref, st, rb = _encode_with_chunks(P, enc, data, boff, good, guard)
    assert not st.any()
    off = enc.off.cpu().numpy()
    h2 = torch.empty_like(enc.hist)
    # other data of the same size
    other = np.random.default_rng(3).integers(0, 256, w.data.size).astype(np.uint8)
    stale = torch.empty_like(good)
    P.histogram_chunks(dev(other), boff, h2, stale)
    c, st2, _ = _encode_with_chunks(P, enc, data, boff, stale, guard)
    assert (st2 == P.ERR_INVALID_ARG).all(), st2
    assert (c[:guard] == 0xA5).all() and (c[guard + total:] == 0xA5).all()
    # odd blocks get the chunk counts of their reversed bytes
    rev = np.concatenate([w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])][::-1] for b in range(w.nblk)])
    P.histogram_chunks(dev(rev), boff, h2, stale)
    mixed = good.clone().view(w.nblk, -1)
    mixed[1::2] = stale.view(w.nblk, -1)[1::2]
    c, st3, rb3 = _encode_with_chunks(P, enc, data, boff, mixed.view(-1), guard)
    assert (c[:guard] == 0xA5).all() and (c[guard + total:] == 0xA5).all()
    n_refused = 0
    for b in range(w.nblk):
        lo, hi = guard + int(off[b]), guard + int(off[b]) + int(rb[b])
        if b % 2 and st3[b] == P.ERR_INVALID_ARG:
            n_refused += 1
            continue
        assert st3[b] == 0 and rb3[b] == rb[b], (b, st3)
        assert np.array_equal(c[lo:hi], ref[lo:hi]), b
    assert n_refused >= 1    # (some odd block is cut where its chunk counts matter)
    # the right counts again: the records decode
    comp = torch.from_numpy(ref[guard:guard + total].copy()).cuda()
    out, st4 = P.decode(comp, enc.off, boff)
    assert not st4.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)


def test_misaligned_records_rejected(P):
    """A record placed off a 16-byte boundary is an argument error, for the
    encoder (nothing written) and for every decode path (not read as words)."""
    import torch
    w = workloads.skew80(nblk=4, bs=65536)
    data, boff = dev(w.data), off64(w.blk_off)
    enc = P.Encoder(w.nblk)
    total = enc.plan(data, boff)
    enc.ensure(total)
    comp = torch.full((total + 64,), 0x77, dtype=torch.uint8, device="cuda")
    P.encode_blocks_chunked(data, boff, w.nblk, enc.layout, enc.chunk_hist, comp, enc.off + 4, enc.rec_bytes,
                            enc.status)
    assert (enc.status.cpu().numpy() == P.ERR_INVALID_ARG).all()
    assert (comp.cpu().numpy() == 0x77).all()
    # good records, then the same bytes 4 bytes further on
    good = P.encode(data, boff)
    rec = good.comp[:total]
    shifted = torch.zeros(total + 64, dtype=torch.uint8, device="cuda")
    shifted[4:4 + total] = rec
    for batched in (False, True):
        out, st = P.decode(shifted, good.off + 4, boff, batched=batched)
        assert (st.cpu().numpy() == P.ERR_INVALID_ARG).all(), (batched, st)
        out, st = P.decode(rec.contiguous(), good.off, boff, batched=batched)
        assert not st.cpu().numpy().any()
        assert np.array_equal(out.cpu().numpy()[: w.data.size], w.data)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
@pytest.mark.parametrize("ans", [False, True])
def test_plan_blocks_equals_steps(P, name, ans, flat):
    """The one-launch plan writes what the histogram, code-length and layout
    calls write one after another."""
    import torch
    w = WORKLOADS[name]()
    n = w.nblk
    data, boff = dev(w.data), off64(w.blk_off)
    prm = P.params(ans=ans, flat=flat)

    def bufs():
        return (torch.zeros(n * 256, dtype=torch.int32, device="cuda"),
                torch.zeros(n * P.CHUNKS * 256, dtype=torch.int32, device="cuda"),
                torch.zeros(n * 256, dtype=torch.uint8, device="cuda"),
                torch.zeros(n * P.layout_bytes(), dtype=torch.uint8, device="cuda"),
                torch.zeros(n, dtype=torch.int64, device="cuda"),
                torch.full((n,), 77, dtype=torch.int32, device="cuda"))

    h1, c1, l1, y1, r1, s1 = bufs()
    P.histogram_chunks(data, boff, h1, c1)
    P.code_lengths(h1, n, prm.max_len, l1, s1)
    P.build_layout(h1, l1, n, prm, y1, r1, s1)
    h2, c2, l2, y2, r2, s2 = bufs()
    P.plan_blocks(data, boff, prm, h2, c2, l2, y2, r2, s2)
    for a, b in [(h1, h2), (c1, c2), (l1, l2), (y1, y2), (r1, r2), (s1, s2)]:
        assert torch.equal(a, b)


@pytest.mark.parametrize("shift", [1, 3, 8, 13])
def test_unaligned_input(P, oracle, shift):
    """Blocks read through an input pointer at any byte offset: histograms,
    plan and records are the same as from an aligned buffer."""
    import torch
    w = WORKLOADS["mixed_24"]()
    buf = torch.zeros(w.data.size + 32, dtype=torch.uint8, device="cuda")
    buf[shift:shift + w.data.size] = dev(w.data)
    data = buf[shift:shift + w.data.size]
    assert data.data_ptr() % 16 == shift % 16
    boff = off64(w.blk_off)
    h = torch.empty(w.nblk * 256, dtype=torch.int32, device="cuda")
    P.histogram(data, boff, h)
    got = h.cpu().numpy().view(np.uint32).reshape(w.nblk, 256)
    for b in range(w.nblk):
        assert np.array_equal(got[b], oracle.histogram(w.data[int(w.blk_off[b]):int(w.blk_off[b + 1])])), b
    enc = P.encode(data, boff, P.params(ans=True))
    ref = P.encode(dev(w.data), boff, P.params(ans=True))
    assert not enc.status.cpu().numpy().any()
    assert torch.equal(enc.off, ref.off) and torch.equal(enc.rec_bytes, ref.rec_bytes)
    off, rb = ref.off.cpu().numpy(), ref.rec_bytes.cpu().numpy()
    a, r = enc.comp.cpu().numpy(), ref.comp.cpu().numpy()
    for b in range(w.nblk):
        lo = int(off[b])
        assert np.array_equal(a[lo:lo + int(rb[b])], r[lo:lo + int(rb[b])]), b


@pytest.mark.parametrize("flat", [False, True])
def test_big_blocks_coded_chunk_by_chunk(P, oracle, flat):
    """Blocks whose levels do not fit the encoder's buffers are coded one
    plan chunk per work item, possibly by different CTAs at once; their
    records are the oracle's byte for byte, beside small blocks coded whole,
    ragged sizes included, and they decode."""
    rng = np.random.default_rng(41)
    blocks = [rng.integers(0, 200, 200001).astype(np.uint8),                         # high entropy, 8 chunks
              rng.choice(256, 131072, p=rng.dirichlet(np.ones(256) * 0.3)).astype(np.uint8),
              rng.integers(0, 5, 16383).astype(np.uint8),                            # 3 chunks, ragged end
              np.full(5000, 4, np.uint8),                                            # constant, whole
              rng.integers(0, 3, 4000).astype(np.uint8),                             # small, whole
              rng.integers(0, 97, 65536 + 33).astype(np.uint8)]
    off = np.zeros(len(blocks) + 1, np.uint64)
    off[1:] = np.cumsum([b.size for b in blocks])
    data = np.concatenate(blocks)
    enc = P.encode(dev(data), off64(off), P.params(flat=flat))
    st = enc.status.cpu().numpy()
    assert not st.any(), st
    comp, coff, rb = enc.comp.cpu().numpy(), enc.off.cpu().numpy(), enc.rec_bytes.cpu().numpy()
    for b, x in enumerate(blocks):
        ref = oracle.encode_block(x, oracle.params(flat=flat))
        got = comp[int(coff[b]):int(coff[b]) + int(rb[b])]
        assert got.size == ref.size and np.array_equal(got, ref), b
    out, st = P.decode(enc.comp, enc.off, off64(off))
    assert not st.cpu().numpy().any()
    assert np.array_equal(out.cpu().numpy()[: data.size], data)
