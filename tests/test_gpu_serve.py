"""GPU: the decompression server (device-resident request loop, admission by
device-memory budget, continuous batching).

Every request's result must be exactly what pivco_decode_blocks gives for it
alone (whose bytes the oracle pins in the parity tests), whatever else is in
flight: bytes and status, for valid and corrupt requests alike."""
import time

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
    P.set_tuning()
    return P


def _encode_requests(P, reqs):
    """Records of every request (host), plus its decode alone (host); every
    other request coded with the regrouped tree (PVC2), so the server decodes
    both kinds of record in one mix."""
    import torch
    out = []
    for i, r in enumerate(reqs):
        data = torch.from_numpy(r.data).cuda()
        boff = torch.from_numpy(r.blk_off.astype(np.int64)).cuda()
        enc = P.encode(data, boff, P.params(ans=r.ans, flat=bool(i % 2)))
        assert not enc.status.cpu().numpy().any()
        alone, st = P.decode(enc.comp, enc.off, boff)
        comp = enc.comp[: int(enc.off[-1].item())].cpu().numpy()
        out.append({"comp": comp, "coff": enc.off.cpu().numpy().astype(np.uint64),
                    "ooff": r.blk_off.astype(np.uint64), "alone": alone.cpu().numpy()[: r.data.size],
                    "alone_status": st.cpu().numpy(), "data": r.data})
    return out


def _pinned(a):
    import torch
    t = torch.empty(max(a.size, 1), dtype=torch.uint8, pin_memory=True)
    t[: a.size] = torch.from_numpy(a)
    return t


def _serve(P, items, arena_bytes, budget=0, gap_s=0.0):
    import torch
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    outs, ids = [], []
    with P.Server(arena, budget_bytes=budget) as srv:
        for it in items:
            comp = _pinned(it["comp"])
            out = torch.zeros(max(it["data"].size, 1), dtype=torch.uint8, pin_memory=True)
            ids.append(srv.submit(comp, it["coff"], it["ooff"], out))
            outs.append((comp, out))
            if gap_s:
                time.sleep(gap_s)
        srv.drain(120000)
        res = []
        for rid, (comp, out) in zip(ids, outs):
            state, status, lat = srv.poll(rid)
            assert state == P.DONE
            res.append((status, out.numpy()[: len(out)], lat))
    return res


@pytest.fixture(scope="module")
def items(P):
    reqs = workloads.serving_requests(24, 200.0, seed=4, hi=3 << 20)
    return _encode_requests(P, reqs)


def test_serve_burst_equals_alone(P, items):
    res = _serve(P, items, 1 << 30)
    for it, (status, out, lat) in zip(items, res):
        assert status == 0
        n = it["data"].size
        assert np.array_equal(out[:n], it["alone"]) and np.array_equal(out[:n], it["data"])
        assert lat > 0


def test_serve_staggered_small_budget(P, items):
    # room for roughly one large request at a time: admission must wait for retirements
    big = max(it["comp"].size + 3 * it["data"].size for it in items)
    res = _serve(P, items, 512 << 20, budget=big + (8 << 20), gap_s=0.002)
    for it, (status, out, lat) in zip(items, res):
        assert status == 0
        assert np.array_equal(out[: it["data"].size], it["alone"])


def test_serve_corrupt_and_empty_in_mix(P, items):
    mix = [dict(it) for it in items[:8]]
    bad = dict(mix[3])
    comp = bad["comp"].copy()
    comp[int(bad["coff"][0]) + 144] ^= 2            # n_v of the first block's root
    bad["comp"] = comp
    mix[3] = bad
    empty = {"comp": np.zeros(0, np.uint8), "coff": np.zeros(1, np.uint64), "ooff": np.zeros(1, np.uint64),
             "data": np.zeros(0, np.uint8), "alone": np.zeros(0, np.uint8)}
    mix.insert(5, empty)
    # the corrupt request decoded alone through the plain entry point
    import torch
    alone, st = P.decode(torch.from_numpy(comp).cuda(), torch.from_numpy(bad["coff"].astype(np.int64)).cuda(),
                         torch.from_numpy(bad["ooff"].astype(np.int64)).cuda())
    st = st.cpu().numpy()
    first_bad = int(st[np.nonzero(st)[0][0]])
    res = _serve(P, mix, 1 << 30)
    for i, (it, (status, out, lat)) in enumerate(zip(mix, res)):
        if i == 3:
            assert status == first_bad
            ok = st == 0
            for b in np.nonzero(ok)[0]:          # the intact blocks still decode as alone
                lo, hi = int(it["ooff"][b]), int(it["ooff"][b + 1])
                assert np.array_equal(out[lo:hi], alone.cpu().numpy()[lo:hi])
        else:
            assert status == 0
            assert np.array_equal(out[: it["data"].size], it["alone"])


def test_serve_rejects_oversized(P, items):
    import torch
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    it = max(items, key=lambda x: x["data"].size)
    with P.Server(arena, budget_bytes=it["data"].size // 2) as srv:
        out = torch.zeros(it["data"].size, dtype=torch.uint8, pin_memory=True)
        with pytest.raises(P.PivcoError, match="CAPACITY"):
            srv.submit(_pinned(it["comp"]), it["coff"], it["ooff"], out)
