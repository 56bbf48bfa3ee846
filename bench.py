"""PivCo-Huffman benchmark on GB300: encode + decode throughput of the hot path.

One step = one pass of the whole path over one batch of synthetic blocks:
histogram -> code lengths -> layout -> record placement (scan) -> encode
(-> selective ANS) and then decode (plan -> ANS decode -> rank directories ->
bottom-up merge).  Each leg is timed with CUDA events on the launching
stream; L2 is flushed before each leg.  `value` is raw bytes / (encode time +
decode time) summed over all ranks' blocks (weak scaling: every rank codes
its own batch).  The headline workload is skew80 (4096 x 64 KiB); the other
configurations (zipf1, skew95, mixed) are measured the same way and reported
under `per_config`.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload skew80]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm

Prints one JSON line on rank 0.
"""
import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PivCo decode/encode GB/s on 1 GB300 (% HBM peak), batched vs plain; p99 ms"
WORKLOADS = {
    "skew80": "4096 blocks x 64 KiB (256 MiB), byte 0 with P=0.8, 255 others uniform, no ANS, seed 1",
    "skew95": "2048 blocks x 128 KiB (256 MiB), P(top)=0.95 + Zipf(1.3) tail, selective ANS, seed 2",
    "mixed": "4096 blocks log-uniform 4 KiB-1 MiB, per-block alphabet/Zipf, selective ANS, seed 3",
    "zipf1": "1 block of 2^20 symbols, Zipf(1.0) over 256, no ANS, seed 0",
}
# the kernels whose source a committed ncu record (profiles/traffic.json) belongs to
KERNEL_SOURCES = {"encode_kernel": "paper_2606_05765_gb300/csrc/k_encode.cu",
                  "decode_batch_kernel": "paper_2606_05765_gb300/csrc/k_decode.cu"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pivco", choices=["pivco", "reference"])
    ap.add_argument("--workload", default="skew80", choices=sorted(WORKLOADS))
    ap.add_argument("--tree", default="flat", choices=["flat", "canonical"],
                    help="records of the regrouped tree with flat subtrees (PVC2, Sec. 2.2.3-2.2.4) or of the "
                         "canonical tree (PVC1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-config", action="store_true", help="measure the headline workload only")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-segments", type=int, default=8)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default decode tuning")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="offered-load time per arrival rate")
    ap.add_argument("--serve-repeats", type=int, default=3, help="runs per arrival rate (p99 reported per run)")
    return ap.parse_args(argv)


def shard_blocks(nblk, rank, world):
    """Contiguous block range of this rank (blocks are independent units)."""
    per = (nblk + world - 1) // world
    lo = min(nblk, rank * per)
    return lo, min(nblk, lo + per)


def reduce_max(value, device=None):
    """Max over ranks of a per-rank figure (the timed region's duration); the
    only collective of the multi-GPU bench (blocks shard with no exchange)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(raw_per_rank, steps, tot_ms_max, world):
    """Whole-job throughput: the bytes all ranks processed / the slowest rank's time."""
    return world * raw_per_rank * steps / (tot_ms_max / 1e3) / 1e9


def kernel_record(kernel, workload):
    """DRAM bytes and warp instructions per launch of `kernel` on `workload`
    (records of the tree --tree names: "skew80", "skew80/canonical") from the
    committed ncu summary (profiles/traffic.json), only while the kernel's
    source file is byte-identical to the one profiled (else {})."""
    import hashlib
    key = workload if FLAT else workload + "/canonical"
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key][kernel]
        src = open(os.path.join(ROOT, KERNEL_SOURCES[kernel]), "rb").read()
    except (OSError, KeyError, ValueError):
        return {}
    return rec if hashlib.sha256(src).hexdigest() == rec.get("source_sha256") else {}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index, period_ms=20):
        self.cmd = ["nvidia-smi", "-i", str(gpu_index),
                    "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                    "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                    "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", str(period_ms)]
        self.lines, self.proc = [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            time.sleep(0.1)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Cores this process may run on (read at run time)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_round_trip(oracle, prm, x, sub_off):
    buf, rec_off, sizes = oracle.encode_batch(x, sub_off, prm)
    st, out = oracle.decode_batch(buf, rec_off[:-1], sizes, sub_off)
    assert not st.any() and np.array_equal(out, x)


# tree of the records every leg codes (set from --tree): regrouped with flat subtrees, or canonical
FLAT = True
TREE_DESC = {"flat": "regrouped tree with flat subtrees (records PVC2, Sec. 2.2.3-2.2.4)",
             "canonical": "canonical tree (records PVC1)"}


def cpu_baseline(w, budget_s=10.0, ans=False):
    """The oracle as it stands, on the host: single-threaded over a bounded
    prefix of the same blocks (about budget_s), then on every host core
    (one block per task, threads over blocks: the oracle's C calls run
    without the interpreter lock) over a prefix of the same size per core.
    Returns GB/s of raw bytes per (encode + decode)."""
    import oracle
    oracle.build()
    prm = oracle.params(ans=ans, flat=FLAT)
    nb, t_all, raw_all, used = 1, 0.0, 0, 0
    while used < w.nblk and t_all < budget_s:
        take = min(nb, w.nblk - used)
        lo, hi = int(w.blk_off[used]), int(w.blk_off[used + take])
        sub_off = (w.blk_off[used:used + take + 1] - w.blk_off[used]).astype(np.uint64)
        t0 = time.perf_counter()
        _oracle_round_trip(oracle, prm, w.data[lo:hi], sub_off)
        t_all += time.perf_counter() - t0
        raw_all += hi - lo
        used += take
        nb *= 2
    single = raw_all / t_all / 1e9
    cores = host_cores()
    # all cores: blocks handed out one per task, up to `cores` times the
    # single-threaded sample (so the run stays about budget_s long)
    want = min(w.nblk, max(used, 1) * cores)
    jobs = []
    for b in range(want):
        lo, hi = int(w.blk_off[b]), int(w.blk_off[b + 1])
        jobs.append((w.data[lo:hi], np.array([0, hi - lo], np.uint64)))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda j: _oracle_round_trip(oracle, prm, j[0], j[1]), jobs))
    t_par = time.perf_counter() - t0
    raw_par = int(w.blk_off[want])
    return {"value": raw_par / t_par / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of %d blocks (%.1f MB), encode+decode, %.1f s on %d threads (one block per task); "
                      "single-threaded: %.4f GB/s on the first %d blocks (%.1f MB, %.1f s)"
                      % (want, w.nblk, raw_par / 1e6, t_par, cores, single, used, raw_all / 1e6, t_all),
            "single_thread_gbs": single}


def serving_leg(P, seconds=2.0, budget=8 << 30, pool_n=48, seed=4, repeats=3):
    """Poisson decompression requests through the server (device-resident
    loop, admission by an 8 GiB device budget).  A pool of distinct requests
    (sizes log-uniform 1 KiB-16 MiB, each drawn from the skew80 / skew95 /
    mixed distributions) is encoded once; arrivals pick pool entries.  The
    capacity is measured first (everything submitted at once), then arrivals
    are offered at 0.5, 0.8 and 0.95 of it, `repeats` runs each.  Latency =
    result in host memory minus the scheduled arrival."""
    import ctypes as C
    import torch
    import workloads
    reqs = workloads.serving_requests(pool_n, 1.0, seed=seed)
    pool = []
    for r in reqs:
        data = torch.from_numpy(r.data).cuda()
        boff = torch.from_numpy(r.blk_off.astype(np.int64)).cuda()
        enc = P.encode(data, boff, P.params(ans=r.ans, flat=FLAT))
        tot = int(enc.off[-1].item())
        comp = torch.empty(max(tot, 1), dtype=torch.uint8, pin_memory=True)
        comp[:tot].copy_(enc.comp[:tot])
        out = torch.zeros(max(r.data.size, 1), dtype=torch.uint8, pin_memory=True)
        coff = enc.off.cpu().numpy().astype(np.uint64)
        ooff = r.blk_off.astype(np.uint64)
        pool.append({"data": r.data, "comp": comp, "out": out, "coff": coff, "ooff": ooff,
                     "raw": int(r.data.size), "nblk": int(coff.size - 1)})
    torch.cuda.synchronize()
    arena = torch.empty(budget + (16 << 20), dtype=torch.uint8, device="cuda")
    lib = P.lib()
    rid = C.c_uint64()

    def run(order, arrivals):
        srv = P.Server(arena, budget_bytes=budget)
        t_sub, ids = [], []
        try:
            t0 = time.perf_counter()
            i = 0
            while i < len(order):
                now = time.perf_counter() - t0
                if arrivals[i] > now:
                    if arrivals[i] - now > 2e-4:
                        time.sleep(1e-4)
                    continue
                e = pool[order[i]]
                rc = lib.pivco_server_submit(srv.handle, C.c_void_p(e["comp"].data_ptr()),
                                             C.c_void_p(e["coff"].ctypes.data), e["nblk"],
                                             C.c_void_p(e["ooff"].ctypes.data), C.c_void_p(e["out"].data_ptr()),
                                             C.byref(rid))
                if rc != 0:
                    raise P.PivcoError("pivco_server_submit: %s" % P.STATUS_NAMES.get(rc, rc))
                t_sub.append(time.perf_counter() - t0)
                ids.append(rid.value)
                i += 1
            srv.drain(600000)
            t_end = time.perf_counter() - t0
            lat, bad = [], 0
            for k, q in enumerate(ids):
                st, status, l_ms = srv.poll(q)
                bad += status != 0 or st != P.DONE
                lat.append(l_ms + 1e3 * (t_sub[k] - arrivals[k]))
        finally:
            srv.close()
        raw = sum(pool[j]["raw"] for j in order)
        return {"n": len(order), "raw_bytes": raw, "wall_s": t_end, "lat_ms": lat, "bad": bad,
                "last_done_s": max(arrivals[k] + lat[k] / 1e3 for k in range(len(order)))}

    rng = np.random.Generator(np.random.PCG64(seed))
    burst = [j % pool_n for j in range(4 * pool_n)]
    run(burst[:pool_n], np.zeros(pool_n))                      # warm-up
    cap = run(burst, np.zeros(len(burst)))
    cap_gbs = cap["raw_bytes"] / cap["wall_s"] / 1e9
    # what the copies alone take: every request of the burst, its records in
    # and its output back between pinned host memory and the device, one
    # request after the other on one stream (no decode)
    dcomp = torch.empty(max(int(e["comp"].numel()) for e in pool), dtype=torch.uint8, device="cuda")
    dout = torch.empty(max(e["raw"] for e in pool), dtype=torch.uint8, device="cuda")
    hout = torch.empty(dout.numel(), dtype=torch.uint8, pin_memory=True)
    cs = torch.cuda.Stream()
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(cs):
            for j in burst:
                e = pool[j]
                nc = int(e["comp"].numel())
                dcomp[:nc].copy_(e["comp"], non_blocking=True)
                hout[:e["raw"]].copy_(dout[:e["raw"]], non_blocking=True)
        cs.synchronize()
        t_copy = time.perf_counter() - t0
    copy_gbs = cap["raw_bytes"] / t_copy / 1e9
    mean_raw = np.mean([e["raw"] for e in pool])
    rates = []
    ok = cap["bad"] == 0
    for frac in (0.5, 0.8, 0.95):
        lam = frac * cap_gbs * 1e9 / mean_raw                  # requests per second
        n = int(min(10000, max(200, lam * seconds)))
        runs = []
        for _ in range(max(1, repeats)):
            order = rng.integers(0, pool_n, n)
            arrivals = np.cumsum(rng.exponential(1.0 / lam, n))
            r = run(order, arrivals)
            ok = ok and r["bad"] == 0
            span = max(r["last_done_s"], arrivals[-1])
            runs.append({"offered_gbs": r["raw_bytes"] / arrivals[-1] / 1e9, "gbs": r["raw_bytes"] / span / 1e9,
                         "p50": float(np.percentile(r["lat_ms"], 50)), "p99": float(np.percentile(r["lat_ms"], 99))})
        p99s = [x["p99"] for x in runs]
        rates.append({"load": frac, "requests": n, "runs": len(runs),
                      "offered_gbs": round(statistics.mean(x["offered_gbs"] for x in runs), 3),
                      "gbs": round(statistics.mean(x["gbs"] for x in runs), 3),
                      "p50_ms": round(statistics.median(x["p50"] for x in runs), 4),
                      "p99_ms": round(statistics.median(p99s), 4),
                      "p99_ms_runs": [round(x, 4) for x in p99s]})
    for e in pool:
        n = e["raw"]
        ok = ok and bool(np.array_equal(e["out"].numpy()[:n], e["data"]))
    return {"budget_bytes": budget, "pool_requests": pool_n, "capacity_gbs": round(cap_gbs, 3),
            "capacity_requests": len(burst), "copies_only_gbs": round(copy_gbs, 3), "rates": rates, "verified": ok,
            "latency": "result in pinned host memory minus scheduled arrival; p99_ms is the median over runs",
            "sizes": "log-uniform 1 KiB-16 MiB; skew80 64 KiB / skew95 128 KiB / mixed 1 MiB blocks"}


def make_workload(name):
    import workloads
    return workloads.by_name(name)


def run_reference(args):
    """Reference arm: the oracle (the paper's method restated plainly in C)."""
    global FLAT
    FLAT = args.tree == "flat"
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make_workload(args.workload)
    import oracle
    oracle.build()
    prm = oracle.params(ans=w.ans, flat=FLAT)
    # each step: a bounded sample of the workload (16 blocks, <= a few MB)
    take = min(w.nblk, 16)
    lo, hi = 0, int(w.blk_off[take])
    sub_off = w.blk_off[:take + 1].astype(np.uint64)
    x = w.data[lo:hi]
    for _ in range(args.warmup):
        buf, rec_off, sizes = oracle.encode_batch(x, sub_off, prm)
        oracle.decode_batch(buf, rec_off[:-1], sizes, sub_off)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        buf, rec_off, sizes = oracle.encode_batch(x, sub_off, prm)
        st, out = oracle.decode_batch(buf, rec_off[:-1], sizes, sub_off)
        times.append(time.perf_counter() - t0)
        assert not st.any()
    tot = sum(times)
    value = (hi - lo) * len(times) / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload], "sample_blocks": take,
                       "sample_bytes": hi - lo, "tree": args.tree},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first %d blocks (%d bytes) per step, single-threaded" % (take, hi - lo)},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _stats(xs):
    """mean, median, best (the paper's App. C keeps the best run) of a list of ms."""
    return {"mean": statistics.mean(xs), "median": statistics.median(xs), "best": min(xs)}


def measure(P, torch, w, dev, stream, flush, steps, warmup, autotune):
    """Times one workload: the batched path (encode sequence and persistent
    decode, each a CUDA graph) and the plain path (one launch per pipeline
    step), plus the encode kernel alone.  Returns times (ms per step) and
    checks."""
    raw = int(w.data.size)
    nblk = w.nblk
    data = torch.from_numpy(w.data).to(dev)
    blk_off = torch.from_numpy(w.blk_off.astype(np.int64)).to(dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        enc = P.Encoder(nblk, P.params(ans=w.ans, flat=FLAT), dev)
        enc.ensure(enc.plan(data, blk_off, stream))
        res = enc.run(data, blk_off, stream, replan=False)
        dec = P.Decoder(nblk, dev)
        P.set_tuning(16384, 64, 0)         # the largest workspace any autotuner candidate needs
        dec.prepare(res.comp, res.off, stream)
        P.set_tuning()
        out = torch.empty(raw, dtype=torch.uint8, device=dev)
        # pick the decode launch tuning for this batch (does not change the bytes)
        if autotune:
            tuned, _ = P.autotune_decode(res.comp, res.off, nblk, out, blk_off, dec.ws, dec.status, reps=2,
                                         stream=stream)
        else:
            tuned = P.get_tuning()
        dec.prepare(res.comp, res.off, stream)
        n0 = P.launch_count()
        g_enc = P.Graph(stream)
        with g_enc:
            enc.run(data, blk_off, stream)
        n_enc_graph = P.launch_count() - n0
        n0 = P.launch_count()
        g_dec = P.Graph(stream)
        with g_dec:
            P.decode_batched(res.comp, res.off, nblk, out, blk_off, dec.ws, dec.status, stream)
        n_dec_graph = P.launch_count() - n0
    stream.synchronize()
    E = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def plain_step():
        flush.zero_()
        E[0].record(stream)
        enc.run(data, blk_off, stream)
        E[1].record(stream)
        flush.zero_()
        E[2].record(stream)
        P.decode_plan(res.comp, res.off, nblk, dec.ws, dec.status, stream)
        P.decode_ans(res.comp, res.off, nblk, dec.ws, dec.status, stream)
        E[3].record(stream)
        P.decode_merge(res.comp, res.off, nblk, out, blk_off, dec.ws, dec.status, stream)
        E[4].record(stream)

    def batched_step():
        flush.zero_()
        E[0].record(stream)
        g_enc.launch(stream)
        E[1].record(stream)
        flush.zero_()
        E[2].record(stream)
        g_dec.launch(stream)
        E[4].record(stream)

    def timed(step_fn, n):
        t_enc, t_dec, t_mid = [], [], []
        with torch.cuda.stream(stream):
            for _ in range(n):
                step_fn()
                E[4].synchronize()
                t_enc.append(E[0].elapsed_time(E[1]))
                t_dec.append(E[2].elapsed_time(E[4]))
                t_mid.append(E[3].elapsed_time(E[4]) if step_fn is plain_step else t_dec[-1])
        return t_enc, t_dec, t_mid

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plain_step()
            batched_step()
    torch.cuda.synchronize()
    r = {"w": w, "raw": raw, "nblk": nblk, "tuning": tuned.as_dict(),
         "launches_per_step": n_enc_graph + n_dec_graph}
    r["b_enc"], r["b_dec"], _ = timed(batched_step, steps)
    torch.cuda.synchronize()
    ok_b = (not enc.status.cpu().numpy().any()) and (not dec.status.cpu().numpy().any()) and bool(torch.equal(out, data))
    out.zero_()
    r["p_enc"], r["p_dec"], r["p_merge"] = timed(plain_step, max(3, steps // 2))
    torch.cuda.synchronize()
    ok_p = (not enc.status.cpu().numpy().any()) and (not dec.status.cpu().numpy().any()) and bool(torch.equal(out, data))
    # the encode kernel alone (statistics already on the device)
    Ek = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    t_enck = []
    with torch.cuda.stream(stream):
        for _ in range(max(3, steps // 4)):
            flush.zero_()
            Ek[0].record(stream)
            P.encode_blocks_chunked(data, blk_off, nblk, enc.layout, enc.chunk_hist, enc.comp, enc.off, enc.rec_bytes,
                                    enc.status, stream)
            Ek[1].record(stream)
            Ek[1].synchronize()
            t_enck.append(Ek[0].elapsed_time(Ek[1]))
        enc.run(data, blk_off, stream)          # the final records (with ANS) again
    torch.cuda.synchronize()
    r["enc_kernel"] = t_enck
    r["rec_bytes"] = int(enc.rec_bytes.sum().item())
    r["ok"] = ok_b and ok_p and not enc.status.cpu().numpy().any()
    r["checks"] = {"batched": ok_b, "plain": ok_p}
    del g_enc, g_dec
    return r


def roofline(r, workload, peak_gbs, issue_peak):
    """Rooflines of the two big kernels of the batched step.  Both are bound
    by the integer/shared-memory instruction issue rate, so `bound` is "alu":
    achieved = warp instructions per launch (committed ncu capture of this
    source) / event-timed duration, against the SM issue peak (SMs x 4
    schedulers x SM clock).  The HBM figure (algorithmic bytes / duration
    against the measured copy bandwidth) is given beside it."""
    algo = r["raw"] + r["rec_bytes"]
    ks = {"decode_batch_kernel": statistics.mean(r["b_dec"]), "encode_kernel": statistics.mean(r["enc_kernel"])}
    out = {}
    for k, ms in ks.items():
        rec = kernel_record(k, workload)
        gbs = algo / (ms / 1e3) / 1e9
        e = {"ms": round(ms, 4), "bytes": algo, "hbm_gbs": round(gbs, 2), "hbm_frac": round(gbs / peak_gbs, 4),
             "traffic": rec.get("bytes")}
        if rec.get("inst"):
            ips = rec["inst"] / (ms / 1e3)
            e.update({"warp_inst": rec["inst"], "issue_tinst_s": round(ips / 1e12, 4),
                      "issue_frac": round(ips / issue_peak, 4)})
        out[k] = e
    dom = max(ks, key=ks.get)
    d = out[dom]
    line = {"bound": "alu" if "issue_frac" in d else "hbm", "kernel": dom}
    if "issue_frac" in d:
        line.update({"achieved": d["issue_tinst_s"], "peak": round(issue_peak / 1e12, 4), "unit": "Twarp-inst/s",
                     "frac": d["issue_frac"], "traffic": d["traffic"],
                     "hbm": {"achieved": d["hbm_gbs"], "peak": peak_gbs, "unit": "GB/s", "frac": d["hbm_frac"]}})
    else:
        line.update({"achieved": d["hbm_gbs"], "peak": peak_gbs, "unit": "GB/s", "frac": d["hbm_frac"],
                     "traffic": d["traffic"]})
    line["kernels"] = out
    return line


def summarize(r, world, dev, peak_gbs, issue_peak, workload):
    raw = r["raw"]
    r4 = lambda x: round(x, 4)
    b_step = [a + b for a, b in zip(r["b_enc"], r["b_dec"])]
    tot_b = reduce_max(sum(b_step), dev)
    tot_p = reduce_max(sum(a + b for a, b in zip(r["p_enc"], r["p_dec"])), dev)
    gbs = lambda ms: raw / (ms / 1e3) / 1e9
    return {
        "value": round(whole_job_gbs(raw, len(b_step), tot_b, world), 3),
        "ms_per_step": r4(tot_b / len(b_step)),
        "encode_gbs": round(gbs(statistics.mean(r["b_enc"])), 3),
        "decode_gbs": round(gbs(statistics.mean(r["b_dec"])), 3),
        "best_of_runs": {"value": round(raw / (min(b_step) / 1e3) / 1e9, 3),
                         "encode_gbs": round(gbs(min(r["b_enc"])), 3), "decode_gbs": round(gbs(min(r["b_dec"])), 3)},
        "p50_ms": r4(float(np.percentile(b_step, 50))), "p99_ms": r4(float(np.percentile(b_step, 99))),
        "batched": {"value": round(whole_job_gbs(raw, len(b_step), tot_b, world), 3),
                    "encode_ms": {k: r4(v) for k, v in _stats(r["b_enc"]).items()},
                    "decode_ms": {k: r4(v) for k, v in _stats(r["b_dec"]).items()}},
        "plain": {"value": round(whole_job_gbs(raw, len(r["p_enc"]), tot_p, world), 3),
                  "ms_per_step": r4(tot_p / len(r["p_enc"])),
                  "encode_gbs": round(gbs(statistics.mean(r["p_enc"])), 3),
                  "decode_gbs": round(gbs(statistics.mean(r["p_dec"])), 3),
                  "encode_ms": {k: r4(v) for k, v in _stats(r["p_enc"]).items()},
                  "decode_ms": {k: r4(v) for k, v in _stats(r["p_dec"]).items()}},
        "roofline": roofline(r, workload, peak_gbs, issue_peak),
        "tuning": r["tuning"],
    }


def main(argv=None):
    global FLAT
    args = parse_args(argv)
    FLAT = args.tree == "flat"
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_2606_05765_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2606_05765_gb300 import build as B
    B.build()
    peak_gbs, sm_mhz_max, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 4 * sm_mhz_max * 1e6          # warp instructions per second
    stream = torch.cuda.Stream(dev)                  # everything runs here (graphs need a capturable stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    # the headline workload, with clocks sampled during its timed region
    w = make_workload(args.workload)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = P.launch_count()
    with ClockSampler(local) as clk:
        r = measure(P, torch, w, dev, stream, flush, args.steps, args.warmup, not args.no_autotune)
    n_launch = r["launches_per_step"] * args.steps
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    head = summarize(r, world, dev, peak_gbs, issue_peak, args.workload)
    ok = r["ok"]

    # the other configurations, measured the same way (fewer steps)
    per_config = {}
    if not args.no_per_config:
        for name in [n for n in ("zipf1", "skew95", "mixed") if n != args.workload]:
            wc = make_workload(name)
            rc = measure(P, torch, wc, dev, stream, flush, max(3, args.steps // 4), 3, not args.no_autotune)
            s = summarize(rc, world, dev, peak_gbs, issue_peak, name)
            s["desc"] = WORKLOADS[name]
            s["blocks"] = rc["nblk"]
            s["raw_bytes"] = rc["raw"]
            s["compressed_bytes"] = rc["rec_bytes"]
            s["verified"] = rc["ok"]
            ok = ok and rc["ok"]
            per_config[name] = s
            del wc, rc
            torch.cuda.empty_cache()

    # the same workload coded with the other tree (canonical against the
    # regrouped one with flat subtrees, Sec. 2.2.3-2.2.4)
    other_tree = None
    if not args.no_per_config:
        FLAT = not FLAT
        ro = measure(P, torch, w, dev, stream, flush, max(3, args.steps // 4), 3, not args.no_autotune)
        so = summarize(ro, world, dev, peak_gbs, issue_peak, args.workload)
        FLAT = not FLAT
        other_tree = {"tree": TREE_DESC["canonical" if FLAT else "flat"], "value": so["value"],
                      "encode_gbs": so["encode_gbs"], "decode_gbs": so["decode_gbs"],
                      "compressed_bytes": ro["rec_bytes"], "verified": ro["ok"],
                      "encode_kernel_ms": so["roofline"]["kernels"]["encode_kernel"]["ms"],
                      "decode_batch_kernel_ms": so["roofline"]["kernels"]["decode_batch_kernel"]["ms"]}
        ok = ok and ro["ok"]
        del ro
        torch.cuda.empty_cache()

    # end to end through the public host-buffer API (pivco_host_compress /
    # pivco_host_decompress) with pinned host buffers: every step copies the
    # raw bytes in and the records out, then the records in and the bytes out
    e2e = None
    raw = r["raw"]
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        h_in = torch.from_numpy(w.data).pin_memory()
        h_out = torch.empty(raw, dtype=torch.uint8).pin_memory()
        with P.HostCodec(w.blk_off, P.params(ans=w.ans, flat=FLAT), segments=args.e2e_segments) as hc:
            h_comp = torch.empty(max(hc.capacity, 1), dtype=torch.uint8).pin_memory()
            e2e_t = []
            e2e_ok = True
            for i in range(args.e2e_steps + 1):
                t0 = time.perf_counter()
                comp_off, st_c = hc.compress(h_in, h_comp)
                comp_bytes = int(comp_off[-1])
                st_d = hc.decompress(h_comp, comp_off, h_out)
                if i:
                    e2e_t.append(time.perf_counter() - t0)
                e2e_ok = e2e_ok and not st_c.any() and not st_d.any()
        ok = ok and e2e_ok and bool(torch.equal(h_out, h_in))
        e2e = {"value": round(raw / statistics.mean(e2e_t) / 1e9 * world, 3), "unit": "GB/s",
               "h2d_bytes_per_step": raw + comp_bytes, "d2h_bytes_per_step": comp_bytes + raw,
               "api": "pivco_host_compress + pivco_host_decompress, %d pieces" % args.e2e_segments}

    serving = None
    if world == 1 and not args.no_serving:
        serving = serving_leg(P, seconds=args.serve_seconds, repeats=args.serve_repeats)
        ok = ok and serving["verified"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, ans=w.ans)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": head["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload], "blocks": r["nblk"],
                       "tree": TREE_DESC[args.tree],
                       "raw_bytes_per_gpu": raw, "compressed_bytes": r["rec_bytes"],
                       "ratio": round(raw / r["rec_bytes"], 4),
                       "l2": "L2 flushed (256 MiB write) before each leg; inputs 256 MiB > 129 MB L2",
                       "path": "batched: encode launch sequence and persistent work-queue decode, each one CUDA graph",
                       "tuning": head["tuning"], "parallelism": "blocks sharded per GPU"},
            "encode_gbs": head["encode_gbs"], "decode_gbs": head["decode_gbs"],
            "best_of_runs": head["best_of_runs"], "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "batched": head["batched"], "plain": head["plain"],
            "roofline": dict(head["roofline"], peak_source="%s (MEASURED_PEAKS.json hbm_gbs, sm_max_mhz; %d SMs)"
                             % (peak_kind, sms)),
            "per_config": per_config,
            "other_tree": other_tree,
            "serving": serving,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch, "clocks": clocks, "verified": ok,
            "checks": r["checks"],
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
