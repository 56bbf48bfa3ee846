"""PivCo-Huffman benchmark on GB300: encode + decode throughput of the hot path.

One step = one pass of the whole path over one batch of synthetic blocks:
histogram -> code lengths -> layout -> record placement (scan) -> encode
(-> selective ANS) and then decode (plan -> ANS decode -> bottom-up merge).
Each leg is timed with CUDA events on the launching stream; L2 is flushed
before each leg.  `value` is raw bytes / (encode time + decode time) summed
over all ranks' blocks (weak scaling: every rank codes its own batch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload skew80]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm

Prints one JSON line on rank 0.
"""
import argparse
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
    # name: (generator kwargs, description)
    "skew80": ({}, "4096 blocks x 64 KiB (256 MiB), byte 0 with P=0.8, 255 others uniform, no ANS, seed 1"),
    "skew95": ({}, "2048 blocks x 128 KiB (256 MiB), P(top)=0.95 + Zipf(1.3) tail, selective ANS, seed 2"),
    "mixed": ({}, "4096 blocks log-uniform 4 KiB-1 MiB, per-block alphabet/Zipf, selective ANS, seed 3"),
    "zipf1": ({}, "1 block of 2^20 symbols, Zipf(1.0) over 256, no ANS, seed 0"),
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pivco", choices=["pivco", "reference"])
    ap.add_argument("--workload", default="skew80", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-segments", type=int, default=4)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default decode tuning")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="offered-load time per arrival rate")
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


KERNEL_SOURCES = {"encode_kernel": "paper_2606_05765_gb300/csrc/k_encode.cu",
                  "decode_batch_kernel": "paper_2606_05765_gb300/csrc/k_decode.cu"}


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/traffic.json), only while the kernel's source file is
    byte-identical to the one profiled (else None)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[workload][kernel]
        src = open(os.path.join(ROOT, KERNEL_SOURCES[kernel]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    return rec["bytes"] if hashlib.sha256(src).hexdigest() == rec["source_sha256"] else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


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


def cpu_baseline(w, budget_s=10.0, ans=False):
    """The oracle as it stands, single-threaded on the host, on a bounded
    prefix of the same blocks; returns GB/s of raw bytes per (encode+decode)."""
    import oracle
    oracle.build()
    prm = oracle.params(ans=ans)
    nb = 1
    t_all, raw_all, used = 0.0, 0, 0
    while used < w.nblk and t_all < budget_s:
        take = min(nb, w.nblk - used)
        lo, hi = int(w.blk_off[used]), int(w.blk_off[used + take])
        sub_off = (w.blk_off[used:used + take + 1] - w.blk_off[used]).astype(np.uint64)
        x = w.data[lo:hi]
        t0 = time.perf_counter()
        buf, rec_off, sizes = oracle.encode_batch(x, sub_off, prm)
        st, out = oracle.decode_batch(buf, rec_off[:-1], sizes, sub_off)
        t_all += time.perf_counter() - t0
        assert not st.any() and np.array_equal(out, x)
        raw_all += hi - lo
        used += take
        nb *= 2
    return {"value": raw_all / t_all / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d of %d blocks (%.1f MB), encode+decode, %.1f s single-threaded"
                      % (used, w.nblk, raw_all / 1e6, t_all)}


def serving_leg(P, seconds=2.0, budget=8 << 30, pool_n=48, seed=4):
    """Poisson decompression requests through the server (device-resident
    loop, admission by an 8 GiB device budget).  A pool of distinct requests
    (sizes log-uniform 1 KiB-16 MiB, each drawn from the skew80 / skew95 /
    mixed distributions) is encoded once; arrivals pick pool entries.  The
    capacity is measured first (everything submitted at once), then arrivals
    are offered at 0.5, 0.8 and 0.95 of it.  Latency = result in host memory
    minus the scheduled arrival."""
    import ctypes as C
    import torch
    import workloads
    reqs = workloads.serving_requests(pool_n, 1.0, seed=seed)
    pool = []
    for r in reqs:
        data = torch.from_numpy(r.data).cuda()
        boff = torch.from_numpy(r.blk_off.astype(np.int64)).cuda()
        enc = P.encode(data, boff, P.params(ans=r.ans))
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
    mean_raw = np.mean([e["raw"] for e in pool])
    rates = []
    ok = cap["bad"] == 0
    for frac in (0.5, 0.8, 0.95):
        lam = frac * cap_gbs * 1e9 / mean_raw                  # requests per second
        n = int(min(10000, max(200, lam * seconds)))
        order = rng.integers(0, pool_n, n)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n))
        r = run(order, arrivals)
        ok = ok and r["bad"] == 0
        span = max(r["last_done_s"], arrivals[-1])
        rates.append({"load": frac, "requests": n, "offered_gbs": round(r["raw_bytes"] / arrivals[-1] / 1e9, 3),
                      "gbs": round(r["raw_bytes"] / span / 1e9, 3),
                      "p50_ms": round(float(np.percentile(r["lat_ms"], 50)), 4),
                      "p99_ms": round(float(np.percentile(r["lat_ms"], 99)), 4)})
    for e in pool:
        n = e["raw"]
        ok = ok and bool(np.array_equal(e["out"].numpy()[:n], e["data"]))
    return {"budget_bytes": budget, "pool_requests": pool_n, "capacity_gbs": round(cap_gbs, 3),
            "capacity_requests": len(burst), "rates": rates, "verified": ok,
            "latency": "result in pinned host memory minus scheduled arrival",
            "sizes": "log-uniform 1 KiB-16 MiB; skew80 64 KiB / skew95 128 KiB / mixed 1 MiB blocks"}


def make_workload(name, rank=0):
    import workloads
    return workloads.by_name(name)


def run_reference(args):
    """Reference arm: the oracle (the paper's method restated plainly in C)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make_workload(args.workload)
    import oracle
    oracle.build()
    prm = oracle.params(ans=w.ans)
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
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload][1], "sample_blocks": take,
                       "sample_bytes": hi - lo},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first %d blocks (%d bytes) per step" % (take, hi - lo)},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main(argv=None):
    args = parse_args(argv)
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

    w = make_workload(args.workload)
    raw = int(w.data.size)
    nblk = w.nblk
    data = torch.from_numpy(w.data).to(dev)
    blk_off = torch.from_numpy(w.blk_off.astype(np.int64)).to(dev)
    stream = torch.cuda.Stream(dev)          # everything runs here (graphs need a capturable stream)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        enc = P.Encoder(nblk, P.params(ans=w.ans), dev)
        enc.ensure(enc.plan(data, blk_off, stream))
        res = enc.run(data, blk_off, stream, replan=False)
        dec = P.Decoder(nblk, dev)
        P.set_tuning(16384, 64, 0)         # the largest workspace any autotuner candidate needs
        dec.prepare(res.comp, res.off, stream)
        P.set_tuning()
        out = torch.empty(raw, dtype=torch.uint8, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
        # pick the decode launch tuning for this batch (does not change the bytes)
        if args.no_autotune:
            tuned = P.get_tuning()
        else:
            tuned, _ = P.autotune_decode(res.comp, res.off, nblk, out, blk_off, dec.ws, dec.status, reps=2,
                                         stream=stream)
        dec.prepare(res.comp, res.off, stream)
        # batched path: the encode launch sequence and the persistent decode, each a CUDA graph
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

    E = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

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

    def timed(step_fn, steps, clk=None):
        t_enc, t_dec, t_mid = [], [], []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                step_fn()
                E[4].synchronize()
                t_enc.append(E[0].elapsed_time(E[1]))
                t_dec.append(E[2].elapsed_time(E[4]))
                t_mid.append(E[3].elapsed_time(E[4]) if step_fn is plain_step else t_dec[-1])
        return t_enc, t_dec, t_mid

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plain_step()
            batched_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # headline: the batched path, with clocks sampled during the timed region
    n_launch0 = P.launch_count()
    with ClockSampler(local) as clk:
        b_enc, b_dec, _ = timed(batched_step, args.steps)
    n_launch = P.launch_count() - n_launch0 + args.steps * (n_enc_graph + n_dec_graph)
    torch.cuda.synchronize()
    ok_b = (not enc.status.cpu().numpy().any()) and (not dec.status.cpu().numpy().any()) and bool(torch.equal(out, data))
    # the plain path (one launch per step of the pipeline) on the same batch
    out.zero_()
    p_steps = max(3, args.steps // 2)
    p_enc, p_dec, p_merge = timed(plain_step, p_steps)
    torch.cuda.synchronize()
    ok_p = (not enc.status.cpu().numpy().any()) and (not dec.status.cpu().numpy().any()) and bool(torch.equal(out, data))
    # the encode kernel alone, for its roofline (statistics already on the device)
    Ek = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    t_enck = []
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.steps // 4)):
            flush.zero_()
            Ek[0].record(stream)
            P.encode_blocks_chunked(data, blk_off, nblk, enc.layout, enc.chunk_hist, enc.comp, enc.off, enc.rec_bytes,
                                    enc.status, stream)
            Ek[1].record(stream)
            Ek[1].synchronize()
            t_enck.append(Ek[0].elapsed_time(Ek[1]))
        enc.run(data, blk_off, stream)          # the final records (with ANS) again
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ok = ok_b and ok_p and not enc.status.cpu().numpy().any()
    rec_bytes = int(enc.rec_bytes.sum().item())

    def agg(te, td):
        tot = reduce_max(sum(a + b for a, b in zip(te, td)), dev)
        return whole_job_gbs(raw, len(te), tot, world), tot / len(te)

    value, ms_step = agg(b_enc, b_dec)
    plain_value, plain_ms = agg(p_enc, p_dec)
    step_ms = [a + b for a, b in zip(b_enc, b_dec)]

    # roofline of the dominant kernel of the headline (batched) step
    peak, peak_kind = measured_peaks()
    kernels = {
        "decode_batch_kernel": {"ms": statistics.mean(b_dec), "bytes": rec_bytes + raw},
        "encode_kernel": {"ms": statistics.mean(t_enck), "bytes": raw + rec_bytes},
        "decode_merge (plain)": {"ms": statistics.mean(p_merge), "bytes": rec_bytes + raw},
    }
    for k in kernels:
        kernels[k]["gbs"] = kernels[k]["bytes"] / (kernels[k]["ms"] / 1e3) / 1e9
        kernels[k]["frac"] = kernels[k]["gbs"] / peak
    dom = max(["decode_batch_kernel", "encode_kernel"], key=lambda k: kernels[k]["ms"])
    ach = kernels[dom]["gbs"]

    # end to end through the public host-buffer API (pivco_host_compress /
    # pivco_host_decompress) with pinned host buffers: every step copies the
    # raw bytes in and the records out, then the records in and the bytes out
    e2e = None
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        h_in = torch.from_numpy(w.data).pin_memory()
        h_out = torch.empty(raw, dtype=torch.uint8).pin_memory()
        with P.HostCodec(w.blk_off, P.params(ans=w.ans), segments=args.e2e_segments) as hc:
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
        serving = serving_leg(P, seconds=args.serve_seconds)
        ok = ok and serving["verified"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, ans=w.ans)

    if rank == 0:
        clocks = clk.summary()
        r4 = lambda x: round(x, 4)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r4(ms_step), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload][1], "blocks": nblk,
                       "raw_bytes_per_gpu": raw, "compressed_bytes": rec_bytes, "ratio": r4(raw / rec_bytes),
                       "l2": "L2 flushed (256 MiB write) before each leg; inputs 256 MiB > 129 MB L2",
                       "path": "batched: encode launch sequence and persistent work-queue decode, each one CUDA graph",
                       "tuning": tuned.as_dict(), "parallelism": "blocks sharded per GPU"},
            "encode_gbs": round(raw / (statistics.mean(b_enc) / 1e3) / 1e9, 3),
            "decode_gbs": round(raw / (statistics.mean(b_dec) / 1e3) / 1e9, 3),
            "p50_ms": r4(float(np.percentile(step_ms, 50))), "p99_ms": r4(float(np.percentile(step_ms, 99))),
            "batched": {"value": round(value, 3), "decode_gbs": round(raw / (statistics.mean(b_dec) / 1e3) / 1e9, 3)},
            "plain": {"value": round(plain_value, 3), "ms_per_step": r4(plain_ms),
                      "encode_gbs": round(raw / (statistics.mean(p_enc) / 1e3) / 1e9, 3),
                      "decode_gbs": round(raw / (statistics.mean(p_dec) / 1e3) / 1e9, 3)},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(ach, 2), "peak": peak,
                         "unit": "GB/s", "frac": r4(ach / peak), "traffic": kernel_traffic(dom, args.workload),
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                         "kernels": {k: {kk: r4(vv) for kk, vv in v.items()} for k, v in kernels.items()}},
            "serving": serving,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch, "clocks": clocks, "verified": ok,
            "checks": {"batched": ok_b, "plain": ok_p},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
