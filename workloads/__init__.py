"""Seeded synthetic workloads for PivCo-Huffman (no codec arithmetic here).

These generators stand in for the paper's datasets (App. A: proba80, text and
DNA corpora), which are not available: i.i.d. skewed and Zipf byte streams with
the shapes of the five benchmark configurations.  Both the CUDA path's tests
and the oracle's tests draw their inputs from here, and nothing else is shared.

Recipe (numpy ``PCG64(seed)``; inverse-CDF sampling with ``searchsorted`` on a
float64 CDF; the rank-k symbol is byte k-1 unless ``permute`` is given):

  zipf1      1 block of 2^20 symbols, P(k) ~ 1/k over 256 symbols, seed 0
  skew80     4096 blocks x 64 KiB, byte 0 with P = 0.8, the other 255 uniform, seed 1
  skew95     2048 blocks x 128 KiB, byte 0 with P = 0.95, bytes 1..255 ~ k^-1.3
             carrying the remaining 0.05, seed 2
  mixed      4096 blocks, size floor(exp(U(ln 4096, ln 2^20))); per block an
             alphabet A ~ U{2..256} and exponent s ~ U(0.5, 2.0), P(k) ~ k^-s, seed 3
  serving    Poisson request stream, sizes floor(exp(U(ln 1 KiB, ln 16 MiB))),
             each request drawn from skew80 / skew95 / mixed, seed 4
  golomb     PivCo-Golomb values: 4096 blocks x 32 KiB, i.i.d. geometric with
             mean unary code length 1.25 .. 5 (App. G, Table 18), seed 5
"""
import hashlib
from dataclasses import dataclass, field

import numpy as np

KiB, MiB = 1024, 1024 * 1024
_CHUNK = 1 << 24


@dataclass
class Workload:
    name: str
    data: np.ndarray          # uint8, all blocks back to back
    blk_off: np.ndarray       # uint64[nblk + 1]
    ans: bool                 # whether the configuration enables selective ANS
    desc: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nblk(self):
        return self.blk_off.size - 1

    def sha256(self):
        return hashlib.sha256(self.data.tobytes()).hexdigest()


def _sample(rng, probs, n, out=None):
    """n i.i.d. draws of ranks 0..len(probs)-1 by inverse CDF (uint8)."""
    p = np.asarray(probs, np.float64)
    cdf = np.cumsum(p / p.sum())
    out = np.empty(n, np.uint8) if out is None else out
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        u = rng.random(hi - lo)
        idx = np.searchsorted(cdf, u, side="right")
        np.minimum(idx, p.size - 1, out=idx)
        out[lo:hi] = idx.astype(np.uint8)
    return out


def _uniform_blocks(nblk, bs):
    return (np.arange(nblk + 1, dtype=np.uint64) * np.uint64(bs)).astype(np.uint64)


def _permute(rng_seed, data):
    perm = np.random.Generator(np.random.PCG64(rng_seed + 1000)).permutation(256).astype(np.uint8)
    return perm[data]


def zipf1(n=1 << 20, seed=0, permute=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.arange(1, 257, dtype=np.float64)
    data = _sample(rng, 1.0 / k, n)
    if permute:
        data = _permute(seed, data)
    return Workload("zipf1", data, _uniform_blocks(1, n), False,
                    "1 block of %d symbols, P(k)~1/k over 256, seed %d" % (n, seed))


def skew80(nblk=4096, bs=64 * KiB, seed=1, permute=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.full(256, 0.2 / 255)
    p[0] = 0.8
    data = _sample(rng, p, nblk * bs)
    if permute:
        data = _permute(seed, data)
    return Workload("skew80", data, _uniform_blocks(nblk, bs), False,
                    "%d x %d B blocks, P(byte0)=0.8, 255 others uniform, seed %d" % (nblk, bs, seed))


def _skew95_probs():
    k = np.arange(1, 256, dtype=np.float64)
    tail = k ** -1.3
    p = np.empty(256)
    p[0] = 0.95
    p[1:] = 0.05 * tail / tail.sum()
    return p


def skew95(nblk=2048, bs=128 * KiB, seed=2, permute=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    data = _sample(rng, _skew95_probs(), nblk * bs)
    if permute:
        data = _permute(seed, data)
    return Workload("skew95", data, _uniform_blocks(nblk, bs), True,
                    "%d x %d B blocks, P(byte0)=0.95 + k^-1.3 tail, selective ANS, seed %d" % (nblk, bs, seed))


def mixed_sizes(nblk, rng, lo=4 * KiB, hi=MiB):
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), nblk))).astype(np.uint64)


def mixed(nblk=4096, seed=3, lo=4 * KiB, hi=MiB, permute=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = mixed_sizes(nblk, rng, lo, hi)
    alpha = rng.integers(2, 257, nblk)
    expo = rng.uniform(0.5, 2.0, nblk)
    blk_off = np.zeros(nblk + 1, np.uint64)
    blk_off[1:] = np.cumsum(sizes)
    data = np.empty(int(blk_off[-1]), np.uint8)
    for b in range(nblk):
        k = np.arange(1, int(alpha[b]) + 1, dtype=np.float64)
        _sample(rng, k ** -expo[b], int(sizes[b]), out=data[int(blk_off[b]):int(blk_off[b + 1])])
    if permute:
        data = _permute(seed, data)
    return Workload("mixed", data, blk_off, True,
                    "%d blocks, log-uniform %d..%d B, alphabet U{2..256}, Zipf s~U(0.5,2), seed %d"
                    % (nblk, lo, hi, seed), {"alpha": alpha, "expo": expo})


@dataclass
class Request:
    arrival_s: float
    kind: str                 # "skew80" | "skew95" | "mixed"
    data: np.ndarray
    blk_off: np.ndarray
    ans: bool


def serving_requests(n_req, rate_per_s, seed=4, lo=KiB, hi=16 * MiB):
    """Poisson arrivals at ``rate_per_s``; each request picks a distribution."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, n_req)
    arr = np.cumsum(gaps)
    sizes = mixed_sizes(n_req, rng, lo, hi)
    kinds = rng.integers(0, 3, n_req)
    reqs = []
    p80 = np.full(256, 0.2 / 255)
    p80[0] = 0.8
    for i in range(n_req):
        n = int(sizes[i])
        if kinds[i] == 0:
            kind, bs, p, ans = "skew80", 64 * KiB, p80, False
        elif kinds[i] == 1:
            kind, bs, p, ans = "skew95", 128 * KiB, _skew95_probs(), True
        else:
            a = int(rng.integers(2, 257))
            s = float(rng.uniform(0.5, 2.0))
            kind, bs, p, ans = "mixed", MiB, np.arange(1, a + 1, dtype=np.float64) ** -s, True
        data = _sample(rng, p, n)
        nb = (n + bs - 1) // bs
        off = np.minimum(np.arange(nb + 1, dtype=np.uint64) * np.uint64(bs), np.uint64(n)).astype(np.uint64)
        reqs.append(Request(float(arr[i]), kind, data, off, ans))
    return reqs


def golomb(nblk=4096, bs=32 * KiB, avg_len=2.0, seed=5):
    """PivCo-Golomb values (App. G, Table 18's sweep of average code lengths):
    i.i.d. geometric values v >= 0 with P(v) = p (1 - p)^v, p = 1 / avg_len,
    so the unary code length v + 1 has mean avg_len; capped at 255."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nblk * bs
    data = np.minimum(rng.geometric(1.0 / avg_len, n) - 1, 255).astype(np.uint8)
    return Workload("golomb", data, _uniform_blocks(nblk, bs), False,
                    "%d blocks x %d values, geometric with mean code length %.2f, seed %d" % (nblk, bs, avg_len, seed),
                    {"avg_len": avg_len})


def by_name(name, **kw):
    return {"zipf1": zipf1, "skew80": skew80, "skew95": skew95, "mixed": mixed, "golomb": golomb}[name](**kw)
