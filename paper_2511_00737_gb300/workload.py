"""Seeded synthetic inputs for EP-HDC client-side inference.

This module only draws data; it contains none of the method's arithmetic, so both
the CUDA path and the CPU oracle may take their inputs from it.  The shapes follow
the paper's workloads (Sec. 6): HOG-sized feature vectors (F = 608 / 768 / 1024),
hypervector dimension D up to 16K, 2 to 16 classes.  The paper's datasets (Face,
Emotion, MNIST) are not available; uniformly drawn features stand in for them.

* features  X[B][F] int8 = floor(128 u), u ~ U[0, 1)        (values 0..127)
* projection Wt[D][F] int8 in {-1, +1}, equiprobable           (Sec. 2.1 random base)
* classes   C[k][D] int8 uniform in {-8, ..., 7}               (4-bit class HVs)
* client batch sizes  B_c = min(4096, floor(exp(u ln 4097)))   (log-uniform 1..4096)
* serving requests    Poisson arrivals, lognormal batch sizes (median 32, sigma 1,
  clipped to [1, 8192])
"""
import math
from dataclasses import dataclass, field

import numpy as np

# numpy's PCG64 streams, one per kind of input, so each array is independent of
# the shapes of the others
_STREAM = {"X": 16, "W": 17, "C": 18, "clients": 19, "arrivals": 20}


def _rng(seed, kind, extra=0):
    return np.random.Generator(np.random.PCG64([int(seed), _STREAM[kind], int(extra)]))


def features(seed, B, F, batch=0):
    u = _rng(seed, "X", batch).random((B, F))
    return np.floor(128.0 * u).astype(np.int8)


def projection(seed, D, F):
    bits = _rng(seed, "W").integers(0, 2, size=(D, F), dtype=np.int8)
    return (2 * bits - 1).astype(np.int8)


def classes(seed, k, D, lo=-8, hi=7):
    return _rng(seed, "C").integers(lo, hi + 1, size=(k, D), dtype=np.int8)


def client_batches(seed, clients=64, max_batch=4096):
    u = _rng(seed, "clients").random(clients)
    b = np.floor(np.exp(u * math.log(max_batch + 1))).astype(np.int64)
    return np.clip(b, 1, max_batch)


def arrivals(seed, count, rate_per_s=2000.0, median=32, sigma=1.0, max_batch=8192):
    """(arrival times in seconds, batch sizes) of a Poisson request stream."""
    g = _rng(seed, "arrivals")
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    sizes = np.floor(g.lognormal(math.log(median), sigma, size=count)).astype(np.int64)
    return np.cumsum(gaps), np.clip(sizes, 1, max_batch)


def default_shift(F, bits):
    """Quantiser shift s = max(0, round(log2 sigma_A) - (b - 2)), where sigma_A is the
    standard deviation of a projected feature sum for features uniform on 0..127."""
    ex2 = 127.0 * 255.0 / 6.0
    sigma_a = math.sqrt(F * ex2)
    return max(0, int(round(math.log2(sigma_a))) - (bits - 2))


@dataclass
class Workload:
    """One named configuration: BFV parameters, slot layout and input shapes."""
    name: str
    n: int
    L: int
    k: int
    k_in: int
    r: int
    D: int
    F: int
    bits: int
    B: int
    seed: int = 2511
    shift: int = -1
    clients: list = field(default_factory=list)

    def __post_init__(self):
        if self.shift < 0:
            self.shift = default_shift(self.F, self.bits)


def config(name, **over):
    """Named workloads with the shapes of the paper's experiments, with optional overrides."""
    base = {
        # 16 queries, F=608, D=2048, 4-bit HVs, 2 classes, n=4096, 3 primes; packed
        # layout A with r=128 (7 rotations).  Small enough for the oracle in seconds.
        "small": dict(n=4096, L=3, k=2, k_in=2, r=128, D=2048, F=608, bits=4, B=16),
        # 1024 queries, F=608, D=10000, 8-bit HVs, 2 classes, n=8192, 4 primes
        "face1024": dict(n=8192, L=4, k=2, k_in=1, r=8, D=10000, F=608, bits=8, B=1024),
        # the same batch in the paper's packed layout A: both classes in one ciphertext
        # (k_in = k = 2), r = 4 (P = 2500 plaintexts, 2 rotations)
        "face1024_a": dict(n=8192, L=4, k=2, k_in=2, r=4, D=10000, F=608, bits=8, B=1024),
        # the same batch in the per-query form: one query at a time, D folded over
        # n/(2 k_in) chunks (HE-HDC's dense shape, log2 r rotations per query)
        "face1024_perquery": dict(n=8192, L=4, k=2, k_in=2, r=2048, D=10000, F=608, bits=8,
                                  B=1),
        # 64 clients with log-uniform batch sizes, F=768, D=10000, 4-bit HVs, 7 classes
        "clients64": dict(n=8192, L=4, k=7, k_in=1, r=8, D=10000, F=768, bits=4, B=0),
        # 65536 queries, F=1024, D=16384, 8-bit HVs, 16 classes, n=16384, 6 primes
        "dense65536": dict(n=16384, L=6, k=16, k_in=1, r=16, D=16384, F=1024, bits=8, B=65536),
        # the same batch with r = 8: 32 groups of 2048 queries, P = 2048 (a 25.8 GB
        # model), 3 rotations on half as many ciphertexts
        "dense65536_r8": dict(n=16384, L=6, k=16, k_in=1, r=8, D=16384, F=1024, bits=8,
                              B=65536),
        # serving: F=608, D=10000, 7 classes, n=8192, 4 primes
        "serve": dict(n=8192, L=4, k=7, k_in=1, r=8, D=10000, F=608, bits=8, B=0),
    }[name]
    base.update(over)
    w = Workload(name=name, **base)
    if name == "clients64" and not w.clients:
        w.clients = [int(b) for b in client_batches(w.seed)]
        w.B = int(sum(w.clients))
    return w
