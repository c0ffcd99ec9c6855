"""The noise-growth experiment of Sec. 5.2 (Alg. 1, findDmax) on the GPU.

For a ring degree n and a plaintext modulus t of log2 t bits, findDmax repeats a
trial many times (1000 in the paper) and averages D_i, the number of products
the client-side dot product can accumulate before decryption goes wrong.  A trial
here is the method's own computation at the paper's layout (one class, k_in = k =
1, r = 1): fresh keys, an encrypted class hypervector of D_lim dimensions, one group
of n query hypervectors, and `ephdc_find_dmax_trial`, which decrypts the
accumulator after every prefix on the device.  The RNS modulus q is the largest the
128-bit table of Sec. 6 allows at n (27-bit primes: 2 at n = 2048, 4 at 4096, 8 at
8192), or a fixed size for a second series.

Inputs are synthetic and seeded: query values uniform on [-128, 127] (8-bit
hypervectors) and class values uniform on [-8, 7] (4-bit class hypervectors), drawn
on the device from PyTorch's generator; the keys and encryption randomness come
from the library's ChaCha20 streams keyed by the trial's seed.

    python -m paper_2511_00737_gb300.noise --n 2048 --log-t 18 25 --trials 1000
"""
import argparse
import json
import math
import time

import torch

from . import ephdc as E

# log2 q at the 128-bit security level (Sec. 6, the parameter table)
LOGQ_128 = {1024: 27, 2048: 54, 4096: 109, 8192: 218, 16384: 438}


def is_prime(v):
    """Deterministic Miller-Rabin for v < 2^32 (bases 2, 7, 61)."""
    if v < 2:
        return False
    for b in (2, 7, 61):
        if v % b == 0:
            return v == b
    d, s = v - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for b in (2, 7, 61):
        x = pow(b, d, v)
        if x in (1, v - 1):
            continue
        for _ in range(s - 1):
            x = x * x % v
            if x == v - 1:
                break
        else:
            return False
    return True


def plaintext_modulus(n, log_t):
    """The smallest prime t >= 2^log_t with t = 1 (mod 2n) (slot packing needs it)."""
    c = ((1 << log_t) + 2 * n - 1) // (2 * n) * (2 * n) + 1
    while not is_prime(c):
        c += 2 * n
    return c


def rns_at_bound(n, prime_bits=27):
    """(L, prime_bits) with L primes of prime_bits bits inside the 128-bit bound.
    The plaintext modulus must stay below the primes (log2 t < prime_bits)."""
    return max(2, min(8, LOGQ_128[n] // prime_bits)), prime_bits


class Trials:
    """One (n, t, q, D_lim) configuration; runs seeded trials on the current device."""

    def __init__(self, n, t, L, prime_bits, d_lim, device=None):
        self.n, self.t, self.L, self.prime_bits, self.d_lim = n, t, L, prime_bits, d_lim
        self.dev = torch.device(device or "cuda")
        self.ctx = E.Context(n, L, 1, 1, 1, d_lim, 16, 8, 0, n, t=t, prime_bits=prime_bits,
                             device=self.dev)
        self.logq = sum(math.log2(p) for p in self.ctx.q)

    def inputs(self, seed):
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        H = torch.randint(-128, 128, (self.n, self.d_lim), generator=g, device=self.dev,
                          dtype=torch.int8)
        cls = torch.randint(-8, 8, (1, self.d_lim), generator=g, device=self.dev,
                            dtype=torch.int8)
        return H, cls

    def trial(self, seed, H=None, cls=None):
        if H is None:
            H, cls = self.inputs(seed)
        c = self.ctx
        sk, _ = c.keygen(seed)
        model = c.encrypt_model(cls, sk, seed)
        pt = c.encode_plain(H)
        return E.ephdc_find_dmax_trial(c.ctx, sk, H, cls, pt, model)

    def close(self):
        self.ctx.close()


def find_dmax(n, log_t, trials, L=None, prime_bits=27, d_lim=None, seed=1, d_cap=1 << 16):
    """Alg. 1's findDmax: mean and spread of D_i over `trials` trials.  Without an
    explicit d_lim the prefix limit doubles from 64 until two probe trials end below
    it (up to d_cap); trials that reach the limit are counted as censored."""
    if L is None:
        L, prime_bits = rns_at_bound(n, prime_bits)
    t = plaintext_modulus(n, log_t)
    if t >= (1 << (prime_bits - 1)):
        raise ValueError("t = %d is not below the %d-bit primes" % (t, prime_bits))
    t0 = time.time()
    if d_lim is None:
        d_lim = 64
        while True:
            tr = Trials(n, t, L, prime_bits, d_lim)
            probe = [tr.trial(seed + 10 ** 6 + k) for k in range(2)]
            tr.close()
            if max(probe) < d_lim or d_lim >= d_cap:
                break
            d_lim *= 2
        d_lim = min(d_cap, max(64, 2 * max(probe) + 16))
    tr = Trials(n, t, L, prime_bits, d_lim)
    vals = [tr.trial(seed + k) for k in range(trials)]
    logq = tr.logq
    tr.close()
    mean = sum(vals) / len(vals)
    std = math.sqrt(sum((v - mean) ** 2 for v in vals) / max(1, len(vals) - 1))
    return {"n": n, "log2_t": round(math.log2(t), 3), "t": t, "L": L, "prime_bits": prime_bits,
            "log2_q": round(logq, 2), "trials": trials, "d_lim": d_lim,
            "dmax_mean": mean, "dmax_std": std, "dmax_min": min(vals), "dmax_max": max(vals),
            "censored": sum(v >= d_lim for v in vals), "seconds": round(time.time() - t0, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[2048])
    ap.add_argument("--log-t", type=int, nargs=2, default=[18, 25])
    ap.add_argument("--trials", type=int, default=1000)
    ap.add_argument("--L", type=int, default=None, help="fixed number of primes (else the bound)")
    ap.add_argument("--prime-bits", type=int, default=27)
    ap.add_argument("--d-cap", type=int, default=1 << 16)
    a = ap.parse_args()
    for n in a.n:
        for T in range(a.log_t[0], a.log_t[1] + 1):
            r = find_dmax(n, T, a.trials, L=a.L, prime_bits=a.prime_bits, d_cap=a.d_cap)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
