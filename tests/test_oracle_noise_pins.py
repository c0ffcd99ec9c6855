"""Pins of the oracle's findDmax (Sec. 5.2, Alg. 1): the noise-growth experiment on
small parameters (n = 1024, two 20- or 21-bit primes) where decryption fails after
tens to hundreds of products.  D_i is checked against its definition with an independent
decryption (Python big-integer CRT), and the mean D_max against the growth law the
mathematics fixes: the accumulated noise grows like t sqrt(D) while the budget
q/(2t) shrinks like 1/t, so D_max scales as q^2 / t^4."""
import math

import numpy as np
import pytest

import oracle as O


def trial(t, k, D=200, n=1024, bits=20):
    o = O.Oracle(n, 2, 1, 1, 1, D, t=t, prime_bits=bits)
    rng = np.random.default_rng(1000 + k)
    H = rng.integers(-128, 128, (o.cap, D)).astype(np.int8)
    cls = rng.integers(-8, 8, (1, D)).astype(np.int8)
    s, _ = o.keygen(500 + k)
    model = o.encrypt_model(500 + k, cls, s)
    m = o.encode_plain(H)
    return o, H, cls, s, model, m


def bigint_decrypt_scores(o, s, acc, B):
    """Decryption written out with Python integers: CRT of c0 + c1 s, then
    round(t x / q) mod t, then the slot values of the one class."""
    Q = math.prod(o.q)
    xs = []
    for l, p in enumerate(o.q):
        sl = np.asarray(s, np.int64) % p
        xs.append((acc[0, l].astype(np.int64) + O.polymul(acc[1, l], sl, p, o.psi[l])) % p)
    coeff = np.zeros(o.n, np.int64)
    for kk in range(o.n):
        x = sum(int(xs[l][kk]) * pow(Q // p, -1, p) * (Q // p) for l, p in enumerate(o.q)) % Q
        coeff[kk] = ((o.t * x + Q // 2) // Q) % o.t
    slots = O.slot_decode(coeff.astype(np.uint32), o.zeta, o.t)
    half = o.n // 2
    # slot (rho, qq) holds query rho * cap_row + qq (k_in = 1, r = 1)
    return np.concatenate([slots[:half], slots[half:]])[:B]


def test_dmax_is_the_first_failure():
    o, H, cls, s, model, m = trial(40961, 0)
    Di = o.find_dmax_trial(m, model, s, H, cls)
    assert 0 < Di < o.D
    for Dp, ok in [(Di, True), (Di + 1, False)]:
        sub = O.Oracle(o.n, o.L, 1, 1, 1, Dp, t=o.t, prime_bits=20)
        acc = sub.ptct_mac(np.ascontiguousarray(m[:, :Dp]), o.cap, np.ascontiguousarray(model[:Dp]))
        got = bigint_decrypt_scores(o, s, acc[0, 0], o.cap)
        clear = O.clear_scores(H[:, :Dp], cls[:, :Dp], o.t)[:, 0]
        assert np.array_equal(got, clear) == ok


def mean_dmax(t, bits, trials=4, D=1000):
    vals = []
    for k in range(trials):
        o, H, cls, s, model, m = trial(t, k, D=D, bits=bits)
        vals.append(o.find_dmax_trial(m, model, s, H, cls))
        assert vals[-1] < o.D
    return float(np.mean(vals))


def test_dmax_scales_as_t_to_the_minus_four():
    t1, t2 = 18433, 40961
    ratio = mean_dmax(t1, 20) / mean_dmax(t2, 20)
    want = (t2 / t1) ** 4  # 24.4
    assert want / 2 < ratio < want * 2, ratio


def test_dmax_scales_as_q_squared():
    """One more bit per prime (q about 4 times larger) allows about 16 times more
    products."""
    o20, o21 = O.Oracle(1024, 2, 1, 1, 1, 1, prime_bits=20), O.Oracle(1024, 2, 1, 1, 1, 1,
                                                                      prime_bits=21)
    want = (math.prod(o21.q) / math.prod(o20.q)) ** 2
    ratio = mean_dmax(40961, 21) / mean_dmax(40961, 20)
    assert want / 2 < ratio < want * 2, ratio
