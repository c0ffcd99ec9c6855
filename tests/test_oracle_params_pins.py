"""Pins of the oracle's parameter generality and of the scaling operation:
plaintext moduli other than 65537, smaller RNS primes (the prime size the 128-bit
table of Sec. 6 allows at small N), and the scaling operation of Sec. 5.1 against
its closed form."""
import numpy as np
import pytest
import sympy

import oracle as O


@pytest.mark.parametrize("n,L,bits", [(2048, 2, 27), (4096, 4, 27), (8192, 8, 27), (1024, 3, 20)])
def test_primes_below_any_bit_size(n, L, bits):
    q = [int(v) for v in O.find_primes(n, L, bits)]
    want, c = [], (1 << bits) - 2 * n + 1
    while len(want) < L:
        if sympy.isprime(c):
            want.append(c)
        c -= 2 * n
    assert q == want


@pytest.mark.parametrize("t", [40961, 786433, 536903681])
def test_scores_for_other_plaintext_moduli(t):
    """End to end at n = 32 (t = 1 mod 64): decrypted scores = clear dot products mod t,
    and decrypt(encrypt(v)) = v for slot values spanning [0, t)."""
    assert sympy.isprime(t) and t % 64 == 1
    o = O.Oracle(32, 3, 3, 1, 2, 9, t=t)
    assert o.t == t and o.zeta ** 0 == 1
    rng = np.random.default_rng(t % 1000)
    H = rng.integers(-128, 128, (20, 9)).astype(np.int8)
    cls = rng.integers(-8, 8, (3, 9)).astype(np.int8)
    s, gk = o.keygen(4)
    out = o.rotate_sum(gk, o.ptct_mac(o.encode_plain(H), 20, o.encrypt_model(4, cls, s)))
    assert np.array_equal(o.decrypt_scores(s, out, 20), O.clear_scores(H, cls, t))
    v = rng.integers(0, t, 32)
    assert np.array_equal(o.decrypt_slots(s, o.encrypt_slots(4, 1, s, v)), v)
    # the slot encoder mod t is still the O(n^2) definition
    assert np.array_equal(O.slot_encode(v, o.zeta, t), O.slot_encode_definition(v, o.zeta, t))


def test_small_primes_end_to_end():
    """Three 20-bit primes (q ~ 2^60): a short dot product still decrypts exactly."""
    o = O.Oracle(64, 3, 2, 2, 1, 5, prime_bits=20)
    assert all(p < (1 << 20) for p in o.q)
    rng = np.random.default_rng(5)
    H = rng.integers(-8, 8, (30, 5)).astype(np.int8)
    cls = rng.integers(-8, 8, (2, 5)).astype(np.int8)
    s, gk = o.keygen(8)
    out = o.rotate_sum(gk, o.ptct_mac(o.encode_plain(H), 30, o.encrypt_model(8, cls, s)))
    assert np.array_equal(o.decrypt_scores(s, out, 30), O.clear_scores(H, cls))
    assert o.noise_budget(s, out[0, 0]) > 0


def scaled_scores(H, cls, r, P, s_, g, t):
    """Closed form of the scaling operation: the accumulator is multiplied by
    u = (2^s)^-1 mod t after products i = g-1, 2g-1, ... (i < P), so the product of
    plaintext i is scaled floor(P/g) - floor(i/g) times; rotate-and-sum then adds the
    r chunks."""
    u = pow(pow(2, s_, t), -1, t)
    B, D = H.shape
    out = np.zeros((B, cls.shape[0]), np.int64)
    for d in range(D):
        i = d // r
        w = pow(u, P // g - i // g, t)
        out = (out + np.outer(H[:, d].astype(np.int64), cls[:, d].astype(np.int64)) % t * w) % t
    return out.astype(np.uint32)


@pytest.mark.parametrize("n,L,k,k_in,r,D,B,s_,g", [
    (32, 3, 2, 2, 1, 7, 9, 3, 2),      # paper form, P = 7: scalings after i = 1, 3, 5
    (32, 3, 3, 1, 2, 11, 20, 5, 3),    # P = 6, g = 3: after i = 2, 5 (the last product)
    (64, 4, 2, 1, 4, 33, 40, 1, 4),    # P = 9, g = 4: after i = 3, 7
])
def test_scaling_operation_matches_closed_form(n, L, k, k_in, r, D, B, s_, g):
    o = O.Oracle(n, L, k, k_in, r, D, scale_shift=s_, scale_group=g)
    assert (o.scale_u * (1 << s_)) % o.t == 1
    rng = np.random.default_rng(n + g)
    H = rng.integers(-128, 128, (B, D)).astype(np.int8)
    cls = rng.integers(-8, 8, (k, D)).astype(np.int8)
    s, gk = o.keygen(6)
    out = o.rotate_sum(gk, o.ptct_mac(o.encode_plain(H), B, o.encrypt_model(6, cls, s)))
    got = o.decrypt_scores(s, out, B)
    assert np.array_equal(got, scaled_scores(H, cls, r, o.P, s_, g, o.t))
    # without the operation the same inputs give the plain dot products
    o0 = O.Oracle(n, L, k, k_in, r, D)
    out0 = o0.rotate_sum(gk, o0.ptct_mac(o0.encode_plain(H), B, o0.encrypt_model(6, cls, s)))
    assert np.array_equal(o0.decrypt_scores(s, out0, B), O.clear_scores(H, cls))


def test_scaling_divides_exactly_when_partial_sums_are_multiples():
    """The case the operation is meant for (Sec. 5.1): with class values that are
    multiples of 2^(2s), both scaled partial sums are exact divisions by 2^s."""
    s_, g = 2, 2
    o = O.Oracle(32, 3, 1, 1, 1, 4, scale_shift=s_, scale_group=g)
    rng = np.random.default_rng(1)
    H = rng.integers(-8, 8, (16, 4)).astype(np.int8)
    cls = (rng.integers(-2, 2, (1, 4)) * 16).astype(np.int8)
    s, gk = o.keygen(2)
    out = o.ptct_mac(o.encode_plain(H), 16, o.encrypt_model(2, cls, s))
    got = o.decrypt_scores(s, out, 16).astype(np.int64)
    # ((p0 + p1) / 4 + p2 + p3) / 4 with exact divisions
    prod = H.astype(np.int64) * cls[0].astype(np.int64)
    want = ((prod[:, 0] + prod[:, 1]) // 4 + prod[:, 2] + prod[:, 3])
    assert np.all(want % 4 == 0)
    assert np.array_equal(got[:, 0], (want // 4) % o.t)
