"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is against a printed
value (RFC 8439 vectors, the paper's batch sizes, security bounds and operation
counts), a textbook definition evaluated independently (direct polynomial
evaluation, schoolbook convolution, Python big-integer CRT), a closed form or an
invariant (round trips, slot products, rotations, decryption of encryptions).
"""
import math

import numpy as np
import pytest
import sympy

import oracle as O
from oracle import tiny
from tests.conftest import read_golden

from paper_2511_00737_gb300 import workload as WL


def _golden_chacha():
    rows = {r[0]: r[1:] for r in read_golden("rfc8439_chacha20.txt")}
    h = lambda xs: [int(x, 16) for x in xs]
    return {k: h(v) for k, v in rows.items()}


# ---------------------------------------------------------------- ChaCha20 (RFC 8439)
def test_quarter_round_rfc8439():
    g = _golden_chacha()
    assert O.quarter_round(*g["quarter_in"]) == g["quarter_out"]
    x = list(g["quarter_in"])
    tiny._qr(x, 0, 1, 2, 3)
    assert x == g["quarter_out"]


def test_block_function_rfc8439():
    g = _golden_chacha()
    out = O.chacha20_block(g["key"], g["counter"][0], g["nonce"])
    assert [int(v) for v in out] == g["block"]
    assert tiny.chacha20_block(g["key"], g["counter"][0], g["nonce"]) == g["block"]


def test_stream_word_layout():
    """word w of a stream = word w%16 of block w//16, key = seed, nonce = (domain, obj)."""
    seed, dom, obj = 0x0123456789ABCDEF, 3, (7 << 32) | 11
    words = O.stream_words(seed, dom, obj, 5, 40)
    key = [seed & 0xFFFFFFFF, seed >> 32] + [0] * 6
    nonce = [dom, obj >> 32, obj & 0xFFFFFFFF]
    ref = []
    for w in range(5, 45):
        ref.append(tiny.chacha20_block(key, w // 16, nonce)[w % 16])
    assert [int(v) for v in words] == ref


# ---------------------------------------------------------------- primes and roots
def test_is_prime_matches_library():
    rng = np.random.default_rng(1)
    vals = list(rng.integers(2, 2**32 - 1, size=3000)) + [2, 3, 4, 5, 7, 61, 2147483647,
                                                           4294967291, 3215031751, 25326001]
    for v in vals:
        assert O.is_prime(int(v)) == sympy.isprime(int(v)), v


@pytest.mark.parametrize("n,L", [(16, 3), (2048, 2), (4096, 3), (8192, 4), (16384, 6)])
def test_find_primes(n, L):
    q = [int(v) for v in O.find_primes(n, L)]
    assert q == sorted(q, reverse=True)
    for p in q:
        assert p < 2**30 and p % (2 * n) == 1 and sympy.isprime(p)
    # no admissible prime skipped between 2^30 and the smallest chosen one
    c = 2**30 - 2 * n + 1
    expect = []
    while len(expect) < L:
        if sympy.isprime(c):
            expect.append(c)
        c -= 2 * n
    assert q == expect
    assert q == tiny.primes(n, L) if n <= 64 else True


@pytest.mark.parametrize("n", [8, 64, 4096, 8192, 16384])
def test_root_has_order_2n(n):
    for p in list(O.find_primes(n, 2)) + [65537]:
        p = int(p)
        psi = O.root_2n(p, n)
        assert pow(psi, n, p) == p - 1 and pow(psi, 2 * n, p) == 1
        # psi is x^((p-1)/2n) for the least quadratic non-residue x
        x = 2
        while sympy.legendre_symbol(x, p) != -1:
            x += 1
        assert psi == pow(x, (p - 1) // (2 * n), p)


# ---------------------------------------------------------------- NTT
@pytest.mark.parametrize("n", [8, 16, 64])
def test_ntt_is_evaluation_at_odd_powers(n):
    rng = np.random.default_rng(n)
    p = int(O.find_primes(n, 1)[0])
    psi = O.root_2n(p, n)
    a = rng.integers(0, p, n)
    got = O.ntt(a, p, psi)
    for j in range(n):
        ref = sum(int(a[k]) * pow(psi, (2 * j + 1) * k, p) for k in range(n)) % p
        assert int(got[j]) == ref


@pytest.mark.parametrize("n", [8, 32, 64])
def test_polymul_matches_python_schoolbook(n):
    rng = np.random.default_rng(100 + n)
    p = int(O.find_primes(n, 1)[0])
    psi = O.root_2n(p, n)
    a, b = rng.integers(0, p, n), rng.integers(0, p, n)
    ref = tiny.negamul([int(v) for v in a], [int(v) for v in b], p)
    assert [int(v) for v in O.polymul(a, b, p, psi)] == ref
    assert [int(v) for v in O.negacyclic_mul_schoolbook(a, b, p)] == ref


def test_tiny_negamul_matches_numpy_convolution():
    rng = np.random.default_rng(5)
    n, p = 32, 97
    a, b = rng.integers(0, p, n), rng.integers(0, p, n)
    full = np.convolve(a.astype(object), b.astype(object))
    ref = [(full[i] - (full[i + n] if i + n < len(full) else 0)) % p for i in range(n)]
    assert tiny.negamul([int(v) for v in a], [int(v) for v in b], p) == ref


@pytest.mark.parametrize("n", [1024, 4096])
def test_polymul_matches_schoolbook_full_size(n):
    rng = np.random.default_rng(n)
    p = int(O.find_primes(n, 1)[0])
    psi = O.root_2n(p, n)
    a, b = rng.integers(0, p, n), rng.integers(0, p, n)
    assert np.array_equal(O.polymul(a, b, p, psi), O.negacyclic_mul_schoolbook(a, b, p))


@pytest.mark.parametrize("n,L", [(8192, 4), (16384, 6)])
def test_ntt_roundtrip_full_size(n, L):
    rng = np.random.default_rng(7)
    for p in O.find_primes(n, L):
        p = int(p)
        psi = O.root_2n(p, n)
        a = rng.integers(0, p, n)
        assert np.array_equal(O.intt(O.ntt(a, p, psi), p, psi), a)


# ---------------------------------------------------------------- slots mod t
@pytest.mark.parametrize("n", [16, 64, 256])
def test_slot_encoder_matches_definition(n):
    rng = np.random.default_rng(n)
    zeta = O.root_2n(65537, n)
    v = rng.integers(0, 65537, n)
    m = O.slot_encode(v, zeta)
    assert np.array_equal(m, O.slot_encode_definition(v, zeta))
    if n <= 64:
        assert [int(x) for x in m] == tiny.encode([int(x) for x in v], zeta)
        assert tiny.decode([int(x) for x in m], zeta) == [int(x) for x in v]


def test_slot_roundtrip_and_product_n4096():
    n, t = 4096, 65537
    rng = np.random.default_rng(11)
    zeta = O.root_2n(t, n)
    v, w = rng.integers(0, t, n), rng.integers(0, t, n)
    mv, mw = O.slot_encode(v, zeta), O.slot_encode(w, zeta)
    assert np.array_equal(O.slot_decode(mv, zeta), v)
    prod = O.negacyclic_mul_schoolbook(mv, mw, t)
    assert np.array_equal(O.slot_decode(prod, zeta), (v.astype(np.int64) * w) % t)


@pytest.mark.parametrize("n", [32, 1024])
def test_galois_rotates_rows(n):
    t = 65537
    rng = np.random.default_rng(n + 3)
    zeta = O.root_2n(t, n)
    v = rng.integers(0, t, n)
    m = O.slot_encode(v, zeta)
    half = n // 2
    for s in [1, 3, half // 4]:
        g = pow(3, s, 2 * n)
        got = O.slot_decode(O.automorphism(m, g, t), zeta)
        ref = np.concatenate([np.roll(v[:half], -s), np.roll(v[half:], -s)])
        assert np.array_equal(got, ref)
    got = O.slot_decode(O.automorphism(m, 2 * n - 1, t), zeta)
    assert np.array_equal(got, np.concatenate([v[half:], v[:half]]))


# ---------------------------------------------------------------- samplers
def test_cdt_table_and_gaussian_moments():
    T_ = O.cdt_table(3.2)
    assert [int(x) for x in T_] == tiny.cdt_table(3.2)
    assert np.all(np.diff(T_.astype(np.float64)) >= 0)
    e = np.concatenate([O.sample_gauss(9, 3, o, 1 << 17) for o in range(8)])
    assert e.size >= 10**6
    assert np.abs(e).max() <= 19
    assert abs(e.mean()) < 0.02
    assert abs(e.std() - 3.2) / 3.2 < 0.01


def test_ternary_and_uniform():
    s = O.sample_ternary(12345, 1 << 16)
    assert set(np.unique(s)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs((s == v).mean() - 1 / 3) < 0.01
    assert [int(x) for x in s[:64]] == tiny.ternary(12345, 64)
    q = O.find_primes(8192, 4)
    a = O.sample_uniform(12345, 2, 5, 8192, q)
    for l in range(4):
        assert a[l].max() < q[l]
        assert abs(a[l].mean() / q[l] - 0.5) < 0.01
    ref = tiny.uniform_poly(12345, 2, 5, 8192, [int(x) for x in q])
    assert [int(x) for x in a[3][:50]] == ref[3][:50]


# ---------------------------------------------------------------- parameters
def test_delta_is_floor_q_over_t():
    o = O.Oracle(8192, 4, 2, 1, 8, 10000)
    Q = math.prod(o.q)
    for l, p in enumerate(o.q):
        assert o.delta[l] == (Q // 65537) % p


def test_security_bounds_from_paper_table():
    bound = {int(a): int(b) for a, b in read_golden("paper_security_bounds.txt")}
    for n, L in [(4096, 3), (8192, 4)]:
        logq = sum(math.log2(int(p)) for p in O.find_primes(n, L))
        assert logq <= bound[int(math.log2(n))]


def test_batch_size_matches_paper():
    for N, k, batch in read_golden("paper_batch_sizes.txt"):
        o = O.Oracle(int(N), 2, int(k), int(k), 1, 64)
        assert o.cap == int(batch)


def test_operation_counts_match_paper_table():
    """(k_in = k, r = 1) is EP-HDC's SIMD form; (k_in = 1, r = N/2) is HE-HDC's."""
    for method, N, D, k, mulcp, rot in read_golden("paper_op_counts.txt"):
        N, D, k, mulcp, rot = map(int, (N, D, k, mulcp, rot))
        if method == "ephdc":
            o = O.Oracle(N, 2, k, k, 1, D)
            assert o.cap == 2 * (N // (2 * k))
        else:
            o = O.Oracle(N, 2, k, 1, N // 2, D)
        assert o.P * o.Kp == mulcp and o.logr == rot


# ---------------------------------------------------------------- BFV invariants
@pytest.fixture(scope="module")
def c1():
    o = O.Oracle(4096, 3, 2, 2, 128, 2048)
    s, gk = o.keygen(77)
    return o, s, gk


def test_encrypt_decrypt_roundtrip(c1):
    o, s, _ = c1
    rng = np.random.default_rng(3)
    v = rng.integers(0, 65537, o.n)
    ct = o.encrypt_slots(77, 999, s, v)
    assert np.array_equal(o.decrypt_slots(s, ct), v)
    assert o.noise_budget(s, ct) > 40


def test_plaintext_times_ciphertext(c1):
    """decrypt(lift(m_w) * ct_v) = v * w slot-wise (one MulCP)."""
    o, s, _ = c1
    rng = np.random.default_rng(4)
    v, w = rng.integers(0, 65537, o.n), rng.integers(0, 65537, o.n)
    ct = o.encrypt_slots(77, 5, s, v)
    mw = O.slot_encode(w, o.zeta)
    prod = np.zeros_like(ct)
    for l, p in enumerate(o.q):
        lm = np.where(mw <= 32768, mw.astype(np.int64), mw.astype(np.int64) - 65537) % p
        for poly in range(2):
            prod[poly, l] = O.polymul(lm, ct[poly, l], p, o.psi[l])
    assert np.array_equal(o.decrypt_slots(s, prod), (v.astype(np.int64) * w) % 65537)


def test_rotation_with_key_switching(c1):
    o, s, gk = c1
    rng = np.random.default_rng(6)
    v = rng.integers(0, 65537, o.n)
    ct = o.encrypt_slots(77, 6, s, v)
    half = o.n // 2
    for j in range(o.logr):
        rc = o.rotate(o.fold_galois(j), gk[j], ct)
        sh = o.W << j
        ref = np.concatenate([np.roll(v[:half], -sh), np.roll(v[half:], -sh)])
        assert np.array_equal(o.decrypt_slots(s, rc), ref)
        assert o.noise_budget(s, rc) > 20


def test_decrypt_matches_python_bigint_crt(c1):
    o, s, _ = c1
    rng = np.random.default_rng(8)
    ct = np.stack([np.stack([rng.integers(0, p, o.n) for p in o.q]) for _ in range(2)])
    got = o.decrypt(s, ct)
    Q = math.prod(o.q)
    xs = []
    for l, p in enumerate(o.q):
        sl = np.asarray(s, np.int64) % p
        xs.append((ct[0, l].astype(np.int64) + O.polymul(ct[1, l], sl, p, o.psi[l])) % p)
    for kk in range(0, o.n, 97):
        x = sum(int(xs[l][kk]) * pow(Q // p, -1, p) * (Q // p) for l, p in enumerate(o.q)) % Q
        assert int(got[kk]) == ((65537 * x + Q // 2) // Q) % 65537


# ---------------------------------------------------------------- HDC encode
@pytest.mark.parametrize("shift,bits", [(0, 8), (5, 8), (9, 4), (3, 2)])
def test_hdc_encode_matches_float64_matmul(shift, bits):
    X = WL.features(1, 37, 96)
    Wt = WL.projection(1, 300, 96)
    X[0, :] = 127  # extremes of the projection
    Wt[0, :] = -1
    H = O.hdc_encode(X, Wt, shift, bits)
    A = X.astype(np.float64) @ Wt.astype(np.float64).T  # exact: |A| < 2^53
    v = np.floor((A + (2.0 ** (shift - 1) if shift else 0.0)) / 2.0 ** shift)
    v = np.clip(v, -(2 ** (bits - 1)), 2 ** (bits - 1) - 1)
    assert np.array_equal(H, v.astype(np.int8))
    assert H.min() == -(2 ** (bits - 1)) or shift == 0


# ---------------------------------------------------------------- two implementations
@pytest.mark.parametrize("n,L,k,k_in,r,D,B", [
    (32, 3, 2, 2, 2, 11, 13),     # packed classes, ragged D (11 = 5*2 + 1)
    (32, 2, 3, 1, 4, 9, 5),       # one class per ciphertext, 2 rotations
    (16, 3, 2, 1, 1, 6, 17),      # paper form (r = 1, no rotation), 2 groups + tail
])
def test_c_oracle_matches_tiny_bfv_word_for_word(n, L, k, k_in, r, D, B):
    seed = 4242
    o = O.Oracle(n, L, k, k_in, r, D)
    tb = tiny.TinyBFV(n, L, k, k_in, r, D)
    assert o.q == tb.q and o.zeta == tb.zeta and o.cap == tb.cap
    rng = np.random.default_rng(n * 31 + r)
    cls = rng.integers(-8, 8, size=(k, D)).astype(np.int8)
    H = rng.integers(-128, 128, size=(B, D)).astype(np.int8)

    s, gk = o.keygen(seed)
    ts, tgk = tb.keygen(seed)
    assert [int(v) for v in s] == ts
    for j in range(o.logr):
        for i in range(L):
            assert gk[j, i, 0].tolist() == tgk[j][i][0]
            assert gk[j, i, 1].tolist() == tgk[j][i][1]

    model = o.encrypt_model(seed, cls, s)
    tmodel = tb.encrypt_model(seed, cls.tolist(), ts)
    for i in range(o.P):
        for jp in range(o.Kp):
            assert model[i, jp, 0].tolist() == tmodel[i][jp][0]
            assert model[i, jp, 1].tolist() == tmodel[i][jp][1]

    m = o.encode_plain(H)
    tm = tb.encode_plain(H.tolist())
    assert m.tolist() == tm

    acc = o.ptct_mac(m, B, model)
    tacc = tb.ptct_mac(tm, tmodel)
    out = o.rotate_sum(gk, acc)
    for g in range(o.groups(B)):
        for jp in range(o.Kp):
            assert acc[g, jp, 0].tolist() == tacc[g][jp][0]
            assert acc[g, jp, 1].tolist() == tacc[g][jp][1]
            tout = tb.rotate_sum(tacc[g][jp], tgk)
            assert out[g, jp, 0].tolist() == tout[0]
            assert out[g, jp, 1].tolist() == tout[1]

    clear = O.clear_scores(H, cls)
    assert np.array_equal(o.decrypt_scores(s, out, B), clear)
    tout_all = [[tb.rotate_sum(tacc[g][jp], tgk) for jp in range(o.Kp)]
                for g in range(o.groups(B))]
    assert np.array_equal(np.array(tb.scores(ts, tout_all, B), np.uint32), clear)


def test_end_to_end_small_config_matches_clear_scores():
    """16 queries, F=608, D=2048, 4-bit HVs, 2 classes, n=4096, 3 primes."""
    w = WL.config("small")
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    cls = WL.classes(w.seed, w.k, w.D)
    s, gk = o.keygen(w.seed)
    model = o.encrypt_model(w.seed, cls, s)
    H, m, out = o.infer(X, Wt, model, gk, w.shift, w.bits)
    assert np.array_equal(o.decrypt_scores(s, out, w.B), O.clear_scores(H, cls))
    assert o.noise_budget(s, out[0, 0]) > 20
    # 4-bit quantised hypervectors use the full range
    assert H.min() == -8 and H.max() == 7
