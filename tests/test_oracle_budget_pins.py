"""Pins of the oracle's noise budget (the decryption-correctness margin of Alg. 1
and Sec. 5.2: a BFV ciphertext decrypts correctly while its noise stays below
q/(2t)).

The budget is log2(q/(2t)) - log2(max_k |t x_k - q m'_k| / t), x = CRT of the phase
c0 + c1 s, m' its rounded message.  Two independent routes fix it:
- a hand-built ciphertext whose phase is a known error polynomial e (c1 = 0,
  c0 = e mod q_l, message 0): the noise term is t max|e| / t, so the budget is the
  closed form log2(q/(2t)) - log2(max|e|);
- the same quantity recomputed with Python integers (a ternary-secret negacyclic
  product by signed shifts, CRT by exact big-integer arithmetic) on ciphertexts the
  oracle encrypts and rotates, at n = 16 and n = 4096.
A dropped factor t, a wrong logarithm or a missing centring fails one of them.
"""
import math

import numpy as np

import oracle as O


def _phase_bigint(o, s, ct):
    """x_k = CRT([c0 + c1 s]_{q_l}) in [0, q), by Python integers only."""
    n = o.n
    s = np.asarray(s, np.int64)
    xs = []
    for l, p in enumerate(o.q):
        c0 = ct[0, l].astype(np.int64)
        c1 = ct[1, l].astype(np.int64)
        acc = c0 % p
        # c1 * s in Z[x]/(x^n + 1): x^j c1 is c1 shifted up by j, the wrapped part negated
        for j in np.nonzero(s)[0]:
            sh = np.concatenate([-c1[n - j:], c1[:n - j]]) if j else c1
            acc = (acc + int(s[j]) * sh) % p
        xs.append([int(v) for v in acc])
    Q = math.prod(int(p) for p in o.q)
    out = []
    for k in range(n):
        x = 0
        for l, p in enumerate(o.q):
            Ql = Q // int(p)
            x += xs[l][k] * Ql * pow(Ql, -1, int(p))
        out.append(x % Q)
    return out, Q


def _budget_bigint(o, s, ct):
    xs, Q = _phase_bigint(o, s, ct)
    t = o.t
    worst = 0
    for x in xs:
        v = (t * x) % Q
        worst = max(worst, min(v, Q - v))
    return math.log2(Q) - math.log2(2 * t) - math.log2(worst / t)


def test_budget_of_a_known_error_is_the_closed_form():
    o = O.Oracle(1024, 3, 2, 2, 1, 16)
    rng = np.random.default_rng(21)
    s = rng.integers(-1, 2, o.n).astype(np.int32)
    Q = math.prod(int(p) for p in o.q)
    for emax in (1, 7, 19, 1000, 123457):
        e = rng.integers(-emax, emax + 1, o.n)
        e[rng.integers(0, o.n)] = emax * (1 if rng.integers(0, 2) else -1)
        ct = np.zeros((2, o.L, o.n), np.uint32)
        for l, p in enumerate(o.q):
            ct[0, l] = np.mod(e, p)
        want = math.log2(Q / (2 * o.t)) - math.log2(emax)
        assert abs(o.noise_budget(s, ct) - want) < 1e-9, emax


def test_budget_equals_python_bigint_at_n16():
    o = O.Oracle(16, 2, 2, 2, 2, 8)
    s, gk = o.keygen(5)
    rng = np.random.default_rng(22)
    v = rng.integers(0, o.t, o.n)
    ct = o.encrypt_slots(5, 31, s, v)
    assert abs(o.noise_budget(s, ct) - _budget_bigint(o, s, ct)) < 1e-9
    rc = o.rotate(o.fold_galois(0), gk[0], ct)
    assert abs(o.noise_budget(s, rc) - _budget_bigint(o, s, rc)) < 1e-9


def test_budget_equals_python_bigint_at_n4096():
    o = O.Oracle(4096, 3, 2, 2, 128, 2048)
    s, gk = o.keygen(77)
    rng = np.random.default_rng(23)
    v = rng.integers(0, o.t, o.n)
    ct = o.encrypt_slots(77, 41, s, v)
    fresh = o.noise_budget(s, ct)
    assert abs(fresh - _budget_bigint(o, s, ct)) < 1e-9
    # one plaintext product (a centred lifted slot vector) costs about log2(n t / 2) bits
    w = rng.integers(0, o.t, o.n)
    mw = O.slot_encode(w, o.zeta).astype(np.int64)
    lm = np.where(mw <= o.t // 2, mw, mw - o.t)
    prod = np.zeros_like(ct)
    for l, p in enumerate(o.q):
        for poly in range(2):
            prod[poly, l] = O.polymul(lm % p, ct[poly, l], p, o.psi[l])
    after = o.noise_budget(s, prod)
    assert abs(after - _budget_bigint(o, s, prod)) < 1e-9
    assert 0 < fresh - after < math.log2(o.n * o.t)
