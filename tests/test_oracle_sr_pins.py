"""Pins of the oracle's server-side variant (HE-HDC-SR, Sec. 3 and the comparison
of Sec. 6, Table t:clientrt): the client encrypts its query hypervectors in the SIMD
form, the server holds the class hypervectors as plaintexts.  Checked against the
slot layout written out by brute force, the clear dot products, the ChaCha20 streams
of the samplers, and the message-size ratio the paper reports."""
import math

import numpy as np
import pytest

import oracle as O
from tests.conftest import read_golden


def _slots_of_queries(o, H, g, i):
    """Slot vector of query plaintext (g, i), written out from the layout definition."""
    v = np.zeros(o.n, np.int64)
    half = o.n // 2
    for rho in range(2):
        for ch in range(o.r):
            d = i * o.r + ch
            if d >= o.D:
                continue
            for qq in range(o.cap_row):
                beta = g * o.cap + rho * o.cap_row + qq
                if beta >= H.shape[0]:
                    continue
                for jin in range(o.k_in):
                    v[rho * half + ch * o.W + jin * o.cap_row + qq] = int(H[beta, d]) % 65537
    return v


def _slots_of_classes(o, cls, jp, i):
    v = np.zeros(o.n, np.int64)
    half = o.n // 2
    for rho in range(2):
        for ch in range(o.r):
            d = i * o.r + ch
            if d >= o.D:
                continue
            for jin in range(o.k_in):
                for qq in range(o.cap_row):
                    v[rho * half + ch * o.W + jin * o.cap_row + qq] = \
                        int(cls[jp * o.k_in + jin, d]) % 65537
    return v


CASES = [
    (32, 3, 3, 1, 2, 9, 20),    # one class per ciphertext, 1 rotation, 2 groups
    (32, 3, 2, 2, 4, 11, 5),    # packed classes, ragged D, 2 rotations
    (16, 2, 2, 2, 1, 6, 9),     # the paper's form: r = 1, no rotation, 2 groups
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,B", CASES)
def test_query_ciphertexts_decrypt_to_query_slots(n, L, k, k_in, r, D, B):
    o = O.Oracle(n, L, k, k_in, r, D)
    rng = np.random.default_rng(n + r)
    H = rng.integers(-128, 128, (B, D)).astype(np.int8)
    s, _ = o.keygen(11)
    ctq = o.encrypt_queries(11, H, s)
    assert ctq.shape == (o.groups(B), o.P, 2, L, n)
    for g in range(o.groups(B)):
        for i in range(o.P):
            assert np.array_equal(o.decrypt_slots(s, ctq[g, i]), _slots_of_queries(o, H, g, i))
            assert o.noise_budget(s, ctq[g, i]) > 20


def test_query_ciphertext_is_secret_key_rlwe_with_its_own_streams():
    """c1 is the uniform stream of domain 6 and c0 + c1 s = round(q m / t) + e with e the
    Gaussian stream of domain 7, for ciphertext number g*P + i."""
    o = O.Oracle(32, 2, 2, 1, 2, 10)
    H = np.random.default_rng(2).integers(-8, 8, (40, 10)).astype(np.int8)
    s, _ = o.keygen(5)
    ctq = o.encrypt_queries(5, H, s)
    for g, i in [(0, 0), (1, 3), (2, 4)]:
        gi = g * o.P + i
        a = O.sample_uniform(5, 6, gi, o.n, o.q)
        e = O.sample_gauss(5, 7, gi, o.n).astype(np.int64)
        m = O.slot_encode(_slots_of_queries(o, H, g, i), o.zeta)
        Q = math.prod(o.q)
        scaled = [(Q * int(v) + (o.t + 1) // 2) // o.t for v in m]  # round(Q m / t)
        for l, p in enumerate(o.q):
            assert np.array_equal(ctq[g, i, 1, l], a[l])
            sl = np.asarray(s, np.int64) % p
            phase = (ctq[g, i, 0, l].astype(np.int64) + O.polymul(a[l], sl, p, o.psi[l])) % p
            want = (np.array([v % p for v in scaled], np.int64) + e) % p
            assert np.array_equal(phase, want)


@pytest.mark.parametrize("n,L,k,k_in,r,D,B", CASES)
def test_model_plaintexts_decode_to_class_slots(n, L, k, k_in, r, D, B):
    o = O.Oracle(n, L, k, k_in, r, D)
    cls = np.random.default_rng(7).integers(-8, 8, (k, D)).astype(np.int8)
    mm = o.encode_model_plain(cls)
    assert mm.shape == (o.Kp, o.P, n)
    for jp in range(o.Kp):
        for i in range(o.P):
            assert np.array_equal(O.slot_decode(mm[jp, i], o.zeta), _slots_of_classes(o, cls, jp, i))


@pytest.mark.parametrize("n,L,k,k_in,r,D,B", CASES)
def test_server_side_scores_equal_clear_dot_products(n, L, k, k_in, r, D, B):
    o = O.Oracle(n, L, k, k_in, r, D)
    rng = np.random.default_rng(n * 7 + B)
    H = rng.integers(-128, 128, (B, D)).astype(np.int8)
    cls = rng.integers(-8, 8, (k, D)).astype(np.int8)
    s, gk = o.keygen(21)
    ctq = o.encrypt_queries(21, H, s)
    acc = o.ctpt_mac(ctq, B, o.encode_model_plain(cls))
    out = o.rotate_sum(gk, acc)
    clear = O.clear_scores(H, cls)
    assert np.array_equal(o.decrypt_scores(s, out, B), clear)
    # the same scores as the client-side path, through different ciphertexts
    model = o.encrypt_model(21, cls, s)
    out_client = o.rotate_sum(gk, o.ptct_mac(o.encode_plain(H), B, model))
    assert np.array_equal(o.decrypt_scores(s, out_client, B), clear)
    assert not np.array_equal(out, out_client)
    assert o.noise_budget(s, out[0, 0]) > 5


def test_ct_times_pt_is_slotwise_product():
    """One MulCP of the server side: decrypt(ct(v) * pt(w)) = v * w slot-wise, for one
    query ciphertext and one model plaintext (B = cap, P = 1)."""
    o = O.Oracle(64, 3, 1, 1, 1, 1)
    rng = np.random.default_rng(9)
    H = rng.integers(-128, 128, (o.cap, 1)).astype(np.int8)
    cls = np.array([[5]], np.int8)
    s, _ = o.keygen(3)
    ctq = o.encrypt_queries(3, H, s)
    acc = o.ctpt_mac(ctq, o.cap, o.encode_model_plain(cls))
    v = _slots_of_queries(o, H, 0, 0)
    w = _slots_of_classes(o, cls, 0, 0)
    assert np.array_equal(o.decrypt_slots(s, acc[0, 0]), (v * w) % 65537)


def test_message_ratio_is_D_as_the_paper_reports():
    """At the paper's form (r = 1, k_in = k) the server-side client uploads G*P = G*D
    query ciphertexts, the client-side client sends G*(k/k_in) = G score ciphertexts:
    the ratio is D.  The paper's byte counts give D to within its serialisation
    overhead (Table t:clientrt)."""
    for N, D, sr, ep in read_golden("paper_message_sizes.txt"):
        N, D, sr, ep = int(N), int(D), float(sr), float(ep)
        o = O.Oracle(N, 2, 2, 2, 1, D)
        assert o.P == D and o.Kp == 1
        assert D <= sr / ep <= 1.1 * D
