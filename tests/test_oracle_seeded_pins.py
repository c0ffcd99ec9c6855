"""The seeded model message: every model ciphertext's c1 is the uniform polynomial of
ChaCha20 domain 2 for its ciphertext number, so c0 and the seed determine the model
(half the bytes of the full message).  Pinned against the stream itself and against
decryption of the rebuilt ciphertexts."""
import numpy as np

import oracle as O


def test_c1_is_the_domain_2_stream_and_the_rebuilt_model_decrypts():
    o = O.Oracle(64, 3, 4, 2, 2, 13)
    cls = np.random.default_rng(4).integers(-8, 8, (4, 13)).astype(np.int8)
    s, _ = o.keygen(77)
    model = o.encrypt_model(77, cls, s)
    rebuilt = model.copy()
    for i in range(o.P):
        for jp in range(o.Kp):
            a = O.sample_uniform(77, 2, i * o.Kp + jp, o.n, o.q)
            assert np.array_equal(model[i, jp, 1], a)
            rebuilt[i, jp, 1] = a
    assert np.array_equal(rebuilt, model)
    # a wrong seed gives ciphertexts that no longer decrypt to the class slots
    bad = model.copy()
    bad[0, 0, 1] = O.sample_uniform(78, 2, 0, o.n, o.q)
    assert not np.array_equal(o.decrypt_slots(s, bad[0, 0]), o.decrypt_slots(s, model[0, 0]))
    assert model[:, :, 0].nbytes * 2 == model.nbytes


def _brv(j, bits):
    return int(format(j, "0%db" % bits)[::-1], 2)


def test_compact_model_c1_is_the_domain_8_stream_in_the_evaluation_domain():
    """The compact model regenerated while multiplying: c1 evaluated at psi^(2j+1) is
    64-bit word l*n + brv(j) of the domain-8 stream mod q_l.  Checked by evaluating the
    coefficient-domain c1 directly with Python integers (n = 16), and through the
    oracle's transform at n = 64; and every ciphertext decrypts to the class slots of
    the standard model."""
    for n, L, direct in ((16, 2, True), (64, 3, False)):
        o = O.Oracle(n, L, 4, 2, 2, 13)
        cls = np.random.default_rng(5).integers(-8, 8, (4, 13)).astype(np.int8)
        s, _ = o.keygen(91)
        model = o.encrypt_model_seeded_ntt(91, cls, s)
        standard = o.encrypt_model(91, cls, s)
        bits = n.bit_length() - 1
        for i in range(o.P):
            for jp in range(o.Kp):
                cidx = i * o.Kp + jp
                w = O.stream_words(91, 8, cidx, 0, 2 * L * n).astype(np.uint64)
                words = w[0::2] | (w[1::2] << np.uint64(32))
                for l, p in enumerate(o.q):
                    want = [int(words[l * n + _brv(j, bits)]) % p for j in range(n)]
                    c1 = [int(v) for v in model[i, jp, 1, l]]
                    if direct:
                        psi = o.psi[l]
                        got = [sum(c1[k] * pow(psi, (2 * j + 1) * k, p) for k in range(n)) % p
                               for j in range(n)]
                    else:
                        got = [int(v) for v in O.ntt(model[i, jp, 1, l], p, o.psi[l])]
                    assert got == want, (n, i, jp, l)
                assert np.array_equal(o.decrypt_slots(s, model[i, jp]),
                                      o.decrypt_slots(s, standard[i, jp]))
        assert not np.array_equal(model[:, :, 1], standard[:, :, 1])


def test_compact_model_scores_equal_the_clear_dot_products():
    w = dict(n=1024, L=3, k=3, k_in=1, r=4, D=100)
    o = O.Oracle(w["n"], w["L"], w["k"], w["k_in"], w["r"], w["D"])
    rng = np.random.default_rng(6)
    cls = rng.integers(-8, 8, (3, 100)).astype(np.int8)
    X = rng.integers(0, 128, (300, 32)).astype(np.int8)
    Wt = (2 * rng.integers(0, 2, (100, 32)) - 1).astype(np.int8)
    s, gk = o.keygen(12)
    model = o.encrypt_model_seeded_ntt(12, cls, s)
    H, _, out = o.infer(X, Wt, model, gk, 5, 8)
    assert np.array_equal(o.decrypt_scores(s, out, 300), O.clear_scores(H, cls))
