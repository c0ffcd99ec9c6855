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
