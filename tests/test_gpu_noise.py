"""The noise-growth experiment (Sec. 5.2, Alg. 1 findDmax) on the GPU against the
oracle: the same seeded trial gives the same D_i, exactly."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import noise as N

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("t,D", [(40961, 64), (18433, 600)])
def test_trial_dmax_equals_oracle(t, D):
    n = 1024
    o = O.Oracle(n, 2, 1, 1, 1, D, t=t, prime_bits=20)
    tr = N.Trials(n, t, 2, 20, D)
    assert tr.ctx.q == o.q
    got, want = [], []
    for k in range(3):
        rng = np.random.default_rng(700 + k)
        H = rng.integers(-128, 128, (n, D)).astype(np.int8)
        cls = rng.integers(-8, 8, (1, D)).astype(np.int8)
        s, _ = o.keygen(900 + k)
        want.append(o.find_dmax_trial(o.encode_plain(H), o.encrypt_model(900 + k, cls, s), s, H,
                                      cls))
        got.append(tr.trial(900 + k, _dev(H), _dev(cls)))
    tr.close()
    assert got == want
    assert all(0 < v < D for v in want)


def test_no_failure_within_a_large_budget():
    """At the default parameters (four 30-bit primes, t = 65537) 200 products are far
    inside the budget: D_i = D."""
    tr = N.Trials(1024, 65537, 4, 30, 200)
    assert tr.trial(5) == 200
    tr.close()


def test_find_dmax_driver():
    r = N.find_dmax(2048, 22, trials=8)
    assert r["log2_q"] <= 54 and r["L"] == 2 and r["censored"] == 0
    assert 0 < r["dmax_mean"] < r["d_lim"]
    assert r["t"] % 4096 == 1 and N.is_prime(r["t"])


def test_plaintext_modulus_rule():
    assert N.plaintext_modulus(2048, 16) == 65537
    assert N.plaintext_modulus(1024, 14) == 18433 and N.plaintext_modulus(1024, 13) == 12289
