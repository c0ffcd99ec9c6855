"""GPU parity beyond the default parameters: other plaintext moduli t, smaller RNS
primes, and the scaling operation of Sec. 5.1 (folded into the encoded plaintexts on
the GPU, applied to the running accumulator by the oracle), bit for bit against the
oracle, on both the client-side path and the server-side variant."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def scaled_scores(H, cls, r, P, s_, g, t):
    """sum_d h[d] c[d] u^(floor(P/g) - floor(i/g)) mod t, i = d // r, u = (2^s)^-1 mod t"""
    u = pow(pow(2, s_, t), -1, t)
    out = np.zeros((H.shape[0], cls.shape[0]), np.int64)
    for d in range(H.shape[1]):
        w = pow(u, P // g - (d // r) // g, t)
        out = (out + np.outer(H[:, d].astype(np.int64), cls[:, d].astype(np.int64)) % t * w) % t
    return out.astype(np.uint32)


CASES = [
    # n, L, k, k_in, r, D, F, bits, B, t, prime_bits, scale_shift, scale_group
    (1024, 3, 3, 1, 4, 100, 32, 8, 300, 40961, 27, 0, 0),
    (2048, 3, 2, 2, 8, 64, 48, 4, 70, 1073153, 30, 0, 0),
    (1024, 4, 2, 1, 2, 50, 16, 8, 600, 536881153, 30, 0, 0),
    (1024, 4, 3, 1, 4, 100, 32, 8, 300, 65537, 30, 3, 10),     # P = 25: 2 scalings
    (2048, 4, 2, 2, 1, 40, 32, 4, 100, 65537, 30, 2, 16),      # paper form, P = 40
]


def _oracle_and_gpu(case, seed=31):
    n, L, k, k_in, r, D, F, bits, B, t, pb, ss, sg = case
    kw = dict(t=t, prime_bits=pb, scale_shift=ss, scale_group=sg or 512)
    o = O.Oracle(n, L, k, k_in, r, D, **kw)
    ctx = E.Context(n, L, k, k_in, r, D, F, bits, 0, B, t=t, prime_bits=pb, scale_shift=ss,
                    scale_group=sg)
    assert ctx.t == t and ctx.q == o.q
    X = WL.features(seed, B, F)
    Wt = WL.projection(seed, D, F)
    cls = WL.classes(seed, k, D)
    return o, ctx, X, Wt, cls, (r, o.P, ss, sg or 512, t)


@pytest.mark.parametrize("case", CASES)
def test_client_side_path_matches_oracle(case):
    o, ctx, X, Wt, cls, sc = _oracle_and_gpu(case)
    seed, B = 31, X.shape[0]
    s, ogk = o.keygen(seed)
    omodel = o.encrypt_model(seed, cls, s)
    H, m, oout = o.infer(X, Wt, omodel, ogk, 0, ctx.hv_bits)
    sk, gk = ctx.keygen(seed)
    model = ctx.encrypt_model(_dev(cls), sk, seed)
    out = ctx.infer(_dev(X), _dev(Wt), model, gk)
    torch.cuda.synchronize()
    assert np.array_equal(ctx.ct_to_host_coeff(model, o.P * o.Kp),
                          omodel.reshape(o.P * o.Kp, 2, o.L, o.n))
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    scores = _u32(ctx.decrypt_scores(sk, out, B))
    r, P, ss, sg, t = sc
    want = scaled_scores(H, cls, r, P, ss, sg, t) if ss else O.clear_scores(H, cls, t)
    assert np.array_equal(scores, want)
    assert np.array_equal(o.decrypt_scores(s, oout, B), want)
    ctx.device_status()
    ctx.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[3]])
def test_server_side_variant_matches_oracle(case):
    o, ctx, X, Wt, cls, sc = _oracle_and_gpu(case)
    seed, B = 31, X.shape[0]
    H = O.hdc_encode(X, Wt, 0, ctx.hv_bits)
    s, ogk = o.keygen(seed)
    oout = o.rotate_sum(ogk, o.ctpt_mac(o.encrypt_queries(seed, H, s), B,
                                        o.encode_model_plain(cls)))
    sk, gk = ctx.keygen(seed)
    ctq = ctx.encrypt_queries(_dev(H), sk, seed)
    out = ctx.ctpt_similarity(ctq, B, ctx.encode_model_plain(_dev(cls)), gk)
    torch.cuda.synchronize()
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    r, P, ss, sg, t = sc
    want = scaled_scores(H, cls, r, P, ss, sg, t) if ss else O.clear_scores(H, cls, t)
    assert np.array_equal(_u32(ctx.decrypt_scores(sk, out, B)), want)
    ctx.close()
