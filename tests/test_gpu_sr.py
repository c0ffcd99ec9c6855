"""GPU parity of the server-side variant (HE-HDC-SR, Sec. 3; the comparison of
Sec. 6, Table t:clientrt): encrypted query ciphertexts, the plaintext model, and
the score ciphertexts after ct x pt accumulate + rotate-and-sum, bit for bit against
the CPU oracle, and decrypted scores equal to the clear dot products mod t."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu

T = 65537


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _lifted(m, q):
    mm = m.astype(np.int64)
    v = np.where(mm <= (T - 1) // 2, mm, mm - T)
    return np.stack([np.mod(v, p) for p in q], axis=-2).astype(np.uint32)


def _run(w, B, seed, check_plain=True):
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, max(B, 1))
    X = WL.features(seed, B, w.F)
    Wt = WL.projection(seed, w.D, w.F)
    cls = WL.classes(seed, w.k, w.D)
    H = O.hdc_encode(X, Wt, w.shift, w.bits)
    s, ogk = o.keygen(seed)
    octq = o.encrypt_queries(seed, H, s)
    omm = o.encode_model_plain(cls)
    oout = o.rotate_sum(ogk, o.ctpt_mac(octq, B, omm))

    sk, gk = ctx.keygen(seed)
    gH = ctx.hdc_encode(_dev(X), _dev(Wt))
    ctq = ctx.encrypt_queries(gH, sk, seed)
    mm = ctx.encode_model_plain(_dev(cls))
    out = ctx.ctpt_similarity(ctq, B, mm, gk)
    torch.cuda.synchronize()
    G = o.groups(B)
    assert np.array_equal(gH.cpu().numpy(), H)
    got_ctq = ctx.ct_to_host_coeff(ctq, G * o.P)
    assert np.array_equal(got_ctq, octq.reshape(G * o.P, 2, w.L, w.n))
    if check_plain:
        got_mm = ctx.plain_to_host_coeff(mm, o.Kp * o.P)
        assert np.array_equal(got_mm, _lifted(omm.reshape(o.Kp * o.P, w.n), o.q))
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    scores = _u32(ctx.decrypt_scores(sk, out, B))
    assert np.array_equal(scores, O.clear_scores(H, cls))
    ctx.device_status()
    ctx.close()


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B", [
    (1024, 3, 3, 1, 4, 100, 32, 8, 300),      # one class per ct, 2 rotations, ragged tail
    (2048, 2, 2, 2, 1, 37, 48, 4, 1500),      # the paper's form: r = 1, no rotation
    (4096, 3, 7, 7, 8, 300, 64, 4, 20),       # packed classes, 3 rotations, one partial group
    (1024, 2, 5, 1, 2, 64, 16, 8, 1),         # a single query; Kp = 5 > 4 outputs per thread
])
def test_server_side_path_matches_oracle(n, L, k, k_in, r, D, F, bits, B):
    w = WL.Workload(name="t", B=B, seed=99, n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F,
                    bits=bits)
    _run(w, B, 99)


@pytest.mark.parametrize("plan", [0, 1, 2])
def test_query_encryption_same_for_every_ntt_plan(plan):
    w = WL.Workload(name="t", B=70, seed=5, n=8192, L=4, k=2, k_in=1, r=8, D=40, F=32, bits=8)
    ctx = E.Context.for_workload(w)
    H = _dev(np.random.default_rng(1).integers(-128, 128, (70, 40)).astype(np.int8))
    sk, _ = ctx.keygen(5)
    ctx.tune_set("ntt_plan", 0)
    ref = ctx.encrypt_queries(H, sk, 5)
    ctx.tune_set("ntt_plan", plan)
    assert torch.equal(ctx.encrypt_queries(H, sk, 5), ref)
    ctx.close()


def test_server_side_errors_are_reported():
    w = WL.Workload(name="t", B=4, seed=5, n=1024, L=2, k=2, k_in=1, r=2, D=8, F=16, bits=8)
    ctx = E.Context.for_workload(w)
    H = torch.zeros((4, 8), dtype=torch.int8, device="cuda")
    sk, gk = ctx.keygen(1)
    with pytest.raises(E.EphdcError):
        ctx.encrypt_queries(torch.zeros((5, 8), dtype=torch.int8, device="cuda"), sk, 1)
    ctq = ctx.encrypt_queries(H, sk, 1)
    mm = ctx.encode_model_plain(torch.zeros((2, 8), dtype=torch.int8, device="cuda"))
    with pytest.raises(E.EphdcError):
        ctx.ctpt_similarity(ctq, 0, mm, gk)
    ctx.device_status()
    ctx.close()


@pytest.mark.slow
def test_face1024_server_side_full_size_bit_exact():
    """1024 queries, D=10000, 8-bit HVs, 2 classes, n=8192, 4 primes, k_in=1 r=8: all
    1250 query ciphertexts and both score ciphertexts bit-exact."""
    w = WL.config("face1024")
    _run(w, w.B, w.seed)
