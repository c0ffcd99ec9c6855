"""The coefficient-blocked storage layout ("layout" 1): plaintexts [L][n/4][G][P][4]
and model [L][n/4][P][O][4], read by the tensor-core multiply-accumulate.  Every
result must equal the oracle's exactly, as in the standard layout: the encrypted
model and the plaintexts (converted back to the host formats), the score
ciphertexts, the decrypted scores; the packed multi-client pass, the scaling
operation and the full-size dense batch (by the oracle's digests); and the entry
points that do not take this layout must refuse it."""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu

T = 65537
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _lifted(m, q):
    mm = m.astype(np.int64)
    v = np.where(mm <= (T - 1) // 2, mm, mm - T)
    return np.stack([np.mod(v, p) for p in q], axis=-2).astype(np.uint32)


def _blocked_ctx(w, B, **kw):
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, max(B, 1), **kw)
    ctx.tune_set("layout", 1)
    assert ctx.tune_get("layout") == 1
    return ctx


LAYOUTS = [
    # n, L, k, k_in, r, D, F, bits, B
    (1024, 2, 2, 2, 1, 50, 32, 8, 700),     # paper layout, no rotation, 2 groups
    (1024, 3, 3, 1, 4, 41, 16, 4, 600),     # ragged D, 3 groups
    (2048, 2, 7, 7, 2, 33, 64, 8, 300),     # 7 packed classes
    (4096, 3, 2, 1, 16, 300, 48, 6, 1000),  # 4 rotations, G = 4 with a partial tail
    (1024, 4, 16, 1, 2, 700, 32, 8, 17),    # 32 outputs (every row of a digit block), B < cap
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B", LAYOUTS)
def test_blocked_layout_matches_oracle(n, L, k, k_in, r, D, F, bits, B):
    w = WL.Workload(name="t", n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F, bits=bits, B=B,
                    seed=2000 + n + r)
    o = O.Oracle(n, L, k, k_in, r, D)
    X, Wt, cls = WL.features(w.seed, B, F), WL.projection(w.seed, D, F), WL.classes(w.seed, k, D)
    s, ogk = o.keygen(w.seed)
    omodel = o.encrypt_model(w.seed, cls, s)
    H, m, out = o.infer(X, Wt, omodel, ogk, w.shift, bits)

    ctx = _blocked_ctx(w, B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    assert np.array_equal(ctx.model_to_host_coeff(model), omodel)
    gX, gW = _dev(X), _dev(Wt)
    pt = ctx.encode_plain(ctx.hdc_encode(gX, gW))
    G = o.groups(B)
    got_pt = ctx.plain_to_host_coeff(pt, G * o.P)
    assert np.array_equal(got_pt, _lifted(m.reshape(G * o.P, n), o.q))
    g_out = ctx.ptct_similarity(pt, B, model, gk)
    ctx.device_status()
    assert np.array_equal(_u32(g_out).reshape(out.shape), out)
    assert torch.equal(ctx.infer(gX, gW, model, gk), g_out)
    assert np.array_equal(_u32(ctx.decrypt_scores(sk, g_out, B)), O.clear_scores(H, cls))
    ctx.close()


def test_blocked_layout_packed_clients_match_oracle():
    sizes = [5, 0, 300, 17, 64, 1, 129]
    w = WL.Workload(name="t", n=1024, L=3, k=3, k_in=1, r=4, D=100, F=32, bits=8,
                    B=sum(sizes), seed=77)
    Xs = [WL.features(w.seed, b, w.F, batch=i) for i, b in enumerate(sizes)]
    Wt, cls = WL.projection(w.seed, w.D, w.F), WL.classes(w.seed, w.k, w.D)
    ctx = _blocked_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    out = ctx.infer_multi([_dev(x) for x in Xs], _dev(Wt), model, gk)
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    s, ogk = o.keygen(w.seed)
    _, _, oout = o.infer(np.concatenate(Xs), Wt, o.encrypt_model(w.seed, cls, s), ogk,
                         w.shift, w.bits)
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    ctx.close()


def test_blocked_layout_with_the_scaling_operation():
    w = WL.Workload(name="t", n=1024, L=3, k=2, k_in=1, r=4, D=200, F=32, bits=4, B=300,
                    seed=31)
    kw = dict(scale_shift=3, scale_group=16)
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D, **kw)
    X, Wt, cls = WL.features(w.seed, w.B, w.F), WL.projection(w.seed, w.D, w.F), \
        WL.classes(w.seed, w.k, w.D)
    s, ogk = o.keygen(w.seed)
    _, _, oout = o.infer(X, Wt, o.encrypt_model(w.seed, cls, s), ogk, w.shift, w.bits)
    ctx = _blocked_ctx(w, w.B, **kw)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    out = ctx.infer(_dev(X), _dev(Wt), model, gk)
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    ctx.close()


def test_entry_points_without_the_blocked_layout_refuse_it():
    w = WL.config("small")
    ctx = _blocked_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(WL.features(w.seed, w.B, w.F)),
                                         _dev(WL.projection(w.seed, w.D, w.F))))
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    for mode in (1, 2):
        ctx.tune_set("mac_mode", mode)
        with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
            ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.tune_set("mac_mode", 3)
    assert torch.equal(ctx.ptct_similarity(pt, w.B, model, gk), ref)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, w.B, model, gk, torch.empty_like(ref))
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        ctx.model_to_seeded(model)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        ctx.encode_model_plain(_dev(WL.classes(w.seed, w.k, w.D)))
    ctx.close()


@pytest.mark.slow
def test_dense65536_blocked_full_size_digests():
    """65536 queries, n = 16384, 6 primes, 16 classes, 64 groups in the blocked layout:
    the score ciphertexts of groups 0 and 63 against the oracle's digests."""
    w = WL.config("dense65536")
    ctx = _blocked_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    out = ctx.infer(_dev(WL.features(w.seed, w.B, w.F)), _dev(WL.projection(w.seed, w.D, w.F)),
                    model, gk)
    ctx.device_status()
    words = _u32(out).reshape(-1, ctx.Kp, 2, w.L, w.n)
    with open(os.path.join(GOLDEN, "dense65536_group_digests.txt")) as f:
        digests = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(digests) == 2
    for g, _, _, digest in digests:
        got = np.ascontiguousarray(words[int(g)], dtype="<u4")
        assert hashlib.sha256(got.tobytes()).hexdigest() == digest, g
    ctx.close()
