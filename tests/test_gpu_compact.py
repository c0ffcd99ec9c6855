"""The compact model (only c0 stored; c1 drawn in the evaluation domain from the model
seed and regenerated by the tiled multiply-accumulate while it stages the model),
against the oracle's compact model word for word: the stored model (expanded back to
the host format), every output ciphertext, the decrypted scores; also through the
chunked pass and the packed multi-client pass, and the refusals of the paths that do
not take it."""
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


def _compact_ctx(w, B):
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, max(B, 1))
    full = E.lib().ephdc_model_bytes(ctx.ctx)
    ctx.tune_set("model_seed", w.seed)
    assert ctx.tune_get("model_seed") == w.seed
    assert 2 * E.lib().ephdc_model_bytes(ctx.ctx) == full
    return ctx


LAYOUTS = [
    # n, L, k, k_in, r, D, F, bits, B
    (1024, 2, 2, 2, 1, 50, 32, 8, 700),     # paper layout, no rotation, 2 groups
    (1024, 3, 3, 1, 4, 41, 16, 4, 600),     # ragged D, 3 groups, 3 ciphertexts per group
    (2048, 2, 7, 7, 2, 33, 64, 8, 300),     # 7 packed classes, 3 groups of 146
    (4096, 3, 2, 1, 16, 300, 48, 6, 1000),  # 4 rotations, G = 4 with a partial tail
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B", LAYOUTS)
def test_compact_model_matches_oracle(n, L, k, k_in, r, D, F, bits, B):
    w = WL.Workload(name="t", n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F, bits=bits, B=B,
                    seed=3000 + n + r)
    o = O.Oracle(n, L, k, k_in, r, D)
    X, Wt, cls = WL.features(w.seed, B, F), WL.projection(w.seed, D, F), WL.classes(w.seed, k, D)
    s, ogk = o.keygen(w.seed)
    omodel = o.encrypt_model_seeded_ntt(w.seed, cls, s)
    H, _, out = o.infer(X, Wt, omodel, ogk, w.shift, bits)

    ctx = _compact_ctx(w, B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    assert np.array_equal(ctx.model_to_host_coeff(model), omodel)
    gX, gW = _dev(X), _dev(Wt)
    got = ctx.infer(gX, gW, model, gk)
    ctx.device_status()
    assert np.array_equal(_u32(got).reshape(out.shape), out)
    assert np.array_equal(_u32(ctx.decrypt_scores(sk, got, B)), O.clear_scores(H, cls))
    if o.groups(B) >= 2:  # the chunked pass regenerates the same c1 per chunk
        ctx.tune_set("chunk", 7)
        assert torch.equal(ctx.infer(gX, gW, model, gk), got)
    ctx.close()


def test_compact_model_packed_clients_match_oracle():
    sizes = [5, 0, 300, 17, 64, 1, 129]
    w = WL.Workload(name="t", n=1024, L=3, k=3, k_in=1, r=4, D=100, F=32, bits=8,
                    B=sum(sizes), seed=78)
    Xs = [WL.features(w.seed, b, w.F, batch=i) for i, b in enumerate(sizes)]
    Wt, cls = WL.projection(w.seed, w.D, w.F), WL.classes(w.seed, w.k, w.D)
    ctx = _compact_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    out = ctx.infer_multi([_dev(x) for x in Xs], _dev(Wt), model, gk)
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    s, ogk = o.keygen(w.seed)
    _, _, oout = o.infer(np.concatenate(Xs), Wt, o.encrypt_model_seeded_ntt(w.seed, cls, s),
                         ogk, w.shift, w.bits)
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    ctx.close()


def test_paths_without_the_compact_model_refuse_it():
    w = WL.config("small")
    ctx = _compact_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(WL.features(w.seed, w.B, w.F)),
                                         _dev(WL.projection(w.seed, w.D, w.F))))
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    for mode in (1, 3):
        ctx.tune_set("mac_mode", mode)
        with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
            ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.tune_set("mac_mode", 2)
    assert torch.equal(ctx.ptct_similarity(pt, w.B, model, gk), ref)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, w.B, model, gk, torch.empty_like(ref))
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        ctx.model_to_seeded(model)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        ctx.tune_set("layout", 1)
    ctx.tune_set("model_seed", -1)   # back to the full model
    assert ctx.tune_get("model_seed") == -1
    ctx.close()
