"""The digit model ("model_digits" 1): the encrypted model stored as the fp16 tensor-core
operand of its signed base-256 digits and read by the digit-outer-product
multiply-accumulate (8 coefficients x 16 groups per CTA, model blocks multicast across
a cluster of group blocks).  Every result must equal the oracle's exactly: the model
converted back to residues, the score ciphertexts (ragged group blocks, every cluster
size, two exact windows of plaintexts, 2 to 32 outputs), the decrypted scores, the
packed multi-client pass and the full-size dense batch (by the oracle's digests); and
the entry points that do not take the digit model must refuse it."""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _digit_ctx(w, B, cluster=0, **kw):
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, max(B, 1), **kw)
    ctx.tune_set("model_digits", 1)
    assert ctx.tune_get("model_digits") == 1
    ctx.tune_set("mac_cluster", cluster)
    # per (limb, coefficient, 16 plaintexts) an operand tile of 4 digits x 16 outputs
    # (k/k_in <= 8) or x 32 outputs, 16 fp16 columns
    rows = 64 if 2 * ctx.Kp <= 16 else 128
    assert E.lib().ephdc_model_bytes(ctx.ctx) == w.L * w.n * ((ctx.P + 15) // 16) * rows * 32
    return ctx


LAYOUTS = [
    # n, L, k, k_in, r, D, F, bits, B, cluster
    (1024, 2, 2, 2, 1, 50, 32, 8, 700, 0),       # 2 outputs, 2 groups, ragged step
    (1024, 3, 3, 1, 4, 41, 16, 4, 600, 0),       # 6 outputs, 3 groups, P = 11 (one step)
    (2048, 2, 7, 7, 2, 33, 64, 8, 300, 0),       # 7 packed classes, 3 groups of 146
    (4096, 3, 2, 1, 16, 300, 48, 6, 1000, 0),    # 4 rotations, G = 4 with a partial tail
    (1024, 4, 16, 1, 2, 700, 32, 8, 17, 0),      # 32 outputs (every model row), B < cap
    (1024, 2, 4, 1, 1, 1100, 32, 8, 1500, 0),    # P = 1100: two exact windows
    (1024, 2, 12, 1, 4, 64, 32, 8, 5120, 0),     # P = 16 exactly, 24 outputs, 2 group blocks
    (1024, 2, 4, 1, 8, 160, 32, 8, 5115, 0),     # G = 40: 3 group blocks in a cluster of 4
    (1024, 2, 4, 1, 8, 160, 32, 8, 8957, 0),     # G = 70: clusters of 4, 3 CTAs without groups
    (1024, 2, 4, 1, 8, 160, 32, 8, 8957, 1),     # the same without clusters
    (1024, 2, 4, 1, 8, 160, 32, 8, 8957, 2),     # clusters of 2
    (1024, 2, 4, 1, 8, 160, 32, 8, 8957, 8),     # one cluster of 8 (3 CTAs without groups)
    (1024, 2, 8, 1, 4, 200, 32, 8, 4000, 0),     # 16 outputs: every lane 0-15 of a 64-row tile
    (1024, 2, 9, 1, 4, 200, 32, 8, 4000, 0),     # 18 outputs: the smallest 128-row tile
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B,cluster", LAYOUTS)
def test_digit_model_matches_oracle(n, L, k, k_in, r, D, F, bits, B, cluster):
    w = WL.Workload(name="t", n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F, bits=bits, B=B,
                    seed=4000 + n + r + k)
    o = O.Oracle(n, L, k, k_in, r, D)
    X, Wt, cls = WL.features(w.seed, B, F), WL.projection(w.seed, D, F), WL.classes(w.seed, k, D)
    s, ogk = o.keygen(w.seed)
    omodel = o.encrypt_model(w.seed, cls, s)
    H, _, out = o.infer(X, Wt, omodel, ogk, w.shift, bits)

    ctx = _digit_ctx(w, B, cluster)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    assert np.array_equal(ctx.model_to_host_coeff(model), omodel)
    gX, gW = _dev(X), _dev(Wt)
    got = ctx.infer(gX, gW, model, gk)
    ctx.device_status()
    assert np.array_equal(_u32(got).reshape(out.shape), out)
    pt = ctx.encode_plain(ctx.hdc_encode(gX, gW))
    ctx.tune_set("mac_mode", 4)
    assert torch.equal(ctx.ptct_similarity(pt, B, model, gk), got)
    assert np.array_equal(_u32(ctx.decrypt_scores(sk, got, B)), O.clear_scores(H, cls))
    ctx.close()


@pytest.mark.parametrize("fill", ["q_minus_1", "max_negative_digits", "random"])
def test_digit_model_exact_at_extreme_residues(fill):
    """The digit-model product against the 64-bit CUDA-core one on hand-made plaintexts
    and models (converted to digits by bfv_model_to_digits): every residue q_l - 1, every
    residue with the most negative balanced digits a residue below 2^30 can have
    (8355712: digits -128, -128, -128, 1; a full window of them sums 1024 x 2^14 = 2^24
    in one accumulator), or random residues; 32 outputs, 40 groups (3 group blocks in a
    cluster of 4), P = 1100 (a full and a partial window)."""
    w = WL.Workload(name="t", n=1024, L=2, k=16, k_in=1, r=1, D=1100, F=32, bits=8,
                    B=40 * 1024, seed=6)
    std = E.Context.for_workload(w)
    G, P, L, n = std.groups(w.B), std.P, w.L, w.n
    assert G == 40 and P == 1100
    rng = np.random.default_rng(10)
    q = np.array(std.q, dtype=np.uint64)

    def make(shape):
        if fill == "q_minus_1":
            a = np.broadcast_to((q - 1).reshape(L, 1), shape[:-2] + (L, n))
        elif fill == "max_negative_digits":
            a = np.full(shape, 8355712, np.uint64)
        else:
            a = rng.integers(0, 1 << 62, size=shape, dtype=np.uint64) % q.reshape(L, 1)
        return _dev(np.ascontiguousarray(a).astype(np.uint32).view(np.int32))

    pt = make((G, P, L, n))
    model = make((P, std.Kp, 2, L, n))
    std.tune_set("mac_mode", 1)
    ref = std.ptct_similarity(pt, w.B, model, None)
    dig = _digit_ctx(w, w.B)
    mdig = dig.model_to_digits(model)
    assert np.array_equal(dig.model_to_host_coeff(mdig), std.model_to_host_coeff(model))
    got = dig.ptct_similarity(pt, w.B, mdig, None)
    dig.device_status()
    assert torch.equal(got, ref)
    std.close()
    dig.close()


def test_digit_model_packed_clients_match_oracle():
    sizes = [5, 0, 300, 17, 64, 1, 129]
    w = WL.Workload(name="t", n=1024, L=3, k=3, k_in=1, r=4, D=100, F=32, bits=8,
                    B=sum(sizes), seed=79)
    Xs = [WL.features(w.seed, b, w.F, batch=i) for i, b in enumerate(sizes)]
    Wt, cls = WL.projection(w.seed, w.D, w.F), WL.classes(w.seed, w.k, w.D)
    ctx = _digit_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    out = ctx.infer_multi([_dev(x) for x in Xs], _dev(Wt), model, gk)
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    s, ogk = o.keygen(w.seed)
    _, _, oout = o.infer(np.concatenate(Xs), Wt, o.encrypt_model(w.seed, cls, s), ogk,
                         w.shift, w.bits)
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    ctx.close()


def test_entry_points_without_the_digit_model_refuse_it():
    w = WL.config("small")
    ctx = _digit_ctx(w, w.B)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(WL.features(w.seed, w.B, w.F)),
                                         _dev(WL.projection(w.seed, w.D, w.F))))
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    for mode in (1, 2, 3):
        ctx.tune_set("mac_mode", mode)
        with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
            ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.tune_set("mac_mode", 4)
    assert torch.equal(ctx.ptct_similarity(pt, w.B, model, gk), ref)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, w.B, model, gk, torch.empty_like(ref))
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
        ctx.model_to_seeded(model)
    for knob, v in (("layout", 1), ("model_seed", 5)):
        with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):
            ctx.tune_set(knob, v)
    ctx.tune_set("model_digits", 0)
    with pytest.raises(E.EphdcError, match="EPHDC_EUNSUPPORTED"):   # mode 4 needs digits
        ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.close()


@pytest.mark.slow
def test_dense65536_digit_model_full_size_digests():
    """65536 queries, n = 16384, 6 primes, 16 classes, 64 groups with the digit model:
    the score ciphertexts of groups 0 and 63 against the oracle's digests."""
    w = WL.config("dense65536")
    ctx = _digit_ctx(w, w.B)
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
