"""Batching of many clients' uneven batches: packing, the tiled multi-group
multiply-accumulate, CUDA-graph replay and the autotuner, against the oracle."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import autotune as AT
from paper_2511_00737_gb300 import batching as BT
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


# n, L, k, k_in, r, D, F, bits; cap = n / r for k_in = 1
SMALL = dict(n=1024, L=3, k=3, k_in=1, r=4, D=100, F=32, bits=8)
SIZES = [5, 0, 300, 17, 64, 1, 129]


def _setup(sizes, seed=77, max_batch=None, **over):
    prm = dict(SMALL, **over)
    w = WL.Workload(name="t", B=sum(sizes), seed=seed, **prm)
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift,
                    max_batch or max(1, w.B))
    Xs = [WL.features(seed, b, w.F, batch=i) for i, b in enumerate(sizes)]
    Wt = WL.projection(seed, w.D, w.F)
    cls = WL.classes(seed, w.k, w.D)
    sk, gk = ctx.keygen(seed)
    model = ctx.encrypt_model(_dev(cls), sk, seed)
    return w, ctx, Xs, Wt, cls, sk, gk, model


def test_packed_requests_match_oracle_on_concatenated_batch():
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(SIZES)
    out = ctx.infer_multi([_dev(x) for x in Xs], _dev(Wt), model, gk)
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    s, ogk = o.keygen(w.seed)
    omodel = o.encrypt_model(w.seed, cls, s)
    Xcat = np.concatenate(Xs)
    H, _, oout = o.infer(Xcat, Wt, omodel, ogk, w.shift, w.bits)
    assert np.array_equal(_u32(out).reshape(oout.shape), oout)
    scores = _u32(ctx.decrypt_scores(sk, out, w.B))
    assert np.array_equal(scores, O.clear_scores(H, cls))
    ctx.device_status()
    ctx.close()


def test_each_request_same_alone_and_in_the_mix():
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(SIZES)
    Wd = _dev(Wt)
    mixed = ctx.infer_multi([_dev(x) for x in Xs], Wd, model, gk)
    mixed_scores = _u32(ctx.decrypt_scores(sk, mixed, w.B))
    pb = BT.PackedBatch(SIZES, ctx.cap)
    for r, x in enumerate(Xs):
        if not len(x):
            continue
        alone = ctx.infer(_dev(x), Wd, model, gk)
        alone_scores = _u32(ctx.decrypt_scores(sk, alone, len(x)))
        assert np.array_equal(mixed_scores[pb.rows(r)], alone_scores)
        assert np.array_equal(alone_scores,
                              O.clear_scores(O.hdc_encode(x, Wt, w.shift, w.bits), cls))
    ctx.close()


def test_tiled_mac_equals_streaming_for_every_tiling():
    sizes = [900, 700, 1000, 33]  # 11 groups of 256
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(sizes, k=7, D=64)
    H = ctx.hdc_encode(_dev(np.concatenate(Xs)), _dev(Wt))
    pt = ctx.encode_plain(H)
    ctx.tune_set("mac_mode", 1)
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    for knobs in AT.candidates(ctx, ctx.groups(w.B)):
        AT.apply(ctx, {"mac_mode": 0, "mac_splits": 0, **knobs})
        got = ctx.ptct_similarity(pt, w.B, model, gk)
        assert torch.equal(got, ref), knobs
    ctx.device_status()
    ctx.close()


def test_graph_replay_equals_eager_and_is_reused():
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(SIZES, max_batch=4 * 256)
    Wd = _dev(Wt)
    eager = BT.GraphedPipeline(ctx, Wd, model, gk, max_groups=4, use_graphs=False)
    graphed = BT.GraphedPipeline(ctx, Wd, model, gk, max_groups=4, use_graphs=True)
    mixes = [Xs, Xs[::-1], [Xs[2], Xs[6]], [Xs[2]]]
    for mix in mixes:
        dmix = [_dev(x) for x in mix]
        a, pa = eager.run(dmix)
        a = a.clone()
        b, pb = graphed.run(dmix)
        torch.cuda.synchronize()
        assert pa.groups == pb.groups
        assert torch.equal(a, b)
        scores = _u32(ctx.decrypt_scores(sk, b, pb.total))
        for r, x in enumerate(mix):
            clear = O.clear_scores(O.hdc_encode(x, Wt, w.shift, w.bits), cls)
            assert np.array_equal(scores[pb.rows(r)], clear)
    assert set(graphed.graphs) == {2, 3}  # 516 queries need 3 groups of 256, 429 and 300 need 2
    ctx.close()


def test_pipelines_on_several_streams_give_the_same_ciphertexts():
    """Consecutive packed steps alternating over three pipelines (each its own context,
    graphs and stream, all sharing the model and keys), launched without any
    synchronisation between them, give each step the ciphertexts of running it alone."""
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(SIZES, max_batch=4 * 256)
    Wd = _dev(Wt)
    ctxs = [ctx] + [E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, 4 * 256)
                    for _ in range(2)]
    pipes = [BT.GraphedPipeline(cx, Wd, model, gk, max_groups=4) for cx in ctxs]
    streams = [torch.cuda.Stream() for _ in ctxs]
    mixes = [Xs, Xs[::-1], [Xs[2], Xs[6]], [Xs[2]], Xs[1:], [Xs[4]]]
    dmixes = [[_dev(x) for x in mix] for mix in mixes]
    alone = []
    for dmix in dmixes:
        out, _ = pipes[0].run(dmix)
        torch.cuda.synchronize()
        alone.append(out.clone())
    torch.cuda.synchronize()
    got = []
    for i, dmix in enumerate(dmixes):    # no synchronisation between the steps
        j = i % 3
        out, _ = pipes[j].launch(dmix, streams[j])
        with torch.cuda.stream(streams[j]):
            got.append(out.clone())      # before this pipeline's next step overwrites it
    torch.cuda.synchronize()
    for i, out in enumerate(got):
        assert torch.equal(out, alone[i]), i
    for cx in ctxs[1:]:
        cx.close()
    ctx.close()


def test_autotuner_picks_a_schedule_and_results_do_not_change(tmp_path, monkeypatch):
    monkeypatch.setattr(AT, "CACHE", str(tmp_path / "tune.json"))
    sizes = [600, 600, 600]
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(sizes, k=2)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(np.concatenate(Xs)), _dev(Wt)))
    ctx.tune_set("mac_mode", 1)
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    best, ms, table = AT.tune_similarity(ctx, pt, w.B, model, gk, reps=2, max_candidates=12)
    assert ms > 0 and len(table) == 12
    assert torch.equal(ctx.ptct_similarity(pt, w.B, model, gk), ref)
    best2, ms2, table2 = AT.tune_similarity(ctx, pt, w.B, model, gk)  # from the cache
    assert best2 == best and table2 == []
    ctx.close()


@pytest.mark.slow
def test_clients64_full_size_sampled():
    """64 clients, log-uniform batch sizes (sum ~ 31.5K), F=768, D=10000, 4-bit HVs,
    7 classes, n=8192, 4 primes: sampled queries' decrypted scores against the clear
    dot products, and the score ciphertexts of three groups (one partial) bit for bit
    against the oracle's (by digest)."""
    w = WL.config("clients64")
    ctx = E.Context.for_workload(w)
    dev = torch.device("cuda")
    Xs = [WL.features(w.seed, b, w.F, batch=i) for i, b in enumerate(w.clients)]
    Wt = WL.projection(w.seed, w.D, w.F)
    cls = WL.classes(w.seed, w.k, w.D)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    out = ctx.infer_multi([_dev(x) for x in Xs], _dev(Wt), model, gk)
    scores = _u32(ctx.decrypt_scores(sk, out, w.B))
    ctx.device_status()
    Xcat = np.concatenate(Xs)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, w.B, 256), [0, w.B - 1]]))
    H = O.hdc_encode(Xcat[rows], Wt, w.shift, w.bits)
    assert np.array_equal(scores[rows], O.clear_scores(H, cls))
    # groups 0, 15 and the partial group 31 bit for bit: digests of the oracle's score
    # ciphertexts on those rows of the concatenated batch
    # (tests/golden/make_clients64_digests.py, oracle only)
    import hashlib
    words = _u32(out).reshape(-1, ctx.Kp, 2, w.L, w.n)
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                          "clients64_group_digests.txt")
    with open(golden) as f:
        digests = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(digests) == 3
    for g, first, count, digest in digests:
        assert int(first) == int(g) * ctx.cap
        assert int(count) == min(ctx.cap, w.B - int(first))
        got = np.ascontiguousarray(words[int(g)], dtype="<u4")
        assert hashlib.sha256(got.tobytes()).hexdigest() == digest, g
    ctx.close()


@pytest.mark.parametrize("k,groups,D", [
    (7, 11, 1200),   # 14 outputs (rows past O zero); P = 300: two 256-windows, ragged chunk
    (5, 40, 300),    # 10 outputs, 40 groups (columns past G zero)
    (16, 9, 520),    # 32 outputs: all 32 rows of every digit block
    (16, 70, 64),    # 32 outputs, 70 groups: two group blocks of 64
    (2, 3, 2100),    # 4 outputs, P = 525: three windows, the last one partial
])
def test_tensor_core_mac_equals_streaming(k, groups, D):
    """The exact byte-split tensor-core product gives the same accumulators (and so the
    same score ciphertexts) as the 64-bit CUDA-core multiply-accumulate."""
    sizes = [256] * groups
    w, ctx, Xs, Wt, cls, sk, gk, model = _setup(sizes, k=k, D=D)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(np.concatenate(Xs)), _dev(Wt)))
    ctx.tune_set("mac_mode", 1)
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.tune_set("mac_mode", 3)
    got = ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.device_status()
    assert torch.equal(got, ref)
    if groups <= 11:
        H = O.hdc_encode(np.concatenate(Xs), Wt, w.shift, w.bits)
        assert np.array_equal(_u32(ctx.decrypt_scores(sk, got, w.B)), O.clear_scores(H, cls))
    ctx.close()


@pytest.mark.parametrize("fill", ["max_negative_digits", "q_minus_1", "random"])
def test_tensor_core_mac_exact_at_extreme_residues(fill):
    """The signed-digit tensor-core product against the 64-bit CUDA-core one on
    hand-made plaintexts and models: every residue q_l - 1, every residue with the
    most negative balanced digits a residue below 2^30 can have (8355712: digits
    -128, -128, -128, 1), or random residues; 32 outputs, 70 groups (two group blocks),
    P = 300 (a full and a partial window)."""
    w = WL.Workload(name="t", n=1024, L=3, k=16, k_in=1, r=4, D=1200, F=32, bits=8,
                    B=70 * 256, seed=5)
    ctx = E.Context.for_workload(w)
    sk, gk = ctx.keygen(w.seed)
    G, P, L, n = ctx.groups(w.B), ctx.P, w.L, w.n
    assert G == 70 and P == 300
    rng = np.random.default_rng(9)
    q = np.array(ctx.q, dtype=np.uint64)

    def make(shape):
        if fill == "q_minus_1":
            a = np.broadcast_to((q - 1).reshape(L, 1), shape[:-2] + (L, n))
        elif fill == "max_negative_digits":
            a = np.full(shape, 8355712, np.uint64)
        else:
            a = rng.integers(0, 1 << 62, size=shape, dtype=np.uint64) % q.reshape(L, 1)
        return _dev(np.ascontiguousarray(a).astype(np.uint32).view(np.int32))

    pt = make((G, P, L, n))
    model = make((P, ctx.Kp, 2, L, n))
    assert (-8421504 + 16777216) == 8355712  # -128 (1 + 2^8 + 2^16) + 2^24
    ctx.tune_set("mac_mode", 1)
    ref = ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.tune_set("mac_mode", 3)
    got = ctx.ptct_similarity(pt, w.B, model, gk)
    ctx.device_status()
    assert torch.equal(got, ref)
    ctx.close()
