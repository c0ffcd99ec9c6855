"""GPU parity: every stage of the CUDA path against the CPU oracle, bit for bit.

All comparisons are exact (integer work): secret key, Galois keys, encrypted model
and every output ciphertext in the coefficient domain, quantised hypervectors,
plaintext polynomials, and decrypted scores, which must also equal the clear
integer dot products mod t.  Calls go through the C ABI (via the ctypes binding).
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

pytestmark = pytest.mark.gpu

T = 65537


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _lifted(m, q):
    """centred lift of plaintext coefficients (mod t) into each limb, [..][L][n]"""
    mm = m.astype(np.int64)
    v = np.where(mm <= (T - 1) // 2, mm, mm - T)
    return np.stack([np.mod(v, p) for p in q], axis=-2).astype(np.uint32)


class Case:
    """One configuration run on both sides from the same seeded inputs."""

    def __init__(self, w, B=None, seed=None):
        self.w = w
        self.B = B if B is not None else w.B
        self.seed = seed if seed is not None else w.seed
        self.o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
        self.ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift,
                             max(self.B, 1))
        self.X = WL.features(self.seed, self.B, w.F)
        self.Wt = WL.projection(self.seed, w.D, w.F)
        self.cls = WL.classes(self.seed, w.k, w.D)

    def oracle_all(self):
        o = self.o
        self.s, self.gk = o.keygen(self.seed)
        self.model = o.encrypt_model(self.seed, self.cls, self.s)
        self.H, self.m, self.out = o.infer(self.X, self.Wt, self.model, self.gk, self.w.shift,
                                           self.w.bits)
        return self

    def gpu_all(self):
        c = self.ctx
        self.g_sk, self.g_gk = c.keygen(self.seed)
        self.g_model = c.encrypt_model(_dev(self.cls), self.g_sk, self.seed)
        self.g_X, self.g_Wt = _dev(self.X), _dev(self.Wt)
        self.g_H = c.hdc_encode(self.g_X, self.g_Wt)
        self.g_pt = c.encode_plain(self.g_H)
        self.g_out = c.ptct_similarity(self.g_pt, self.B, self.g_model, self.g_gk)
        torch.cuda.synchronize()
        return self


@pytest.fixture(scope="module")
def small():
    return Case(WL.config("small")).oracle_all().gpu_all()


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("n,L", [(1024, 2), (4096, 3), (8192, 4), (16384, 6)])
def test_ntt_natural_order_matches_oracle(n, L):
    ctx = E.Context(n, L, 2, 1, 1, 64, 16, 8, 0, 4)
    rng = np.random.default_rng(n)
    for limb in range(L + 1):
        p = ctx.q[limb] if limb < L else T
        psi = O.root_2n(p, n)
        a = rng.integers(0, p, size=(3, n)).astype(np.uint32)
        ga = _dev(a.view(np.int32))
        ctx.ntt_natural(ga, limb)
        got = _u32(ga)
        for r in range(3):
            assert np.array_equal(got[r], O.ntt(a[r], p, psi))
        ctx.ntt_natural(ga, limb, inverse=True)
        assert np.array_equal(_u32(ga), a)
    ctx.close()


# ---------------------------------------------------------------- server side
def test_secret_and_galois_keys_match_oracle(small):
    c = small
    assert np.array_equal(c.ctx.sk_to_host(c.g_sk), c.s)
    assert np.array_equal(c.ctx.gk_to_host_coeff(c.g_gk), c.gk)


def test_encrypted_model_matches_oracle(small):
    c = small
    got = c.ctx.ct_to_host_coeff(c.g_model, c.o.P * c.o.Kp)
    assert np.array_equal(got.reshape(c.model.shape), c.model)


# ---------------------------------------------------------------- client path
def test_hdc_encode_matches_oracle(small):
    assert np.array_equal(small.g_H.cpu().numpy(), small.H)


# persistent 128x256 (3 / 4 stages: 0 / 3; clusters of two sharing each W slice: 4), one
# tile per CTA (1), persistent 128x128 (2)
@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("B,D,F,bits,shift", [(1, 257, 16, 8, 0), (300, 1000, 96, 4, 6),
                                              (129, 130, 608, 8, 5), (2000, 64, 1024, 2, 9),
                                              (8000, 1200, 608, 8, 5)])
def test_hdc_encode_ragged_shapes(B, D, F, bits, shift, mode):
    """Ragged rows and columns; the last shape has 630 output tiles, so each persistent
    CTA (two per SM) takes two or three tiles and reuses its TMEM accumulators.  In
    clusters of two (mode 4) an odd count of 128-row blocks leaves the second CTA of
    the last pairs without rows, and D = 64 leaves its half of every W slice empty."""
    ctx = E.Context(1024, 2, 2, 1, 1, D, F, bits, shift, B)
    ctx.tune_set("hdc_mode", mode)
    X = WL.features(B + D, B, F)
    Wt = WL.projection(B + D, D, F)
    X[0] = 127
    H = ctx.hdc_encode(_dev(X), _dev(Wt))
    assert np.array_equal(H.cpu().numpy(), O.hdc_encode(X, Wt, shift, bits))
    ctx.device_status()
    ctx.close()


def test_hdc_encode_extreme_magnitudes_exact():
    """|X Wt^T| up to 127 * F with F = 1024: the fp16-operand tensor-core product must
    still be the exact integer (all partial sums < 2^24)."""
    B, D, F = 256, 384, 1024
    X = WL.features(5, B, F)
    Wt = WL.projection(5, D, F)
    X[:64] = 127
    Wt[:100] = -1
    Wt[100:200] = 1
    for shift, bits, mode in [(0, 8, 0), (10, 8, 1), (14, 4, 2), (5, 8, 4)]:
        ctx = E.Context(1024, 2, 2, 1, 1, D, F, bits, shift, B)
        ctx.tune_set("hdc_mode", mode)
        H = ctx.hdc_encode(_dev(X), _dev(Wt))
        assert np.array_equal(H.cpu().numpy(), O.hdc_encode(X, Wt, shift, bits))
        ctx.device_status()
        ctx.close()


def test_plaintexts_match_oracle(small):
    c = small
    G = c.o.groups(c.B)
    got = c.ctx.plain_to_host_coeff(c.g_pt, G * c.o.P)
    assert np.array_equal(got, _lifted(c.m.reshape(G * c.o.P, c.o.n), c.o.q))


def test_score_ciphertexts_match_oracle(small):
    c = small
    got = _u32(c.g_out).reshape(c.out.shape)
    assert np.array_equal(got, c.out)


def test_decrypted_scores_equal_clear_dot_products(small):
    c = small
    scores = c.ctx.decrypt_scores(c.g_sk, c.g_out, c.B)
    clear = O.clear_scores(c.H, c.cls)
    assert np.array_equal(_u32(scores), clear)
    assert np.array_equal(c.o.decrypt_scores(c.s, c.out, c.B), clear)


def test_fused_infer_equals_step_calls(small):
    c = small
    out = c.ctx.infer(c.g_X, c.g_Wt, c.g_model, c.g_gk)
    assert torch.equal(out, c.g_out)


# ---------------------------------------------------------------- layouts and tails
LAYOUTS = [
    # n, L, k, k_in, r, D, F, bits, B
    (1024, 2, 2, 2, 1, 50, 32, 8, 700),     # paper layout, r = 1, no rotation, 2 groups
    (1024, 3, 3, 1, 4, 41, 16, 4, 600),     # one class per ct, ragged D (41 = 10*4 + 1)
    (2048, 2, 7, 7, 2, 33, 64, 8, 300),     # 7 packed classes, cap_row = floor(512/7)
    (4096, 3, 2, 1, 16, 300, 48, 6, 1000),  # 4 rotations, G = 4 with a partial tail
    (1024, 4, 5, 5, 8, 100, 32, 8, 17),     # 3 rotations, cap_row = 12, B < cap
    # D a multiple of r: whole query rows packed by vector loads, partial last group
    (2048, 2, 3, 1, 8, 96, 32, 8, 300),     # 8-byte rows, G = 2 (256 + 44)
    (4096, 3, 2, 1, 16, 320, 48, 8, 200),   # 16-byte rows, B < cap
    (2048, 2, 2, 2, 4, 100, 32, 8, 300),    # layout A rows: 4 bytes, 2 positions each
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B", LAYOUTS)
def test_layouts_end_to_end(n, L, k, k_in, r, D, F, bits, B):
    w = WL.Workload(name="t", n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F, bits=bits, B=B,
                    seed=1000 + n + r)
    c = Case(w).oracle_all().gpu_all()
    assert np.array_equal(c.g_H.cpu().numpy(), c.H)
    assert np.array_equal(_u32(c.g_out).reshape(c.out.shape), c.out)
    got = c.ctx.ct_to_host_coeff(c.g_model, c.o.P * c.o.Kp)
    assert np.array_equal(got.reshape(c.model.shape), c.model)
    scores = _u32(c.ctx.decrypt_scores(c.g_sk, c.g_out, B))
    assert np.array_equal(scores, O.clear_scores(c.H, c.cls))
    c.ctx.close()


def test_batch_of_one_and_partial_group():
    w = WL.config("small")
    for B in (1, 9):
        c = Case(w, B=B).oracle_all().gpu_all()
        assert np.array_equal(_u32(c.g_out).reshape(c.out.shape), c.out)
        c.ctx.close()


# ---------------------------------------------------------------- errors
def test_errors_are_reported_not_faulted(small):
    c = small
    with pytest.raises(E.EphdcError, match="EPHDC_ENOMEM"):
        E.hdc_encode(c.ctx.ctx, c.g_X, c.g_Wt, c.B + 1000, c.g_H)
    bad = torch.empty(c.g_H.numel() + 16, dtype=torch.int8, device="cuda")[1:]
    with pytest.raises(E.EphdcError, match="EPHDC_EINVAL"):
        E.hdc_encode(c.ctx.ctx, c.g_X, c.g_Wt, c.B, bad)
    with pytest.raises(E.EphdcError, match="EPHDC_EINVAL"):
        E.Context(1000, 2, 2, 1, 1, 10, 16, 8, 0, 4)


# ---------------------------------------------------------------- full size
@pytest.mark.slow
@pytest.mark.parametrize("name", ["face1024", "face1024_a"])
def test_face1024_full_size_bit_exact(name):
    """1024 queries, F=608, D=10000, 8-bit HVs, 2 classes, n=8192, 4 primes, in layout B
    (k_in = 1, r = 8) and the paper's layout A (k_in = 2, r = 4): every score ciphertext
    bit-exact, scores equal to the clear dot products mod t."""
    c = Case(WL.config(name)).oracle_all().gpu_all()
    assert np.array_equal(c.g_H.cpu().numpy(), c.H)
    assert np.array_equal(_u32(c.g_out).reshape(c.out.shape), c.out)
    scores = _u32(c.ctx.decrypt_scores(c.g_sk, c.g_out, c.B))
    assert np.array_equal(scores, O.clear_scores(c.H, c.cls))
    # the fused call agrees with the step calls
    out = c.ctx.infer(c.g_X, c.g_Wt, c.g_model, c.g_gk)
    assert torch.equal(out, c.g_out)
    c.ctx.close()


@pytest.mark.slow
def test_dense65536_full_size_sampled():
    """65536 queries, F=1024, D=16384, 8-bit HVs, 16 classes, n=16384, 6 primes, layout
    k_in=1 r=16 (64 groups, 4 rotations): sampled hypervector rows against the oracle's
    projection, every sampled query's 16 decrypted scores against the clear dot
    products mod t, and the score ciphertexts of groups 0 and 63 bit for bit against
    the oracle's (by digest)."""
    w = WL.config("dense65536")
    ctx = E.Context.for_workload(w)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    cls = WL.classes(w.seed, w.k, w.D)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(cls), sk, w.seed)
    gX, gW = _dev(X), _dev(Wt)
    H = ctx.hdc_encode(gX, gW)
    out = ctx.infer(gX, gW, model, gk)
    scores = _u32(ctx.decrypt_scores(sk, out, w.B))
    ctx.device_status()
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([rng.integers(0, w.B, 192), [0, 1023, 1024, w.B - 1]]))
    Ho = O.hdc_encode(X[rows], Wt, w.shift, w.bits)
    assert np.array_equal(H.cpu().numpy()[rows], Ho)
    assert np.array_equal(scores[rows], O.clear_scores(Ho, cls))
    # groups 0 and 63 bit for bit: the digests of the oracle's score ciphertexts for
    # those groups (tests/golden/make_dense65536_digests.py, oracle only)
    import hashlib
    words = _u32(out).reshape(-1, ctx.Kp, 2, w.L, w.n)
    with open(os.path.join(GOLDEN, "dense65536_group_digests.txt")) as f:
        digests = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(digests) == 2
    for g, first, count, digest in digests:
        assert int(first) == int(g) * ctx.cap and int(count) == ctx.cap
        got = np.ascontiguousarray(words[int(g)], dtype="<u4")
        assert hashlib.sha256(got.tobytes()).hexdigest() == digest, g
    # the tensor-core and the tiled CUDA-core products give the same ciphertexts
    for mode in (3, 2):
        ctx.tune_set("mac_mode", mode)
        assert torch.equal(ctx.infer(gX, gW, model, gk), out), mode
    ctx.device_status()
    ctx.close()


@pytest.mark.parametrize("n,L,r", [(2048, 2, 2), (4096, 3, 8), (8192, 4, 8), (16384, 6, 16)])
def test_every_ntt_plan_gives_the_same_plaintexts(n, L, r):
    """The pass schedules of the encoding transforms differ only in speed."""
    w = WL.Workload(name="t", n=n, L=L, k=2, k_in=1, r=r, D=96, F=32, bits=8, B=300, seed=n)
    ctx = E.Context.for_workload(w)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    H = ctx.hdc_encode(_dev(X), _dev(Wt))
    ref = None
    for v in (0, 1, 2):
        ctx.tune_set("ntt_plan", v)
        pt = ctx.encode_plain(H)
        if ref is None:
            ref = pt
            o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
            m = o.encode_plain(O.hdc_encode(X, Wt, w.shift, w.bits))
            G = o.groups(w.B)
            got = ctx.plain_to_host_coeff(pt, G * o.P)
            assert np.array_equal(got, _lifted(m.reshape(G * o.P, n), o.q))
        else:
            assert torch.equal(pt, ref), v
    ctx.close()


@pytest.mark.parametrize("r,k_in,D,B", [(8, 1, 96, 300), (16, 1, 96, 300), (4, 2, 100, 300),
                                         (8, 1, 96, 1), (4, 2, 100, 257)])
def test_query_row_pack_matches_oracle(r, k_in, D, B):
    """Shapes whose query rows are packed by vector loads (D a multiple of r), with full,
    partial and single-query groups: plaintexts equal to the oracle's."""
    w = WL.Workload(name="t", n=2048, L=2, k=2, k_in=k_in, r=r, D=D, F=32, bits=8, B=B,
                    seed=77 + r + B)
    ctx = E.Context.for_workload(w)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    pt = ctx.encode_plain(ctx.hdc_encode(_dev(X), _dev(Wt)))
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    m = o.encode_plain(O.hdc_encode(X, Wt, w.shift, w.bits))
    G = o.groups(w.B)
    got = ctx.plain_to_host_coeff(pt, G * o.P)
    assert np.array_equal(got, _lifted(m.reshape(G * o.P, w.n), o.q))
    ctx.close()


@pytest.mark.parametrize("name", ["small", "face1024"])
def test_launch_count_matches_profiler(name):
    """The library's own kernel-launch count for one fused call (the figure bench.py
    reports as gpu_launches) equals the number of this library's kernels a CUDA
    activity trace sees."""
    w = WL.config(name)
    ctx = E.Context.for_workload(w)
    X = _dev(WL.features(w.seed, w.B, w.F))
    Wt = _dev(WL.projection(w.seed, w.D, w.F))
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    ctx.infer(X, Wt, model, gk)  # first call: lazy set-up outside the trace
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]):  # the first session may come up late
        torch.zeros(1, device="cuda").add_(1)
        torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        ctx.infer(X, Wt, model, gk)
        torch.cuda.synchronize()
    _, _, claimed = ctx.profile_read()
    ctx.profile(False)
    # raw activity records: kernels launched outside torch ops have no CPU-side parent
    raw = []
    try:
        for e in prof.profiler.kineto_results.events():
            raw.append((e.name(), str(e.device_type())))
    except AttributeError:
        raw = [(e.name, str(e.device_type)) for e in prof.events()]

    def ours(n):
        for pre in ("void ", "(anonymous namespace)::", "<unnamed>::", "ephdc::"):
            n = n.replace(pre, "")
        return n.startswith("k_")
    names = [n for n, d in raw if "CUDA" in d and ours(n)]
    if not names:
        pytest.skip("the CUDA activity trace recorded none of this library's kernels "
                    "(%d records, e.g. %s)" % (len(raw), raw[:3]))
    assert claimed == len(names), sorted(set(names))
    ctx.close()


def test_launch_count_of_packed_requests_matches_profiler():
    """The same check for many clients' batches packed into one call (70 requests: two
    gathers of up to 64 requests each)."""
    w = WL.config("small")
    sizes = [1 + (7 * i) % 13 for i in range(70)]
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, sum(sizes) + 64)
    Wt = _dev(WL.projection(w.seed, w.D, w.F))
    Xs = [_dev(WL.features(w.seed, b, w.F, batch=i)) for i, b in enumerate(sizes)]
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(_dev(WL.classes(w.seed, w.k, w.D)), sk, w.seed)
    ctx.infer_multi(Xs, Wt, model, gk)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]):
        torch.zeros(1, device="cuda").add_(1)
        torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        ctx.infer_multi(Xs, Wt, model, gk)
        torch.cuda.synchronize()
    _, _, claimed = ctx.profile_read()
    ctx.profile(False)
    raw = []
    try:
        for e in prof.profiler.kineto_results.events():
            raw.append((e.name(), str(e.device_type())))
    except AttributeError:
        raw = [(e.name, str(e.device_type)) for e in prof.events()]

    def ours(n):
        for pre in ("void ", "(anonymous namespace)::", "<unnamed>::", "ephdc::"):
            n = n.replace(pre, "")
        return n.startswith("k_")
    names = [n for n, d in raw if "CUDA" in d and ours(n)]
    if not names:
        pytest.skip("the CUDA activity trace recorded none of this library's kernels")
    assert sum("gather_widen" in n for n in names) == 2
    assert claimed == len(names), sorted(set(names))
    ctx.close()
