"""Host logic of the multiply-accumulate autotuner (no GPU): which schedules it offers
for each storage form of the plaintexts and the model, so that it never times a
schedule the context would refuse, and the cache key separates the forms."""
import pytest

from paper_2511_00737_gb300 import autotune as AT


class FakeCtx:
    """The knobs and sizes candidates() and _key() read."""

    def __init__(self, Kp=16, layout=0, model_seed=-1, model_digits=0):
        self.Kp, self.n, self.L, self.k, self.k_in, self.r, self.device = Kp, 8192, 4, Kp, 1, 8, 0
        self.knobs = {"layout": layout, "model_seed": model_seed, "model_digits": model_digits}

    def tune_get(self, k):
        return self.knobs[k]


def modes(cands):
    return sorted({c["mac_mode"] for c in cands})


def test_residue_model_offers_streaming_tiled_and_tensor_cores():
    c = AT.candidates(FakeCtx(Kp=16), 64)
    assert modes(c) == [1, 2, 3]
    assert all("mac_cluster" not in k for k in c)
    # a single group: no multi-group schedules
    assert modes(AT.candidates(FakeCtx(Kp=16), 1)) == [1]
    # more than 32 outputs: no tensor-core schedule
    assert 3 not in modes(AT.candidates(FakeCtx(Kp=17), 64))


def test_blocked_layout_offers_only_the_tensor_core_product():
    assert AT.candidates(FakeCtx(layout=1), 64) == [{"mac_mode": 3}]


def test_compact_model_offers_only_the_tiled_product():
    assert modes(AT.candidates(FakeCtx(model_seed=7), 64)) == [2]
    assert AT.candidates(FakeCtx(model_seed=7), 1) == [{"mac_mode": 2}]


@pytest.mark.parametrize("G,clusters", [(1, [1]), (16, [1]), (17, [1, 2]), (32, [1, 2]),
                                        (33, [1, 2, 4]), (64, [1, 2, 4]), (500, [1, 2, 4])])
def test_digit_model_offers_the_digit_product_per_cluster_size(G, clusters):
    c = AT.candidates(FakeCtx(model_digits=1), G)
    assert modes(c) == [4]
    # cluster sizes up to the power of two that covers the 16-group blocks
    assert [k["mac_cluster"] for k in c] == clusters


def test_cache_key_separates_storage_forms(monkeypatch):
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda d: "GPU X")
    keys = {AT._key(FakeCtx(**kw), 64) for kw in
            ({}, {"layout": 1}, {"model_seed": 3}, {"model_digits": 1})}
    assert len(keys) == 4


def test_tuner_skips_schedules_the_device_refuses(monkeypatch):
    """A candidate whose launch fails (EphdcError, e.g. a cluster shape the device cannot
    place) is skipped and the fastest of the others is applied; if none runs, it says so."""
    from paper_2511_00737_gb300.ephdc import EphdcError

    class TunableCtx(FakeCtx):
        def __init__(self, refuse):
            super().__init__(model_digits=1)
            self.refuse, self.set = refuse, {}

        def groups(self, B):
            return B

        def out_ct(self, B):
            return None

        def tune_set(self, k, v):
            self.set[k] = v

        def ptct_similarity_into(self, *a):
            if self.set.get("mac_cluster") in self.refuse:
                raise EphdcError(-4, "cluster cannot be placed")

    # time = cluster size: the refused cluster 1 would have been the fastest
    def timed(fn, reps):
        fn()
        return {1: 1.0, 2: 2.0, 4: 4.0}[ctx.set["mac_cluster"]]

    monkeypatch.setattr(AT, "_time", timed)
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda d: "GPU X")
    ctx = TunableCtx(refuse={1})
    best, ms, table = AT.tune_similarity(ctx, None, 64, None, None, use_cache=False)
    assert best == {"mac_mode": 4, "mac_cluster": 2} and ms == 2.0
    assert [k["mac_cluster"] for _, k in table] == [2, 4]
    assert ctx.set["mac_cluster"] == 2   # the winner is applied last
    ctx = TunableCtx(refuse={1, 2, 4})
    with pytest.raises(RuntimeError, match="no multiply-accumulate schedule"):
        AT.tune_similarity(ctx, None, 64, None, None, use_cache=False)


def test_hdc_tuner_picks_the_fastest_kernel_and_skips_refused_ones(monkeypatch):
    """tune_hdc times every HDC projection kernel (hdc_mode 0..4), skips one the device
    refuses (e.g. a cluster it cannot place), applies the fastest and keys its cache by
    the projection's shape as well."""
    from paper_2511_00737_gb300.ephdc import EphdcError

    class HdcCtx(FakeCtx):
        def __init__(self, refuse):
            super().__init__()
            self.D, self.F, self.refuse = 10000, 608, refuse
            self.knobs["hdc_mode"] = 0

        def groups(self, B):
            return B // 1024

        def tune_set(self, k, v):
            self.knobs[k] = v

        def hdc_encode(self, X, Wt):
            if self.knobs["hdc_mode"] in self.refuse:
                raise EphdcError(-4, "cluster cannot be placed")

    times = {0: 0.20, 1: 0.26, 2: 0.23, 3: 0.21, 4: 0.19}

    def timed(fn, reps):
        fn()
        return times[ctx.knobs["hdc_mode"]]

    class X:
        shape = (16384, 608)

    monkeypatch.setattr(AT, "_time", timed)
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda d: "GPU X")
    ctx = HdcCtx(refuse=set())
    best, ms, table = AT.tune_hdc(ctx, X, None, use_cache=False)
    assert best == {"hdc_mode": 4} and ms == 0.19 and len(table) == 5
    assert ctx.knobs["hdc_mode"] == 4
    ctx = HdcCtx(refuse={4})
    best, ms, table = AT.tune_hdc(ctx, X, None, use_cache=False)
    assert best == {"hdc_mode": 0} and [k["hdc_mode"] for _, k in table] == [0, 3, 2, 1]
    assert ctx.knobs["hdc_mode"] == 0
    ctx = HdcCtx(refuse={0, 1, 2, 3, 4})
    with pytest.raises(RuntimeError, match="no HDC projection kernel"):
        AT.tune_hdc(ctx, X, None, use_cache=False)
