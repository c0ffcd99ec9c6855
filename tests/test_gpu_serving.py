"""Serving loop: continuous batching with memory admission; every request's result
equals the clear scores and the result of running it alone."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import serving as SV
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _serve(budget=None, n_req=60, rate=4000.0, slots=2, use_graphs=True, sizes=None):
    w = WL.Workload(name="t", n=1024, L=3, k=3, k_in=1, r=4, D=120, F=32, bits=8, B=0, seed=9)
    dev = torch.device("cuda")
    Wt = WL.projection(w.seed, w.D, w.F)
    cls = WL.classes(w.seed, w.k, w.D)
    keyctx = E.Context.for_workload(w, max_batch=256)
    sk, gk = keyctx.keygen(w.seed)
    model = keyctx.encrypt_model(torch.from_numpy(cls).to(dev), sk, w.seed)
    t, drawn = WL.arrivals(w.seed, n_req, rate_per_s=rate, median=40, max_batch=700)
    if sizes is None:
        sizes = drawn
    t = t[:len(sizes)]
    Xs = [WL.features(w.seed, int(b), w.F, batch=i) for i, b in enumerate(sizes)]
    Xd = [torch.from_numpy(x).to(dev) for x in Xs]
    srv = SV.Server(w, torch.from_numpy(Wt).to(dev), model, gk, slots=slots, max_groups=3,
                    budget_bytes=budget, use_graphs=use_graphs, keep_outputs=True)
    srv.warm()
    wall = srv.run(t, lambda rid: Xd[rid])
    return w, keyctx, sk, gk, model, Wt, cls, Xs, Xd, srv, srv.report(wall)


def _check_results(w, keyctx, sk, srv, Wt, cls, Xs):
    for st in srv.steps:
        out = torch.from_numpy(st.host_out.numpy()).cuda()
        scores = _u32(srv.slots[0].ctx.decrypt_scores(sk, out, st.packed.total))
        for r in st.reqs:
            clear = O.clear_scores(O.hdc_encode(Xs[r.rid], Wt, w.shift, w.bits), cls)
            assert np.array_equal(scores[r.rows], clear), r.rid


def test_serving_results_equal_clear_scores_and_alone():
    w, keyctx, sk, gk, model, Wt, cls, Xs, Xd, srv, rep = _serve()
    assert rep["completed"] + rep["rejected"] == len(Xs) and rep["rejected"] == 0
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    assert any(len(st.reqs) > 1 for st in srv.steps)  # requests were batched together
    _check_results(w, keyctx, sk, srv, Wt, cls, Xs)
    # a few requests alone give the same scores as in their mixed step
    ctx = srv.slots[0].ctx
    for st in srv.steps[:3]:
        out = torch.from_numpy(st.host_out.numpy()).cuda()
        mixed = _u32(ctx.decrypt_scores(sk, out, st.packed.total))
        for r in st.reqs:
            alone = ctx.infer(Xd[r.rid], srv.slots[0].pipe.Wt, model, gk)
            assert np.array_equal(_u32(ctx.decrypt_scores(sk, alone, r.B)), mixed[r.rows])


def test_admission_bounded_by_memory_budget():
    # a 40-query request needs ~73 KB (features + one group of 3 score ciphertexts):
    # 160 KB admits two at a time; the 600-query request (3 groups) never fits
    sizes = [40] * 20 + [600] + [40] * 10
    w, keyctx, sk, gk, model, Wt, cls, Xs, Xd, srv, rep = _serve(budget=160 * 1024, sizes=sizes)
    assert [r.B for r in srv.rejected] == [600]
    assert rep["completed"] == len(sizes) - 1
    assert max(len(st.reqs) for st in srv.steps) <= 2
    assert srv.used == 0
    _check_results(w, keyctx, sk, srv, Wt, cls, Xs)
