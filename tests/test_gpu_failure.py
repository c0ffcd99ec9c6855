"""Failure detection on the device without a fault: a bounded wait that runs out.

`ephdc_wait_selfcheck` launches one thread that waits, through the same bounded
mbarrier wait as the tensor-core pipelines, on a barrier nothing arrives on, with a
limit of 10^5 cycles.  The wait must give up, the status word must report
EPHDC_ETIMEOUT with the self-check's code, the word must clear once read, and the
context must stay usable: the whole client path (tcgen05 projection included) run
after the timeout gives the same ciphertexts as before it, and they decrypt to the
clear scores."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    w = WL.config("small")
    dev = torch.device("cuda")
    ctx = E.Context.for_workload(w)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    cls = WL.classes(w.seed, w.k, w.D)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(torch.from_numpy(cls).to(dev), sk, w.seed)
    Xd, Wd = torch.from_numpy(X).to(dev), torch.from_numpy(Wt).to(dev)
    before = ctx.infer(Xd, Wd, model, gk)
    ctx.device_status()                       # nothing gave up so far

    for limit in (1, 100000):
        ctx.wait_selfcheck(limit)
        with pytest.raises(E.EphdcError) as err:
            ctx.device_status()
        assert err.value.status == -5 and "code 99" in str(err.value)
        ctx.device_status()                   # the word was cleared by the read

    with pytest.raises(E.EphdcError) as err:  # limits out of range are refused on the host
        ctx.wait_selfcheck(0)
    assert err.value.status == -1
    with pytest.raises(E.EphdcError):
        ctx.wait_selfcheck((1 << 31) + 1)

    after = ctx.infer(Xd, Wd, model, gk)
    ctx.device_status()
    assert torch.equal(after, before)
    H = O.hdc_encode(X, Wt, w.shift, w.bits)
    scores = _u32(ctx.decrypt_scores(sk, after, w.B))
    assert np.array_equal(scores, O.clear_scores(H, cls))
    ctx.close()
