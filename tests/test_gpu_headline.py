"""The face1024 throughput step exactly as it is timed: 16 consecutive 1024-query
batches (one 16384-row feature array) packed into one pass of 16 groups, the
multi-group MAC under every tiled schedule the autotuner may pick for 16 groups,
four contexts with their own scratch on four streams sharing the resident model and
rotation keys.  Groups 0 and 15 of every run are compared word for word with SHA-256
digests of the oracle's score ciphertexts (tests/golden/make_face1024x16_digests.py,
oracle only), and all 16 groups of every run with each other."""
import hashlib
import os

import numpy as np
import pytest
import torch

from paper_2511_00737_gb300 import autotune as AT
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "face1024x16_group_digests.txt")
BATCHES = 16
STREAMS = 4


def _digests():
    with open(GOLDEN) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return [(int(g), int(first), int(count), d) for g, first, count, d in rows]


def _check_groups(ctx, w, out, digests):
    words = out.cpu().numpy().view(np.uint32).reshape(-1, ctx.Kp, 2, w.L, w.n)
    assert words.shape[0] == BATCHES
    for g, first, count, digest in digests:
        assert first == g * ctx.cap and count == ctx.cap
        got = np.ascontiguousarray(words[g], dtype="<u4")
        assert hashlib.sha256(got.tobytes()).hexdigest() == digest, g


@pytest.mark.slow
def test_face1024_throughput_step_every_tiled_schedule():
    w = WL.config("face1024")
    B = BATCHES * w.B
    dev = torch.device("cuda")
    ctxs = [E.Context.for_workload(w, max_batch=B) for _ in range(STREAMS)]
    ctx = ctxs[0]
    assert ctx.groups(B) == BATCHES
    sk, gk = ctx.keygen(w.seed)
    cls = torch.from_numpy(WL.classes(w.seed, w.k, w.D)).to(dev)
    model = ctx.encrypt_model(cls, sk, w.seed)
    Wt = torch.from_numpy(WL.projection(w.seed, w.D, w.F)).to(dev)
    X = torch.from_numpy(WL.features(w.seed, B, w.F, batch=0)).to(dev)
    digests = _digests()
    assert [d[0] for d in digests] == [0, BATCHES - 1]

    tiled = [c for c in AT.candidates(ctx, BATCHES) if c["mac_mode"] == 2]
    assert {"mac_mode": 2, "mac_tile": 4043215} in tiled
    # the streaming kernel and the tensor-core product ride along as further schedules
    scheds = tiled + [{"mac_mode": 1, "mac_splits": 0}, {"mac_mode": 3}]
    streams = [torch.cuda.Stream(device=dev) for _ in range(STREAMS)]
    outs = [cx.out_ct(B) for cx in ctxs]
    ref = None
    for first in range(0, len(scheds), STREAMS):
        batch = scheds[first:first + STREAMS]
        torch.cuda.synchronize()
        for j, knobs in enumerate(batch):
            AT.apply(ctxs[j], {"mac_mode": 0, "mac_splits": 0, **knobs})
            ctxs[j].tune_set("ntt_plan", (first // STREAMS + j) % 3)
            outs[j].fill_(-1)
        torch.cuda.synchronize()
        for j in range(len(batch)):
            with torch.cuda.stream(streams[j]):
                ctxs[j].infer(X, Wt, model, gk, out=outs[j])
        torch.cuda.synchronize()
        for j, knobs in enumerate(batch):
            ctxs[j].device_status()
            if ref is None:
                _check_groups(ctx, w, outs[j], digests)
                ref = outs[j].clone()
            assert torch.equal(outs[j], ref), knobs
    # digests once more on the tiling the autotuner picks for this step on a GB300
    # (4 groups and 4 outputs per warp, 32 groups per CTA, 15 plaintexts per chunk)
    AT.apply(ctx, {"mac_mode": 2, "mac_tile": 4043215})
    _check_groups(ctx, w, ctx.infer(X, Wt, model, gk), digests)
    # the pass in plaintext-index chunks (encode a chunk of every group, accumulate it,
    # next chunk): the same ciphertexts, with a ragged last chunk (1250 = 52 x 24 + 2)
    for chunk in (24, 125):
        ctx.tune_set("chunk", chunk)
        got = ctx.infer(X, Wt, model, gk)
        ctx.device_status()
        assert torch.equal(got, ref), chunk
    ctx.tune_set("chunk", 0)
    for cx in ctxs:
        cx.close()
