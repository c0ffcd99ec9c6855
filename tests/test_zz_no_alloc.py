"""The no-allocation similarity entry point against the allocating one.

bfv_ptct_similarity_noalloc exists for callers that must not allocate device
memory while they serve (a loop whose admission control has already budgeted all
of HBM, a process whose memory pool owns the device, or a latency-critical loop
that cannot take the device-wide synchronisation a cudaMalloc/cudaFree may cause).
Its scratch is a fixed array compiled into the library.  This file is collected
last so that a failure here leaves every other test already run; it needs nothing
from the other tests and passes in a fresh process too.
"""
import numpy as np
import pytest
import torch

from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


def _setup(w, B):
    ctx = E.Context(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift, B)
    dev = torch.device("cuda")
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(torch.from_numpy(WL.classes(w.seed, w.k, w.D)).to(dev), sk, w.seed)
    X = torch.from_numpy(WL.features(w.seed, B, w.F)).to(dev)
    Wt = torch.from_numpy(WL.projection(w.seed, w.D, w.F)).to(dev)
    pt = ctx.encode_plain(ctx.hdc_encode(X, Wt))
    return ctx, model, gk, pt


@pytest.mark.parametrize("name,B", [("small", 16), ("face1024", 1024), ("face1024", 700)])
def test_noalloc_matches_allocating_entry_point_twice(name, B):
    w = WL.config(name)
    ctx, model, gk, pt = _setup(w, B)
    ref = ctx.ptct_similarity(pt, B, model, gk)
    torch.cuda.synchronize()
    for _ in range(2):  # the array keeps the previous call's contents
        out = torch.full_like(ref, -1)
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, B, model, gk, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)  # exact integer ciphertexts: zero tolerance
    ctx.close()


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    w = WL.config("serve")  # 7 ciphertexts per group of 1024 queries at n = 8192, L = 4
    B = 2048
    ctx, model, gk, pt = _setup(w, B)
    out = ctx.out_ct(B)
    with pytest.raises(E.EphdcError, match="EPHDC_EINVAL.*static scratch"):
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, B, model, gk, out)
    ctx.close()
