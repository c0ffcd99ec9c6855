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

import oracle as O
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


# face1024 (r = 8) ends its rotate-and-sum ping-pong after 3 steps, face1024_a (the
# paper's layout A, r = 4) after 2, so both ends of the ping-pong are covered
@pytest.mark.parametrize("name,B", [("small", 16), ("face1024", 1024), ("face1024", 700),
                                    ("face1024_a", 1024)])
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


# (n, L, k, k_in, r, D, F, bits, B): an odd and an even number of rotate-and-sum
# steps, and r = 1 (the paper's layout: no rotation, no Galois keys, gk = NULL)
ORACLE_LAYOUTS = [
    (4096, 3, 2, 2, 128, 2048, 608, 4, 16),  # 7 steps
    (2048, 2, 3, 1, 4, 100, 32, 8, 300),     # 2 steps, 3 ciphertexts per group, 2 groups
    (1024, 2, 2, 2, 1, 50, 32, 8, 700),      # no rotation, 2 groups
]


@pytest.mark.parametrize("n,L,k,k_in,r,D,F,bits,B", ORACLE_LAYOUTS)
def test_noalloc_matches_the_oracle_twice(n, L, k, k_in, r, D, F, bits, B):
    w = WL.Workload(name="t", n=n, L=L, k=k, k_in=k_in, r=r, D=D, F=F, bits=bits, B=B,
                    seed=4242 + n + r)
    ctx, model, gk, pt = _setup(w, B)
    if r == 1:
        assert gk is None
    o = O.Oracle(n, L, k, k_in, r, D)
    s, ogk = o.keygen(w.seed)
    omodel = o.encrypt_model(w.seed, WL.classes(w.seed, k, D), s)
    _, _, want = o.infer(WL.features(w.seed, B, F), WL.projection(w.seed, D, F), omodel, ogk,
                         w.shift, bits)
    out = ctx.out_ct(B)
    for _ in range(2):  # the second call starts from the first call's scratch contents
        out.fill_(-1)
        E.bfv_ptct_similarity_noalloc(ctx.ctx, pt, B, model, gk, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(want.shape)
        assert np.array_equal(got, want)  # exact integer ciphertexts: zero tolerance
    ctx.close()
