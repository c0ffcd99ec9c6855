"""GPU seeded model message: the c0 halves in the coefficient domain equal the
oracle's, and the model rebuilt from them and the seed equals the encrypted model
word for word."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2511_00737_gb300 import ephdc as E
from paper_2511_00737_gb300 import workload as WL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["small", "face1024"])
def test_seeded_model_roundtrip(name):
    w = WL.config(name)
    ctx = E.Context.for_workload(w, max_batch=16)
    cls = WL.classes(w.seed, w.k, w.D)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(torch.from_numpy(cls).cuda(), sk, w.seed)
    seeded = ctx.model_to_seeded(model)
    assert seeded.numel() * 2 == model.numel()
    rebuilt = ctx.model_from_seeded(seeded, w.seed)
    torch.cuda.synchronize()
    assert torch.equal(rebuilt, model)
    if name == "small":
        o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
        s, _ = o.keygen(w.seed)
        om = o.encrypt_model(w.seed, cls, s)
        got = seeded.cpu().numpy().view(np.uint32).reshape(o.P, o.Kp, o.L, o.n)
        assert np.array_equal(got, om[:, :, 0])
    ctx.close()
