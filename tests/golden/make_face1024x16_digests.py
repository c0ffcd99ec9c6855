"""Writes face1024x16_group_digests.txt: SHA-256 digests of the oracle's score
ciphertexts for query groups 0 and 15 of the face1024 throughput step: 16
consecutive 1024-query batches (16384 feature rows drawn as one array, F = 608,
D = 10000, 8-bit hypervectors, 2 classes, n = 8192, L = 4 primes, layout k_in = 1,
r = 8) packed into one pass, so the encrypted model is streamed once for all 16
groups.

Only the oracle and the seeded input generators run here.  Groups are independent
given the keys and the model, so the oracle runs groups 0 and 15 alone: group g
holds rows g*1024 .. g*1024 + 1023 of the step's feature array.  Each group's output
is the uint32 words [k/k_in][2][L][n] of its score ciphertexts in the coefficient
domain, little-endian.

    python tests/golden/make_face1024x16_digests.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2511_00737_gb300 import workload as WL  # noqa: E402

BATCHES = 16
GROUPS = (0, 15)


def main():
    w = WL.config("face1024")
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    cap = o.cap
    s, gk = o.keygen(w.seed)
    cls = WL.classes(w.seed, w.k, w.D)
    model = o.encrypt_model(w.seed, cls, s)
    X = WL.features(w.seed, BATCHES * w.B, w.F, batch=0)
    Wt = WL.projection(w.seed, w.D, w.F)
    lines = ["# SHA-256 of the oracle's score ciphertexts (uint32 [k/k_in][2][L][n], coefficient",
             "# domain, little-endian) for query groups of the face1024 throughput step (16",
             "# 1024-query batches drawn as one 16384-row feature array, packed into one pass),",
             "# written by tests/golden/make_face1024x16_digests.py (oracle only).",
             "# columns: group first_query queries sha256"]
    for g in GROUPS:
        rows = X[g * cap:(g + 1) * cap]
        _, _, out = o.infer(rows, Wt, model, gk, w.shift, w.bits)
        words = np.ascontiguousarray(out[0], dtype="<u4")
        lines.append("%d %d %d %s" % (g, g * cap, len(rows),
                                      hashlib.sha256(words.tobytes()).hexdigest()))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "face1024x16_group_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
