"""Writes clients64_group_digests.txt: SHA-256 digests of the oracle's score ciphertexts
for query groups 0, 15 and 31 of the clients64 workload (64 clients with log-uniform
batch sizes packed back to back, F = 768, D = 10000, 4-bit hypervectors, 7 classes,
n = 8192, L = 4 primes, layout k_in = 1, r = 8; 1024 queries per group, the last group
partial).

Only the oracle and the seeded input generators run here.  The packed query space is
the clients' rows concatenated in order, so group g of the packed pass holds rows
g*1024 .. of that concatenation.  Each group's output is the uint32 words
[k/k_in][2][L][n] of its score ciphertexts in the coefficient domain, little-endian.

    python tests/golden/make_clients64_digests.py
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

GROUPS = (0, 15, 31)


def main():
    w = WL.config("clients64")
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    cap = o.cap
    s, gk = o.keygen(w.seed)
    cls = WL.classes(w.seed, w.k, w.D)
    model = o.encrypt_model(w.seed, cls, s)
    X = np.concatenate([WL.features(w.seed, b, w.F, batch=i) for i, b in enumerate(w.clients)])
    Wt = WL.projection(w.seed, w.D, w.F)
    lines = ["# SHA-256 of the oracle's score ciphertexts (uint32 [k/k_in][2][L][n], coefficient",
             "# domain, little-endian) for query groups of the clients64 workload (the clients'",
             "# batches packed back to back), written by tests/golden/make_clients64_digests.py",
             "# (oracle only).",
             "# columns: group first_query queries sha256"]
    for g in GROUPS:
        rows = X[g * cap:(g + 1) * cap]
        _, _, out = o.infer(rows, Wt, model, gk, w.shift, w.bits)
        words = np.ascontiguousarray(out[0], dtype="<u4")
        lines.append("%d %d %d %s" % (g, g * cap, len(rows), hashlib.sha256(words.tobytes()).hexdigest()))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "clients64_group_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
