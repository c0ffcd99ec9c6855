"""Writes dense65536_group_digests.txt: SHA-256 digests of the oracle's score
ciphertexts for query groups 0 and 63 of the dense65536 workload (65536 queries,
F = 1024, D = 16384, 8-bit hypervectors, 16 classes, n = 16384, L = 6 primes, layout
k_in = 1, r = 16; 1024 queries per group).

Only the oracle and the seeded input generators run here.  Each group's output is the
uint32 words [k/k_in][2][L][n] of its score ciphertexts in the coefficient domain,
little-endian, the layout bfv_ptct_similarity writes for that group.  The full
ciphertexts (6.3 MB per group) are too large to store; the GPU test hashes the same
words of its own full-size run and compares.  The oracle takes several minutes here.

    python tests/golden/make_dense65536_digests.py
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

GROUPS = (0, 63)


def main():
    w = WL.config("dense65536")
    o = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, w.D)
    cap = o.cap
    s, gk = o.keygen(w.seed)
    cls = WL.classes(w.seed, w.k, w.D)
    model = o.encrypt_model(w.seed, cls, s)
    X = WL.features(w.seed, w.B, w.F)
    Wt = WL.projection(w.seed, w.D, w.F)
    lines = ["# SHA-256 of the oracle's score ciphertexts (uint32 [k/k_in][2][L][n], coefficient",
             "# domain, little-endian) for query groups of the dense65536 workload, written by",
             "# tests/golden/make_dense65536_digests.py (oracle only).",
             "# columns: group first_query queries sha256"]
    for g in GROUPS:
        rows = X[g * cap:(g + 1) * cap]
        _, _, out = o.infer(rows, Wt, model, gk, w.shift, w.bits)
        words = np.ascontiguousarray(out[0], dtype="<u4")
        lines.append("%d %d %d %s" % (g, g * cap, len(rows), hashlib.sha256(words.tobytes()).hexdigest()))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "dense65536_group_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
