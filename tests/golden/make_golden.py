"""Write tests/golden/tiny_oracle.json: the CPU oracle's answers on the seeded
tiny workload (10 classes, 5,000 references, 20 query images of 100
descriptors, k = 10), with SHA-256 digests of the generated input bytes.

Calls only the oracle and the seeded generator.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1112_0059_gb300 import synth  # noqa: E402


def digest(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def main() -> None:
    w = synth.workload("tiny")
    ref, labels = synth.reference_set(w)
    q, offsets, _ = synth.query_set(w)
    k = 10
    lt, lc = oracle.local_nbnn(ref, labels, w.n_classes, q, offsets, k)
    nt, nc = oracle.nbnn(ref, labels, w.n_classes, q, offsets)
    d, j = oracle.knn(ref, q[:8], k + 1)
    out = {
        "workload": "tiny (10 classes x 5 ref images x 100; 20 query images x 100; seed 0)",
        "k": k,
        "sha256": {"ref": digest(ref), "labels": digest(labels), "queries": digest(q),
                   "offsets": digest(offsets)},
        "local_nbnn": {"totals": lt.tolist(), "classes": lc.tolist()},
        "nbnn": {"totals": nt.tolist(), "classes": nc.tolist()},
        "knn_first_8_rows": {"dist": d.tolist(), "idx": j.tolist()},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
