"""Write tests/golden/small_dense_seed0.json from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
It records SHA-256 digests of the seeded inputs and of the oracle's product
for the small dense workload (two degree-1023 polynomials, |coefficients| <
2^255, seed 0), plus a few coefficients in decimal for readability.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    sh, a, b = W.small_dense(seed=0)
    c, cn = oracle.polymul(a, b, sh.lc)
    out = {
        "workload": "small_dense: na=nb=1024, |coeff| < 2^255, seed 0; lc=%d" % sh.lc,
        "written_by": "tests/golden/make_golden.py (oracle only)",
        "inputs_sha256": hashlib.sha256(a[0].tobytes() + a[1].tobytes() +
                                        b[0].tobytes() + b[1].tobytes()).hexdigest(),
        "sha256": hashlib.sha256(c.tobytes() + cn.tobytes()).hexdigest(),
        "samples": {},
    }
    for k in (0, 1, 1023, 2046):
        v = int.from_bytes(c[k].astype("<u4").tobytes(), "little")
        out["samples"][str(k)] = str(-v if cn[k] else v)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_dense_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
