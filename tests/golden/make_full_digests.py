"""Write tests/golden/full_size_digests.json from the CPU oracle only.

Run from the repository root:  python tests/golden/make_full_digests.py
For every full-size workload it records the SHA-256 digest of the oracle's
complete product -- every limb and every sign, c as little-endian uint32
rows of Lc limbs followed by the sign bytes -- computed by Kronecker
substitution with the oracle's own Karatsuba (oracle.polymul_kron, pinned
to the schoolbook definition in tests/test_oracle_pins.py), plus digests of
the seeded inputs and a few coefficients in decimal.  Minutes of CPU time
per workload on a few cores.
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

WORKLOADS = {
    "large_dense": ("na=nb=32768, |coeff| < 2^4096, signed uniform, seed 1", lambda: W.large_dense(seed=1)),
    "huge_dense": ("na=nb=262144, |coeff| < 2^1024, signed uniform, seed 2", lambda: W.huge_dense(seed=2)),
    "huge_mixed": ("na=nb=262144, half the positions < 2^64, the rest < 2^2048, signed, seed 2",
                   lambda: W.huge_mixed(seed=2)),
}
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_digests.json")


def digest_inputs(a, b):
    return hashlib.sha256(a[0].tobytes() + a[1].tobytes() + b[0].tobytes() + b[1].tobytes()).hexdigest()


def main(names):
    out = {}
    if os.path.exists(PATH):
        out = json.load(open(PATH))
    for name in names:
        what, make = WORKLOADS[name]
        sh, a, b = make()
        t0 = time.time()
        c, cn = oracle.polymul_kron(a, b, sh.lc)
        dt = time.time() - t0
        samples = {}
        for k in (0, 1, sh.nc // 2, sh.nc - 1):
            v = int.from_bytes(c[k].astype("<u4").tobytes(), "little")
            samples[str(k)] = str(-v if cn[k] else v)
        out[name] = {
            "workload": "%s: %s; lc=%d" % (name, what, sh.lc),
            "written_by": "tests/golden/make_full_digests.py (oracle.polymul_kron only)",
            "nc": sh.nc, "lc": sh.lc,
            "inputs_sha256": digest_inputs(a, b),
            "sha256": hashlib.sha256(c.astype("<u4").tobytes() + cn.tobytes()).hexdigest(),
            "negative_coefficients": int(cn.sum()),
            "samples": samples,
            "oracle_seconds": round(dt, 1), "oracle_threads": oracle.default_threads(),
        }
        print(name, out[name]["sha256"], "%.1f s" % dt, flush=True)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
