"""Writes crossings.json: voxel crossings per cascade of one wavelength for the plans the
benchmark and tests use, counted by the FP64 oracle (geometry only).  These are the
algorithmic work units of the roofline: each crossing reads chi and eta (8 bytes in FP32)."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

PLANS = [
    # (nx, nz, n_cascades, dirs0, branching, interval0, rule)
    (64, 64, 5, 4, 4, 1.0, 0),
    (256, 256, 7, 4, 4, 1.0, 0),
    (512, 512, 7, 4, 4, 1.0, 0),
    (1024, 1024, 8, 4, 4, 1.0, 0),
]


def key(p):
    return "{}x{}_C{}_W{}_B{}_L{}_r{}".format(*p)


def main():
    out = {}
    for p in PLANS:
        t = time.time()
        tot, per = oracle.count_crossings(p[0], p[1], p[2], p[3], p[4], p[5], p[6])
        out[key(p)] = {"total": tot, "per_cascade": [int(x) for x in per]}
        print(key(p), tot, list(per), f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, "crossings.json"), "w") as f:
        json.dump({"source": "oracle.count_crossings (FP64 exact ray/face intersections)",
                   "plans": out}, f, indent=1)


if __name__ == "__main__":
    main()
