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
# the 16 domains of the uneven multi-domain workload (sides of batched_domains(), 8 cascades)
BATCH_SIDES = [256, 320, 640, 768, 1152, 1280, 1408, 1472, 1664, 1728, 1792, 1856, 1920, 1984]
PLANS += [(s, s, 8, 4, 4, 1.0, 0) for s in BATCH_SIDES if s != 1024]
# the headline recipe at other sizes (8 cascades), for the size sweep of the benchmark
PLANS += [(512, 512, 8, 4, 4, 1.0, 0), (2048, 2048, 8, 4, 4, 1.0, 0)]


def key(p):
    return "{}x{}_C{}_W{}_B{}_L{}_r{}".format(*p)


def main():
    path = os.path.join(HERE, "crossings.json")
    out = json.load(open(path))["plans"] if os.path.exists(path) else {}
    for p in PLANS:
        if key(p) in out:
            continue
        t = time.time()
        tot, per = oracle.count_crossings(p[0], p[1], p[2], p[3], p[4], p[5], p[6])
        out[key(p)] = {"total": tot, "per_cascade": [int(x) for x in per]}
        print(key(p), tot, list(per), f"{time.time() - t:.1f}s", flush=True)
        with open(path, "w") as f:
            json.dump({"source": "oracle.count_crossings (FP64 exact ray/face intersections)",
                       "plans": out}, f, indent=1)


if __name__ == "__main__":
    main()
