"""Write tests/golden/fullsize_oracle.json: the FP64 oracle's counts for the
full-size workloads whose exact counts take the host minutes (the
cell-pruned oracle of Sec. 3.3, itself pinned to the brute force of the
serial loop of Sec. 3.1 by tests/test_oracle.py).

This script calls only oracle/ (and the seeded input generators); no value
it writes comes from the CUDA library.  Each entry is keyed by workload,
seed and a SHA-256 of the generated inputs, so a test that regenerates the
inputs on another machine uses the stored counts only when its inputs are
byte-identical (else it counts with the oracle itself).

Stored per count: the SHA-256 of the uint64 histogram (little-endian,
row-major), its sum, and for the small histograms the values themselves;
for weighted counts the FP64 weighted sums.

    python tests/golden/make_fullsize.py c2 c4 c5     # any subset
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1210_1833_gb300 import synthetic  # noqa: E402

OUT = os.path.join(HERE, "fullsize_oracle.json")


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def counts_record(c, keep_values=False):
    c = np.ascontiguousarray(c, dtype="<u8")
    rec = {"sha256": sha(c), "sum": int(c.sum()), "nonzero": int(np.count_nonzero(c))}
    if keep_values:
        rec["counts"] = [int(v) for v in c.ravel()]
    return rec


def c2():
    """xi(r, mu) light cone: DD, DR, RR of 500k data and 2M randoms (Eq. 15
    inputs), 40 x 40 bins."""
    w = synthetic.c2_rmu_lightcone()
    reach = [w.edges0[-1]] * 3
    out = {"cite": "Sec. 2.2 Eq. 11 (pair counts) and Eq. 15; cell-pruned oracle (Sec. 3.3)",
           "workload": w.name, "seed": 1,
           "inputs": {"data": sha(w.data), "randoms": sha(w.randoms)}}
    for name, a, b in (("DD", w.data, None), ("DR", w.data, w.randoms), ("RR", w.randoms, None)):
        c, _, _ = oracle.count("rmu", a, b, edges0=w.edges0, edges1=w.edges1, cells=reach)
        out[name] = counts_record(c)
    return out


def c4():
    """Batched xi(sigma, pi): DD, DR, RR of each of the 64 periodic boxes,
    50 x 50 bins."""
    boxes = synthetic.c4_batched_sigpi()
    e0, e1 = boxes[0].edges0, boxes[0].edges1
    reach = [e0[-1], e0[-1], e1[-1]]
    out = {"cite": "Sec. 2.1 Eq. 2 (sigma, pi split), Sec. 2.2 Eq. 11; cell-pruned oracle "
                   "(Sec. 3.3) per box", "workload": "c4_batched_sigpi", "seed": 3,
           "inputs": {"boxes": sha(*[b.data for b in boxes] + [b.randoms for b in boxes])},
           "boxes": []}
    for b in boxes:
        rec = {"name": b.name, "n_data": len(b.data), "n_randoms": len(b.randoms)}
        for name, xa, xb in (("DD", b.data, None), ("DR", b.data, b.randoms),
                             ("RR", b.randoms, None)):
            c, _, _ = oracle.count("sigpi", xa, xb, edges0=e0, edges1=e1, periodic=True, L=b.L,
                                   cells=reach)
            rec[name] = counts_record(c)
        out["boxes"].append(rec)
    return out


def c5():
    """Weighted DD of 4M objects in a periodic cube: counts and the weighted
    sums W_b = sum of w_i w_j per bin (Neumaier-compensated FP64), 30 bins."""
    w = synthetic.c5_weighted()
    c, _, ws = oracle.count("mono", w.data, edges0=w.edges0, periodic=True, L=w.L, wa=w.weights,
                            weighted=True, cells=[w.edges0[-1]] * 3)
    rec = counts_record(c, keep_values=True)
    rec["wsum"] = [float(v) for v in ws.ravel()]
    return {"cite": "Sec. 2.2 Eq. 11 with the object weights of Sec. 3.4; cell-pruned oracle "
                    "(Sec. 3.3)", "workload": w.name, "seed": 4,
            "inputs": {"data": sha(w.data), "weights": sha(w.weights)}, "DD": rec}


MAKERS = {"c2": c2, "c4": c4, "c5": c5}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        t0 = time.time()
        rec = MAKERS[n]()
        rec["oracle_threads"] = oracle.max_threads()
        rec["seconds"] = round(time.time() - t0, 1)
        data[n] = rec
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")
        print(n, "done in %.1f s" % rec["seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(MAKERS))
