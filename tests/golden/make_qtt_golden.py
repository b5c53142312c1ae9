"""Writes the FP64-oracle summary of the banded QTT workload that the GPU tests
compare against at a size where the oracle takes minutes (2^12 x 2^12 matrix,
12 modes of size 4, eps = 1e-6).

Only the oracle and the input generators are called.  The file keeps, per bond,
the rank, the largest and the smallest kept singular value, the first discarded
one and the discarded tail sum of squares, plus the oracle TT's values at seeded
sample positions (half of them nonzeros of the input, half uniform positions).

    python tests/golden/make_qtt_golden.py 12
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fasttt as O            # noqa: E402
from oracle import tteval as OT           # noqa: E402
from paper_1908_02721_gb300 import workloads as W   # noqa: E402

SAMPLE_SEED = 31
N_SAMPLES = 1024


def main(m):
    w = W.banded_qtt(m, eps=1e-6)
    t0 = time.time()
    res = O.fasttt(w.idx, w.vals, w.dims, w.eps)
    secs = time.time() - t0
    bonds = {}
    for b, s in sorted(res.sigmas.items()):
        r = res.ranks[b]
        bonds[str(b)] = {
            "n_sigma": int(s.size),
            "rank": int(r),
            "sigma_first": float(s[0]).hex(),
            "sigma_last_kept": float(s[r - 1]).hex(),
            "sigma_first_dropped": float(s[r]).hex() if r < s.size else None,
            "tail2": float(sum(float(x) ** 2 for x in s[r:][::-1])).hex(),
            "delta": float(res.deltas[b]).hex(),
        }
    pos = W.sample_positions(w, N_SAMPLES // 2, N_SAMPLES // 2, SAMPLE_SEED)
    vals = OT.tt_eval_at(res.cores, pos)
    out = {
        "workload": w.name,
        "m": m,
        "eps": w.eps,
        "oracle_seconds": round(secs, 1),
        "p": res.p,
        "R": int(res.R),
        "rt": [int(x) for x in res.rt],
        "ranks": [int(x) for x in res.ranks],
        "norm2": float(res.norm2).hex(),
        "err2": float(res.err2).hex(),
        "bonds": bonds,
        "sample_seed": SAMPLE_SEED,
        "n_samples": int(pos.shape[1]),
        "tt_at_samples": [float(v).hex() for v in vals],
    }
    path = os.path.join(HERE, f"qtt{m}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path}: oracle {secs:.0f} s, ranks {res.ranks}")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 12)
