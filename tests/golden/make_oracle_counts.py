"""Writes tests/golden/oracle_counts.json: the CPU oracle's own iteration
counts for the benchmark workloads.  Calls only oracle/ and the seeded
input generators.

The paper prints no worked numerical example (no residuals, no iteration
counts for a given field); these counts are the oracle's, recorded so that a
bounded CPU sample (a few oracle iterations) can be scaled to a whole solve.

Usage: python tests/golden/make_oracle_counts.py [threads]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1701_00426_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "mscg_32x32x32x32_m0.01_15shifts_tol1e-10": dict(dims=(32, 32, 32, 32), mass=0.01, n_shift=15, tol=1e-10),
    "mscg_8x8x8x8_m0.01_15shifts_tol1e-10": dict(dims=(8, 8, 8, 8), mass=0.01, n_shift=15, tol=1e-10),
    "cg_8x8x8x8_m0.1_tol1e-10": dict(dims=(8, 8, 8, 8), mass=0.1, n_shift=1, tol=1e-10),
}


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    orc = oracle()
    used = orc.set_threads(threads)
    out_path = os.path.join(HERE, "oracle_counts.json")
    res = json.load(open(out_path)) if os.path.exists(out_path) else {}
    for name, w in WORKLOADS.items():
        if name in res:
            continue
        U = inputs.random_links(w["dims"])
        b = inputs.gaussian_field(w["dims"], k=0)
        shifts = inputs.log_shifts(w["n_shift"]) if w["n_shift"] > 1 else [0.0]
        t = time.time()
        x, info = orc.mscg(w["dims"], U, w["mass"], shifts, b, w["tol"])
        res[name] = {"iters": info["iters"], "refine_iters": info["refine_iters"],
                     "shift_iters": info["shift_iters"], "max_true_resid": float(max(info["true_resid"])),
                     "status": info["status"], "seconds": round(time.time() - t, 1), "threads": used,
                     "links_seed": inputs.LINK_SEED, "source_seed": inputs.SOURCE_SEED}
        print(name, res[name], flush=True)
        json.dump(res, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main()
