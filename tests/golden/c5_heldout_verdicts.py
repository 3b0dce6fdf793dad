"""Writes c5_heldout_verdicts.json: the CPU oracle's verdict on each of the
2,000 held-out kernels of the learned-ranker workload (corpus-shaped kernels,
seeds 200000.., up to 10^6 instances each).  It calls only oracle/ and the
seeded input generators; the GPU tests and the bench's ranked suite compare
every form of the check (plain, batched, ranked) with these verdicts.

    python tests/golden/c5_heldout_verdicts.py [--jobs N]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c5_heldout_verdicts.json")
FIRST, COUNT, HI_EXP = 200000, 2000, 6.0


def heldout(j):
    import workloads
    return workloads.config4(FIRST + j, hi_exp=HI_EXP)


def verdict(j):
    import oracle
    w = heldout(j)
    o = oracle.check(w.text, w.binding, cap=1 << 22, pair=False)
    pairs = {}
    for x in o.witnesses:
        pairs[f"{x[3]},{x[4]}"] = pairs.get(f"{x[3]},{x[4]}", 0) | x[5]
    return {"item": FIRST + j, "racy": o.racy, "n_witness": o.n_witness, "n_by_kind": list(o.n_by_kind),
            "n_instances": o.n_instances, "n_keys": o.n_keys, "n_oob": o.n_oob, "pairs": pairs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(a.jobs) as p:
        rows = p.map(verdict, range(COUNT), chunksize=8)
    with open(OUT, "w") as f:
        json.dump({"workload": f"config4 items {FIRST}..{FIRST + COUNT - 1}, hi_exp {HI_EXP}",
                   "written_by": "tests/golden/c5_heldout_verdicts.py (CPU oracle only)", "verdicts": rows}, f)
        f.write("\n")
    print(f"{sum(r['racy'] for r in rows)} racy of {len(rows)}; {sum(r['n_instances'] for r in rows):,} instances")


if __name__ == "__main__":
    main()
