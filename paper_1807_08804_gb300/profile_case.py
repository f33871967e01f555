"""Run one batch of a named workload once, for profiling under ncu.

  python -m paper_1807_08804_gb300.profile_case --workload single-1m --queries 1000

Keeps device memory small (one batch, no comparison modes) so that a full
ncu capture of a few kernels ends quickly.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="single-1m")
    ap.add_argument("--queries", type=int, default=0)
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--wave", type=int, default=0)
    ap.add_argument("--group", type=int, default=0, help="lanes per work item (0 = library default)")
    ap.add_argument("--rounds", type=int, default=0, help="refinement rounds (0 = library default)")
    a = ap.parse_args()
    import paper_1807_08804_gb300 as gs
    from paper_1807_08804_gb300 import inputs as I
    w = I.WORKLOADS[a.workload]
    g = w.graph()
    qs = w.queries(g, a.queries or None)
    dg = gs.DeviceGraph(g)
    if a.group or a.rounds:
        gs.tune_set(dg, a.group, a.rounds)
    b = gs.Batch(dg, qs, cap=w.cap, wave_queries=a.wave)
    for _ in range(a.runs):
        b.run()
        b.finish()
    res = b.fetch()
    print(f"{len(qs)} queries, {sum(r.count for r in res)} embeddings, "
          f"{sum(r.status != 0 for r in res)} not ok")
    b.close()
    dg.free()


if __name__ == "__main__":
    main()
