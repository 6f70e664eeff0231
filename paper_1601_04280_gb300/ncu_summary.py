"""Summarize an ncu launch list (CSV of gpu__time_duration.sum) per kernel of this library.

usage: python -m paper_1601_04280_gb300.ncu_summary launches.csv "<title>" > profiles/<name>.md
"""
import collections
import csv
import sys


def main(path, title):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if r and r[0] == "ID"][0]
    hdr, data = rows[hi], rows[hi + 1:]
    ki, vi, mi = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Name")
    agg = collections.OrderedDict()
    for r in data:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0].replace("void ", "")
        if not (name.startswith("rlu::") or name.startswith("tc::")):
            continue
        a = agg.setdefault(name[:64], [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", ""))
    tot = sum(v[1] for v in agg.values())
    nfact = max((c for k, (c, t) in agg.items() if "k_pivoted_lu<double" in k), default=0)
    print("# %s\n" % title)
    print("Per-kernel device time of this library's kernels over the whole command (%d factorizations: warm-up,"
          % nfact)
    print("timed steps, graph replays, stage-timing and e2e repetitions). ncu serializes launches and runs them")
    print("cold: compare the")
    print("SHARES with bench.py's live `stage_ms`, not the absolute times.\n")
    print("| kernel | launches | total ms | mean us/launch | share |")
    print("|---|---|---|---|---|")
    for k, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print("| `%s` | %d | %.2f | %.1f | %.1f%% |" % (k, c, t / 1e6, t / c / 1e3, 100 * t / tot))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
