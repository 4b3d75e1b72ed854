"""Summarise an ncu launch list (CSV of gpu__time_duration.sum) per kernel.

Usage: python -m paper_2102_11910_gb300.profiling launches.csv
Prints, per kernel, the number of launches, total device time and share.
"""
import collections
import csv
import re
import sys


STEP_KERNELS = {"k_bin_count", "k_bin_scan", "k_bin_scatter", "k_regularize", "k_rows_fwd", "k_cols", "k_rows_inv",
                "k_interpolate"}


def kernel_name(raw):
    s = raw.replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    s = re.sub(r"^void\s+", "", s)
    s = s.replace("<unnamed>::", "")
    return re.split(r"[<(]", s, maxsplit=1)[0].strip()


def main(path):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    h = rows[hi]
    ki, mi, ui = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Unit")
    tot, cnt = collections.OrderedDict(), collections.Counter()
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "s": 1e6,
             "second": 1e6}
    for r in rows[hi + 1:]:
        if len(r) <= mi or not r[mi]:
            continue
        us = float(r[mi].replace(",", "")) * scale.get(r[ui], 1.0)
        name = kernel_name(r[ki])
        tot[name] = tot.get(name, 0.0) + us
        cnt[name] += 1
    def table(names, title):
        T = sum(tot[k] for k in names)
        print(title)
        print("%-34s %8s %12s %7s" % ("kernel", "launches", "total_us", "share"))
        for k in sorted(names, key=lambda x: -tot[x]):
            print("%-34s %8d %12.1f %6.1f%%" % (k, cnt[k], tot[k], 100 * tot[k] / T))
        print()

    table(list(tot), "all launches")
    step = [k for k in tot if k in STEP_KERNELS]
    if step:
        table(step, "kernels of the VIC step only (plan set-up and torch fills excluded)")


if __name__ == "__main__":
    main(sys.argv[1])
