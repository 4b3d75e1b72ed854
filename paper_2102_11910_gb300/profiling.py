"""Summaries of ncu output for the step kernels.

Usage:
  python -m paper_2102_11910_gb300.profiling launches launches.csv [N]
      per kernel: launches, total device time and share, from an ncu CSV of
      gpu__time_duration.sum (one pass; cold-cache, serialised launches);
      with N, the step-kernel table counts only the first N launches of each
      step kernel (the device-resident steps a bench run starts with);
  python -m paper_2102_11910_gb300.profiling traffic traffic.csv
      per step kernel: DRAM bytes read + written per launch, from
      `ncu -i report --page raw --csv` or `ncu --metrics ... --csv`, as the
      JSON that bench.py reads (keyed by the source hash of csrc/, so a stale
      capture is ignored).
"""
import collections
import csv
import glob
import hashlib
import json
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))

# kernel function -> name used by the per-kernel timing of the library
STEP_KERNELS = {
    "k_locate": "bin_locate", "k_offsets": "bin_offsets", "k_scatter": "bin_scatter", "k_deposit": "regularize",
    "k_rows_fwd_r": "fft_rows_fwd", "k_cols_r": "fft_cols_conv", "k_rows_inv_r": "fft_rows_inv",
    "k_interp_tiles_f32": "interpolate", "k_interp_tiles": "interpolate",
}


def csrc_sha():
    """Hash of the CUDA sources; counters taken from another build do not apply."""
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(HERE, "csrc", "*"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def kernel_name(raw):
    s = raw.replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    s = re.sub(r"^void\s+", "", s)
    return re.split(r"[<(]", s, maxsplit=1)[0].strip()


def _rows(path):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    return rows[hi], rows[hi + 1:]


def launches(path, first=None):
    h, body = _rows(path)
    ki, mi, ui = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Unit")
    tot, cnt = collections.OrderedDict(), collections.Counter()
    ftot, fcnt = collections.OrderedDict(), collections.Counter()
    first = int(first) if first is not None else None
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "s": 1e6,
             "second": 1e6}
    for r in body:
        if len(r) <= mi or not r[mi]:
            continue
        us = float(r[mi].replace(",", "")) * scale.get(r[ui], 1.0)
        name = kernel_name(r[ki])
        tot[name] = tot.get(name, 0.0) + us
        cnt[name] += 1
        if name in STEP_KERNELS and (first is None or fcnt[name] < first):
            ftot[name] = ftot.get(name, 0.0) + us
            fcnt[name] += 1

    def table(tot, cnt, names, title):
        T = sum(tot[k] for k in names)
        print(title)
        print("%-34s %8s %12s %7s %9s" % ("kernel", "launches", "total_us", "share", "avg_us"))
        for k in sorted(names, key=lambda x: -tot[x]):
            print("%-34s %8d %12.1f %6.1f%% %9.2f" % (k, cnt[k], tot[k], 100 * tot[k] / T, tot[k] / cnt[k]))
        print()

    table(tot, cnt, list(tot), "all launches")
    if ftot:
        title = "kernels of the VIC step only (plan set-up and torch fills excluded)"
        if first is not None:
            title += ", first %d launches of each" % first
        table(ftot, fcnt, list(ftot), title)


def traffic(path):
    """DRAM bytes per launch of each step kernel, from either CSV layout of
    ncu: one column per metric (`ncu -i report --page raw --csv`) or one row
    per metric (`ncu --metrics ... --csv`)."""
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    want = ("dram__bytes_read.sum", "dram__bytes_write.sum")
    h, body = _rows(path)
    ki = h.index("Kernel Name")
    per_launch = collections.OrderedDict()         # (launch id, kernel) -> bytes
    if "Metric Name" in h:
        ii, ni, ui, vi = h.index("ID"), h.index("Metric Name"), h.index("Metric Unit"), h.index("Metric Value")
        for r in body:
            if len(r) <= vi or r[ni] not in want:
                continue
            name = STEP_KERNELS.get(kernel_name(r[ki]))
            if name:
                key = (r[ii], name)
                per_launch[key] = per_launch.get(key, 0.0) + float(r[vi].replace(",", "")) * unit.get(r[ui], 1.0)
    else:
        units, body = body[0], body[1:]
        cols = {m: h.index(m) for m in want}
        for n, r in enumerate(body):
            name = STEP_KERNELS.get(kernel_name(r[ki]))
            if name:
                per_launch[(n, name)] = sum(float(r[cols[m]].replace(",", "")) * unit.get(units[cols[m]], 1.0)
                                            for m in want)
    acc = collections.defaultdict(lambda: [0.0, 0])
    for (_, name), b in per_launch.items():
        acc[name][0] += b
        acc[name][1] += 1
    out = {"csrc_sha": csrc_sha(), "source": os.path.basename(path),
           "kernels": {k: {"dram_bytes": v[0] / v[1], "launches": v[1]} for k, v in acc.items()}}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    {"launches": launches, "traffic": traffic}[sys.argv[1]](*sys.argv[2:])
