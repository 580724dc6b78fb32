"""Summaries of Nsight Compute output for the text files kept under profiles/.

    python -m paper_2412_10789_gb300.ncu_summary launches LAUNCHES.csv [--exclude REGEX]
        per kernel: launches, total device time and share, from a launch list
        taken with `ncu --metrics gpu__time_duration.sum --csv --log-file ...`
        (cold-cache, serialised launches: compare shares, not absolute times).

    python -m paper_2412_10789_gb300.ncu_summary report REPORT.ncu-rep [--json OUT --units-scale S]
        per captured launch: duration, DRAM bytes, L2 hit rate, issue activity,
        warp stall reasons, registers; with --json, also writes the mean DRAM
        bytes per launch (scaled by S when the capture ran a smaller case) and a
        hash of the kernel's source files, which bench.py compares before it
        reports the figure as the kernel's traffic.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
import subprocess
from collections import OrderedDict

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")

# Source files each profiled kernel is built from (for the staleness hash).
KERNEL_SOURCES = {
    "cheb_step_kernel": ["step.cuh", "cheb.cu", "gp_internal.h", "schedule.cpp"],
    "spmm_step_kernel": ["batch.cu", "batch.h", "gp_internal.h"],
}

REPORT_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("dram__throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__throughput.avg.pct_of_peak_sustained_elapsed", "L2 throughput % of peak"),
    ("lts__t_sector_hit_rate.pct", "L2 sector hit rate %"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % (occupancy)"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__block_size", "block size"),
    ("launch__grid_size", "grid size"),
    ("launch__shared_mem_per_block", "shared memory/block"),
]
STALL_PREFIX = "smsp__average_warps_issue_stalled_"
STALL_SUFFIX = "_per_issue_active.ratio"


def source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _to_bytes(value: str, unit: str) -> float:
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    return float(value) * scale.get(unit, 1.0)


def _to_us(value: str, unit: str) -> float:
    scale = {"ns": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "nsecond": 1e-3, "s": 1e6}
    return float(value) * scale.get(unit, 1.0)


def launches(path: str, exclude: str | None = None) -> str:
    with open(path) as f:
        rows = list(csv.reader(f))
    start = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[start]
    agg: "OrderedDict[str, list]" = OrderedDict()
    for r in rows[start + 1:]:
        d = dict(zip(hdr, r))
        if d.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = d["Kernel Name"].split("(")[0].replace("void ", "").replace("unnamed>::", "")
        if exclude and re.search(exclude, name):
            continue
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += _to_us(d["Metric Value"], d["Metric Unit"]) / 1e3
    total = sum(v[1] for v in agg.values())
    lines = ["| kernel | launches | total ms | mean us | share |", "|---|---:|---:|---:|---:|"]
    for name, (n, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        lines.append(f"| `{name}` | {n} | {ms:.3f} | {1e3 * ms / n:.1f} | {ms / total:.3f} |")
    lines.append(f"| total | {sum(v[0] for v in agg.values())} | {total:.3f} | | 1.000 |")
    return "\n".join(lines)


def _raw_rows(rep: str):
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr, units = rows[0], rows[1]
    return [(dict(zip(hdr, r)), dict(zip(hdr, units))) for r in rows[2:]]


def report(rep: str, json_out: str | None = None, units_scale: float = 1.0, kernel: str | None = None) -> str:
    recs = _raw_rows(rep)
    lines = []
    dram = []
    for i, (d, u) in enumerate(recs):
        name = d.get("Kernel Name", "").split("(")[0].replace("void ", "").replace("unnamed>::", "")
        lines.append(f"### launch {i}: `{name}`")
        lines.append("| metric | value |")
        lines.append("|---|---:|")
        for key, label in REPORT_METRICS:
            if key in d and d[key] != "":
                lines.append(f"| {label} (`{key}`) | {d[key]} {u.get(key, '')} |")
        stalls = []
        for key, val in d.items():
            if key.startswith(STALL_PREFIX) and key.endswith(STALL_SUFFIX):
                try:
                    stalls.append((float(val), key[len(STALL_PREFIX):-len(STALL_SUFFIX)]))
                except ValueError:
                    pass
        stalls.sort(reverse=True)
        if stalls:
            lines.append("| top warp stalls (cycles per issued instruction) | " +
                         ", ".join(f"{n} {v:.2f}" for v, n in stalls[:5]) + " |")
        if "dram__bytes_read.sum" in d:
            dram.append(_to_bytes(d["dram__bytes_read.sum"], u["dram__bytes_read.sum"]) +
                        _to_bytes(d["dram__bytes_write.sum"], u["dram__bytes_write.sum"]))
        lines.append("")
    if json_out and dram:
        mean = sum(dram) / len(dram)
        kname = kernel or next(k for k in KERNEL_SOURCES if k in recs[0][0].get("Kernel Name", ""))
        with open(json_out, "w") as f:
            json.dump({"kernel": kname, "launches_captured": len(dram), "dram_bytes_per_launch": mean,
                       "units_scale": units_scale, "dram_bytes_per_launch_full_size": mean * units_scale,
                       "kernel_source_hash": source_hash(kname)}, f, indent=1)
            f.write("\n")
    return "\n".join(lines)


def main():
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("launches")
    a.add_argument("csv")
    a.add_argument("--exclude", default=None, help="regex of kernel names to leave out")
    b = sub.add_parser("report")
    b.add_argument("rep")
    b.add_argument("--json", default=None)
    b.add_argument("--units-scale", type=float, default=1.0)
    b.add_argument("--kernel", default=None)
    args = p.parse_args()
    if args.cmd == "launches":
        print(launches(args.csv, args.exclude))
    else:
        print(report(args.rep, args.json, args.units_scale, args.kernel))


if __name__ == "__main__":
    main()
