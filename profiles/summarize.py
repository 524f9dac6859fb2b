"""Turn raw ncu output into the short text summaries kept in this folder.

  python profiles/summarize.py launches <launches.csv> <out.md> "<command>"
  python profiles/summarize.py kernel <capture.ncu-rep> <out.md> "<command>"

`launches` groups a `--metrics gpu__time_duration.sum` launch list by kernel
(launches, total time, share); `kernel` extracts the DRAM, tensor-pipe and
occupancy counters of each captured launch (needs `ncu -i`, no GPU).
"""
from __future__ import annotations

import collections
import csv
import io
import re
import subprocess
import sys


def _short(name: str) -> str:
    name = re.sub(r"\(CUtensorMap_st.*|\((const |float|int|lr::|double|unsigned|long).*\)$", "", name)
    name = re.sub(r"\(anonymous namespace\)::|<?unnamed>::|^void ", "", name)
    return name.strip()


def launches(src: str, out: str, cmd: str) -> None:
    lines = [ln for ln in open(src) if ln.startswith('"')]
    rows = list(csv.reader(lines))
    hdr, rows = rows[0], rows[1:]
    i_name, i_val = hdr.index("Kernel Name"), hdr.index("Metric Value")
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows:
        a = agg[_short(r[i_name])]
        a[0] += 1
        a[1] += float(r[i_val])
    tot = sum(t for _, t in agg.values())
    with open(out, "w") as f:
        f.write(f"# Launch list: {len(rows)} launches, {tot / 1e6:.3f} ms summed device time\n\n")
        f.write(f"Command:\n\n    {cmd}\n\n")
        f.write("Per-launch times under ncu are serialised and cold-cache; compare shares.\n\n")
        f.write("| kernel | launches | total ms | share |\n|---|---:|---:|---:|\n")
        for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
            f.write(f"| `{k}` | {n} | {t / 1e6:.3f} | {100 * t / tot:.1f}% |\n")


WANT = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed",
    "sm__throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__warps_active.avg.pct_of_peak_sustained_active",
    "launch__registers_per_thread", "launch__grid_size", "launch__block_size",
    "launch__shared_mem_per_block_dynamic", "lts__t_sector_hit_rate.pct",
]


def kernel(rep: str, out: str, cmd: str) -> None:
    raw = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(io.StringIO(raw)))
    hdr, units, data = rows[0], rows[1], rows[2:]
    with open(out, "w") as f:
        f.write(f"# ncu capture: {len(data)} launch(es)\n\nCommand:\n\n    {cmd}\n\n")
        for d in data:
            f.write(f"## `{_short(d[hdr.index('Kernel Name')])}`\n\n| metric | value | unit |\n|---|---:|---|\n")
            for k in WANT:
                if k in hdr:
                    i = hdr.index(k)
                    f.write(f"| {k} | {d[i]} | {units[i]} |\n")
            f.write("\n")


if __name__ == "__main__":
    {"launches": launches, "kernel": kernel}[sys.argv[1]](*sys.argv[2:5])
