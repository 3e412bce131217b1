"""Summaries of Nsight Compute exports for the files under profiles/.

    python -m paper_2203_15561_gb300.ncu_summary launches <launches.csv> [first:last]
        per kernel: launches, total device time, share (from a
        `--metrics gpu__time_duration.sum --csv --log-file` run), optionally
        over a slice of the launch list only
    python -m paper_2203_15561_gb300.ncu_summary full <raw.csv>
        selected counters of each captured launch (from
        `ncu -i <report> --page raw --csv`)
    python -m paper_2203_15561_gb300.ncu_summary source-hash
        hash of the batched kernel's sources, recorded next to counters so that stale
        counters are recognised

Reads only the files it is given; runs nothing.
"""
from __future__ import annotations

import collections
import csv
import hashlib
import re
import sys
from pathlib import Path

CSRC = Path(__file__).resolve().parent / "csrc"

FULL_METRICS = [
    "gpu__time_duration.sum",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
    "smsp__inst_executed.sum",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "sm__warps_active.avg.per_cycle_active",
    "launch__registers_per_thread",
    "launch__grid_size",
    "launch__block_size",
    "launch__occupancy_limit_shared_mem",
    "smsp__sass_inst_executed_op_shared_ld.sum",
    "smsp__sass_inst_executed_op_shared_st.sum",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared_op_ld.sum",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared_op_st.sum",
    "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum",
    "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum.pct_of_peak_sustained_elapsed",
    "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_branch_resolving_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_not_selected_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
]


# The translation unit of the batched alignment kernel: the sources its
# counters depend on.
KERNEL_SOURCES = [CSRC / "genasm_align.cu", CSRC / "genasm_window.cuh", CSRC / "genasm_pair.cuh",
                  CSRC / "genasm_internal.h", CSRC.parent.parent / "include" / "genasm.h"]


def _code_only(text: str) -> str:
    """C/C++ source without its comments and blank space: the counters depend
    on the code alone, so editing a comment does not retire them."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "".join(text.split())


def source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(p.name.encode())
        h.update(_code_only(p.read_text()).encode())
    return h.hexdigest()[:16]


def _rows(path: str):
    lines = Path(path).read_text(errors="replace").splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith('"ID"') or l.startswith("ID,"))
    return list(csv.reader(lines[start:]))


def launches(path: str, first: int | None = None, last: int | None = None) -> str:
    """Per-kernel totals over the launches with position first..last-1 in
    the list (Python slice semantics; negative counts from the end)."""
    rows = _rows(path)
    hdr = rows[0]
    ki, mi, vi, ui = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    scale = {"nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "second": 1e3}
    agg = collections.defaultdict(lambda: [0, 0.0])
    timed = [r for r in rows[1:] if len(r) > vi and r[mi] == "gpu__time_duration.sum"]
    for r in timed[first:last]:
        name = r[ki].split("(")[0].replace("void ", "").strip()
        agg[name][0] += 1
        agg[name][1] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1e-6)
    total = sum(v[1] for v in agg.values()) or 1.0
    out = ["| kernel | launches | total ms | share |", "|---|---:|---:|---:|"]
    for name, (n, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"| `{name}` | {n} | {ms:.3f} | {100 * ms / total:.1f}% |")
    return "\n".join(out)


def full(path: str) -> str:
    rows = _rows(path)
    hdr, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        name = r[hdr.index("Kernel Name")] if "Kernel Name" in hdr else "?"
        out.append(f"### `{name.split('(')[0]}`\n")
        out.append("| counter | value | unit |\n|---|---:|---|")
        for m in FULL_METRICS:
            if m in hdr:
                i = hdr.index(m)
                out.append(f"| `{m}` | {r[i]} | {units[i]} |")
        out.append("")
    return "\n".join(out)


def main(argv):
    if len(argv) >= 1 and argv[0] == "source-hash":
        print(source_hash())
    elif len(argv) in (2, 3) and argv[0] == "launches":
        a = b = None
        if len(argv) == 3:  # "first:last"
            fa, fb = argv[2].split(":")
            a, b = (int(fa) if fa else None), (int(fb) if fb else None)
        print(launches(argv[1], a, b))
    elif len(argv) == 2 and argv[0] == "full":
        print(full(argv[1]))
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
