"""Hash of the batched alignment kernel's sources.

Profiler counters of the batched kernel (DRAM bytes per launch) are committed
next to the hash of the sources they were taken from; ``bench.py`` reports
them only while the hash still matches, so a changed kernel never carries
stale counters. The hash covers code only: editing a comment or blank space
keeps the counters.
"""
from __future__ import annotations

import hashlib
import re
from pathlib import Path

CSRC = Path(__file__).resolve().parent / "csrc"

# The translation unit of the batched alignment kernel: the sources its
# counters depend on.
KERNEL_SOURCES = [CSRC / "genasm_align.cu", CSRC / "genasm_window.cuh", CSRC / "genasm_pair.cuh",
                  CSRC / "genasm_internal.h", CSRC.parent.parent / "include" / "genasm.h"]


def _code_only(text: str) -> str:
    """C/C++ source without its comments and blank space."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "".join(text.split())


def source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for p in sources or KERNEL_SOURCES:
        h.update(p.name.encode())
        h.update(_code_only(p.read_text()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    print(source_hash())
