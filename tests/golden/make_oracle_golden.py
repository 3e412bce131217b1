"""Writes oracle_workload1_first100.tsv: the CPU oracle's output (plain
four-vector GenASM, W=64, O=24, k=64) for pairs 0..99 of workload 1.

It calls only the oracle and the seeded input generator. Regenerate it only
when the oracle's arithmetic changes, and name in the commit message the
passage of the paper (or the reading of it) that justifies the change.
"""
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2203_15561_gb300 import datagen  # noqa: E402


def main():
    b = datagen.make_batch(1, pair_ids=range(100))
    r = oracle.align(b, W=64, O=24, k=64, variant="unimproved")
    lines = ["# pair_id\tdistance\tref_consumed\tcigar  (workload 1, seed 1, W=64 O=24 k=64)"]
    for p in range(b.n_pairs):
        lines.append(f"{int(b.pair_ids[p])}\t{int(r.dist[p])}\t{int(r.ref_consumed[p])}\t{r.cigar_str(p) or '-'}")
    (Path(__file__).resolve().parent / "oracle_workload1_first100.tsv").write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
