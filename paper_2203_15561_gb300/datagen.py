"""Seeded synthetic (read, reference) pairs for the five alignment workloads.

This module is the one piece of code that both the CPU oracle and the GPU path
consume. It holds none of the alignment arithmetic: it only draws random
sequences and applies sequencing-error models to them.

The paper evaluates on 138,929 (read, reference) pairs taken from minimap2
chains of 500 simulated 10 kb PacBio human reads (Sec. II). Neither the human
genome nor PBSIM2 nor minimap2 is available, so the generators below stand in
for that data set with the same shapes: read length, pair count and error
profile.

Every pair is drawn from its own ``numpy.random.default_rng([seed, pair_id])``
stream (PCG64), so any subset of a workload can be regenerated without drawing
the rest, and the result does not depend on which other pairs were requested.

Sequences are returned as ASCII bytes (``b"ACGT"``), laid out back to back with
each sequence starting at a multiple of four characters, so that a 2-bit packer
maps the start of every sequence to a whole byte.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterable, Sequence

import numpy as np

ALPHABET = np.frombuffer(b"ACGT", dtype=np.uint8)

# Window geometry and error cap used by every workload: W = 64, O = 24, k = 64.
DEFAULT_W = 64
DEFAULT_O = 24
DEFAULT_K = 64


@dataclasses.dataclass
class Batch:
    """A batch of pairs in the ASCII layout described in the module docstring."""

    reads: np.ndarray      # uint8 ASCII, concatenated, each start 4-aligned
    read_off: np.ndarray   # uint64 character offset of each read (multiple of 4)
    read_len: np.ndarray   # uint32 read length in bases
    refs: np.ndarray       # uint8 ASCII, concatenated, each start 4-aligned
    ref_off: np.ndarray    # uint64 character offset of each reference
    ref_len: np.ndarray    # uint32 reference length in bases
    pair_ids: np.ndarray   # uint64 pair index inside the workload
    name: str = ""

    @property
    def n_pairs(self) -> int:
        return int(self.read_len.shape[0])

    @property
    def read_bases(self) -> int:
        return int(self.read_len.sum(dtype=np.uint64))

    @property
    def ref_bases(self) -> int:
        return int(self.ref_len.sum(dtype=np.uint64))

    def read(self, p: int) -> bytes:
        o = int(self.read_off[p])
        return self.reads[o:o + int(self.read_len[p])].tobytes()

    def ref(self, p: int) -> bytes:
        o = int(self.ref_off[p])
        return self.refs[o:o + int(self.ref_len[p])].tobytes()

    def slice(self, a: int, b: int) -> "Batch":
        """Pairs a..b-1 as a Batch of their own, sharing no offsets with this one.
        Sequences are laid out back to back in pair order, so the pairs' bytes
        are one contiguous range of each buffer; offsets are rebased to it."""
        a, b = max(0, a), min(self.n_pairs, b)
        if b <= a:
            return from_pairs([], pair_ids=[], name=self.name)

        def part(buf, off, ln):
            lo = int(off[a])
            hi = max(lo, int((off[b - 1] + (ln[b - 1] + 3) // 4 * 4)))
            return buf[lo:max(hi, lo + 4)].copy(), (off[a:b] - np.uint64(lo)).astype(np.uint64)

        rb, ro = part(self.reads, self.read_off, self.read_len.astype(np.uint64))
        fb, fo = part(self.refs, self.ref_off, self.ref_len.astype(np.uint64))
        if rb.shape[0] < 4:
            rb = np.concatenate([rb, np.full(4 - rb.shape[0], ord("A"), np.uint8)])
        if fb.shape[0] < 4:
            fb = np.concatenate([fb, np.full(4 - fb.shape[0], ord("A"), np.uint8)])
        return Batch(rb, ro, self.read_len[a:b].copy(), fb, fo, self.ref_len[a:b].copy(),
                     self.pair_ids[a:b].copy(), self.name)

    def subset(self, idx: Sequence[int]) -> "Batch":
        return from_pairs([(self.read(int(p)), self.ref(int(p))) for p in idx],
                          pair_ids=[int(self.pair_ids[int(p)]) for p in idx],
                          name=self.name)


def _layout(seqs: Sequence[np.ndarray]) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Concatenate code arrays into ASCII with 4-aligned starts."""
    lens = np.fromiter((len(s) for s in seqs), dtype=np.uint64, count=len(seqs))
    padded = (lens + 3) // 4 * 4
    off = np.zeros(len(seqs), dtype=np.uint64)
    if len(seqs) > 1:
        off[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum()) if len(seqs) else 0
    buf = np.full(max(total, 4), ord("A"), dtype=np.uint8)
    for s, o in zip(seqs, off):
        if len(s):
            buf[int(o):int(o) + len(s)] = ALPHABET[s]
    return buf, off, lens.astype(np.uint32)


def from_pairs(pairs: Iterable[tuple[bytes | str, bytes | str]], pair_ids=None, name: str = "") -> Batch:
    """Build a Batch from explicit (read, reference) strings over ACGT."""
    lut = np.full(256, 255, dtype=np.uint8)
    for c, v in zip(b"ACGTacgt", (0, 1, 2, 3, 0, 1, 2, 3)):
        lut[c] = v
    reads, refs = [], []
    for r, f in pairs:
        r = r.encode() if isinstance(r, str) else bytes(r)
        f = f.encode() if isinstance(f, str) else bytes(f)
        rc = lut[np.frombuffer(r, dtype=np.uint8)] if r else np.zeros(0, np.uint8)
        fc = lut[np.frombuffer(f, dtype=np.uint8)] if f else np.zeros(0, np.uint8)
        if (rc == 255).any() or (fc == 255).any():
            raise ValueError("sequences must be over ACGT")
        reads.append(rc)
        refs.append(fc)
    return _assemble(reads, refs, pair_ids, name)


def _assemble(reads, refs, pair_ids, name) -> Batch:
    rb, ro, rl = _layout(reads)
    fb, fo, fl = _layout(refs)
    if pair_ids is None:
        pair_ids = np.arange(len(reads), dtype=np.uint64)
    return Batch(rb, ro, rl, fb, fo, fl, np.asarray(pair_ids, dtype=np.uint64), name)


# ---------------------------------------------------------------------------
# Error models
# ---------------------------------------------------------------------------

def _random_codes(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(0, 4, size=n, dtype=np.uint8)


def _substitute(rng, base: np.ndarray) -> np.ndarray:
    """Uniform replacement among the three other bases."""
    return ((base.astype(np.int64) + rng.integers(1, 4, size=base.shape[0])) % 4).astype(np.uint8)


def mutate_point(rng, src: np.ndarray, p_sub: float, p_ins: float, p_del: float) -> np.ndarray:
    """Short-read model: per source base, delete it with p_del, otherwise substitute
    it with p_sub; then insert one random base after it with p_ins."""
    n = src.shape[0]
    u = rng.random(n)
    deleted = u < p_del
    subst = (~deleted) & (u < p_del + p_sub)
    base = src.copy()
    if subst.any():
        base[subst] = _substitute(rng, src[subst])
    ins = rng.random(n) < p_ins
    ins_base = _random_codes(rng, n)
    keep = ~deleted
    count = keep.astype(np.int64) + ins.astype(np.int64)
    total = int(count.sum())
    start = np.cumsum(count) - count
    out = np.empty(total, dtype=np.uint8)
    out[start[keep]] = base[keep]
    out[(start + keep)[ins]] = ins_base[ins]
    return out


def mutate_long(rng, read_len: int, p_sub: float, p_del: float, p_ins: float,
                mean_indel: float = 1.5) -> tuple[np.ndarray, np.ndarray]:
    """Long-read model (PacBio-like).

    Per source base: a deletion event starts there with rate p_del / mean_indel,
    otherwise the base is substituted with p_sub; an insertion event follows it
    with rate p_ins / mean_indel. Event lengths are geometric on {1, 2, ...} with
    mean ``mean_indel``. Source bases are drawn until the read reaches
    ``read_len``. Returns (read codes, true source span codes)."""
    gp = 1.0 / mean_indel
    r_del = p_del / mean_indel
    r_ins = p_ins / mean_indel
    est = int(read_len / max(0.2, 1.0 - p_del + p_ins) * 1.05) + 64
    while True:
        n = est
        src = _random_codes(rng, n)
        s_idx = np.flatnonzero(rng.random(n) < r_del)
        del_len = rng.geometric(gp, size=s_idx.shape[0])
        diff = np.zeros(n + 1, dtype=np.int64)
        np.add.at(diff, s_idx, 1)
        np.add.at(diff, np.minimum(s_idx + del_len, n), -1)
        deleted = np.cumsum(diff[:n]) > 0
        subst = (~deleted) & (rng.random(n) < p_sub)
        base = src.copy()
        if subst.any():
            base[subst] = _substitute(rng, src[subst])
        i_idx = np.flatnonzero(rng.random(n) < r_ins)
        ins_len = np.zeros(n, dtype=np.int64)
        ins_len[i_idx] = rng.geometric(gp, size=i_idx.shape[0])
        keep = ~deleted
        count = keep.astype(np.int64) + ins_len
        cum = np.cumsum(count)
        if cum[-1] < read_len:
            est = int(est * 1.5) + 64
            continue
        span = int(np.searchsorted(cum, read_len)) + 1
        count = count[:span]
        keep = keep[:span]
        total = int(cum[span - 1])
        start = cum[:span] - count
        out = _random_codes(rng, total)          # inserted bases are random
        out[start[keep]] = base[:span][keep]
        return out[:read_len], src[:span]


def _flanked(rng, span: np.ndarray, flank_frac: float) -> np.ndarray:
    f = int(round(flank_frac * span.shape[0]))
    return np.concatenate([_random_codes(rng, f), span, _random_codes(rng, f)])


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

CONFIG_N_PAIRS = {1: 1_000, 2: 10_000, 3: 138_929, 4: 200_000}
CONFIG_NAMES = {
    1: "short-100bp-1000pairs",
    2: "long-10kb-10000pairs",
    3: "paper-scale-138929pairs",
    4: "mixed-100bp-50kb-200000pairs",
    5: "serving-poisson-2000rps-60s",
}


def _pair_short(rng) -> tuple[np.ndarray, np.ndarray]:
    # Workload 1: 100 bp random reference; read = reference with 2% substitutions,
    # 0.2% insertions and 0.2% deletions at uniform positions.
    ref = _random_codes(rng, 100)
    return mutate_point(rng, ref, 0.02, 0.002, 0.002), ref


def _pair_long(rng, read_len: int, p_sub=0.02, p_del=0.04, p_ins=0.06) -> tuple[np.ndarray, np.ndarray]:
    # 12% total: 2% substitutions, 4% deletions, 6% insertions (indel mean 1.5);
    # reference = true span plus a 5% random flank on each side.
    read, span = mutate_long(rng, read_len, p_sub, p_del, p_ins)
    return read, _flanked(rng, span, 0.05)


def _pair_paper_scale(rng) -> tuple[np.ndarray, np.ndarray]:
    # Workload 3: lengths normal(10000, 1500) clipped to [2000, 20000]; the
    # long-read error model; 20% decoys whose reference is unrelated.
    n = int(np.clip(round(rng.normal(10_000, 1_500)), 2_000, 20_000))
    decoy = rng.random() < 0.2
    read, ref = _pair_long(rng, n)
    if decoy:
        ref = _random_codes(rng, ref.shape[0])
    return read, ref


def _pair_mixed(rng) -> tuple[np.ndarray, np.ndarray]:
    # Workload 4: lengths log-uniform over [100, 50000]. Reads under 1 kb use the
    # short-read model (1.5% substitutions, 0.05% insertions, 0.05% deletions);
    # longer reads use the long-read model at a per-read total error rate drawn
    # uniformly from [8%, 15%], split 1:2:3 between substitutions, deletions and
    # insertions, with the 5% flank.
    n = int(round(math.exp(rng.uniform(math.log(100), math.log(50_000)))))
    if n < 1000:
        ref = _random_codes(rng, n)
        read = mutate_point(rng, ref, 0.015, 0.0005, 0.0005)
        return read, ref
    e = rng.uniform(0.08, 0.15)
    return _pair_long(rng, n, p_sub=e / 6, p_del=2 * e / 6, p_ins=3 * e / 6)


def make_pair(config: int, pair_id: int, seed: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """(read codes, reference codes) of one pair of workload ``config`` (1-4)."""
    seed = config if seed is None else seed
    rng = np.random.default_rng([seed, pair_id])
    if config == 1:
        return _pair_short(rng)
    if config == 2:
        return _pair_long(rng, 10_000)
    if config == 3:
        return _pair_paper_scale(rng)
    if config == 4:
        return _pair_mixed(rng)
    raise ValueError(f"no pair generator for workload {config}")


def _make_chunk(args):
    config, ids, seed = args
    return [make_pair(config, int(p), seed) for p in ids]


def make_batch(config: int, pair_ids: Sequence[int] | None = None, n_pairs: int | None = None,
               seed: int | None = None, workers: int = 0) -> Batch:
    """Pairs of workload ``config``. By default all of its pairs; ``pair_ids``
    selects a subset, ``n_pairs`` the first n. ``workers`` > 1 draws the pairs
    in that many spawned processes (the result does not depend on it)."""
    if pair_ids is None:
        n = CONFIG_N_PAIRS[config] if n_pairs is None else n_pairs
        pair_ids = range(n)
    ids = [int(p) for p in pair_ids]
    if workers > 1 and len(ids) >= 4 * workers:
        import concurrent.futures as cf
        import multiprocessing as mp
        step = (len(ids) + 4 * workers - 1) // (4 * workers)
        chunks = [(config, ids[x:x + step], seed) for x in range(0, len(ids), step)]
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            pairs = [pr for part in ex.map(_make_chunk, chunks) for pr in part]
    else:
        pairs = _make_chunk((config, ids, seed))
    return _assemble([r for r, _ in pairs], [f for _, f in pairs], ids, CONFIG_NAMES[config])


@dataclasses.dataclass
class Request:
    arrival_s: float
    pair_ids: np.ndarray     # ids of the workload-4-style pairs it carries


def make_requests(rate_per_s: float = 2000.0, duration_s: float = 60.0, seed: int = 5,
                  max_pairs: int = 64) -> list[Request]:
    """Workload 5: open-loop Poisson arrivals; each request carries 1..64
    (uniform) pairs drawn from the workload-4 distribution. Pair j of the
    stream is ``make_pair(4, j, seed=seed)``."""
    rng = np.random.default_rng([seed, 1 << 40])
    t, nxt, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return out
        k = int(rng.integers(1, max_pairs + 1))
        out.append(Request(t, np.arange(nxt, nxt + k, dtype=np.uint64)))
        nxt += k
