"""GPU tests of the alignment server (continuous batching): every request's
result is the same when it runs alone and when it shares steps with others,
and equals the CPU oracle; requests wait for memory when the budget is tight."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2203_15561_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_15561_gb300 as ga  # noqa: E402
from paper_2203_15561_gb300.serving import Server  # noqa: E402


def request_batches(n_requests: int, seed: int = 5):
    reqs = datagen.make_requests(rate_per_s=2000.0, duration_s=n_requests / 1500.0, seed=seed)[:n_requests]
    return [datagen.make_batch(4, pair_ids=list(r.pair_ids), seed=seed) for r in reqs]


def drain(server, want: int, max_steps: int = 100000):
    got = {}
    for _ in range(max_steps):
        if len(got) >= want:
            break
        server.step()
        for r in server.poll():
            got[r.tag] = r
    return got


def check_against_oracle(batch, res):
    ref = oracle.align(batch)
    np.testing.assert_array_equal(res.dist, ref.dist)
    np.testing.assert_array_equal(res.status, ref.status)
    np.testing.assert_array_equal(res.ref_consumed, ref.ref_consumed)
    for p in range(batch.n_pairs):
        np.testing.assert_array_equal(res.runs(p), ref.runs(p))


def test_same_alone_and_in_the_mix():
    batches = request_batches(12)
    # In the mix: staggered submissions so requests join while others run.
    srv = Server(2 << 30, step_windows=8)
    got = {}
    for t, b in enumerate(batches):
        srv.submit(b, tag=t)
        srv.step()
        for r in srv.poll():
            got[r.tag] = r
    got.update(drain(srv, len(batches) - len(got)))
    srv.close()
    assert len(got) == len(batches)
    # Alone: one request at a time in a fresh server.
    for t, b in enumerate(batches):
        one = Server(2 << 30, step_windows=64)
        one.submit(b, tag=t)
        alone = drain(one, 1)[t]
        one.close()
        mix = got[t]
        np.testing.assert_array_equal(alone.dist, mix.dist)
        np.testing.assert_array_equal(alone.cigar_off, mix.cigar_off)
        np.testing.assert_array_equal(alone.cigar, mix.cigar)
        check_against_oracle(b, mix)


def test_workload5_two_seconds_every_request_against_oracle():
    # Workload 5 as it arrives: Poisson requests at 2,000/s, each 1-64 fresh pairs of the
    # workload-4 distribution (pair j of the stream is make_pair(4, j, seed=5)), submitted
    # in real time for 2 s of arrivals while the server steps, then drained. Every served
    # request must equal the oracle on the same pairs.
    import os
    import time

    from fullparity import oracle_dense

    reqs = datagen.make_requests(2000.0, 2.0, seed=5)
    bounds = np.cumsum([0] + [len(r.pair_ids) for r in reqs])
    assert bounds[-1] > 100_000
    batch = datagen.make_batch(4, pair_ids=range(int(bounds[-1])), seed=5,
                               workers=min(16, len(os.sched_getaffinity(0))))
    parts = [batch.slice(int(bounds[i]), int(bounds[i + 1])) for i in range(len(reqs))]
    srv = Server(8 << 30, step_windows=48)
    got, nxt = {}, 0
    t0 = time.perf_counter()
    while len(got) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
            srv.submit(parts[nxt], tag=nxt)
            nxt += 1
        srv.step()
        for r in srv.poll(1024):
            got[r.tag] = r
        assert time.perf_counter() - t0 < 600, "server did not drain"
    srv.close()
    ref = oracle.align(batch)
    dist = np.concatenate([got[i].dist for i in range(len(reqs))])
    status = np.concatenate([got[i].status for i in range(len(reqs))])
    rc = np.concatenate([got[i].ref_consumed for i in range(len(reqs))])
    runs = np.concatenate([got[i].cigar for i in range(len(reqs))])
    np.testing.assert_array_equal(status, ref.status)
    np.testing.assert_array_equal(dist, ref.dist)
    np.testing.assert_array_equal(rc, ref.ref_consumed)
    if not np.array_equal(runs, oracle_dense(ref)):
        for i in range(len(reqs)):
            for q in range(got[i].n_pairs):
                p = int(bounds[i]) + q
                assert np.array_equal(got[i].runs(q), ref.runs(p)), f"request {i}, pair {p}"
        raise AssertionError("CIGAR runs differ")


def test_tight_budget_admits_by_memory():
    batches = request_batches(6, seed=9)
    # Just above the server's fixed needs: requests must wait for memory.
    srv = None
    for budget in (200 << 20, 256 << 20, 400 << 20):
        try:
            srv = Server(budget, step_windows=16)
            break
        except ga.GenasmError:
            continue
    assert srv is not None
    tickets = []
    for t, b in enumerate(batches):
        try:
            tickets.append(srv.submit(b, tag=t))
        except ga.GenasmError as e:  # a request larger than the whole arena
            assert e.code == ga.GA_ENOMEM
    got = drain(srv, len(tickets))
    srv.close()
    assert len(got) == len(tickets)
    for t, r in got.items():
        check_against_oracle(batches[t], r)


def test_empty_request_between_real_ones():
    # A request with no pairs completes at admission, without device space or a
    # launch, and does not hold back the requests around it.
    batches = request_batches(2, seed=11)
    empty = datagen.from_pairs([])
    srv = Server(1 << 30, step_windows=16)
    tickets = [srv.submit(batches[0], tag=0), srv.submit(empty, tag=1), srv.submit(batches[1], tag=2)]
    assert len(set(tickets)) == 3
    got = drain(srv, 3, max_steps=20000)
    waiting, active, _ = srv.pending()
    srv.close()
    assert sorted(got) == [0, 1, 2]
    assert got[1].n_pairs == 0 and got[1].cigar.size == 0
    assert waiting == 0 and active == 0
    check_against_oracle(batches[0], got[0])
    check_against_oracle(batches[1], got[2])


def test_pending_limit_refuses_then_takes_every_request():
    # A pending limit below one request's size: while a request waits for
    # admission every other submission is refused (GA_EAGAIN, nothing copied);
    # the wrapper then steps (admitting the waiting one) and submits again.
    # Every result still equals the oracle.
    batches = request_batches(8, seed=17)
    srv = Server(1 << 30, step_windows=16, pending_limit=1)
    tickets = [srv.submit(b, tag=t) for t, b in enumerate(batches)]
    assert len(set(tickets)) == len(batches)
    assert srv.refusals >= len(batches) - 1
    got = drain(srv, len(batches))
    waiting, active, _ = srv.pending()
    srv.close()
    assert sorted(got) == list(range(len(batches)))
    assert waiting == 0 and active == 0
    for t, r in got.items():
        check_against_oracle(batches[t], r)


def test_oversize_request_refused():
    srv = Server(1 << 30)
    big = datagen.from_pairs([("A" * 10_000_000, "C" * 10_000_000)])  # more runs than a step can return
    with pytest.raises(ga.GenasmError) as e:
        srv.submit(big)
    assert e.value.code == ga.GA_ENOMEM
    srv.close()


def test_results_held_past_the_result_arena():
    # Results stay valid until released. With every result held, a server whose pinned result
    # arena (a sixteenth of the budget) is smaller than the results' runs must hand the later
    # ones out through its heap path; all must still equal the oracle.
    budget = 480 << 20  # a 30 MB result arena; the results' runs take about 45 MB
    srv = Server(budget, step_windows=64)
    batches = request_batches(80, seed=13)
    for t, b in enumerate(batches):
        srv.submit(b, tag=t)
    got = {}
    for _ in range(100000):
        if len(got) == len(batches):
            break
        srv.step()
        for r in srv.poll(release=False):
            got[r.tag] = r
    assert len(got) == len(batches)
    total_runs = sum(int(r.cigar.size) for r in got.values())
    assert 4 * total_runs > budget // 16, "the results fit the arena: the heap path was not taken"
    for t, r in got.items():
        check_against_oracle(batches[t], r)
    for r in got.values():
        srv.release(r.ticket)
    waiting, active, _ = srv.pending()
    srv.close()
    assert waiting == 0 and active == 0

