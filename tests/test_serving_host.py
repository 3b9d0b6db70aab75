"""Serving host logic without a GPU: FIFO admission under a byte budget and a
slot limit, and the seeded request stream."""
import numpy as np

from paper_1709_02733_b300.serving import Admission, make_stream


def test_fifo_admission_blocks_behind_a_large_request():
    adm = Admission(budget_bytes=100, max_slots=8)
    q = [("a", 40), ("b", 50), ("c", 30), ("d", 5)]
    got = adm.admit(q, lambda r: r[1])
    assert [r[0] for r in got] == ["a", "b"]          # c does not fit: FIFO stops there
    assert adm.used == 90 and adm.slots == 2 and [r[0] for r in q] == ["c", "d"]
    adm.release(40)
    got = adm.admit(q, lambda r: r[1])
    assert [r[0] for r in got] == ["c", "d"] and adm.used == 85 and not q


def test_slot_limit():
    adm = Admission(budget_bytes=10 ** 9, max_slots=3)
    q = [(k, 1) for k in range(5)]
    assert len(adm.admit(q, lambda r: r[1])) == 3 and len(q) == 2
    adm.release(1)
    assert len(adm.admit(q, lambda r: r[1])) == 1


def test_release_never_goes_negative():
    adm = Admission(10, 2)
    adm.take(4)
    adm.release(4)
    try:
        adm.release(1)
    except AssertionError:
        return
    raise AssertionError("release below zero was accepted")


def test_stream_is_seeded_and_in_range():
    a, b = make_stream(200, seed=5), make_stream(200, seed=5)
    assert [(r.arrival, r.n, r.nsteps, r.L, r.adjoint) for r in a] == \
           [(r.arrival, r.n, r.nsteps, r.L, r.adjoint) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert 0.015 < gaps.mean() < 0.035                 # Poisson at 40 req/s: mean gap 25 ms
    assert all(96 <= r.n <= 320 and r.n % 8 == 0 for r in a)
    assert all(800 <= r.nsteps <= 2500 and 64 <= r.L <= 512 for r in a)
    frac_adj = np.mean([r.adjoint for r in a])
    assert 0.35 < frac_adj < 0.65


def test_pick_to_advance_shortest_remaining_first():
    from paper_1709_02733_b300.serving import pick_to_advance
    rem = [50.0, 10.0, 30.0, 10.0]
    pts = [8, 2, 4, 2]
    # ascending remaining work, ties by index, until the points reach the bound
    assert pick_to_advance(rem, pts, 1) == [1]
    assert pick_to_advance(rem, pts, 4) == [1, 3]
    assert pick_to_advance(rem, pts, 5) == [1, 3, 2]
    assert pick_to_advance(rem, pts, 10 ** 9) == [1, 3, 2, 0]
    assert pick_to_advance([], [], 4) == []
    # a large solve alone is still advanced
    assert pick_to_advance([5.0], [100], 4) == [0]
