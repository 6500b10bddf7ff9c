"""Host-side logic of the serving loop: pool accounting under a budget (CPU only)."""
import pytest

from paper_2311_05038_b300 import serving


class Fake:
    def __init__(self, key):
        self.key = key
        self.closed = False


def make_pool(budget):
    made, destroyed = [], []

    def create(key):
        m = Fake(key)
        made.append(m)
        return m

    def destroy(m):
        m.closed = True
        destroyed.append(m)

    return serving.ModelPool(budget, create, destroy), made, destroyed


def test_reuses_idle_models_of_the_same_key():
    pool, made, destroyed = make_pool(100)
    a = pool.acquire("a", 40)
    pool.release("a", a)
    assert pool.acquire("a", 40) is a
    assert len(made) == 1 and not destroyed


def test_budget_blocks_until_release():
    pool, made, _ = make_pool(100)
    a1 = pool.acquire("a", 40)
    a2 = pool.acquire("a", 40)
    assert pool.acquire("a", 40) is None          # 120 > 100 and nothing idle
    pool.release("a", a1)
    assert pool.acquire("a", 40) is a1
    assert pool.used == 80 and pool.peak == 80
    del a2


def test_evicts_idle_models_of_other_keys_only():
    pool, made, destroyed = make_pool(100)
    b = pool.acquire("b", 60)
    assert pool.acquire("a", 60) is None          # b is busy: cannot evict
    pool.release("b", b)
    a = pool.acquire("a", 60)                     # now b is idle: evicted
    assert destroyed == [b] and a.key == "a" and pool.used == 60


def test_never_exceeds_budget():
    import random
    rnd = random.Random(0)
    pool, _, _ = make_pool(1000)
    busy = []
    for _ in range(500):
        if busy and rnd.random() < 0.5:
            k, m = busy.pop(rnd.randrange(len(busy)))
            pool.release(k, m)
        else:
            k = rnd.choice("abcd")
            m = pool.acquire(k, {"a": 100, "b": 250, "c": 400, "d": 50}[k])
            if m is not None:
                busy.append((k, m))
        assert pool.used <= 1000
    assert pool.peak <= 1000


def test_single_model_larger_than_budget_is_an_error():
    pool, _, _ = make_pool(10)
    with pytest.raises(ValueError):
        pool.acquire("a", 11)


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert serving.percentile(v, 50) == 50 and serving.percentile(v, 99) == 99
    assert serving.percentile([3.0], 99) == 3.0


# ------------------------------------------------------------------ scheduling policy

class Req:
    def __init__(self, rid, arrival, npoints=1000, nt=100, work_left=None, fits=True):
        self.rid, self.arrival, self.npoints, self.nt = rid, arrival, npoints, nt
        self.work_left = npoints * nt if work_left is None else work_left
        self.fits = fits


def test_admission_keeps_arrival_order_when_everything_fits():
    waiting = [Req(i, 0.1 * i) for i in range(5)]
    got, byp = serving.admit_in_order(waiting, 3, 0, 8, lambda q: q if q.fits else None)
    assert [q.rid for q in got] == [0, 1, 2] and [q.rid for q in waiting] == [3, 4] and byp == 0


def test_admission_lets_fitting_requests_pass_a_blocked_head_up_to_the_bound():
    waiting = [Req(0, 0.0, fits=False)] + [Req(i, 0.1 * i) for i in range(1, 6)]
    got, byp = serving.admit_in_order(waiting, 10, 0, 3, lambda q: q if q.fits else None)
    assert [q.rid for q in got] == [1, 2, 3] and byp == 3          # three passed, then the head blocks
    assert waiting[0].rid == 0
    got, byp = serving.admit_in_order(waiting, 10, byp, 3, lambda q: q if q.fits else None)
    assert got == [] and byp == 3                                  # nothing more passes it
    waiting[0].fits = True
    got, byp = serving.admit_in_order(waiting, 1, byp, 3, lambda q: q if q.fits else None)
    assert [q.rid for q in got] == [0] and byp == 0                # the head goes first, the count resets


def test_priority_rankings():
    a = Req(0, 0.0, npoints=10**6, nt=2000)     # old, big
    b = Req(1, 0.5, npoints=10**3, nt=100)      # newer, tiny
    c = Req(2, 0.2, npoints=10**5, nt=500, work_left=10)
    assert [r.rid for r in serving.rank_active([a, b, c], "age")] == [0, 2, 1]
    assert [r.rid for r in serving.rank_active([a, b, c], "oldest+srpt")] == [0, 2, 1]
    # deadline: arrival + 2 x npoints x nt / 300e9 -> a: 0.0133, b: 0.5, c: 0.2003
    assert [r.rid for r in serving.rank_active([a, b, c], "deadline")] == [0, 2, 1]
    late_big = Req(3, 0.0, npoints=10**8, nt=2000)   # due 1.33 s after arrival
    assert [r.rid for r in serving.rank_active([late_big, b], "deadline")] == [1, 3]
    with pytest.raises(ValueError):
        serving.rank_active([a], "fifo")
