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
