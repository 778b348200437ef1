"""Host logic of the batch autotuner's cache (CPU): a miss runs the tuner and
stores (z chunk, prefetch, tile shape, ms per step) under the members' sizes
and storage; a hit configures the batch without trials; an entry in the
older three-field form (no tile shape) counts as a miss.  The library calls
are replaced by fakes that record what the batch asked for."""
import json
from types import SimpleNamespace

import pytest

from paper_1410_1914_gb300 import batch as B


class FakeLib:
    def __init__(self):
        self.calls = []

    def cl_batch_create(self, handles, z_chunk):
        self.calls.append(("create", tuple(handles), z_chunk))
        return 1234

    def cl_batch_autotune(self, b, steps):
        self.calls.append(("autotune", b, steps))
        return 64, 2, 4, 0.5

    def cl_batch_configure(self, b, zc, pf, tr):
        self.calls.append(("configure", b, zc, pf, tr))

    def cl_batch_destroy(self, b):
        self.calls.append(("destroy", b))


def _solvers(shapes, storage=1):
    return [SimpleNamespace(h=100 + i, shape=s, params=SimpleNamespace(storage=storage))
            for i, s in enumerate(shapes)]


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    for name in ("cl_batch_create", "cl_batch_autotune", "cl_batch_configure", "cl_batch_destroy"):
        monkeypatch.setattr(B.L, name, getattr(lib, name))
    return lib


def test_miss_then_hit(fake, tmp_path):
    cache = str(tmp_path / "sub" / "tune.json")
    b = B.Batch(_solvers([(32, 40, 48), (20, 20, 20)]))
    assert fake.calls[0] == ("create", (100, 101), 0)
    assert b.autotune(steps_per_trial=4, cache=cache) == (64, 2, 4, 0.5, False)
    assert ("autotune", 1234, 4) in fake.calls
    table = json.load(open(cache))
    assert list(table.values()) == [[64, 2, 4, 0.5]]
    fake.calls.clear()
    # the same sizes in another order and another batch: a hit, no trials
    b2 = B.Batch(_solvers([(20, 20, 20), (32, 40, 48)]))
    assert b2.autotune(steps_per_trial=4, cache=cache) == (64, 2, 4, 0.5, True)
    assert ("configure", 1234, 64, 2, 4) in fake.calls
    assert not [c for c in fake.calls if c[0] == "autotune"]
    b.close()
    b2.close()


def test_key_separates_storage_and_sizes(fake, tmp_path):
    a = B.Batch(_solvers([(8, 8, 8)], storage=1)).signature()
    b = B.Batch(_solvers([(8, 8, 8)], storage=2)).signature()
    c = B.Batch(_solvers([(8, 8, 16)], storage=1)).signature()
    assert len({a, b, c}) == 3


def test_three_field_entry_is_a_miss(fake, tmp_path):
    cache = tmp_path / "tune.json"
    b = B.Batch(_solvers([(16, 16, 16)]))
    cache.write_text(json.dumps({b.signature(): [32, 0, 0.7]}))
    assert b.autotune(steps_per_trial=2, cache=str(cache)) == (64, 2, 4, 0.5, False)
    assert json.load(open(cache))[b.signature()] == [64, 2, 4, 0.5]
    b.close()


def test_unreadable_cache_is_ignored(fake, tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{ not json")
    b = B.Batch(_solvers([(16, 16, 16)]))
    assert b.autotune(steps_per_trial=2, cache=str(cache))[-1] is False
    b.close()


def test_no_cache(fake):
    b = B.Batch(_solvers([(16, 16, 16)]))
    assert b.autotune(steps_per_trial=2, cache=None) == (64, 2, 4, 0.5, False)
    b.close()
    assert ("destroy", 1234) in fake.calls
