"""Host-side tests of the launch-shape tuner's cache (no GPU): a cached shape is
used only for the full candidate set and only with the native sources it was
measured on; an unreadable cache means tuning again; the cache file is replaced
atomically."""
import json
import os

import pytest

from paper_1403_1661_gb300 import batch


class Tuned(Exception):
    pass


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(batch, "CACHE", str(path))
    monkeypatch.setattr(batch, "_gpu_key", lambda: "FAKE_GPU")
    pytest.importorskip("torch")

    def no_solver(*a, **k):          # reaching the timing loop means a cache miss
        raise Tuned()
    from paper_1403_1661_gb300 import solver
    monkeypatch.setattr(solver, "solver_from_scenario", no_solver)
    return path


def _entry(shape, sources):
    return {"shape": shape, "ms_per_macro_step": {}, "sources": sources, "when": 0}


def test_hit_needs_the_current_sources(cache):
    key = "FAKE_GPU/N4/fp32tc/shape"
    shape = {"ctas_per_sm": 2, "tc_warps": 4}
    batch._store_cache({key: _entry(shape, batch._sources_key())})
    assert batch.tune(4, "fp32tc") == shape
    # measured on other kernels: tuned again
    batch._store_cache({key: _entry(shape, "0" * 16)})
    with pytest.raises(Tuned):
        batch.tune(4, "fp32tc")
    # an entry without a sources key (older format) is not trusted either
    batch._store_cache({key: {"shape": shape}})
    with pytest.raises(Tuned):
        batch.tune(4, "fp32tc")


def test_narrow_search_and_force_never_read_the_cache(cache):
    key = "FAKE_GPU/N3/fp32/shape"
    batch._store_cache({key: _entry({"ctas_per_sm": 1, "tc_warps": None}, batch._sources_key())})
    with pytest.raises(Tuned):
        batch.tune(3, "fp32", candidates=((1, None),))
    with pytest.raises(Tuned):
        batch.tune(3, "fp32", force=True)


def test_unreadable_cache_means_tuning_again(cache):
    cache.write_text('{"FAKE_GPU/N4/fp32tc/shape": {"shape": ')     # a torn write
    assert batch._load_cache() == {}
    with pytest.raises(Tuned):
        batch.tune(4, "fp32tc")


def test_store_replaces_the_file_whole(cache):
    batch._store_cache({"a": 1})
    batch._store_cache({"b": 2})
    assert json.loads(cache.read_text()) == {"b": 2}
    assert [f for f in os.listdir(cache.parent) if f.startswith(".autotune.")] == []


def test_sources_key_follows_the_native_sources():
    k = batch._sources_key()
    assert len(k) == 16 and k == batch._sources_key()
