"""The autotuner's cache file (host code of libpic, no GPU): entries written by
pic_tune_cache_store read back unchanged by pic_tune_cache_load, another key
left alone when one is replaced, the file a valid JSON object, and missing
keys, missing files and keys with a quote rejected; an entry written before
the sort order was a choice reads as order 0."""
import json

import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    P.load()


def test_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    a = {"sort_every": 4, "tile": [8, 8, 8], "halo": 2, "order": 0}
    b = {"sort_every": 6, "tile": [16, 8, 4], "halo": 1, "order": 1}
    ka = "NVIDIA GB300|256x256x1024|5.0e+08|mixed"
    kb = "NVIDIA GB300|64x64x256|1.0e+07|mixed"
    assert P.pic_tune_cache_load(path, ka) is None            # no file yet
    P.pic_tune_cache_store(path, ka, a)
    P.pic_tune_cache_store(path, kb, b)
    assert P.pic_tune_cache_load(path, ka) == a
    assert P.pic_tune_cache_load(path, kb) == b
    a2 = dict(a, sort_every=3, halo=3, order=1)
    P.pic_tune_cache_store(path, ka, a2)                      # replace one entry
    assert P.pic_tune_cache_load(path, ka) == a2
    assert P.pic_tune_cache_load(path, kb) == b
    doc = json.load(open(path))
    assert doc == {ka: a2, kb: b}
    assert P.pic_tune_cache_load(path, "other|1x1x1|1.0e+00|fp64") is None
    with pytest.raises(P.PicError):
        P.pic_tune_cache_store(path, 'bad"key', a)


def test_entry_without_order_reads_as_cell_order(tmp_path):
    path = tmp_path / "old.json"
    key = "NVIDIA GB300|64x64x256|1.0e+07|mixed"
    path.write_text('{\n"' + key + '": {"sort_every": 8, "tile": [16, 8, 4], "halo": 2}\n}\n')
    assert P.pic_tune_cache_load(str(path), key) == {"sort_every": 8, "tile": [16, 8, 4], "halo": 2, "order": 0}
