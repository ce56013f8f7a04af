"""The autotuner's table on the host (no GPU): what synthpix_tuning_set
writes, synthpix_tuning_lookup reads and synthpix_tuning_clear empties; the
workspace of a tile-0 batch covers every tuning."""
import ctypes as C

import pytest

from paper_2512_09664_b300 import binding as B
from paper_2512_09664_b300 import workloads as W


@pytest.fixture(autouse=True)
def _clean_table():
    B.tuning_clear()
    yield
    B.tuning_clear()


def _lookup(pk):
    t = B.Tuning()
    assert B.lib().synthpix_tuning_lookup(C.byref(pk.batch), pk.pairs, pk.n_pairs, C.byref(t)) == B.OK
    return t.as_dict()


def _set(pk, tile, rps, epi):
    t = B.Tuning()
    for k in range(4):
        t.tile[k] = tile[k]
    t.records_per_stage, t.register_epilogue = rps, epi
    return B.lib().synthpix_tuning_set(C.byref(pk.batch), pk.pairs, pk.n_pairs, C.byref(t))


def test_defaults_by_size_class():
    # classes by frame area: < 2^15, < 2^17, < 2^19, larger
    wl = W.uneven_batch(n_pairs=8, sizes=(64, 256, 512, 1024))
    pk = B.pack(wl)
    got = _lookup(pk)
    present = {B.size_class(p.height, p.width) for p in wl.pairs}
    assert got["tile"] == [e if k in present else 0 for k, e in enumerate((32, 64, 128, 128))]
    assert got["register_epilogue"] == 1 and got["records_per_stage"] > 0
    assert B.size_class(181, 181) == 0 and B.size_class(182, 181) == 1 and B.size_class(512, 512) == 2
    assert B.size_class(1024, 512) == 3


def test_set_lookup_clear_round_trip_and_sharing():
    wl = W.uneven_batch(n_pairs=6, sizes=(128, 512))
    pk = B.pack(wl)
    assert _set(pk, [16, 0, 64, 0], 200, 0) == B.OK
    got = _lookup(pk)
    assert got["tile"] == [16, 0, 64, 0] and got["records_per_stage"] == 200 and got["register_epilogue"] == 0
    # another batch of the same classes, diameters and blur shares the entries
    other = B.pack(W.uneven_batch(n_pairs=3, sizes=(128, 512), seed=9))
    assert _lookup(other)["tile"][2] == 64
    # a batch with a fixed edge ignores the table
    fixed = B.pack(wl, tile=32)
    assert _lookup(fixed)["tile"][0] == 32
    B.tuning_clear()
    assert _lookup(pk)["tile"] == [32, 0, 128, 0]


def test_set_rejects_bad_values():
    pk = B.pack(W.uneven_batch(n_pairs=4, sizes=(128, 512)))
    assert _set(pk, [24, 0, 64, 0], 200, 1) == B.EINVAL
    assert _set(pk, [32, 0, 64, 0], 0, 1) == B.EINVAL
    assert _set(pk, [32, 0, 64, 0], 200, 2) == B.EINVAL
    # more records than the staging buffers of the largest edge hold
    assert _set(pk, [32, 0, 64, 0], 4000, 1) == B.EUNSUPPORTED
    fixed = B.pack(W.uneven_batch(n_pairs=4, sizes=(128, 512)), tile=64)
    assert _set(fixed, [32, 0, 64, 0], 200, 1) == B.EINVAL


def test_tile0_workspace_covers_every_uniform_edge():
    wl = W.uneven_batch(n_pairs=10, sizes=(64, 128, 256, 512, 1024))
    bound = B.workspace_bytes(B.pack(wl))
    for t in (16, 32, 64, 128):
        assert B.workspace_bytes(B.pack(wl, tile=t)) <= bound


def test_cached_record_buffers_fit_a_batch_of_smaller_edges():
    # records per stage tuned with 128-pixel tiles (a 25 KB record region, 1078
    # records) for a batch of two classes; a batch holding only the class cached
    # with edge 32 (19 KB at most, 822 records) resolves the same entry with its
    # record region clamped, not rejected
    wl = W.uneven_batch(n_pairs=12, sizes=(128, 512))
    pk = B.pack(wl)
    c_small, c_big = B.size_class(128, 128), B.size_class(512, 512)
    tile = [0, 0, 0, 0]
    tile[c_small], tile[c_big] = 32, 128
    assert _set(pk, tile, 1000, 1) == B.OK
    big = _lookup(pk)
    assert big["tile"][c_big] == 128 and big["records_per_stage"] == 1000
    small = B.pack(wl.subset([b for b, p in enumerate(wl.pairs) if p.height == 128][:1]))
    got = _lookup(small)
    assert got["tile"][c_small] == 32 and 0 < got["records_per_stage"] < 1000
    assert B.workspace_bytes(small) > 0

