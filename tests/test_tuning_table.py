"""Host side of the launch-shape table (no GPU needed): lookup by grid bits and
the bit length of the element count, validation of shapes, reset, and the JSON
cache round trip of the Python binding."""
import json
import os

import pytest

from paper_2110_11616_gb300 import cga


@pytest.fixture()
def lib():
    lib = cga.load()
    yield lib
    for bits in range(1, 17):
        for nb in range(0, 33):
            cga.tuning_set(bits, (1 << (nb - 1)) if nb else 0, None)


def test_default_shape(lib):
    for bits in (1, 10, 16):
        for n in (0, 1, 4096, 30_000_000):
            assert cga.tuning_get(bits, n) == cga.DEFAULT_TUNING


def test_entries_are_keyed_by_bits_and_bit_length(lib):
    s = {"radix_bits": 9, "sort_threads": 512, "merge_half": 1024}
    cga.tuning_set(12, 20_000_000, s)                       # bit length 25
    assert cga.tuning_get(12, 1 << 24) == s                 # same bucket, lower edge
    assert cga.tuning_get(12, (1 << 25) - 1) == s           # upper edge
    assert cga.tuning_get(12, 1 << 25) == cga.DEFAULT_TUNING
    assert cga.tuning_get(12, (1 << 24) - 1) == cga.DEFAULT_TUNING
    assert cga.tuning_get(11, 20_000_000) == cga.DEFAULT_TUNING
    cga.tuning_set(12, 20_000_000, None)
    assert cga.tuning_get(12, 20_000_000) == cga.DEFAULT_TUNING


@pytest.mark.parametrize("rb,th,half", [(8, 256, 512), (8, 512, 1024), (9, 512, 2048)])
def test_every_candidate_is_accepted(lib, rb, th, half):
    s = {"radix_bits": rb, "sort_threads": th, "merge_half": half}
    cga.tuning_set(16, 1000, s)
    assert cga.tuning_get(16, 1000) == s


@pytest.mark.parametrize("rb,th,half", [(9, 256, 2048), (7, 512, 2048), (10, 512, 2048),
                                        (8, 128, 2048), (8, 1024, 2048), (8, 512, 4096),
                                        (8, 512, 256), (8, 512, 1500), (0, 0, 0)])
def test_invalid_shapes_are_rejected(lib, rb, th, half):
    with pytest.raises(cga.CgaError) as e:
        cga.tuning_set(10, 1000, {"radix_bits": rb, "sort_threads": th, "merge_half": half})
    assert e.value.code == cga.ERR_INVALID_ARG
    assert cga.tuning_get(10, 1000) == cga.DEFAULT_TUNING


def test_bits_out_of_range(lib):
    for bits in (0, 17):
        with pytest.raises(cga.CgaError):
            cga.tuning_get(bits, 10)
        with pytest.raises(cga.CgaError):
            cga.tuning_set(bits, 10, None)


def test_cache_round_trip(lib, tmp_path):
    path = str(tmp_path / "tuning.json")
    a = {"radix_bits": 9, "sort_threads": 512, "merge_half": 512}
    b = {"radix_bits": 8, "sort_threads": 256, "merge_half": 1024}
    cga.tuning_set(12, 30_000_000, a)
    cga.tuning_set(16, 131_072, b)
    cga.tuning_cache_save(path, device="dev-A")
    cga.tuning_cache_save(path, device="dev-B")
    data = json.load(open(path))
    assert set(data) == {"dev-A", "dev-B"} and len(data["dev-A"]) == 2
    cga.tuning_set(12, 30_000_000, None)
    cga.tuning_set(16, 131_072, None)
    assert cga.tuning_cache_load(path, device="dev-C") == 0
    assert cga.tuning_get(12, 30_000_000) == cga.DEFAULT_TUNING
    assert cga.tuning_cache_load(path, device="dev-A") == 2
    assert cga.tuning_get(12, 30_000_000) == a
    assert cga.tuning_get(16, 131_072) == b
    assert not os.path.exists(str(tmp_path / "missing.json"))
    assert cga.tuning_cache_load(str(tmp_path / "missing.json"), device="dev-A") == 0
