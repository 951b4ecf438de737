"""Tuning cache of the autotuner (host-only calls of the C ABI)."""
import pytest


@pytest.fixture(scope="module")
def rg():
    import paper_1810_12163_gb300 as rg
    try:
        rg.lib()
    except OSError as e:  # library not built here
        pytest.skip(str(e))
    return rg


def test_round_trip_and_replacement(rg, tmp_path):
    path = str(tmp_path / "tuning.txt")
    assert rg.tuning_cache_read(path, "gpu|a") is None            # no file yet
    a = dict(hypgen_warps=8, energy_threads=256, leaves_threads=64, mask_threads=128, streams=2)
    b = dict(hypgen_warps=2, energy_threads=32, leaves_threads=512, mask_threads=64, streams=4)
    rg.tuning_cache_write(path, "gpu|a", a)
    rg.tuning_cache_write(path, "gpu|b", b)
    assert rg.tuning_cache_read(path, "gpu|a") == a
    assert rg.tuning_cache_read(path, "gpu|b") == b
    assert rg.tuning_cache_read(path, "gpu|c") is None
    rg.tuning_cache_write(path, "gpu|a", b)                        # replaces the line
    assert rg.tuning_cache_read(path, "gpu|a") == b
    lines = open(path).read().splitlines()
    assert len(lines) == 2 and sum(l.startswith("gpu|a =") for l in lines) == 1


def test_values_outside_the_lists_are_refused(rg, tmp_path):
    path = str(tmp_path / "tuning.txt")
    bad = dict(hypgen_warps=3, energy_threads=128, leaves_threads=128, mask_threads=256)
    with pytest.raises(rg.RelocError) as e:
        rg.tuning_cache_write(path, "k", bad)
    assert e.value.status == 1                                     # RL_ERR_INVALID_ARG
    with pytest.raises(rg.RelocError):
        rg.tuning_cache_write(path, "k", dict(hypgen_warps=4, energy_threads=128, leaves_threads=128,
                                              mask_threads=256, streams=3))
    with open(path, "w") as f:                                     # a corrupt entry is ignored
        f.write("k = 3 128 128 256\nj = 4 128 128\ni = 4 128 128 256 3\n")
    assert rg.tuning_cache_read(path, "k") is None
    assert rg.tuning_cache_read(path, "j") is None
    assert rg.tuning_cache_read(path, "i") is None


def test_every_stream_count_round_trips(rg, tmp_path):
    path = str(tmp_path / "tuning.txt")
    for k in (1, 2, 4, 8):
        t = dict(hypgen_warps=16, energy_threads=128, leaves_threads=128, mask_threads=256, streams=k)
        rg.tuning_cache_write(path, f"k{k}", t)
        assert rg.tuning_cache_read(path, f"k{k}") == t
    with pytest.raises(rg.RelocError):
        rg.tuning_cache_write(path, "k16", dict(hypgen_warps=16, energy_threads=128, leaves_threads=128,
                                                mask_threads=256, streams=16))


def test_entries_without_streams_read_as_one_stream(rg, tmp_path):
    path = str(tmp_path / "tuning.txt")
    with open(path, "w") as f:                                     # written before the streams knob
        f.write("k = 8 64 256 128\n")
    assert rg.tuning_cache_read(path, "k") == dict(hypgen_warps=8, energy_threads=64, leaves_threads=256,
                                                   mask_threads=128, streams=1)
