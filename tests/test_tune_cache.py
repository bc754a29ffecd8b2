"""The autotuner's cache file (host only, no GPU): entries round-trip, the
last line with a key wins, malformed lines and invalid choices are skipped
or refused, keys with tabs or newlines are refused."""
import pytest

from paper_2412_11809_gb300 import TpcError, Tuning, binding


def test_cache_round_trip_and_last_line_wins(tmp_path):
    path = str(tmp_path / "tune.txt")
    key = "NVIDIA GB300|152|256x256:b25|448x512:b24|n16"
    assert binding.tune_cache_lookup(path, key) is None            # no file yet
    t1 = Tuning(ctas_sort=2, ctas_link=1, ctas_acc=3, ctas_out=4, acc_span=512, general_link=2, order=1)
    binding.tune_cache_store(path, key, t1, 3.25)
    binding.tune_cache_store(path, "other|key", {"acc_span": 2048}, 1.0)
    got, ms = binding.tune_cache_lookup(path, key)
    assert got.as_dict() == t1.as_dict() and ms == pytest.approx(3.25)
    t2 = Tuning(acc_span=2048, order=1)
    binding.tune_cache_store(path, key, t2, 2.5)
    got, ms = binding.tune_cache_lookup(path, key)
    assert got.as_dict() == t2.as_dict() and ms == pytest.approx(2.5)
    other, _ = binding.tune_cache_lookup(path, "other|key")
    assert other.acc_span == 2048 and other.ctas_sort == 0
    assert binding.tune_cache_lookup(path, "absent|key") is None
    # a prefix of a stored key is another key
    assert binding.tune_cache_lookup(path, key[:-1]) is None


def test_cache_skips_malformed_lines(tmp_path):
    path = tmp_path / "tune.txt"
    key = "k"
    path.write_text("k\t1 2 3\t1.0\n"               # too few fields
                    "k\t1 1 1 1 777 0 0\t1.0\n"     # acc_span not 512/1024/2048
                    "k\t1 1 1 1 1024 9 0\t1.0\n"    # general_link > 3
                    "garbage line without tabs\n"
                    "k\t0 1 0 2 2048 1 1\t4.5\n")
    got, ms = binding.tune_cache_lookup(str(path), key)
    assert got.as_dict() == {"ctas_sort": 0, "ctas_link": 1, "ctas_acc": 0, "ctas_out": 2,
                             "acc_span": 2048, "general_link": 1, "order": 1} and ms == 4.5


def test_cache_refuses_bad_keys_and_choices(tmp_path):
    path = str(tmp_path / "tune.txt")
    for key in ("", "a\tb", "a\nb"):
        with pytest.raises(TpcError):
            binding.tune_cache_store(path, key, Tuning(), 1.0)
    with pytest.raises(TpcError):
        binding.tune_cache_store(path, "k", Tuning(acc_span=300), 1.0)
    with pytest.raises(TpcError):
        binding.tune_cache_store(path, "k", Tuning(order=2), 1.0)
