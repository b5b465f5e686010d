"""The autotuner's persistent tune cache: host-side file logic only (no GPU).

A line is `<key> <leaf shape> <cone CTAs per SM>`; the last valid line for a key wins,
malformed and out-of-range lines are skipped, keys are single whitespace-free tokens."""
import os

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2010_02857_gb300 import _build
    _build.build()
    import paper_2010_02857_gb300 as p
    return p


def test_missing_file_is_a_miss(pkg, tmp_path):
    assert pkg.tune_cache_lookup(str(tmp_path / "none.txt"), "k") is None


def test_store_then_lookup_round_trip(pkg, tmp_path):
    path = str(tmp_path / "tune.txt")
    pkg.tune_cache_store(path, "dev/sm152;n100", 1, 2)
    pkg.tune_cache_store(path, "dev/sm152;n200", 2, 1)
    assert pkg.tune_cache_lookup(path, "dev/sm152;n100") == (1, 2)
    assert pkg.tune_cache_lookup(path, "dev/sm152;n200") == (2, 1)
    assert pkg.tune_cache_lookup(path, "dev/sm152;n10") is None  # prefixes do not match
    assert open(path).read() == "dev/sm152;n100 1 2\ndev/sm152;n200 2 1\n"


def test_last_valid_line_wins_and_bad_lines_are_skipped(pkg, tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("\n".join([
        "k 0 1",
        "k 1 2",
        "k 3 2",          # leaf shape out of range
        "k 1 0",          # CTAs per SM out of range
        "k 2",            # missing field
        "k 2 1 extra",    # trailing field
        "k x 1",          # not a number
        "   ",
        "other 2 2",
        "k" * 2000 + " 0 1",  # over-long line (longer than any key)
        "",
    ]))
    assert pkg.tune_cache_lookup(str(path), "k") == (1, 2)
    assert pkg.tune_cache_lookup(str(path), "other") == (2, 2)
    pkg.tune_cache_store(str(path), "k", 0, 1)
    assert pkg.tune_cache_lookup(str(path), "k") == (0, 1)


def test_invalid_keys_and_values_are_rejected(pkg, tmp_path):
    path = str(tmp_path / "tune.txt")
    for key in ["", "a b", "a\tb", "a\nb", "k" * 481]:
        with pytest.raises(pkg.IFGFError) as e:
            pkg.tune_cache_store(path, key, 0, 1)
        assert e.value.status == 1
        with pytest.raises(pkg.IFGFError):
            pkg.tune_cache_lookup(path, key)
    for leaf, ctas in [(-1, 1), (3, 1), (0, 0), (0, 3)]:
        with pytest.raises(pkg.IFGFError):
            pkg.tune_cache_store(path, "k", leaf, ctas)
    assert not os.path.exists(path)  # nothing was written
    pkg.tune_cache_store(path, "k" * 480, 2, 2)  # the longest key
    assert pkg.tune_cache_lookup(path, "k" * 480) == (2, 2)


def test_unwritable_cache_is_an_error(pkg, tmp_path):
    with pytest.raises(pkg.IFGFError):
        pkg.tune_cache_store(str(tmp_path / "no_dir" / "tune.txt"), "k", 0, 1)
