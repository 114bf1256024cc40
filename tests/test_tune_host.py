"""The autotuner's host logic (paper_1705_02313_gb300/tune.py), on the CPU:
coordinate descent over the partitioning parameters with a stand-in timer,
the size buckets, and the table text that pg_load_tuning reads."""
import re

from paper_1705_02313_gb300 import tune


def test_coordinate_descent_finds_a_separable_minimum():
    target = {"walk_cap": 32, "switch_block": 512, "loop_ranks": 0, "deep_cut": 16, "ruler_bits": 7}

    def cost(st):  # separable: each parameter adds its own distance from the target
        return 100.0 + sum(abs(tune.CANDIDATES[k].index(st[k]) - tune.CANDIDATES[k].index(target[k])) * 5.0
                           for k in target)

    best, t, seen = tune.coordinate_descent(cost)
    assert best == target and t == 100.0
    key = ",".join("%s=%d" % (f, tune.DEFAULTS[f]) for f in tune.FIELDS)
    assert key in seen  # the defaults are always measured


def test_flat_responses_keep_the_defaults():
    best, _, _ = tune.coordinate_descent(lambda st: 50.0 + 0.5 * (st["walk_cap"] != 64))  # within 2%
    assert best == tune.DEFAULTS


def test_buckets_increase_and_the_last_is_unbounded():
    b = tune.bucket_bounds([10_000, 100_000, 1_000_000, 10_000_000])
    assert all(x < y for x, y in zip(b, b[1:])) and b[-1] >= 2**62
    assert 13_400 < b[0] < 134_000  # between the first two sizes' ids


def test_table_text_is_what_the_library_parses():
    entries = [(1000, dict(tune.DEFAULTS)), (2**62, dict(tune.DEFAULTS, walk_cap=16, loop_ranks=1))]
    text = tune.table_text(entries, "NVIDIA GB300")
    rows = [ln for ln in text.splitlines() if ln and not ln.startswith("#")]
    assert len(rows) == 2
    for (m, st), row in zip(entries, rows):
        f = [int(x) for x in row.split()]
        assert f == [m, st["deep_cut"], st["ruler_bits"], st["walk_cap"], st["switch_block"], st["loop_ranks"]]
    assert tune.device_slug("NVIDIA GB300") == "nvidia_gb300"
    assert re.fullmatch(r".*tuning/nvidia_gb300\.txt", tune.default_table_path("NVIDIA GB300"))
