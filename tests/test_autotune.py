"""Host logic of the autotuner: the search finds the minimum of a known cost surface, the table
round-trips through JSON and lookups fall back to the nearest size class, then to the defaults."""
import itertools
import json

from paper_1907_08817_gb300 import autotune as AT


def _cost(cfg):
    # separable bowl with its minimum at (11, 2, 2) and a small interaction term
    return ((cfg["bucket_log2"] - 11) ** 2 + 3 * (cfg["polish_blocks"] - 2) ** 2
            + 0.5 * (cfg["eps"] - 2) ** 2 + 0.1 * (cfg["bucket_log2"] - 11) * (cfg["eps"] - 2))


def test_coordinate_search_finds_grid_minimum():
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return _cost(cfg)

    best, log = AT.search(measure, repeats=1)
    grid = [dict(zip(AT.DEFAULT_SPACE, v)) for v in itertools.product(*AT.DEFAULT_SPACE.values())]
    assert best == min(grid, key=_cost)
    # each distinct configuration is timed once per repeat and the coordinate search visits fewer
    # configurations than the full grid
    assert len(calls) == len(log) < len(grid)
    full, _ = AT.search(measure, repeats=1, coordinate=False)
    assert full == best


def test_search_takes_median_of_repeats():
    seq = iter([5.0, 1.0, 9.0] + [3.0] * 1000)
    best, log = AT.search(lambda cfg: next(seq), space={"bucket_log2": (12,), "polish_blocks": (3,),
                                                        "eps": (3,)}, repeats=3)
    assert best == AT.DEFAULTS
    assert log == [(AT.DEFAULTS, 5.0)]


def test_table_round_trip_and_fallbacks(tmp_path):
    path = str(tmp_path / "tuned.json")
    assert AT.tuned_options(0, 1 << 20, 1, 32, 0, "fp32", path=path) == AT.DEFAULTS
    AT.save_entry(AT.table_key(0, 1 << 28, 2, 64, 64, "bf16"),
                  {"bucket_log2": 11, "polish_blocks": 2, "eps": 2}, 123.4, path)
    AT.save_entry(AT.table_key(0, 1 << 20, 2, 64, 64, "bf16"),
                  {"bucket_log2": 10, "polish_blocks": 3, "eps": 1}, 1.0, path)
    with open(path) as f:
        t = json.load(f)
    assert t["d0-n28-l2-64x64-bf16"]["sort_ms"] == 123.4
    # exact class
    assert AT.tuned_options(0, (1 << 28) + 5, 2, 64, 64, "bf16", path=path) == \
        {"bucket_log2": 11, "polish_blocks": 2, "eps": 2}
    # nearest size class of the same key type, shape and precision
    assert AT.tuned_options(0, 1 << 26, 2, 64, 64, "bf16", path=path)["bucket_log2"] == 11
    assert AT.tuned_options(0, 1 << 22, 2, 64, 64, "bf16", path=path)["bucket_log2"] == 10
    # a precision never tuned for this key type and shape takes another precision's entry
    assert AT.tuned_options(0, 1 << 28, 2, 64, 64, "fp32", path=path) == \
        {"bucket_log2": 11, "polish_blocks": 2, "eps": 2}
    assert AT.tuned_entry(0, 1 << 28, 2, 64, 64, "fp32", path=path) is None
    # but an entry of the requested precision wins, whatever its size class
    AT.save_entry(AT.table_key(0, 1 << 20, 2, 64, 64, "pwl"),
                  {"bucket_log2": 13, "polish_blocks": 1, "eps": 4}, 2.0, path)
    assert AT.tuned_options(0, 1 << 28, 2, 64, 64, "pwl", path=path)["bucket_log2"] == 13
    # another shape or key type has no entry
    assert AT.tuned_options(0, 1 << 28, 1, 64, 0, "bf16", path=path) == AT.DEFAULTS
    assert AT.tuned_options(1, 1 << 28, 2, 64, 64, "bf16", path=path) == AT.DEFAULTS


def test_shipped_table_is_within_the_space():
    for key, e in AT.load_table().items():
        assert key.count("-") == 4
        for name, values in AT.DEFAULT_SPACE.items():
            assert e[name] in values, (key, name)
