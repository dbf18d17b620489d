"""Host-side pieces of the autotuner (no GPU): candidate sets and size classes."""
from paper_1610_08128_gb300 import tune


def test_candidates_are_valid_option_sets():
    for c in tune.BATCH_CANDIDATES:
        assert c["block_threads"] in (128, 256, 512) and 4 <= c["row_sort_split"] <= 32
    assert len({tuple(sorted(c.items())) for c in tune.BATCH_CANDIDATES}) == len(tune.BATCH_CANDIDATES)
    for c in tune.SINGLE_CANDIDATES:
        assert c["executor"] in (1, 2)
        if c["executor"] == 2:
            assert 32 <= c["block_threads"] <= 512
    assert len({tuple(sorted(c.items())) for c in tune.SINGLE_CANDIDATES}) == len(tune.SINGLE_CANDIDATES)
    from paper_1610_08128_gb300 import rcm

    fields = {f for f, _ in rcm.rcm_options._fields_}
    bfields = {f for f, _ in rcm.rcm_batch_options._fields_}
    for c in tune.SINGLE_CANDIDATES:
        assert set(c) <= fields, c
        # per-level expansion and asynchronous sweeps are separate 512-thread engines
        assert not (c.get("expand_mode", 0) >= 2 and c.get("async_sweeps", 0) == 1), c
    for c in tune.BATCH_CANDIDATES:
        assert set(c) <= bfields, c


def test_size_class_buckets_powers_of_four():
    assert tune.size_class(0) == tune.size_class(1) == tune.size_class(3) == "n<4^1"
    assert tune.size_class(4) == "n<4^2"
    assert tune.size_class(15) == "n<4^2" and tune.size_class(16) == "n<4^3"
    assert tune.size_class(7_077_888) == "n<4^12"
