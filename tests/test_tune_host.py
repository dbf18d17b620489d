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


class _FakeLib:
    """Stands in for the library binding: 'orders' by writing a permutation that depends only on
    the options named in `changes_result`, and reports a time per option set."""
    RCM_OK, RCM_ERR_TOO_LARGE = 0, 4

    def __init__(self, times, changes_result=(), too_large=()):
        from paper_1610_08128_gb300 import rcm as real

        self.rcm_options = real.rcm_options
        self.rcm_batch_options = real.rcm_batch_options
        self.times, self.changes, self.too_large = times, changes_result, too_large
        self.last = None

    @staticmethod
    def _key(o):
        return tuple(sorted((f, getattr(o, f)) for f, _ in o._fields_ if not f.startswith("reserved") and getattr(o, f)))

    def rcm_order_ex(self, n, rp, ci, perm, o, stats, stream=None):
        k = self._key(o)
        if any(dict(k).get(f) == v for f, v in self.too_large):
            return self.RCM_ERR_TOO_LARGE
        shift = sum(1 for f, v in self.changes if dict(k).get(f) == v)
        perm.copy_(perm.new_tensor(list(range(n)))[[(i + shift) % n for i in range(n)]])
        self.last = k
        return self.RCM_OK

    def rcm_order_batch_ex(self, G, n, goff, rp, ci, perm, o, stream=None):
        return self.rcm_order_ex(n, rp, ci, perm, o, None, stream)

    def rcm_stream_status(self, stream=None):
        return self.RCM_OK

    @staticmethod
    def check(st, what=""):
        if st:
            raise RuntimeError(what)


def _patch(monkeypatch, fake):
    monkeypatch.setattr(tune, "rcm", fake)

    def fake_time(fn, torch, repeats):
        fn(None)
        return fake.times.get(fake.last, 10.0)

    monkeypatch.setattr(tune, "_time_ms", fake_time)


def test_tune_single_picks_the_fastest_and_skips_shapes_the_graph_does_not_admit(monkeypatch):
    import pytest as _pytest

    torch = _pytest.importorskip("torch")
    cands = [{"executor": 1, "narrow_threshold": 256}, {"executor": 1, "narrow_threshold": 512},
             {"executor": 2, "block_threads": 128}]
    fast = (("executor", 1), ("narrow_threshold", 512), ("nnz", 5))
    fake = _FakeLib({fast: 1.0}, too_large=(("executor", 2),))
    _patch(monkeypatch, fake)
    perm = torch.zeros(6, dtype=torch.int32)
    best, table = tune.tune_single(6, None, None, perm, nnz=5, candidates=cands)
    assert best == {"executor": 1, "narrow_threshold": 512}
    assert [c for c, _ in table] == cands[:2]          # the shared-memory CTA was refused, not timed


def test_tuners_refuse_a_candidate_that_changes_the_result(monkeypatch):
    import pytest as _pytest

    torch = _pytest.importorskip("torch")
    fake = _FakeLib({}, changes_result=(("narrow_threshold", 512),))
    _patch(monkeypatch, fake)
    perm = torch.zeros(6, dtype=torch.int32)
    with _pytest.raises(RuntimeError, match="changed the result"):
        tune.tune_single(6, None, None, perm, candidates=[{"executor": 1}, {"executor": 1, "narrow_threshold": 512}])
    fake = _FakeLib({}, changes_result=(("row_sort_split", 8),))
    _patch(monkeypatch, fake)
    with _pytest.raises(RuntimeError, match="changed the result"):
        tune.tune_batch(1, 6, None, None, None, perm, candidates=[{"block_threads": 256, "row_sort_split": 32},
                                                                  {"block_threads": 256, "row_sort_split": 8}])
