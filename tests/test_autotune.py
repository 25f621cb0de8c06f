"""Autotuner selection and cache logic, with a fake timer (no GPU)."""
import json

from paper_2412_02413_gb300 import autotune


def test_bucket_and_key():
    assert [autotune.bucket(v) for v in (1, 2, 3, 1024, 1025, 8192)] == [1, 2, 4, 1024, 2048, 8192]
    assert autotune.make_key("split", 128, 4096, 512, 1) == "split:ne128:nt4096:nz512:F1"
    assert autotune.make_key("split", 128, 4000, 300, 1) == "split:ne128:nt4096:nz512:F1"


def test_picks_the_fastest_median_and_caches(tmp_path):
    path = str(tmp_path / "db.json")
    t = autotune.Autotuner(path)
    calls = []
    cost = {1: [3.0, 1.0, 3.0], 2: [2.0, 2.0, 2.0], 4: [5.0, 0.1, 5.0]}   # medians 3, 2, 5

    def run(c):
        calls.append(c)
        return cost[c][sum(1 for x in calls if x == c) - 1]

    assert t.tune("k", [1, 2, 4], run) == 2
    assert len(calls) == 9
    # cached: no more timing, and a fresh tuner reads the file
    assert t.tune("k", [1, 2, 4], run) == 2 and len(calls) == 9
    t2 = autotune.Autotuner(path)
    assert t2.lookup("k") == 2
    db = json.load(open(path))
    assert db["k"]["seconds"] == {"1": 3.0, "2": 2.0, "4": 5.0}


def test_ties_keep_the_first_candidate_and_force_retunes(tmp_path):
    t = autotune.Autotuner(str(tmp_path / "db.json"))
    assert t.tune("k", [8, 4, 2], lambda c: 1.0) == 8
    assert t.tune("k", [8, 4, 2], lambda c: float(c), force=True) == 2


def test_corrupt_cache_is_ignored(tmp_path):
    p = tmp_path / "db.json"
    p.write_text("{not json")
    t = autotune.Autotuner(str(p))
    assert t.lookup("k") is None
    assert t.tune("k", [1], lambda c: 1.0) == 1


def test_stream_grid_candidates():
    assert autotune.stream_grid_candidates(152) == [0, 148, 144, 140, 136, 128]
    assert autotune.stream_grid_candidates(16) == [0, 12, 8]


def test_tune_stream_grid_applies_the_fastest_to_every_plan(tmp_path, monkeypatch):
    class FakePlan:
        def __init__(self):
            self.grid = None

        def set_grid(self, n):
            self.grid = n

    plans = [FakePlan(), FakePlan(), FakePlan()]
    # seconds per step as a function of the grid the plans carry: fastest at 136
    cost = {0: 1.00, 148: 0.98, 144: 0.97, 140: 0.96, 136: 0.95, 128: 0.99}
    monkeypatch.setattr(autotune, "_streams_timer", lambda step, streams: cost[plans[0].grid])

    class W:
        n_elem, nt, nz = 128, 4096, 512

    t = autotune.Autotuner(str(tmp_path / "db.json"))
    best = autotune.tune_stream_grid(t, plans, None, 152, 3, W, 1, [None])
    assert best == 136 and all(p.grid == 136 for p in plans)
    assert t.lookup("stream_grid_S3:ne128:nt4096:nz512:F1") == 136


def test_batch_grid_candidates():
    assert autotune.batch_grid_candidates(2000, 152) == [76, 114, 152]
    assert autotune.batch_grid_candidates(100, 152) == [76, 100]


def test_tune_time_fft_radix_applies_to_every_plan(tmp_path, monkeypatch):
    class FakePlan:
        n_elem, n_samples, nz = 128, 4096, 512

        def __init__(self):
            self.radix = None

        def set_fft_radix(self, r):
            self.radix = r

        def as_tax(self, rf, outs=None):
            pass

    class RF:
        def dim(self):
            return 3

        shape = (1, 128, 4096)

    plans = [FakePlan(), FakePlan()]
    monkeypatch.setattr(autotune, "_event_timer", lambda call, warmup=1, iters=3: {8: 1.0, 4: 2.0}[plans[0].radix])
    t = autotune.Autotuner(str(tmp_path / "db.json"))
    assert autotune.tune_time_fft_radix(t, plans, RF()) == 8
    assert [p.radix for p in plans] == [8, 8]
    assert t.lookup("fft_radix:ne128:nt4096:nz512:F1") == 8


def test_tune_gemm_tile_applies_the_fastest(tmp_path, monkeypatch):
    class FakePlan:
        n_elem, n_samples, nz = 128, 4096, 512
        m = None

        def set_gemm_tile(self, m):
            self.m = m

        def as_tax(self, rf, outs=None):
            pass

    class RF:
        shape = (64, 128, 4096)

        def dim(self):
            return 3

    plan = FakePlan()
    monkeypatch.setattr(autotune, "_event_timer", lambda call, warmup=1, iters=3: {128: 1.0, 256: 1.2}[plan.m])
    t = autotune.Autotuner(str(tmp_path / "db.json"))
    assert autotune.tune_gemm_tile(t, plan, RF(), "fp16split") == 128 and plan.m == 128
    assert t.lookup("gemm_tile_fp16split:ne128:nt4096:nz512:F64") == 128


def test_tune_lane_rows_applies_to_every_plan(tmp_path, monkeypatch):
    class FakePlan:
        n_elem, n_samples, nz = 128, 4096, 512

        def __init__(self):
            self.rows = None

        def set_lane_rows(self, r):
            self.rows = r

        def as_tax(self, rf, outs=None):
            pass

    class RF:
        shape = (1, 128, 4096)

        def dim(self):
            return 3

    plans = [FakePlan(), FakePlan()]
    monkeypatch.setattr(autotune, "_event_timer", lambda call, warmup=1, iters=3: {1: 1.0, 2: 0.9}[plans[0].rows])
    t = autotune.Autotuner(str(tmp_path / "db.json"))
    assert autotune.tune_lane_rows(t, plans, RF()) == 2
    assert [p.rows for p in plans] == [2, 2]
    assert t.lookup("lane_rows:ne128:nt4096:nz512:F1") == 2


def test_tune_gemm_frames_applies_the_fastest(tmp_path, monkeypatch):
    class FakePlan:
        n_elem, n_samples, nz = 128, 4096, 512
        fr = None

        def set_gemm_frames(self, f):
            self.fr = f

        def as_tax(self, rf, outs=None):
            pass

    class RF:
        shape = (8, 128, 4096)

        def dim(self):
            return 3

    plan = FakePlan()
    monkeypatch.setattr(autotune, "_event_timer", lambda call, warmup=1, iters=3: {32: 1.0, 16: 0.6}[plan.fr])
    t = autotune.Autotuner(str(tmp_path / "db.json"))
    assert autotune.tune_gemm_frames(t, plan, RF(), "bf16") == 16 and plan.fr == 16
    assert t.lookup("gemm_frames_bf16:ne128:nt4096:nz512:F8") == 16
