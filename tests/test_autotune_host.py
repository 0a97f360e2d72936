"""Host logic of the schedule autotuner (no GPU): with the C-ABI calls
replaced by a recording fake and a fake clock, `tune` skips the schedules the
handle refuses, keeps each candidate's fastest repeat, sets the fastest
candidate and leaves the handle assembled; `ScheduleCache` tunes a shape once
and hands its choice to later handles of that shape."""
import pytest

from paper_1705_05783_gb300 import autotune, cams


class FakeEngine:
    def __init__(self, cost, refused=()):
        self.cost = cost            # seconds per iterate call under each schedule
        self.refused = set(refused)
        self.now = 0.0
        self.schedule = {}
        self.calls = []

    def clock(self):
        return self.now

    def install(self, monkeypatch):
        def set_schedule(h, ilu_cta=-1, coarse_cluster=-1):
            if (ilu_cta, coarse_cluster) in self.refused:
                raise cams.CamsError(cams.CAMS_EINVAL, "refused")
            self.schedule[h] = (ilu_cta, coarse_cluster)
            self.calls.append(("set", h, (ilu_cta, coarse_cluster)))

        def iterate(h, n):
            self.now += self.cost[self.schedule[h]] * n
            self.calls.append(("iterate", h, n))

        monkeypatch.setattr(cams, "cams_set_schedule", set_schedule)
        monkeypatch.setattr(cams, "cams_iterate", iterate)
        monkeypatch.setattr(cams, "cams_assemble", lambda h, *a: self.calls.append(("assemble", h)))
        monkeypatch.setattr(cams, "cams_update_basis", lambda h, f=False: self.calls.append(("basis", h)))


def test_tune_picks_the_fastest_accepted_schedule(monkeypatch):
    eng = FakeEngine({(0, 0): 3.0, (0, 1): 2.0, (1, 0): 1.0, (1, 1): 0.5}, refused={(1, 1)})
    eng.install(monkeypatch)
    choice, times = autotune.tune("h", None, 0.1, None, iters=2, repeats=2, clock=eng.clock)
    assert choice == (1, 0)
    assert set(times) == {(0, 0), (0, 1), (1, 0)}
    assert times[(1, 0)] == pytest.approx(2.0) and times[(0, 0)] == pytest.approx(6.0)
    assert eng.schedule["h"] == (1, 0)
    assert eng.calls[-1] == ("assemble", "h")               # left assembled at p_n
    assert sum(1 for c in eng.calls if c[0] == "basis") == 1


def test_tune_with_no_accepted_schedule(monkeypatch):
    eng = FakeEngine({}, refused=set(autotune.CANDIDATES))
    eng.install(monkeypatch)
    choice, times = autotune.tune("h", None, 0.1, None, clock=eng.clock)
    assert choice is None and times == {}


def test_cache_tunes_each_shape_once(monkeypatch):
    eng = FakeEngine({(0, 0): 1.0, (0, 1): 2.0, (1, 0): 3.0, (1, 1): 4.0})
    eng.install(monkeypatch)
    cache = autotune.ScheduleCache()
    key = autotune.shape_key(64, 64, 32, (8, 8, 8), 1, 0)
    assert cache.apply("a", key, None, 0.1, None, clock=eng.clock) == (0, 0)
    n_iter = sum(1 for c in eng.calls if c[0] == "iterate")
    assert cache.apply("b", key, None, 0.1, None, clock=eng.clock) == (0, 0)
    assert sum(1 for c in eng.calls if c[0] == "iterate") == n_iter   # not tuned again
    assert eng.schedule["b"] == (0, 0)


def test_tune_ensemble_times_whole_runs(monkeypatch):
    """Every candidate is set on every handle that accepts it and timed over
    whole ensemble runs (after one untimed run); the fastest is kept on
    all handles."""
    eng = FakeEngine({(0, 0): 3.0, (0, 1): 1.0, (1, 0): 2.0, (1, 1): 5.0}, refused={(1, 1)})
    eng.install(monkeypatch)
    handles = ["a", "b", "c"]
    runs = []

    def run():
        # an ensemble run costs the sum of its members under their schedules
        runs.append(dict(eng.schedule))
        eng.now += sum(eng.cost[eng.schedule[h]] for h in handles)

    choice, times = autotune.tune_ensemble(handles, run, repeats=2, clock=eng.clock)
    assert choice == (0, 1)
    assert set(times) == {(0, 0), (0, 1), (1, 0)}
    assert times[(0, 1)] == pytest.approx(3.0)
    assert all(eng.schedule[h] == (0, 1) for h in handles)
    assert len(runs) == 3 * 3                    # one untimed + two timed runs per candidate
