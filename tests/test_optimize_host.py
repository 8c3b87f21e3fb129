"""Host logic of the optimisation driver without a GPU: the continuation
schedule (iterations split evenly over the steps, Sec. 3.3) and the
checkpoint / resume bookkeeping of optimize.run, with a stand-in optimiser
that records what the driver asks of it."""
import pytest

torch = pytest.importorskip("torch")


class FakeOptimizer:
    saved = {}

    def __init__(self, workload, **kw):
        self.k, self.step, self.steps_seen = 0, -1, []
        self.schedule = None

    def set_step(self, step):
        self.step = step

    def iterate(self):
        self.steps_seen.append(self.step)
        self.k += 1
        return {"iter": self.k, "step": self.step}

    def save(self, path):
        FakeOptimizer.saved[path] = (self.k, self.step, list(self.steps_seen), self.schedule)

    @classmethod
    def load(cls, path):
        o = cls("x")
        o.k, o.step, o.steps_seen, o.schedule = FakeOptimizer.saved[path]
        o.steps_seen = list(o.steps_seen)
        return o


@pytest.fixture
def optimize(monkeypatch):
    try:
        from paper_1508_04596_gb300 import optimize as m
    except ImportError as e:  # the binding needs the built library
        pytest.skip(str(e))
    monkeypatch.setattr(m, "Optimizer", FakeOptimizer)
    FakeOptimizer.saved = {}
    return m


def test_continuation_schedule(optimize):
    opt, hist = optimize.run("w", 10, steps=5, log=None)
    assert opt.steps_seen == [0, 0, 1, 1, 2, 2, 3, 3, 4, 4]
    opt, _ = optimize.run("w", 7, steps=3, log=None)
    assert opt.steps_seen == [0, 0, 1, 1, 2, 2, 2]
    opt, _ = optimize.run("w", 3, steps=5, log=None)  # fewer iterations than steps
    assert opt.steps_seen == [0, 1, 2]


def test_checkpoint_every_and_resume(optimize):
    opt, _ = optimize.run("w", 4, steps=2, log=None, checkpoint="ck", every=3)
    assert FakeOptimizer.saved["ck"][0] == 4  # saved at iteration 3, then at the end
    optimize.run("w", 4, steps=2, log=None, checkpoint="half", stop_after=2)
    assert FakeOptimizer.saved["half"] == (2, 0, [0, 0], (4, 2))
    b, hist = optimize.run("w", 4, steps=2, log=None, resume="half")
    assert b.k == 4 and len(hist) == 2
    assert b.steps_seen == opt.steps_seen == [0, 0, 1, 1]


def test_resume_with_another_schedule_is_refused(optimize):
    """The continuation step of iteration k depends on (iters, steps): a run saved
    with one schedule and resumed with another would jump to a different step."""
    optimize.run("w", 2, steps=1, log=None, checkpoint="c1")
    assert FakeOptimizer.saved["c1"][3] == (2, 1)
    with pytest.raises(ValueError, match="iters=2, steps=1"):
        optimize.run("w", 4, steps=2, log=None, resume="c1")
