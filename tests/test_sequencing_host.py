"""Host logic of grid sequencing without a GPU: the pressure pin's node on the
coarser grids, and the order of the solves, prolongations and context releases
of Problem.newton_solve_sequenced, with stand-in problems."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def nc():
    try:
        from paper_1508_04596_gb300 import nc as m
    except ImportError as e:  # the binding needs the built library
        pytest.skip(str(e))
    return m


def test_coarse_pin(nc):
    # quarter cavity pin: node (0, 0, nz) of an 80 x 80 x 160 grid -> (0, 0, 80) of 40 x 40 x 80
    assert nc.coarse_pin((81 * 81) * 160, (80, 80), (40, 40)) == (41 * 41) * 80
    # a general node (6, 4, 2) of a 10 x 8 x 4 grid -> (3, 2, 1) of 5 x 4 x 2
    assert nc.coarse_pin(6 + 11 * (4 + 9 * 2), (10, 8), (5, 4)) == 3 + 6 * (2 + 5 * 1)
    assert nc.coarse_pin(-1, (10, 8), (5, 4)) == -1


class FakeProblem:
    log = []

    def __init__(self, n, levels):
        self.n, self.levels, self.ndof = n, levels, 5 * (n + 1) ** 3
        self.params = type("P", (), {"nx": n, "ny": n, "nz": n})()

    def coarse_problem(self):
        return FakeProblem(self.n // 2, self.levels - 1) if self.levels > 1 else None

    def coarsen(self, g, stream=None):
        FakeProblem.log.append(("coarsen", self.n))
        return g[: (self.n // 2) ** 3]

    fail = ()  # grid sizes whose solve fails

    def newton_solve(self, gam, x, opts=None, stream=None, check=True):
        FakeProblem.log.append(("solve", self.n, float(x.sum())))
        x.fill_(float(self.n))  # "the solution on this grid"
        st = "NC_ERR_MAXIT" if self.n in FakeProblem.fail else "NC_OK"
        return x, {"status": st, "newton_its": 1, "lin_its_total": 2, "seconds": 0.0}

    def prolong(self, xc, stream=None):
        FakeProblem.log.append(("prolong", self.n, float(xc[0])))
        return torch.full((self.ndof,), float(xc[0]), dtype=torch.float64)

    def close(self):
        FakeProblem.log.append(("close", self.n))


def test_sequenced_order(nc):
    FakeProblem.log = []
    fine = FakeProblem(8, 3)  # grids 8, 4, 2
    x = torch.zeros(fine.ndof, dtype=torch.float64)
    gam = torch.ones(8 ** 3, dtype=torch.float64)
    _, info = nc.Problem.newton_solve_sequenced(fine, gam, x)
    assert FakeProblem.log == [
        ("coarsen", 8), ("coarsen", 4),
        ("solve", 2, 0.0), ("prolong", 4, 2.0), ("close", 2),
        ("solve", 4, 2.0 * 5 * 5 ** 3), ("prolong", 8, 4.0), ("close", 4),
        ("solve", 8, 4.0 * 5 * 9 ** 3)]
    assert [lv["dims"] for lv in info["levels"]] == [(2, 2, 2), (4, 4, 4)]


def test_failed_coarse_solve_is_not_prolonged(nc):
    """A coarser solve that does not converge does not seed the finer one: the
    next finer grid starts from zero and the level reports prolonged=False."""
    FakeProblem.log, FakeProblem.fail = [], (2,)
    try:
        fine = FakeProblem(8, 3)
        x = torch.zeros(fine.ndof, dtype=torch.float64)
        _, info = nc.Problem.newton_solve_sequenced(fine, torch.ones(8 ** 3, dtype=torch.float64), x)
    finally:
        FakeProblem.fail = ()
    assert FakeProblem.log == [
        ("coarsen", 8), ("coarsen", 4),
        ("solve", 2, 0.0), ("close", 2),
        ("solve", 4, 0.0), ("prolong", 8, 4.0), ("close", 4),
        ("solve", 8, 4.0 * 5 * 9 ** 3)]
    assert [(lv["status"], lv["prolonged"]) for lv in info["levels"]] == [
        ("NC_ERR_MAXIT", False), ("NC_OK", True)]
