"""Host logic of the learned-scalings fallback (learned.solve_with_scalings)
on a stand-in patch object: the unscaled preconditioner takes over when the
scaled solve breaks down, exceeds the iteration budget, or its scalings
cannot be set up. No GPU: the stand-in records the calls it receives."""
import pytest

from paper_1602_01636_gb300 import igafd, learned


class Info:
    def __init__(self, status, iterations):
        self.status, self.iterations = status, iterations


class StandIn:
    """Answers pcg() with a scripted outcome for the scaled and the unscaled
    preconditioner; scaled_its > cap means 'not converged within the cap'."""

    def __init__(self, scaled_its=5, scaled_status=igafd.OK, setup_fails=False, plain_its=9):
        self.scaled_its, self.scaled_status = scaled_its, scaled_status
        self.setup_fails, self.plain_its = setup_fails, plain_its
        self.scalings = None
        self.calls = []

    def set_scalings(self, logw):
        self.calls.append(("set_scalings", logw))
        if logw is not None and self.setup_fails:
            raise igafd.IgafdError(igafd.ERR_NOT_SPD, "set_scalings")
        self.scalings = logw

    def pcg(self, b, tol, max_iter, dtype, raise_on_error):
        self.calls.append(("pcg", self.scalings, max_iter))
        if self.scalings is None:
            return "x_plain", Info(igafd.OK, self.plain_its)
        if self.scaled_status != igafd.OK:
            return "x_bad", Info(self.scaled_status, 3)
        if self.scaled_its > max_iter:
            return "x_capped", Info(igafd.ERR_NOT_CONVERGED, max_iter)
        return "x_scaled", Info(igafd.OK, self.scaled_its)


def test_scaled_solve_within_budget_is_kept():
    p = StandIn(scaled_its=5)
    x, info, fb = learned.solve_with_scalings(p, "w", None, budget=9)
    assert (x, info.iterations, fb) == ("x_scaled", 5, False)
    assert p.calls == [("set_scalings", "w"), ("pcg", "w", 9)]


@pytest.mark.parametrize("budget,max_iter,cap", [(9, 1000, 9), (None, 40, 40), (500, 40, 40)])
def test_scaled_solve_capped_at_the_budget_then_falls_back(budget, max_iter, cap):
    p = StandIn(scaled_its=cap + 1)
    x, info, fb = learned.solve_with_scalings(p, "w", None, max_iter=max_iter, budget=budget)
    assert fb and x == "x_plain" and info.iterations == 9
    # the scaled run is cut at the budget; the unscaled rerun gets the full cap
    assert p.calls == [("set_scalings", "w"), ("pcg", "w", cap), ("set_scalings", None),
                       ("pcg", None, max_iter)]


def test_breakdown_falls_back():
    p = StandIn(scaled_status=igafd.ERR_BREAKDOWN)
    x, info, fb = learned.solve_with_scalings(p, "w", None, budget=9)
    assert fb and x == "x_plain" and info.status == igafd.OK


def test_failed_scaled_setup_falls_back():
    p = StandIn(setup_fails=True)
    x, info, fb = learned.solve_with_scalings(p, "w", None, budget=9)
    assert fb and x == "x_plain"
    assert p.calls == [("set_scalings", "w"), ("set_scalings", None), ("pcg", None, 1000)]
