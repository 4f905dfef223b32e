"""Host logic of the transition-point search (Gu-Wen ratio X, Sec. III D): bracketing and
refinement on evaluators with a known crossing, and with the oracle as the evaluator."""
import math

import numpy as np
import pytest

from oracle import trg_oracle as O
from paper_2507_21909_b300.tc_scan import bracket_crossing, refine


def step_x(beta_c, width):
    return lambda betas: 1.0 + 1.0 / (1.0 + np.exp(-(np.asarray(betas) - beta_c) / width))


def test_bracket_crossing():
    assert bracket_crossing([0.1, 0.2, 0.3], [1.0, 1.4, 1.9]) == (1, 2)
    assert bracket_crossing([0.1, 0.2, 0.3], [1.0, 1.5, 1.9]) == (0, 1)
    assert bracket_crossing([0.1, 0.2], [1.9, 1.0]) is None
    assert bracket_crossing([0.1, 0.2], [1.0, 1.2]) is None


@pytest.mark.parametrize("beta_c", [0.1311, 0.1497, 0.1899])
def test_refine_narrows_to_a_known_crossing(beta_c):
    out = refine(step_x(beta_c, 1e-3), 0.1, 0.2, points=8, rounds=3)
    lo, hi = out["interval"]
    assert lo <= beta_c <= hi
    assert math.isclose(hi - lo, 0.1 / 7 ** 3, rel_tol=1e-9)
    assert abs(out["beta_c"] - beta_c) < hi - lo
    assert len(out["history"]) == 3


def test_symmetric_crossing_interpolates_exactly():
    """X linear in beta: the interpolated crossing is exact after one round."""
    out = refine(lambda b: 1.0 + (np.asarray(b) - 0.1) * 10.0, 0.1, 0.2, points=5, rounds=1)
    assert abs(out["beta_c"] - 0.15) < 1e-15


def test_no_crossing_and_bad_arguments():
    out = refine(lambda b: np.ones(len(b)), 0.1, 0.2)
    assert out["beta_c"] is None and len(out["history"]) == 1
    with pytest.raises(ValueError):
        refine(lambda b: b, 0.2, 0.1)
    with pytest.raises(ValueError):
        refine(lambda b: b, 0.1, 0.2, points=1)


def test_oracle_evaluator_brackets_the_4d_ising_transition():
    """X of the oracle after 12 steps at D = 5 crosses 1.5 once between beta = 0.13 and
    0.17; the refined interval's end values straddle 1.5, and the crossing lies within
    10 % of the 4D Ising critical coupling 0.1497 (Monte Carlo; at D = 5 it sits near
    0.142, the small-D shift the paper's T_c-versus-D figure shows)."""
    def evaluate(betas):
        out = []
        for b in betas:
            st = O.init_ising(4, float(b), 0.0)
            for n in range(12):
                O.step(st, n % 4, 5, 10, 4, 4, 0x5EED)
            out.append(O.gu_wen_ratio(st))
        return np.array(out)
    res = refine(evaluate, 0.13, 0.17, points=5, rounds=2)
    lo, hi = res["interval"]
    assert hi - lo == pytest.approx(0.01 / 4)
    x_lo, x_hi = evaluate([lo, hi])
    assert x_lo < 1.5 <= x_hi
    assert lo <= res["beta_c"] <= hi
    assert abs(res["beta_c"] - 0.1497) < 0.1 * 0.1497, res["beta_c"]


def test_tc_scan_drives_the_batch_calls(monkeypatch):
    """tc_scan creates one instance per coupling, steps them, reads X and always frees
    the batch (stand-ins for the library calls)."""
    from paper_2507_21909_b300 import _lib as L
    from paper_2507_21909_b300.tc_scan import tc_scan
    calls = []

    def create(model, beta, h, D, lanes=4, precision=0, **kw):
        calls.append(("create", list(model), list(beta), list(h), list(D), lanes, precision))
        calls[-1] = calls[-1] + (len(beta),)
        create.n = len(beta)
        create.betas = np.asarray(beta)
        return len(beta)

    monkeypatch.setattr(L, "trg_batch_create", create)
    monkeypatch.setattr(L, "trg_batch_step", lambda k: calls.append(("step", k)))
    monkeypatch.setattr(L, "trg_batch_gu_wen",
                        lambda n: 1.0 + (create.betas > 0.1497).astype(float))
    monkeypatch.setattr(L, "trg_batch_free", lambda: calls.append(("free",)))
    res = tc_scan(0.14, 0.16, D=8, nsteps=20, points=5, rounds=2, lanes=3, precision=5)
    creates = [c for c in calls if c[0] == "create"]
    assert len(creates) == 2 and all(c[-1] == 5 for c in creates)
    assert creates[0][1] == [0] * 5 and creates[0][4] == [8] * 5 and creates[0][6] == 5
    assert [c for c in calls if c[0] == "step"] == [("step", 20)] * 2
    assert calls.count(("free",)) == 2
    lo, hi = res["interval"]
    assert lo <= 0.1497 <= hi and res["T_c"] == pytest.approx(1 / res["beta_c"])

    def failing_step(k):
        raise L.TrgError(-3, "device error")
    monkeypatch.setattr(L, "trg_batch_step", failing_step)
    calls.clear()
    with pytest.raises(L.TrgError):
        tc_scan(0.14, 0.16, D=8, nsteps=20, points=3, rounds=1)
    assert calls.count(("free",)) == 1
