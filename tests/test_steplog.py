"""Host logic of the step log and the retrying time-step driver, with an injected step
function (no GPU): failures are raised as the library raises them (FrError with
FR_ERR_NONFINITE / FR_ERR_NOT_CONVERGED) or returned as converged == 0; the state is
restored before a retry; a failed step becomes two half steps, up to the halving limit;
other library errors propagate unchanged."""
import io
import json

import numpy as np
import pytest

from paper_2202_09733_gb300 import _native as N
from paper_2202_09733_gb300 import steplog as S


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2202_09733_gb300 import build as B
    B.build()


def make_step(limit, mode="raise", code=-5):
    """a step that adds dt to every entry, and fails (after corrupting q) when dt > limit"""
    calls = []

    def step(q, dt):
        calls.append(dt)
        if dt > limit:
            q += np.nan
            if mode == "raise":
                raise N.FrError(code, "fake step")
            return dict(n_ptc=3, n_gmres=0, converged=0, final_res=1.0)
        q += dt
        return dict(n_ptc=2, n_gmres=7, converged=1, final_res=1e-9)
    return step, calls


def test_plain_march_logs_every_step():
    q = np.zeros(4)
    buf = io.StringIO()
    step, calls = make_step(10.0)
    t = S.march(step, q, 0.0, 0.5, 3, log=S.StepLog(buf), extra={"precision": "fp64"})
    assert t == pytest.approx(1.5) and np.allclose(q, 1.5) and calls == [0.5] * 3
    recs = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [1, 2, 3]
    assert all(r["n_gmres"] == 7 and r["precision"] == "fp64" and r["halvings"] == 0 for r in recs)


@pytest.mark.parametrize("mode,code", [("raise", -5), ("raise", -4), ("flag", 0)])
def test_failed_step_is_restored_and_halved(mode, code):
    q = np.zeros(3)
    buf = io.StringIO()
    step, calls = make_step(0.3, mode, code)
    S.march(step, q, 0.0, 0.5, 1, log=S.StepLog(buf))
    assert np.all(np.isfinite(q)) and np.allclose(q, 0.5)      # restored, then 0.25 + 0.25
    assert calls == [0.5, 0.25, 0.25]
    recs = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert recs[0]["failed"] and recs[0]["halvings"] == 0
    assert [r["dt"] for r in recs[1:]] == [0.25, 0.25] and all(r["halvings"] == 1 for r in recs[1:])


def test_gives_up_after_the_halving_limit():
    q = np.zeros(2)
    step, calls = make_step(0.01)
    with pytest.raises(S.StepFailed):
        S.march(step, q, 0.0, 0.5, 1, max_halvings=2)
    assert calls == [0.5, 0.25, 0.125]
    assert np.all(np.isfinite(q)) and np.allclose(q, 0.0)


def test_other_errors_propagate():
    step, _ = make_step(0.0, "raise", -1)          # FR_ERR_INVALID_ARG is not retried
    with pytest.raises(N.FrError):
        S.march(step, np.zeros(2), 0.0, 0.5, 1)
