"""Per-step JSON-lines log and a time-marching driver that retries a failed step.

The paper reports, per run, the wall time and the average pseudo-time and GMRES counts
per stage (Tables 2-6); `StepLog` writes one JSON object per step with those counters, so
a run can be summarised the same way.  `march` advances a state through `nsteps` steps
of size dt with a caller-supplied step function (for example a closure over
`api.esdirk_step`); a step that raises FR_ERR_NOT_CONVERGED or FR_ERR_NONFINITE, or
returns stats with converged == 0, is undone (the state is restored from a copy taken
before it) and replaced by two steps of dt/2, recursively up to `max_halvings` times.
"""
from __future__ import annotations

import json
import time
from typing import Callable, Optional

from . import _native as N

RETRY_CODES = (-4, -5)     # FR_ERR_NOT_CONVERGED, FR_ERR_NONFINITE


class StepLog:
    """Append-only JSON-lines writer (one object per step, keys sorted)."""

    def __init__(self, target):
        self._own = isinstance(target, str)
        self._f = open(target, "a") if self._own else target

    def write(self, **rec):
        self._f.write(json.dumps(rec, sort_keys=True) + "\n")
        self._f.flush()

    def close(self):
        if self._own:
            self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _snapshot(q):
    return q.clone() if hasattr(q, "clone") else q.copy()


def _restore(q, saved):
    q[...] = saved


class StepFailed(RuntimeError):
    pass


def march(step: Callable, q, t: float, dt: float, nsteps: int, log: Optional[StepLog] = None,
          max_halvings: int = 2, extra: Optional[dict] = None, sync: Optional[Callable] = None):
    """Advance q (updated in place) by nsteps steps of dt from time t; returns the final t.

    step(q, dt) -> stats dict (n_ptc, n_gmres, converged, final_res, ...).  sync, if given,
    is called before reading the clock (e.g. torch.cuda.synchronize)."""
    extra = dict(extra or {})
    counter = [0]

    def one(dt_, depth):
        saved = _snapshot(q)
        if sync:
            sync()
        t0 = time.perf_counter()
        err = None
        try:
            st = step(q, dt_)
        except N.FrError as ex:
            if ex.code not in RETRY_CODES:
                raise
            st, err = None, ex
        if sync:
            sync()
        wall = time.perf_counter() - t0
        ok = st is not None and st.get("converged", 1)
        if ok:
            counter[0] += 1
            if log:
                rec = {k: v for k, v in st.items() if isinstance(v, (int, float, str, list))}
                log.write(step=counter[0], dt=dt_, halvings=depth, wall_s=wall, **rec, **extra)
            return
        _restore(q, saved)
        if log:
            log.write(step=counter[0] + 1, dt=dt_, halvings=depth, wall_s=wall, failed=True,
                      error=str(err) if err else "not converged", **extra)
        if depth >= max_halvings:
            raise StepFailed(f"step of dt={dt_:g} failed after {depth} halvings")
        one(0.5 * dt_, depth + 1)
        one(0.5 * dt_, depth + 1)

    for _ in range(nsteps):
        one(dt, 0)
        t += dt
    return t
