"""Pins of the gap report (oracle/exact.py::gap_report): the depth-buffer marginal gain against
the exact Eq. 2 marginal gain, summarised as the paper does in Sec. V-A / Fig. 4 (overall ratio,
per-depth mean ratio, least-squares slope and R^2).

The expected numbers are worked out by hand in the comments, not by re-running a regression:
- db = 2 ex exactly: every slope 2, R^2 1, every ratio 2;
- a 4-point fit, ex = (1, 2, 3, 4), db = (2, 3, 5, 6): mean ex 2.5, mean db 4,
  Sxx = 2.25 + 0.25 + 0.25 + 2.25 = 5, Sxy = 3 + 0.5 + 0.5 + 3 = 7, slope 7/5 = 1.4,
  intercept 4 - 1.4 * 2.5 = 0.5, fitted (1.9, 3.3, 4.7, 6.1), SS_res = 0.01 + 0.09 + 0.09 + 0.01
  = 0.2, SS_tot = 4 + 1 + 1 + 4 = 10, R^2 = 0.98; through the origin sum(x y) / sum(x^2) =
  (2 + 6 + 15 + 24) / 30 = 47/30; sum ratio 16/10; per depth (0, 0, 1, 1): (2 + 1.5)/2 = 1.75 and
  (5/3 + 6/4)/2 = 19/12;
- a pure offset, db = ex + 10 with ex = (10, 20, 30): slope 1 with intercept 10, R^2 1, but
  through the origin (10*20 + 20*30 + 30*40) / (100 + 400 + 900) = 2000/1400 = 10/7.

Each planted mistake below (made in a copy of the function, on the CPU) must fail one pin.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import exact


def _pin_failures(fn):
    """Runs every pin against `fn`; returns the names of the pins it fails."""
    bad = []

    def check(name, cond):
        if not cond:
            bad.append(name)

    try:
        ex = np.array([3.0, 7.0, 11.0, 20.0, 41.0])
        r = fn(np.array([0, 1, 1, 2, 2]), 2 * ex, ex)
        check("double: slope", np.isclose(r["slope"], 2.0, rtol=0, atol=1e-12))
        check("double: slope through origin", np.isclose(r["slope_through_origin"], 2.0, rtol=0, atol=1e-12))
        check("double: r2", np.isclose(r["r2"], 1.0, rtol=0, atol=1e-12))
        check("double: sum ratio", np.isclose(r["sum_ratio"], 2.0, rtol=0, atol=1e-12))
        check("double: per depth", all(np.isclose(v, 2.0, rtol=0, atol=1e-12) for v in r["per_depth_mean_ratio"].values())
              and sorted(r["per_depth_mean_ratio"]) == [0, 1, 2])

        r = fn(np.array([0, 0, 1, 1]), np.array([2.0, 3.0, 5.0, 6.0]), np.array([1.0, 2.0, 3.0, 4.0]),
               abs_gain=np.array([4.0, 4.0, 6.0, 6.0]))
        check("4-point: slope", np.isclose(r["slope"], 1.4, rtol=0, atol=1e-12))
        check("4-point: r2", np.isclose(r["r2"], 0.98, rtol=0, atol=1e-12))
        check("4-point: slope through origin", np.isclose(r["slope_through_origin"], 47 / 30, rtol=0, atol=1e-12))
        check("4-point: sum ratio", np.isclose(r["sum_ratio"], 1.6, rtol=0, atol=1e-12))
        check("4-point: sums", r["sum_db"] == 16.0 and r["sum_exact"] == 10.0)
        check("4-point: per depth", np.isclose(r["per_depth_mean_ratio"][0], 1.75, rtol=0, atol=1e-12)
              and np.isclose(r["per_depth_mean_ratio"][1], 19 / 12, rtol=0, atol=1e-12))
        check("4-point: abs ratio", np.isclose(r["abs_sum_ratio"], 2.0, rtol=0, atol=1e-12))

        r = fn(np.array([1, 2, 3]), np.array([20.0, 30.0, 40.0]), np.array([10.0, 20.0, 30.0]))
        check("offset: slope", np.isclose(r["slope"], 1.0, rtol=0, atol=1e-12))
        check("offset: r2", np.isclose(r["r2"], 1.0, rtol=0, atol=1e-12))
        check("offset: slope through origin", np.isclose(r["slope_through_origin"], 10 / 7, rtol=0, atol=1e-12))

        # a node with exact gain 0 has no ratio: it is left out of its depth's mean
        r = fn(np.array([0, 0, 1]), np.array([3.0, 5.0, 4.0]), np.array([0.0, 4.0, 2.0]))
        check("zero exact: per depth", np.isclose(r["per_depth_mean_ratio"][0], 1.25, rtol=0, atol=1e-12)
              and np.isclose(r["per_depth_mean_ratio"][1], 2.0, rtol=0, atol=1e-12))
        check("zero exact: sum ratio", np.isclose(r["sum_ratio"], 2.0, rtol=0, atol=1e-12))
    except Exception as e:  # a mutant may also break the arithmetic outright
        bad.append(f"raised {type(e).__name__}")
    return bad


def test_gap_report_pins():
    assert _pin_failures(exact.gap_report) == []


# planted mistakes: (description, text in gap_report, replacement)
MUTANTS = [
    ("intercept column dropped", "np.vstack([ex, np.ones_like(ex)]).T", "np.vstack([ex]).T"),
    ("axes swapped (exact regressed on the depth-buffer gain)", "coef, *_ = np.linalg.lstsq(A, db, rcond=None)",
     "coef, *_ = np.linalg.lstsq(np.vstack([db, np.ones_like(db)]).T, ex, rcond=None)"),
    ("total sum of squares about zero", "np.sum((db - db.mean()) ** 2)", "np.sum(db ** 2)"),
    ("residuals against the mean", "np.sum((db - pred) ** 2)", "np.sum((db - db.mean()) ** 2 * 0.5)"),
    ("origin slope normalised by the other axis", "np.dot(ex, db) / np.dot(ex, ex)", "np.dot(ex, db) / np.dot(db, db)"),
    ("per-depth ratio inverted", "np.mean(db[m] / ex[m])", "np.mean(ex[m] / db[m])"),
    ("per-depth ratio of sums", "np.mean(db[m] / ex[m])", "db[m].sum() / ex[m].sum()"),
    ("zero exact gains kept in the per-depth mean", "(depth == d) & (ex > 0)", "(depth == d)"),
    ("sum ratio inverted", 'out["sum_db"] / out["sum_exact"]', 'out["sum_exact"] / out["sum_db"]'),
]


def _mutant(src_from, src_to):
    src = textwrap.dedent(inspect.getsource(exact.gap_report))
    assert src.count(src_from) == 1, src_from
    ns = {"np": np}
    exec(compile(src.replace(src_from, src_to), "<gap_report mutant>", "exec"), ns)
    return ns["gap_report"]


@pytest.mark.parametrize("desc,src_from,src_to", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_gap_report_mutant_fails_a_pin(desc, src_from, src_to):
    assert _pin_failures(_mutant(src_from, src_to)), f"planted mistake not caught: {desc}"
