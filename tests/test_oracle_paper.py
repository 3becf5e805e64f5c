"""The oracle reproduces the errors the paper prints for its 3D ADR test.

Golden values: tests/golden/paper_adr_errors.txt (Section 4.2, Tables
"adr_order_40" / "adr_order", Figures "adr_ord12_40" / "adr_ord12").  The
paper's PHISPLIT runs form phi_l by Gauss-Lobatto quadrature plus eq. (16); the
oracle uses Pade scaling and squaring, so agreement to many digits pins the
phi matrices, the Tucker operator, K u (grid orientation on the non-cubic grid,
advection sign), both stages of ETD2RK, and the Lawson schemes at once.
"""
import os

import numpy as np
import pytest

import oracle.integrators as oi
from oracle.integrators import OracleProblem, integrate, rel_err_fro, rel_err_inf
from paper_2304_02327_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_adr_errors.txt")
SCHEMES = {"expeuler": oi.EXPEULER, "etd2rk": oi.ETD2RK,
           "lawson_euler": oi.LAWSON_EULER, "lawson2b": oi.LAWSON2B}


def load_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b, c, s, k, e = line.split()
            rows.append(((int(a), int(b), int(c)), s, int(k), float(e)))
    return rows


def run_paper_case(sizes, scheme, steps):
    p = wl.paper_adr_3d(sizes, steps, SCHEMES[scheme])
    op = OracleProblem.from_problem(p, lmax=2)
    U = integrate(op, p.u0, SCHEMES[scheme], steps)
    return rel_err_inf(U, np.exp(1.0) * p.u0)


# Work units ~ N * steps; the default CPU suite runs the cheap points.
CHEAP = {((40, 41, 42), "expeuler", 50), ((40, 41, 42), "expeuler", 450),
         ((40, 41, 42), "etd2rk", 40), ((40, 41, 42), "etd2rk", 140),
         ((40, 41, 42), "lawson_euler", 800), ((40, 41, 42), "lawson2b", 1500),
         ((80, 81, 82), "expeuler", 50), ((80, 81, 82), "etd2rk", 40)}


def _cases():
    out = []
    for sizes, s, k, e in load_golden():
        marks = [] if (sizes, s, k) in CHEAP else [pytest.mark.slow]
        out.append(pytest.param(sizes, s, k, e, marks=marks, id=f"{'x'.join(map(str, sizes))}-{s}-{k}"))
    return out


def test_golden_file_complete():
    rows = load_golden()
    assert len(rows) == 40
    assert {r[1] for r in rows} == set(SCHEMES)


@pytest.mark.parametrize("sizes,scheme,steps,err", _cases())
def test_oracle_reproduces_paper_error(sizes, scheme, steps, err):
    got = run_paper_case(sizes, scheme, steps)
    # The printed values agree with the oracle to ~1e-11 relative; 1e-8 leaves
    # room for the paper's quadrature-based phi_l and BLAS summation order.
    assert abs(got - err) <= 1e-8 * err, (got, err)


def lq_golden(nhat=None):
    """Rows (nhat, scheme, steps, error) of the printed LQ errors, of one nhat if given."""
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_lq_riccati_errors.txt")):
        if line.strip() and not line.startswith("#"):
            nh, scheme, steps, err = line.split()
            if nhat is None or int(nh) == nhat:
                rows.append((int(nh), scheme, int(steps), float(err)))
    return rows


def test_lq_golden_file_complete():
    rows = lq_golden()
    assert len(rows) == 20
    for nhat in (30, 40):
        r = lq_golden(nhat)
        assert sorted({x[2] for x in r}) == [30, 65, 100, 135, 170]
        assert {x[1] for x in r} == {"etd2rk", "exprosenbrock"}
        # the printed errors fall with the step count (second order)
        for sch in ("etd2rk", "exprosenbrock"):
            e = [x[3] for x in sorted(r) if x[1] == sch]
            assert all(a > b for a, b in zip(e, e[1:]))


def lq_reference(nhat, n_coarse):
    """The LQ solution at T: Richardson extrapolation of the oracle's ETD2RK at
    n_coarse and 2 n_coarse steps (a second-order method, so (4 U_fine - U_coarse)/3)."""
    def run(m):
        p = wl.lq_riccati(nhat, m, wl.ETD2RK)
        return integrate(OracleProblem.from_problem(p), p.u0, wl.ETD2RK, m)
    a, b = run(n_coarse), run(2 * n_coarse)
    return (4 * b - a) / 3, rel_err_fro(b, (4 * b - a) / 3)


def test_lq_riccati_printed_error():
    """The oracle's ETD2RK PHISPLIT on the paper's LQ problem (nhat = 30) reproduces
    the printed errors (Figure "riccati"): against a reference extrapolated from 170
    and 340 steps, the 340-step solution's error is a quarter of the printed 170-step
    error (second order), and the 30-step error is the printed 1.7186e-4 to 0.3 %."""
    printed = {(s, n): e for (_, s, n, e) in lq_golden(30)}
    ref, gap = lq_reference(30, 170)
    assert abs(gap / (printed[("etd2rk", 170)] / 4) - 1) < 0.05, gap
    p = wl.lq_riccati(30, 30, wl.ETD2RK)
    got = integrate(OracleProblem.from_problem(p), p.u0, wl.ETD2RK, 30)
    e = rel_err_fro(got, ref)
    assert abs(e / printed[("etd2rk", 30)] - 1) < 3e-3, e


@pytest.mark.slow
def test_lq_riccati_nhat40_printed_error():
    """nhat = 40 (n = 1600): the oracle's ETD2RK at 30 steps reproduces the printed
    1.9744e-4 of Figure "riccati_40" against a reference extrapolated from 100 and 200
    steps (several minutes of host BLAS, hence slow)."""
    printed = {(s, n): e for (_, s, n, e) in lq_golden(40)}
    ref, gap = lq_reference(40, 100)
    p = wl.lq_riccati(40, 30, wl.ETD2RK)
    got = integrate(OracleProblem.from_problem(p), p.u0, wl.ETD2RK, 30)
    e = rel_err_fro(got, ref)
    assert abs(e / printed[("etd2rk", 30)] - 1) < 5e-3, e
