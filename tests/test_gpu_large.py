"""Parity at the full sizes of the measured configurations, through the C ABI.

* 3D ADR at n = 320 (N = 32.8M), 100 ETD2RK steps: the oracle cannot run the whole
  trajectory in a test, so (i) the FP64 GPU form's last step, taken from its own
  state at step 99, is compared with the oracle's step from that state on a seeded
  grid of sampled output entries (the oracle forms K U + G, the first stage and
  G(U2) - G(U) in full and the last Tucker operator only on sampled rows of phi_2,
  `oracle.integrators.step_at`); (ii) each split-precision form's whole 100-step run
  is compared with the FP64 GPU run (itself pinned to the oracle); (iii) each
  split-precision form takes step 100 from the same FP64 state, against the
  oracle's sampled step.
* Matrix Riccati at n = 2048, 50 steps, exponential Euler and ETD2RK: the whole
  trajectory of the oracle (about 10^13 flops, tens of seconds of BLAS on the host
  cores) against all three forms, plus the sampled last ETD2RK step as above.

Tolerances: FP64 1e-12 relative; split-precision forms 1e-6 relative over a whole
run (the stated tolerance of the mixed forms) and 1e-7 on one step (the mixed
error of one increment tau Y, ~1e-6 of |tau Y|, is far below |U|).
"""
import numpy as np
import pytest
import torch

from oracle.integrators import OracleProblem, integrate, rel_err_fro, rel_err_inf, step_at
from paper_2304_02327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_RUN = 1e-6
TOL_ONE_STEP = 1e-7
FORMS = ["bf16x3", "tf32x3"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2304_02327_gb300 import api as _api, build
    build.build()
    _api.lib()
    return _api


def sampled_sets(ns, k, seed):
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(n, min(n, k), replace=False)) for n in ns]


def fp64_run_with_last_step(api, p):
    """FP64 GPU run of p.steps steps; returns (state at step S-1 on the device,
    final state on the host)."""
    plan, g, U = api.setup(p, "fp64")
    api.expint_step(plan, p.scheme, U, p.steps - 1, g=g)
    prev = U.clone()
    api.expint_step(plan, p.scheme, U, 1, t0=(p.steps - 1) * p.tau, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return prev, U.cpu().numpy()


def rel_sampled(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


class Trajectory:
    """The FP64 GPU trajectory of a workload and the oracle's sampled last step."""

    def __init__(self, api, p, k, seed):
        self.p = p
        self.prev, self.final = fp64_run_with_last_step(api, p)
        self.sets = sampled_sets(p.n, k, seed)
        self.ix = np.ix_(*reversed(self.sets))
        self.t_last = (p.steps - 1) * p.tau
        op = OracleProblem.from_problem(p)
        self.ref = step_at(op, self.prev.cpu().numpy(), p.scheme, self.t_last, self.sets)

    def mixed(self, api, prec):
        """(whole run of the form from u0, its last step from the FP64 state) on the host."""
        p = self.p
        plan, g, U = api.setup(p, prec)
        api.expint_step(plan, p.scheme, U, p.steps, g=g)
        torch.cuda.synchronize()
        full = U.cpu().numpy()
        U.copy_(self.prev)
        api.expint_step(plan, p.scheme, U, 1, t0=self.t_last, g=g)
        torch.cuda.synchronize()
        assert plan.status() == 0
        one = U.cpu().numpy()[self.ix]
        del plan, g, U
        torch.cuda.empty_cache()
        return full, one


@pytest.fixture(scope="module")
def adr320(api):
    t = Trajectory(api, wl.workload("adr3d_n320_etd2rk"), 24, 320)
    yield t
    del t
    torch.cuda.empty_cache()


def test_fp64_adr3d_n320_last_step_sampled(adr320):
    """Step 100 of the n = 320 ETD2RK run from the GPU's own state at step 99, FP64
    form, against the oracle on 24^3 sampled entries."""
    assert rel_sampled(adr320.final[adr320.ix], adr320.ref) <= TOL_FP64


@pytest.mark.parametrize("form", FORMS)
def test_mixed_adr3d_n320_full_run(api, adr320, form):
    """All 100 ETD2RK steps at n = 320 in a split-precision form: the whole run against
    the FP64 GPU run, and step 100 from the FP64 state against the oracle."""
    full, one = adr320.mixed(api, form)
    assert rel_err_inf(full, adr320.final) <= TOL_RUN
    assert rel_err_fro(full, adr320.final) <= TOL_RUN
    assert rel_sampled(one, adr320.ref) <= TOL_ONE_STEP


@pytest.fixture(scope="module")
def riccati_etd(api):
    t = Trajectory(api, wl.workload("riccati_n2048_etd2rk"), 64, 2048)
    yield t
    del t
    torch.cuda.empty_cache()


def test_fp64_riccati_n2048_etd2rk_last_step_sampled(riccati_etd):
    """Step 50 of the n = 2048 Riccati ETD2RK run from the GPU's own state at step 49,
    FP64 form, against the oracle on 64 x 64 sampled entries."""
    assert rel_sampled(riccati_etd.final[riccati_etd.ix], riccati_etd.ref) <= TOL_FP64


@pytest.mark.parametrize("form", FORMS)
def test_mixed_riccati_n2048_etd2rk_sampled_last_step(api, riccati_etd, form):
    """Riccati n = 2048 ETD2RK in a split-precision form: the whole 50-step run against
    the FP64 GPU run, and step 50 from the FP64 state against the oracle."""
    full, one = riccati_etd.mixed(api, form)
    assert rel_err_fro(full, riccati_etd.final) <= TOL_RUN
    assert rel_err_inf(full, riccati_etd.final) <= TOL_RUN
    assert rel_sampled(one, riccati_etd.ref) <= TOL_ONE_STEP


@pytest.mark.parametrize("name", ["riccati_n2048_expeuler", "riccati_n2048_etd2rk"])
def test_riccati_n2048_whole_run_against_the_oracle(api, name):
    """The whole 50-step Riccati run at n = 2048 in every form against the oracle's
    whole run (relative errors in the infinity and Frobenius norms)."""
    p = wl.workload(name)
    ref = integrate(OracleProblem.from_problem(p), p.u0, p.scheme, p.steps)
    for form, tol in (("fp64", TOL_FP64), ("bf16x3", TOL_RUN), ("tf32x3", TOL_RUN)):
        plan, g, U = api.setup(p, form)
        api.expint_step(plan, p.scheme, U, p.steps, g=g)
        torch.cuda.synchronize()
        assert plan.status() == 0
        got = U.cpu().numpy()
        assert rel_err_inf(got, ref) <= tol, (form, rel_err_inf(got, ref))
        assert rel_err_fro(got, ref) <= tol, (form, rel_err_fro(got, ref))
        del plan, g, U
        torch.cuda.empty_cache()
