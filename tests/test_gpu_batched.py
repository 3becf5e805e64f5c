"""Parity of the batched mixed-form stepper (many independent 2D problems of uneven
size in one graph-captured run) with the FP64 oracle, instance by instance, and with
the single-problem mixed path.

The batched prepass performs the single-problem mixed prepass's arithmetic and the
grouped tensor-core launch computes every output element with the same sequence of
tensor-core products (K-blocks in order, the main product summed in registers), so
a batch must reproduce the single-problem path bit for bit, whatever the tiling.
"""
import numpy as np
import pytest
import torch

from oracle.integrators import OracleProblem, integrate, rel_err_inf, rel_err_fro
from paper_2304_02327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-6
FORMS = ["tf32x3", "bf16x3"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2304_02327_gb300 import api as _api, build
    build.build()
    _api.lib()
    return _api


@pytest.fixture(params=FORMS)
def form(request):
    return request.param


def small_batch(steps=20):
    """A dozen Allen-Cahn instances: several sizes (two equal, so a class holds more
    than one instance), one non-square, eps log-uniform."""
    probs = wl.batched_allen_cahn(count=10, seed=11, steps=steps,
                                  sizes=(48, 64, 96, 128, 160, 208, 256))
    rng = np.random.default_rng(3)
    A1, A2 = wl.fd_matrix(72, 0.02), wl.fd_matrix(136, 0.02)
    probs.append(wl.Problem(name="ac_nonsquare", A=[A1, A2], u0=rng.uniform(-0.9, 0.9, (136, 72)),
                            g_kind=wl.G_CUBIC, cubic=(0.0, 1.0, 0.0, -1.0), tau=1e-3, steps=steps,
                            scheme=wl.EXPEULER))
    probs.append(probs[2].__class__(**{**probs[2].__dict__, "name": "dup", "u0": -probs[2].u0}))
    return probs


def run_batch(api, probs, form, steps, **kw):
    plans, gs, Us = api.setup_batch(probs, form)
    b = api.Batch(plans, gs, Us, **kw)
    b.run(steps)
    torch.cuda.synchronize()
    assert b.status() == 0
    return [u.cpu().numpy() for u in Us], b


def test_batch_matches_oracle_per_instance(api, form):
    probs = small_batch()
    got, b = run_batch(api, probs, form, 20)
    assert b.info()["classes"] == len({p.u0.shape for p in probs})
    for p, g in zip(probs, got):
        ref = integrate(OracleProblem.from_problem(p, lmax=1), p.u0, p.scheme, p.steps)
        assert rel_err_inf(g, ref) <= TOL_STEP and rel_err_fro(g, ref) <= TOL_STEP, p.name


@pytest.mark.parametrize("nc_cap", [160, 128, 64, 48])
def test_batch_equals_single_problem_path_bitwise(api, form, nc_cap):
    probs = small_batch(steps=5)
    got, _ = run_batch(api, probs, form, 5, autotune=False, nc_cap=nc_cap)
    for p, g in zip(probs, got):
        plan, gg, U = api.setup(p, form)
        api.expint_step(plan, p.scheme, U, 5, g=gg)
        np.testing.assert_array_equal(g, U.cpu().numpy(), err_msg=p.name)


def test_batch_graph_and_plain_launches_agree(api, form):
    probs = small_batch(steps=4)
    g1, b1 = run_batch(api, probs, form, 4, graph=True)
    g2, b2 = run_batch(api, probs, form, 4, graph=False)
    for a, c in zip(g1, g2):
        np.testing.assert_array_equal(a, c)
    # a second run of the captured graph continues from the updated states
    b1.run(4)
    torch.cuda.synchronize()
    b2.run(4)
    torch.cuda.synchronize()
    for a, c in zip(b1.Us, b2.Us):
        assert torch.equal(a, c)


@pytest.mark.parametrize("graph", [True, False])
def test_batch_runs_split_anywhere_agree_bitwise(api, form, graph):
    """Inside a run, each step's update is fused into the next step's prepass and the
    state alternates between the caller's buffers and a second set; the last update
    writes the caller's buffers in place (an even number of fused passes) or from the
    second set (odd).  A run of 5 steps, runs of 2 + 3, of 4 + 1 and five runs of one
    step must all give the same states bit for bit."""
    probs = small_batch(steps=5)
    ref, _ = run_batch(api, probs, form, 5, autotune=False, nc_cap=128, graph=graph)
    for split in ((2, 3), (4, 1), (1, 1, 1, 1, 1)):
        plans, gs, Us = api.setup_batch(probs, form)
        b = api.Batch(plans, gs, Us, autotune=False, nc_cap=128, graph=graph)
        for k in split:
            b.run(k)
        torch.cuda.synchronize()
        assert b.status() == 0
        for a, u, p in zip(ref, Us, probs):
            np.testing.assert_array_equal(a, u.cpu().numpy(), err_msg=f"{p.name} {split}")


def test_batch_paired_and_single_column_prepass_agree_bitwise(api, form):
    """A batch whose instances all have an even n_1 runs the two-columns-per-thread
    prepass; one odd-sized instance switches the whole batch to the one-column kernel.
    Both must give the same states for the shared instances, bit for bit (over a run, so
    the fused update-and-prepass pass is compared too), and the odd instance must match
    the oracle."""
    even = small_batch(steps=4)
    rng = np.random.default_rng(8)
    A1, A2 = wl.fd_matrix(45, 0.03), wl.fd_matrix(38, 0.03)
    odd = wl.Problem(name="ac_odd", A=[A1, A2], u0=rng.uniform(-0.9, 0.9, (38, 45)),
                     g_kind=wl.G_CUBIC, cubic=(0.0, 1.0, 0.0, -1.0), tau=1e-3, steps=4,
                     scheme=wl.EXPEULER)
    got_even, _ = run_batch(api, even, form, 4, autotune=False, nc_cap=128)
    got_mixed, _ = run_batch(api, even + [odd], form, 4, autotune=False, nc_cap=128)
    for a, b, p in zip(got_even, got_mixed, even):
        np.testing.assert_array_equal(a, b, err_msg=p.name)
    ref = integrate(OracleProblem.from_problem(odd, lmax=1), odd.u0, odd.scheme, odd.steps)
    assert rel_err_inf(got_mixed[-1], ref) <= TOL_STEP


def test_batch_autotune_picks_a_candidate(api, form):
    """The autotuner's schedule: a candidate width per size class, kept per class only
    when faster than the best uniform width; the tuned batch still reproduces the
    single-problem path bit for bit (the width never changes an element's products)."""
    probs = small_batch(steps=3)
    got, b = run_batch(api, probs, form, 3, autotune=True)
    sch = b.schedule()
    assert b.info()["nc_cap"] in (160, 128, 96, 64)
    assert len(sch["widths"]) == b.info()["classes"]
    assert set(sch["widths"]) <= {160, 128, 96, 64}
    assert sch["per_class"] or len(set(sch["widths"])) == 1
    assert 0 < sch["tucker_ms_chosen"] <= sch["tucker_ms_uniform"]
    assert sch["tile_order"] in ("round-robin", "alternate rounds reversed")
    for p, g in zip(probs, got):
        plan, gg, U = api.setup(p, form)
        api.expint_step(plan, p.scheme, U, 3, g=gg)
        np.testing.assert_array_equal(g, U.cpu().numpy(), err_msg=p.name)
    # eager launches of the same tuned batch continue exactly like the graph replays
    b2 = run_batch(api, probs, form, 3, autotune=False, nc_cap=64)[1]
    b.set_graph(False)
    b.run(2)
    b2.run(2)
    torch.cuda.synchronize()
    for a, c in zip(b.Us, b2.Us):
        assert torch.equal(a, c)


def test_batch_rejects_unsupported(api):
    p = small_batch(steps=1)[:2]
    plans, gs, Us = api.setup_batch(p, "fp64")
    with pytest.raises(api.PhisplitError) as e:
        api.Batch(plans, gs, Us)
    assert e.value.code == -3
    plans, gs, Us = api.setup_batch(p, "bf16x3")
    with pytest.raises(api.PhisplitError):
        api.Batch(plans, gs, Us, scheme=wl.ETD2RK)


def test_batch_full_config_sampled_instances(api):
    """1024 instances, n uniform over {48, 64, ..., 512}, eps log-uniform in
    [1e-3, 1e-1], 20 exponential Euler steps in BF16x3 with the autotuned tiling and
    the captured graph (the configuration the bench times); eight instances,
    including the largest and the smallest size, are integrated by the oracle."""
    probs = wl.batched_allen_cahn()
    got, b = run_batch(api, probs, "bf16x3", 20)
    assert b.info()["dof"] == sum(p.u0.size for p in probs)
    rng = np.random.default_rng(2024)
    sizes = np.array([p.n[0] for p in probs])
    pick = set(rng.choice(len(probs), 6, replace=False).tolist())
    pick |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for k in sorted(pick):
        p = probs[k]
        ref = integrate(OracleProblem.from_problem(p, lmax=1), p.u0, p.scheme, p.steps)
        assert rel_err_inf(got[k], ref) <= TOL_STEP, (k, p.n[0])


@pytest.mark.parametrize("steps", [1, 3])
def test_batch_nonfinite_state_raises_status(api, steps):
    """A NaN planted (on the host) in one instance's initial state reaches the batch's
    status word, through the closing update pass (one step) and through the fused
    update-and-prepass passes of a longer run; the other instances are unaffected."""
    probs = small_batch(steps=steps)
    probs[3].u0[5, 7] = np.nan
    plans, gs, Us = api.setup_batch(probs, "bf16x3")
    b = api.Batch(plans, gs, Us, autotune=False, nc_cap=128)
    b.run(steps)
    torch.cuda.synchronize()
    assert b.status(reset=True) & api.STATUS_NONFINITE
    assert b.status() == 0
    ref_probs = small_batch(steps=steps)
    got, _ = run_batch(api, ref_probs, "bf16x3", steps, autotune=False, nc_cap=128)
    for k, (u, g) in enumerate(zip(Us, got)):
        if k != 3:
            np.testing.assert_array_equal(u.cpu().numpy(), g)
