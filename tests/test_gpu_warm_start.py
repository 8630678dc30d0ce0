"""Warm start, resume and checkpoint (GPU): a solve stopped by its outer-iteration limit resumes from the
grid's potential; a potential written out (pf_result.phi_V) and set on a fresh grid (pf_set_potential)
restarts the iteration; batches and served requests start from a given potential. The fixed point does not
depend on the start, so every variant meets the oracle's solution."""
import time

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def case(orc):
    prob = W.channel_problem(21, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=7,
                             phi_hi_V=0.06)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12)
    assert ref["status"] == 0
    return prob, ref


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 0.0257)


def test_resume_after_iteration_limit(api, case):
    prob, ref = case
    grid = api.Grid.for_problem(prob)
    part, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, max_outer=10), allow=(3,))
    assert rep["status"] == 3 and rep["outer_iters"] == 10
    assert _rel(part["phi_V"], ref["phi_V"]) > 1e-6  # far from the fixed point
    out, rep2 = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, warm_start=1))
    grid.close()
    assert rep2["status"] == 0 and rep2["lin_iters_first"] == 0
    assert _rel(out["phi_V"], ref["phi_V"]) < TOL_FP64


def test_checkpoint_to_a_fresh_grid(api, case):
    prob, ref = case
    grid = api.Grid.for_problem(prob)
    part, _ = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, max_outer=12), allow=(3,))
    grid.close()
    fresh = api.Grid.for_problem(prob)
    with pytest.raises(api.PFError) as e:  # a fresh grid holds no potential
        fresh.nonlinear_solve(api.nl_opts(warm_start=1))
    assert e.value.status == 1
    fresh.set_potential(part["phi_V"].copy())
    out, rep = fresh.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, warm_start=1))
    fresh.close()
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"]) < TOL_FP64


def test_batch_and_served_requests_from_a_potential(api, case):
    prob, ref = case
    guess = np.linspace(0.0, 0.06, prob.grid.nz).repeat(prob.grid.nx * prob.grid.ny)  # a linear ramp in z (V)
    # batch
    grids = [api.Grid.for_problem(prob) for _ in range(2)]
    for g in grids:
        g.set_potential(guess)
    batch = api.Batch(grids, tiles_per_block=2)
    try:
        res = batch.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, warm_start=1))
    finally:
        batch.close()
        for g in grids:
            g.close()
    for out, rep in res:
        assert rep["status"] == 0 and rep["lin_iters_first"] == 0
        assert _rel(out["phi_V"], ref["phi_V"]) < TOL_FP64
    # server
    srv = api.pf_server_create(4 << 30, 2)
    try:
        t = api.pf_submit(srv, api.make_request(prob, api.nl_opts(tol_outer=1e-11, tol=1e-12), phi0_V=guess))
        t0 = time.time()
        while not api.pf_done(srv, t):
            assert time.time() - t0 < 300
            time.sleep(0.005)
        _, out, rep = api.pf_poll(srv, t, prob.grid.n, len(prob.species))
    finally:
        api.pf_server_destroy(srv)
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"]) < TOL_FP64
