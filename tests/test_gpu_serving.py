"""Serving through pf_submit / pf_poll (GPU): admitted problems share the batched launches, each result is
bitwise that of the same problem in a batch of its own (the engine's 4 tiles per block) and agrees with
pf_nonlinear_solve to the solver tolerance, the HBM budget gates admission, and requests that can never fit
are refused."""
import time

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api as A
    return A


def _problems():
    out = []
    for i, (n, v, salt) in enumerate([(17, 0.05, 0.1), (21, -0.03, 0.2), (25, 0.08, 0.05), (17, -0.1, 0.4),
                                      (29, 0.02, 0.15), (21, 0.0, 0.3)]):
        sp = [W.Species(1, 0.95, salt), W.Species(-1, 1.81, salt), W.WATER]
        out.append(W.channel_problem(n, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=2,
                                     charge_seed=10 + i, phi_hi_V=v, species=sp, name=f"srv{i}"))
    return out


def _wait(api, srv, ticket, prob, timeout=300.0):
    t0 = time.time()
    while True:
        done, out, rep = api.pf_poll(srv, ticket, prob.grid.n, len(prob.species))
        if done:
            return out, rep
        assert time.time() - t0 < timeout
        time.sleep(0.005)


def _alone(api, prob, opts):
    """The problem in a batch of its own with the serving engine's block split."""
    grid = api.Grid.for_problem(prob)
    batch = api.Batch([grid], tiles_per_block=4)
    (out, rep), = batch.nonlinear_solve(opts)
    batch.close()
    grid.close()
    return out, rep


def _single(api, prob, opts):
    grid = api.Grid.for_problem(prob)
    out, rep = grid.nonlinear_solve(opts)
    grid.close()
    return out, rep


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mixed_stream_equals_alone(api, precision):
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    opts = api.nl_opts(tol_outer=1e-9, tol=1e-11, precision=prec)
    probs = _problems()
    srv = api.pf_server_create(8 << 30, 3)
    try:
        reqs = [api.make_request(p, opts) for p in probs]
        tickets = [api.pf_submit(srv, q) for q in reqs]
        results = [_wait(api, srv, t, p) for t, p in zip(tickets, probs)]
    finally:
        api.pf_server_destroy(srv)
    for p, (out, rep) in zip(probs, results):
        assert rep["status"] == 0
        ref, rref = _alone(api, p, opts)
        # same kernels, block split and reduction orders: identical to the problem's own batch
        np.testing.assert_array_equal(out["phi_V"], ref["phi_V"])
        np.testing.assert_array_equal(out["C_M"], ref["C_M"])
        assert rep["outer_iters"] == rref["outer_iters"]
        # and the single-grid solver (another block split) to the solver tolerance
        sref, _ = _single(api, p, opts)
        tol = 1e-8 if precision == "fp64" else 1e-6
        assert np.abs(out["phi_V"] - sref["phi_V"]).max() <= tol * max(np.abs(sref["phi_V"]).max(), 0.0257)


def test_budget_refuses_what_can_never_fit(api):
    srv = api.pf_server_create(1 << 20, 2)  # 1 MiB: no grid fits
    try:
        q = api.make_request(_problems()[0])
        with pytest.raises(api.PFError) as e:
            api.pf_submit(srv, q)
        assert e.value.status == 2  # PF_E_OOM
    finally:
        api.pf_server_destroy(srv)


def test_budget_gates_admission(api):
    """A budget that holds one problem at a time still completes every request correctly."""
    probs = _problems()[:3]
    from paper_1711_04060_gb300 import _binding as B
    opts = api.nl_opts(tol_outer=1e-8, tol=1e-10)
    # just above the device bytes of the largest grid
    one = int(1.05 * max(api.pf_grid_bytes(p.grid.nx, p.grid.ny, p.grid.nz) for p in probs))
    srv = api.pf_server_create(one, 3)
    try:
        tickets = [api.pf_submit(srv, api.make_request(p, opts)) for p in probs]
        results = [_wait(api, srv, t, p) for t, p in zip(tickets, probs)]
        with pytest.raises(api.PFError):
            api.pf_poll(srv, 987654321, 8, 3)  # unknown ticket
    finally:
        api.pf_server_destroy(srv)
    for p, (out, rep) in zip(probs, results):
        ref, _ = _alone(api, p, opts)
        np.testing.assert_array_equal(out["phi_V"], ref["phi_V"])
    assert B.PF_PENDING == 8


def test_mixed_precisions_and_a_failing_request(api):
    """Requests of both precisions share the engine; one that hits its outer-iteration limit ends with
    PF_E_NOCONV while the others finish normally and still equal their own batches."""
    probs = _problems()[:4]
    o64 = api.nl_opts(tol_outer=1e-9, tol=1e-11, precision=api.PF_FP64)
    omx = api.nl_opts(tol_outer=1e-9, tol=1e-11, precision=api.PF_MIXED)
    ofail = api.nl_opts(tol_outer=1e-12, tol=1e-11, max_outer=3)
    opts = [o64, omx, ofail, omx]
    srv = api.pf_server_create(8 << 30, 4)
    try:
        tickets = [api.pf_submit(srv, api.make_request(p, o)) for p, o in zip(probs, opts)]
        results = []
        for t, p in zip(tickets, probs):
            t0 = time.time()
            while not api.pf_done(srv, t):
                assert time.time() - t0 < 300
                time.sleep(0.005)
            results.append(api.pf_poll(srv, t, p.grid.n, len(p.species), allow=(3,)))
    finally:
        api.pf_server_destroy(srv)
    assert [r[2]["status"] for r in results] == [0, 0, 3, 0]
    assert results[2][2]["outer_iters"] == 3
    for k in (0, 1, 3):
        ref, _ = _alone(api, probs[k], opts[k])
        np.testing.assert_array_equal(results[k][1]["phi_V"], ref["phi_V"])
