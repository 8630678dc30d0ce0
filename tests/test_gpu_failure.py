"""Failure detection without a GPU fault: a bounded device wait that runs out reports PF_E_TIMEOUT and leaves
the context usable; a non-finite right-hand side ends the solve with PF_E_BREAKDOWN before the unknown is
touched; a server destroyed with requests in flight and in its queue cancels them cleanly."""
import ctypes

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


def test_bounded_wait_runs_out(api):
    from paper_1711_04060_gb300 import _binding as B
    lib = B.load()
    assert lib.pf_selftest_wait_timeout(2_000_000, None) == B.PF_E_TIMEOUT
    assert b"gave up" in lib.pf_last_error()
    # the context is still usable: a small solve succeeds afterwards
    p = W.linear_problem(n=17, seed=5, n_spheres=2)
    g = p.grid
    grid = api.Grid(g.nx, g.ny, g.nz, g.h, g.origin)
    grid.set_coeffs(p.eps, np.ones(g.n, np.uint8), np.zeros((0, 4)), 0.0, 0.0, [W.NA, W.CL, W.WATER], 78.5, 1.2)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(tol=1e-10))
    grid.close()
    assert rep["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_rhs_is_a_breakdown(api, precision):
    p = W.linear_problem(n=17, seed=6, n_spheres=2)
    g = p.grid
    grid = api.Grid(g.nx, g.ny, g.nz, g.h, g.origin)
    grid.set_coeffs(p.eps, np.ones(g.n, np.uint8), np.zeros((0, 4)), 0.0, 0.0, [W.NA, W.CL, W.WATER], 78.5, 1.2)
    b = p.b.copy()
    b[g.n // 2] = np.nan
    x = np.zeros(g.n)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    rep = grid.linear_solve(api.PF_OP_POISSON, b, x, api.solve_opts(tol=1e-10, precision=prec), allow=(4,))
    assert rep["status"] == 4  # PF_E_BREAKDOWN
    # the grid still works for a finite problem
    x2 = np.zeros(g.n)
    assert grid.linear_solve(api.PF_OP_POISSON, p.b, x2, api.solve_opts(tol=1e-10, precision=prec))["status"] == 0
    grid.close()


def test_server_destroy_cancels_queued_requests(api):
    probs = [W.channel_problem(n, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=2,
                               charge_seed=60 + n) for n in (17, 21, 25, 29, 33, 17)]
    srv = api.pf_server_create(8 << 30, 1)
    tickets = [api.pf_submit(srv, api.make_request(p)) for p in probs]
    assert len(set(tickets)) == len(tickets)
    api.pf_server_destroy(srv)  # one request in flight, the rest queued: returns without waiting for them
