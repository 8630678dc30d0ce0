"""pf_fermi_noalloc: the pointwise step of Eq. (1) for callers that cannot allocate device memory.

It is checked through the C ABI against the outputs of pf_nonlinear_solve, the existing entry point
whose final step computes the same concentrations, steric potential and void fraction from the
converged potential.  Two calls in a row must both match: the second one runs on the scratch array
the first one left behind.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api
    return torch, api


def test_fermi_noalloc_matches_nonlinear_solve(torch_api):
    torch, api = torch_api
    prob = W.channel_problem(21, box_half=10.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=3,
                             species=[W.Species(1, 0.95, 0.1), W.Species(2, 0.99, 0.002), W.Species(-1, 1.81, 0.104),
                                      W.WATER])
    n, ns = prob.grid.n, len(prob.species)
    grid = api.Grid.for_problem(prob)
    dev = {k: torch.zeros(m, dtype=torch.float64, device="cuda")
           for k, m in (("phi_V", n), ("C_M", ns * n), ("S", n), ("Gamma", n))}
    grid.nonlinear_solve(api.nl_opts(tol_outer=1e-10, tol=1e-12), out=dev)
    grid.close()
    torch.cuda.synchronize()
    solvent = torch.from_numpy(prob.solvent.copy()).cuda()
    for call in range(2):
        C = torch.full((ns * n,), -1.0, dtype=torch.float64, device="cuda")
        S = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        G = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        assert api.pf_fermi_noalloc(dev["phi_V"], solvent, prob.species, C, S, G, T_K=prob.T_K) == 0
        torch.cuda.synchronize()
        # the pointwise Newton iteration stops once its step is below 1e-6 max(1, |ln Gamma|); it converges
        # quadratically, so calls from different starting points (here: the bath value against the solve's
        # previous iterate) agree to about 1e-12 max(1, ln^2 Gamma)
        for got, ref in ((C, dev["C_M"]), (S, dev["S"]), (G, dev["Gamma"])):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.abs(g - r).max() <= 1e-10 * max(np.abs(r).max(), 1.0), call


def test_fermi_noalloc_rejects_sizes_beyond_its_scratch(torch_api):
    torch, api = torch_api
    from paper_1711_04060_gb300 import _binding as B
    lib = B.load()
    sp = (B.pf_species * 3)()
    for i, s in enumerate((W.NA, W.CL, W.WATER)):
        sp[i].z, sp[i].radius_A, sp[i].bulk_M = s.z, s.radius_A, s.bulk_M
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    m = torch.ones(4, dtype=torch.uint8, device="cuda")
    st = lib.pf_fermi_noalloc(B.PF_FERMI_NOALLOC_MAX_NODES + 1, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(m.data_ptr()), 3, sp, 298.15, ctypes.c_void_p(x.data_ptr()), None, None,
                              None)
    assert st == B.PF_E_INVAL
    assert b"PF_FERMI_NOALLOC_MAX_NODES" in lib.pf_last_error()
