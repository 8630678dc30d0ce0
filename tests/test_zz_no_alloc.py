"""pf_fermi_noalloc: the pointwise Fermi/steric step for callers that cannot allocate device memory.

Some callers own all device memory themselves (a fixed arena handed to the library, a pool that another
runtime manages) or run where a cudaMalloc is not allowed or would stall; this entry point keeps its
scratch in a fixed device array inside the library instead.  It is checked through the C ABI against
pf_nonlinear_solve, the existing entry point whose final step computes the same concentrations, steric
potential and void fraction from the converged potential, on two calls in a row (the second one starts
from the scratch the first one left behind), and against the CPU oracle's pointwise step at sampled nodes,
up to the largest size the scratch holds.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPECIES = [W.Species(1, 0.95, 0.1), W.Species(2, 0.99, 0.002), W.Species(-1, 1.81, 0.104), W.WATER]


@pytest.fixture(scope="module")
def torch_api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api
    return torch, api


def _oracle_points(orc, species, phi_V, T_K=298.15):
    """The oracle's pointwise step at each potential (volts): C in mol/L, S, Gamma."""
    z = [s.z for s in species]
    sp = orc.species_setup(z, [s.radius_A for s in species], [s.bulk_M for s in species])
    tv, m = orc.thermal_voltage(T_K), orc.molar_to_per_A3()
    C, S, G = [], [], []
    for v in phi_V:
        r = orc.fermi_point(sp, z, float(v) / tv)
        assert r["status"] == 0
        C.append(np.asarray(r["C"]) / m)
        S.append(r["S"])
        G.append(r["Gamma"])
    return np.array(C).T, np.array(S), np.array(G)


def test_fermi_noalloc_matches_nonlinear_solve(torch_api, orc):
    torch, api = torch_api
    prob = W.channel_problem(21, box_half=10.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=3,
                             species=SPECIES)
    n, ns = prob.grid.n, len(prob.species)
    grid = api.Grid.for_problem(prob)
    dev = {k: torch.zeros(m, dtype=torch.float64, device="cuda")
           for k, m in (("phi_V", n), ("C_M", ns * n), ("S", n), ("Gamma", n))}
    grid.nonlinear_solve(api.nl_opts(tol_outer=1e-10, tol=1e-12), out=dev)
    grid.close()
    torch.cuda.synchronize()
    solvent = torch.from_numpy(prob.solvent.copy()).cuda()
    sol = np.flatnonzero(prob.solvent)
    pick = sol[np.linspace(0, len(sol) - 1, 300).astype(np.int64)]
    oC, oS, oG = _oracle_points(orc, prob.species, dev["phi_V"].cpu().numpy()[pick])
    for call in range(2):
        C = torch.full((ns * n,), -1.0, dtype=torch.float64, device="cuda")
        S = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        G = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        # the first call starts every root search from the bath value, the second from the first call's roots
        assert api.pf_fermi_noalloc(dev["phi_V"], solvent, prob.species, C, S, G, T_K=prob.T_K,
                                    warm_start=call == 1) == 0
        torch.cuda.synchronize()
        # the pointwise Newton iteration stops once its step is below 1e-6 max(1, |ln Gamma|); it converges
        # quadratically, so calls from different starting points (the bath value, the previous call's root, the
        # solve's previous outer iterate) agree to about 1e-12 max(1, ln^2 Gamma)
        for got, ref in ((C, dev["C_M"]), (S, dev["S"]), (G, dev["Gamma"])):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.abs(g - r).max() <= 1e-10 * max(np.abs(r).max(), 1.0), call
        Cn = C.cpu().numpy().reshape(ns, n)
        for i in range(ns):
            assert np.abs(Cn[i, pick] - oC[i]).max() <= 1e-9 * np.abs(oC[i]).max(), (call, i)
        assert np.abs(S.cpu().numpy()[pick] - oS).max() <= 1e-9
        assert np.abs(G.cpu().numpy()[pick] - oG).max() <= 1e-9 * oG.max()


def test_fermi_noalloc_at_its_largest_size(torch_api, orc):
    """n = PF_FERMI_NOALLOC_MAX_NODES exactly, potentials over the range the channel solves reach (seeded,
    uniform in [-0.5, 0.5] V, i.e. |phi_hat| < 20) on a seeded 3:1 solvent mask: sampled nodes (the first
    and the last among them) against the oracle, zeros off the solvent, two calls in a row."""
    torch, api = torch_api
    from paper_1711_04060_gb300 import _binding as B
    n = B.PF_FERMI_NOALLOC_MAX_NODES
    ns = len(SPECIES)
    phi = W.uniform(W.substream(77, 1), n, -0.5, 0.5)
    mask = (W.uniform(W.substream(77, 2), n, 0.0, 1.0) < 0.75).astype(np.uint8)
    phi_d = torch.from_numpy(phi).cuda()
    mask_d = torch.from_numpy(mask).cuda()
    sol = np.flatnonzero(mask)
    pick = np.unique(np.concatenate([sol[np.linspace(0, len(sol) - 1, 400).astype(np.int64)], [sol[-1]]]))
    oC, oS, oG = _oracle_points(orc, SPECIES, phi[pick])
    for call in range(2):
        C = torch.full((ns * n,), -1.0, dtype=torch.float64, device="cuda")
        S = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        G = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        assert api.pf_fermi_noalloc(phi_d, mask_d, SPECIES, C, S, G, warm_start=call == 1) == 0
        torch.cuda.synchronize()
        Cn, Sn, Gn = C.cpu().numpy().reshape(ns, n), S.cpu().numpy(), G.cpu().numpy()
        for i in range(ns):
            assert np.abs(Cn[i, pick] - oC[i]).max() <= 1e-9 * np.abs(oC[i]).max(), (call, i)
        assert np.abs(Sn[pick] - oS).max() <= 1e-9
        assert np.abs(Gn[pick] - oG).max() <= 1e-9 * oG.max()
        off = mask == 0
        assert np.all(Cn[:, off] == 0.0) and np.all(Sn[off] == 0.0) and np.all(Gn[off] == 0.0)
        assert np.all(Gn[~off] > 0.0) and np.all(Gn[~off] < 1.0)


def test_fermi_noalloc_rejects_bad_calls(torch_api):
    torch, api = torch_api
    from paper_1711_04060_gb300 import _binding as B
    lib = B.load()
    sp = (B.pf_species * 3)()
    for i, s in enumerate((W.NA, W.CL, W.WATER)):
        sp[i].z, sp[i].radius_A, sp[i].bulk_M = s.z, s.radius_A, s.bulk_M
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    m = torch.ones(4, dtype=torch.uint8, device="cuda")
    px, pm = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr())
    st = lib.pf_fermi_noalloc(B.PF_FERMI_NOALLOC_MAX_NODES + 1, px, pm, 3, sp, 298.15, 0, px, None, None, None)
    assert st == B.PF_E_INVAL
    assert b"PF_FERMI_NOALLOC_MAX_NODES" in lib.pf_last_error()
    # the concentrations are required
    assert lib.pf_fermi_noalloc(4, px, pm, 3, sp, 298.15, 0, None, None, None, None) == B.PF_E_INVAL
    # a charged bath is refused by the same species check as pf_set_coeffs
    sp[0].bulk_M = 0.2
    assert lib.pf_fermi_noalloc(4, px, pm, 3, sp, 298.15, 0, px, None, None, None) == B.PF_E_INVAL
    assert b"electroneutral" in lib.pf_last_error()
