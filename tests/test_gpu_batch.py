"""Batched solves through pf_batch_* (GPU): every problem of a batch of uneven grids matches the oracle,
a problem's result is bitwise the same alone and in a mix (same tiles per block), agrees with
pf_nonlinear_solve to the solver tolerance, and the autotuner reports its candidates."""
import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6
TOL_CONC = 1e-6


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
    """Four channels of different sizes (one non-cubic, with ragged tiles), voltages and salts."""
    out = []
    for i, (n, v, salt) in enumerate([(17, 0.05, 0.1), (21, -0.04, 0.3), (25, 0.08, 0.02), (29, 0.02, 0.15)]):
        sp = [W.Species(1, 0.95, salt), W.Species(-1, 1.81, salt), W.WATER]
        p = W.channel_problem(n, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=2,
                              charge_seed=40 + i, phi_hi_V=v, species=sp, name=f"b{i}")
        out.append(p)
    # non-cubic: 35 x 13 x 21 with an off-centre pore
    p = out[2]
    g = W.Grid(35, 13, 21, 0.5, (-8.5, -3.0, -5.0))
    X, Y, Z = g.coords()
    memb = (np.abs(Z) < 2.0) & ((X - 1.0) ** 2 + Y ** 2 >= 4.0)
    p.grid = g
    p.solvent = (~memb).astype(np.uint8).ravel()
    p.eps = np.where(memb, 2.0, 78.5).ravel()
    p.charges = np.array([[1.0, 2.0, 0.3, 0.5], [-1.0, 1.8, -1.1, -0.5]])
    return out


def _rel(a, b, floor=1e-300):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def _batch_solve(api, probs, opts, tpb):
    grids = [api.Grid.for_problem(p) for p in probs]
    batch = api.Batch(grids, tiles_per_block=tpb)
    try:
        res = batch.nonlinear_solve(opts)
        tune = batch.tune()
    finally:
        batch.close()
        for g in grids:
            g.close()
    return res, tune


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_oracle(api, orc, precision):
    probs = _problems()
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    res, _ = _batch_solve(api, probs, api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec), tpb=2)
    for p, (out, rep) in zip(probs, res):
        assert rep["status"] == 0
        ref = orc.pf_solve_problem(p, tol_outer=1e-11, lin_tol=1e-12)
        assert ref["status"] == 0
        assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)
        ns, n = len(p.species), p.grid.n
        C = out["C_M"].reshape(ns, n)
        for i in range(ns):
            assert _rel(C[i], ref["C_M"][i]) < TOL_CONC, (p.name, i)


def test_other_tile_depths_match_the_oracle(api, orc):
    probs = _problems()[:2]
    grids = [api.Grid.for_problem(p) for p in probs]
    batch = api.Batch(grids)
    try:
        for z in (16, 64):
            batch.set_tiling(2, z)
            res = batch.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12))
            for p, (out, rep) in zip(probs, res):
                ref = orc.pf_solve_problem(p, tol_outer=1e-11, lin_tol=1e-12)
                assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < TOL_FP64
    finally:
        batch.close()
        for g in grids:
            g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alone_equals_in_mix_bitwise(api, precision):
    probs = _problems()
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    opts = api.nl_opts(tol_outer=1e-9, tol=1e-11, precision=prec)
    mix, _ = _batch_solve(api, probs, opts, tpb=2)
    for k in (0, 2):
        alone, _ = _batch_solve(api, [probs[k]], opts, tpb=2)
        np.testing.assert_array_equal(alone[0][0]["phi_V"], mix[k][0]["phi_V"])
        np.testing.assert_array_equal(alone[0][0]["C_M"], mix[k][0]["C_M"])
        assert alone[0][1]["outer_iters"] == mix[k][1]["outer_iters"]


def test_batch_agrees_with_single_grid_solver(api):
    probs = _problems()
    opts = api.nl_opts(tol_outer=1e-11, tol=1e-12)
    res, _ = _batch_solve(api, probs, opts, tpb=4)
    for p, (out, rep) in zip(probs, res):
        grid = api.Grid.for_problem(p)
        ref, rref = grid.nonlinear_solve(opts)
        grid.close()
        assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < TOL_FP64
        assert abs(rep["outer_iters"] - rref["outer_iters"]) <= 1


def test_batch_anderson_same_fixed_point(api, orc):
    probs = _problems()[:2]
    res, _ = _batch_solve(api, probs, api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=api.PF_MIXED,
                                                  accel_depth=5), tpb=2)
    for p, (out, rep) in zip(probs, res):
        ref = orc.pf_solve_problem(p, tol_outer=1e-11, lin_tol=1e-12)
        assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < TOL_MIXED
        assert rep["outer_iters"] < 0.8 * ref["report"]["outer_iters"]


def test_autotuner_record(api):
    probs = _problems()
    grids = [api.Grid.for_problem(p) for p in probs]
    batch = api.Batch(grids)
    try:
        t = batch.autotune()
        assert t["tiles_per_block"] == [1, 2, 4, 8, 16] * 3
        assert t["z_planes"] == [16] * 5 + [32] * 5 + [64] * 5
        assert all(ms > 0 for ms in t["ms"])
        k = int(np.argmin(t["ms"]))
        assert (t["chosen"], t["chosen_z"]) == (t["tiles_per_block"][k], t["z_planes"][k])
        res = batch.nonlinear_solve(api.nl_opts(tol_outer=1e-6, tol=1e-9, precision=api.PF_MIXED))
        assert all(r["status"] == 0 for _, r in res)
        assert (batch.tune()["chosen"], batch.tune()["chosen_z"]) == (t["chosen"], t["chosen_z"])
    finally:
        batch.close()
        for g in grids:
            g.close()


def test_per_problem_status(api):
    """An iteration limit ends every problem with PF_E_NOCONV; the batch reports each one."""
    probs = _problems()[:2]
    grids = [api.Grid.for_problem(p) for p in probs]
    batch = api.Batch(grids, tiles_per_block=2)
    try:
        res = batch.nonlinear_solve(api.nl_opts(tol_outer=1e-12, tol=1e-10, max_outer=2), allow=(3,))
        assert [r["status"] for _, r in res] == [3, 3]
        assert all(r["outer_iters"] == 2 for _, r in res)
    finally:
        batch.close()
        for g in grids:
            g.close()


def test_batch_predicted_starts(api, orc):
    """Extrapolated starting vectors in a batch (pf_nl_opts.predict = 2, the default, as the single-grid solver):
    with the previous iterates instead (predict = 0) the batch reaches the oracle's fixed point too, and at the
    paper's tolerances the extrapolated starts take fewer BiCGSTAB iterations for the same outer iterations."""
    probs = _problems()[:2]
    r0, _ = _batch_solve(api, probs, api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=api.PF_MIXED, predict=0),
                         tpb=2)
    for p, (out, rep) in zip(probs, r0):
        ref = orc.pf_solve_problem(p, tol_outer=1e-11, lin_tol=1e-12)
        assert rep["status"] == 0
        assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < TOL_MIXED
    loose = dict(tol_outer=1e-3, tol=1e-6, precision=api.PF_MIXED)
    a0, _ = _batch_solve(api, probs, api.nl_opts(predict=0, **loose), tpb=2)
    for k in (1, 2):
        a1, _ = _batch_solve(api, probs, api.nl_opts(predict=k, **loose), tpb=2)
        for (o0, p0), (o1, p1) in zip(a0, a1):
            assert p0["status"] == 0 and p1["status"] == 0
            assert abs(p0["outer_iters"] - p1["outer_iters"]) <= 1
            assert _rel(o1["phi_V"], o0["phi_V"], floor=0.0257) < 1e-4
        assert sum(p["lin_iters_total"] for _, p in a1) < sum(p["lin_iters_total"] for _, p in a0), k
