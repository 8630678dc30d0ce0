"""The bench's reference arm on CPU: one JSON line with the contract's keys, the oracle as the timed program,
no host-device traffic, and the workload's L2 statement following the grid size."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "33",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "PF solves/s" and d["unit"] == "solves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "pf_33_four_pores_NaCaCl"
    assert "fits in L2" in d["config"]["l2"]
    # the config names the workload only; the arm's arithmetic is stated beside it
    assert "precision" not in d["config"] and d["precision"].startswith("fp64")
    assert d["cpu_baseline"]["cpu"]["nproc"] >= 1 and d["cpu_baseline"]["cpu"]["model"]


def test_l2_statement_at_the_bench_size():
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), dict(n=257, precision="mixed", tol_outer=1e-3, lin_tol=1e-6, accel_depth=0, inner_tol=0.1,
                              gpus=1))
    assert bench.config_of(args)["l2"].startswith("inputs larger than L2")


def test_accuracy_check_on_an_oracle_solution(orc):
    """The bench's after-the-fact accuracy check, fed the oracle's own converged solution of a small channel:
    the pointwise step agrees to rounding and both residuals are at the solve's tolerance."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1711_04060_gb300 import workloads as W
    prob = W.config2(n=17)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-13)
    assert ref["status"] == 0
    out = {"phi_V": ref["phi_V"], "C_M": ref["C_M"].ravel(), "S": ref["S"], "Gamma": ref["Gamma"], "Psi": ref["Psi"]}
    acc = bench.oracle_accuracy(prob, out, n_sample=500)
    assert max(acc["eq1_conc_rel"]) < 1e-13 and acc["eq1_S_abs"] < 1e-13 and acc["eq1_Gamma_rel"] < 1e-13
    assert acc["pf2_residual_rel2"] < 1e-9 and acc["pf1_residual_rel_inf_sampled"] < 1e-9
    # a perturbed potential shows up in both
    out2 = dict(out, phi_V=out["phi_V"] * (1 + 1e-4))
    acc2 = bench.oracle_accuracy(prob, out2, n_sample=500)
    assert max(acc2["eq1_conc_rel"]) > 1e-7 and acc2["pf2_residual_rel2"] > 1e-6


def test_all_cores_oracle_copy_agrees(orc):
    """The benchmark's OpenMP copy of the oracle runs the same arithmetic: the pointwise node loop bitwise,
    BiCGSTAB to rounding (its reductions run in another order)."""
    from paper_1711_04060_gb300 import workloads as W
    L = orc.load(orc.build_all_cores())
    z, r, b = [1, 2, -1, 0], [0.95, 0.99, 1.81, 1.4], [0.1, 0.001, 0.102, 55.5]
    sp = orc.species_setup(z, r, b)
    ph = W.uniform(W.substream(3, 1), 2000, -12.0, 12.0)
    one = orc.fermi_nodes(sp, z, ph)
    with orc.using(L):
        many = orc.fermi_nodes(sp, z, ph)
    assert one["status"] == 0 and many["status"] == 0
    assert np.array_equal(one["C"], many["C"]) and np.array_equal(one["Gamma"], many["Gamma"])
    for k in (0, 777, 1999):
        pt = orc.fermi_point(sp, z, float(ph[k]))
        assert np.array_equal(pt["C"], one["C"][:, k]) and pt["Gamma"] == one["Gamma"][k]
    p = W.linear_problem(n=17, seed=2, n_spheres=3)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    x1 = orc.bicgstab(g.nx, g.ny, g.nz, A, p.b, tol=1e-12, max_it=2000)["x"]
    with orc.using(L):
        xa = orc.bicgstab(g.nx, g.ny, g.nz, A, p.b, tol=1e-12, max_it=2000)["x"]
    assert np.abs(xa - x1).max() <= 1e-9 * np.abs(x1).max()


def test_ablation_host_step_against_the_oracle(orc):
    """The ablation's host-side pointwise step (numpy, bench.py) and charge spreading agree with the oracle's."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1711_04060_gb300 import workloads as W
    prob = W.config2(n=17)
    sp = bench.host_species(prob)
    assert sp["lam"] == orc.lam(prob.T_K) and abs(sp["Tv"] - orc.thermal_voltage(prob.T_K)) < 1e-18
    phi = W.uniform(W.substream(21, 1), 3000, -15.0, 15.0)
    u = np.full(len(phi), np.log(sp["gB"]))
    rho, kap = bench.host_fermi_chunk(sp, phi, u)
    z = [s.z for s in prob.species]
    osp = orc.species_setup(z, [s.radius_A for s in prob.species], [s.bulk_M for s in prob.species])
    r = orc.fermi_nodes(osp, z, phi)
    orho = (np.asarray(z, float)[:, None] * r["C"]).sum(0)
    okap = orc.lam(prob.T_K) * (np.asarray(z, float)[:, None] ** 2 * r["C"]).sum(0)
    assert np.abs(rho - orho).max() <= 1e-12 * np.abs(orho).max()
    assert np.abs(kap - okap).max() <= 1e-12 * np.abs(okap).max()
    assert np.abs(u - np.log(r["Gamma"])).max() <= 1e-12
    g = prob.grid
    _, ffix = orc.spread_charges(g.nx, g.ny, g.nz, g.h, g.origin, prob.charges, orc.lam(prob.T_K))
    assert np.abs(bench.host_spread(prob, orc.lam(prob.T_K)) - ffix).max() <= 1e-12 * np.abs(ffix).max()


def test_kernel_tables_cover_every_timed_kind():
    """Every kernel kind with algorithmic bytes has a kernel name and a profiler slot, and the per-kind table turns a
    profile into launches, average time and algorithmic GB/s."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1711_04060_gb300 import _binding as B
    assert set(bench.KERNEL_BYTES) <= set(bench.KERNEL_NAMES)
    assert set(bench.KERNEL_BYTES) <= set(B.PROF_NAMES)
    assert len(B.PROF_NAMES) == B.PF_PROF_KINDS
    # phase C+A in FP32 reads one gh array for its faces (12 words); the one-pass CG on PF1 moves 11 words
    assert bench.KERNEL_BYTES["ca_fp32"] == 48 and bench.KERNEL_BYTES["cg_fp32_pf1"] == 44
    prof = {"launches": 3, "ca_fp32": (2, 0.3), "cg_fp32_pf1": (1, 0.1), "fermi": (0, 0.0)}
    t = bench.kernel_table(prof, 10 ** 6)
    assert set(t) == {"ca_fp32", "cg_fp32_pf1"}
    assert t["ca_fp32"]["avg_us"] == 150.0 and t["ca_fp32"]["GB/s"] == round(48e6 / 150e-6 / 1e9, 1)
    assert t["cg_fp32_pf1"]["launches"] == 1


def test_oracle_baseline_charged_its_own_iterations():
    """The CPU baseline extrapolates the oracle's per-iteration cost to the oracle's own solve: on the default 257^3
    workload the counts of its previous-iterate starts, never the fewer iterations of the GPU arm's predicted
    starts; on other workloads the arm's FP64 counts, with the arm's starting vectors named."""
    sys.path.insert(0, ROOT)
    import bench
    fp64 = {"outer_iters": 188, "lin_iters_total": 6152}
    head = {"outer_iters": 188, "lin_iters_total": 6810}
    A = lambda **kw: type("A", (), dict(dict(n=257, tol_outer=1e-3, lin_tol=1e-6, predict=2), **kw))
    o, l, what = bench.oracle_work(A(), fp64, head)
    assert (o, l) == (bench.REF_WORK["outer"], bench.REF_WORK["lin_iters"]) and "previous iterates" in what
    o, l, what = bench.oracle_work(A(n=129), fp64, head)
    assert (o, l) == (188, 6152) and "predict = 2" in what
    o, l, what = bench.oracle_work(A(lin_tol=1e-8), None, head)
    assert (o, l) == (188, 6810)


def test_kernel_traffic_follows_the_source_hash(monkeypatch):
    """roofline.traffic comes from the committed ncu figures only while the stencil sources hash as they did when
    the figures were captured; any other source gives null."""
    sys.path.insert(0, ROOT)
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kind in ("ca_fp32", "b_fp32"):
        e = d[kind]
        assert e["dram_bytes_per_node"] >= e["algorithmic_bytes_per_node"]
        if e["kernel_source_sha256_16"] == bench.kernel_source_hash():
            assert bench.kernel_traffic(kind) == e["dram_bytes_per_node"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.kernel_traffic("ca_fp32") is None and bench.kernel_traffic("b_fp32") is None
    assert bench.kernel_traffic("no_such_kind") is None
