"""Python binding of the C ABI (include/pf_gb300.h): argument marshalling only.

The functions keep the C names (pf_create_grid, pf_set_coeffs, pf_linear_solve,
pf_nonlinear_solve, pf_submit, pf_poll, ...) and take numpy arrays (host memory) or CUDA torch
tensors (device memory; the pointer and the current torch stream are passed through).  Every
step of a solve runs in the CUDA library; nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B
from ._binding import (PF_FP64, PF_MIXED, PF_OP_POISSON, PF_OP_PF1, PF_OP_PF2, PF_MEM_HOST, PF_MEM_DEVICE,  # noqa
                       PF_BICGSTAB, PF_CG_SYMMETRIC, PF_CG_ALL, PF_NORM_REL2, PF_NORM_ABSINF, PF_OK, PF_PENDING,
                       STATUS_NAMES, PF_CHARGES_SPREAD, PF_CHARGES_DECOMPOSED)


class PFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _check(status, allow=()):
    if status != PF_OK and status not in allow:
        raise PFError(status, B.last_error())
    return status


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, mem) of a numpy array (host) or a torch tensor (device when on CUDA)."""
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr()), (PF_MEM_DEVICE if a.is_cuda else PF_MEM_HOST)
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data), PF_MEM_HOST


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # torch missing: use the default stream
        pass
    return ctypes.c_void_p(0)


def solve_opts(max_iter=20000, tol=1e-10, norm=PF_NORM_REL2, precision=PF_FP64, inner_tol=0.1, max_refine=64,
               method=0):
    o = B.pf_solve_opts()
    B.load().pf_default_solve_opts(ctypes.byref(o))
    o.max_iter, o.tol, o.norm, o.precision, o.inner_tol, o.max_refine = max_iter, tol, norm, precision, inner_tol, \
        max_refine
    o.method = method
    return o


def nl_opts(omega=0.3, tol_outer=1e-9, max_outer=500, accel_depth=0, lin_forcing=0.0, warm_start=0, predict=2,
            **lin):
    o = B.pf_nl_opts()
    B.load().pf_default_nl_opts(ctypes.byref(o))
    o.omega, o.tol_outer, o.max_outer = omega, tol_outer, max_outer
    o.accel_depth, o.lin_forcing, o.warm_start, o.predict = accel_depth, lin_forcing, warm_start, predict
    o.lin = solve_opts(**lin)
    return o


class _Coeffs:
    """Keeps the host arrays referenced by a pf_coeffs alive."""

    def __init__(self, eps, solvent, charges, phi_lo_V, phi_hi_V, species, eps_s, lc_A, T_K):
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.solvent = np.ascontiguousarray(solvent, dtype=np.uint8)
        self.charges = np.ascontiguousarray(np.asarray(charges, dtype=np.float64).reshape(-1, 4))
        self.sp = (B.pf_species * max(1, len(species)))()
        for i, s in enumerate(species):
            self.sp[i].z, self.sp[i].radius_A, self.sp[i].bulk_M = int(s.z), float(s.radius_A), float(s.bulk_M)
        c = B.pf_coeffs()
        c.eps = self.eps.ctypes.data
        c.solvent = self.solvent.ctypes.data
        c.n_charges = self.charges.shape[0]
        c.charges = self.charges.ctypes.data if self.charges.size else None
        c.phi_zlo_V, c.phi_zhi_V = float(phi_lo_V), float(phi_hi_V)
        c.n_species = len(species)
        c.species = self.sp
        c.eps_s, c.lc_A, c.T_K = float(eps_s), float(lc_A), float(T_K)
        self.c = c


def coeffs_of(prob) -> _Coeffs:
    return _Coeffs(prob.eps, prob.solvent, prob.charges, prob.phi_lo_V, prob.phi_hi_V, prob.species, prob.eps_s,
                   prob.lc_A, prob.T_K)


# ---------------------------------------------------------------- C names
def pf_create_grid(nx, ny, nz, h_A, origin_A, cuda_stream=None):
    org = (ctypes.c_double * 3)(*origin_A)
    h = ctypes.c_void_p()
    stream = _torch_stream() if cuda_stream is None else ctypes.c_void_p(cuda_stream)
    _check(B.load().pf_create_grid(nx, ny, nz, h_A, org, stream, ctypes.byref(h)))
    return h


def pf_grid_bytes(nx, ny, nz, accel_depth=0):
    """Device bytes of a grid of this size (the serving budget's figure); needs no device."""
    return int(B.load().pf_grid_bytes(nx, ny, nz, accel_depth))


def pf_set_coeffs(grid, coeffs: _Coeffs):
    _check(B.load().pf_set_coeffs(grid, ctypes.byref(coeffs.c)))


def pf_set_filter(grid, fixed=None, phi_V=None):
    """Filter region: nodes with fixed = 1 hold phi_V (volts); fixed None clears it."""
    if fixed is None:
        _check(B.load().pf_set_filter(grid, None, None, PF_MEM_HOST))
        return
    pf_, mf = _ptr(fixed, np.uint8)
    pv, mv = _ptr(phi_V, np.float64)
    if mf != mv:
        raise TypeError("fixed and phi_V must both be host or both be device arrays")
    _check(B.load().pf_set_filter(grid, pf_, pv, mf))


def pf_set_filter_sites(grid, centers, radii, q_ion, occupied, ion_radii, eps_b, eps_p, map_radius_A=0.0,
                        v_sites_A3=1.0):
    """Filter region from the site model (Eqs. 19-20) on the device: returns the site potentials (volts) and
    the site region's steric potential S."""
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    n = len(c) // 3
    r = np.ascontiguousarray(radii, dtype=np.float64)
    q = np.ascontiguousarray(q_ion, dtype=np.float64)
    o = np.ascontiguousarray(occupied, dtype=np.int32)
    ir = np.ascontiguousarray(ion_radii, dtype=np.float64)
    if not (len(r) == len(q) == len(o) == len(ir) == n):
        raise ValueError("one radius, ion charge, occupancy and ion radius per site")
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    st = B.pf_sites(n, vp(c), vp(r), vp(q), vp(o), vp(ir), float(eps_b), float(eps_p), float(map_radius_A),
                    float(v_sites_A3))
    phi = np.zeros(n)
    S = ctypes.c_double(0.0)
    _check(B.load().pf_set_filter_sites(grid, ctypes.byref(st), phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(S)))
    return phi, S.value


def pf_set_charge_mode(grid, mode):
    """PF_CHARGES_SPREAD (Eq. 3) or PF_CHARGES_DECOMPOSED (Eqs. 5-10, built on the device now); returns the
    report of the phi^L solve."""
    rep = B.pf_report()
    _check(B.load().pf_set_charge_mode(grid, int(mode), ctypes.byref(rep)))
    return {"status": rep.status, "iterations": rep.iterations, "residual": rep.residual, "time_ms": rep.time_ms}


def pf_get_decomposition(grid, G_V, b_if):
    """Copies G (volts) and the interface right-hand side into the given arrays (numpy or CUDA; either None)."""
    arrs = [a for a in (G_V, b_if) if a is not None]
    mems = {_ptr(a, np.float64)[1] for a in arrs}
    if len(mems) > 1:
        raise TypeError("G_V and b_if must both be host or both be device arrays")
    mem = mems.pop() if mems else PF_MEM_HOST
    pg = _ptr(G_V, np.float64)[0] if G_V is not None else None
    pb = _ptr(b_if, np.float64)[0] if b_if is not None else None
    _check(B.load().pf_get_decomposition(grid, pg, pb, mem))


def pf_set_kappa(grid, kappa):
    p, mem = _ptr(kappa, np.float64)
    _check(B.load().pf_set_kappa(grid, p, mem))


def pf_linear_solve(grid, op, b, x, opts=None, allow=(), method="bicgstab"):
    """Solves A x = b in place of x (method "bicgstab": pf_linear_solve, "cg": pf_linear_solve_cg); returns
    the report as a dict.  Statuses in `allow` do not raise."""
    pb, mb = _ptr(b, np.float64)
    px, mx = _ptr(x, np.float64)
    if mb != mx:
        raise TypeError("b and x must both be host or both be device arrays")
    if method not in ("bicgstab", "cg"):
        raise ValueError("method is 'bicgstab' or 'cg'")
    fn = B.load().pf_linear_solve if method == "bicgstab" else B.load().pf_linear_solve_cg
    rep = B.pf_report()
    st = fn(grid, op, pb, px, mb, ctypes.byref(opts) if opts is not None else None, ctypes.byref(rep))
    _check(st, allow)
    return {"status": rep.status, "iterations": rep.iterations, "refinements": rep.refinements,
            "residual": rep.residual, "time_ms": rep.time_ms}


def _result_for(res, n_nodes, n_species, out):
    """Fills a pf_result's output pointers from `out` (fresh numpy arrays when None); returns `out`."""
    if out is None:
        out = {"phi_V": np.zeros(n_nodes), "C_M": np.zeros(n_species * n_nodes), "S": np.zeros(n_nodes),
               "Gamma": np.zeros(n_nodes), "Psi": np.zeros(n_nodes)}
    mems = set()
    for k in ("phi_V", "C_M", "S", "Gamma", "Psi"):
        if out.get(k) is not None:
            p, m = _ptr(out[k], np.float64)
            setattr(res, k, p.value)
            mems.add(m)
    if len(mems) > 1:
        raise TypeError("outputs must all be host or all be device arrays")
    res.mem = mems.pop() if mems else PF_MEM_HOST
    return out


def _report(res):
    return {"status": res.status, "outer_iters": res.outer_iters, "lin_iters_total": res.lin_iters_total,
            "lin_iters_first": res.lin_iters_first, "delta": res.delta, "time_ms": res.time_ms}


def pf_nonlinear_solve(grid, n_nodes, n_species, opts=None, out=None, allow=()):
    """Runs the PF iteration; `out` maps phi_V/C_M/S/Gamma/Psi to preallocated arrays (numpy or CUDA
    tensors, all of one kind); by default fresh numpy arrays are returned."""
    res = B.pf_result()
    out = _result_for(res, n_nodes, n_species, out)
    st = B.load().pf_nonlinear_solve(grid, ctypes.byref(opts) if opts is not None else None, ctypes.byref(res))
    _check(st, allow)
    return out, _report(res)


def pf_batch_create(grid_handles, cuda_stream=None):
    arr = (ctypes.c_void_p * len(grid_handles))(*[g.value for g in grid_handles])
    h = ctypes.c_void_p()
    stream = _torch_stream() if cuda_stream is None else ctypes.c_void_p(cuda_stream)
    _check(B.load().pf_batch_create(arr, len(grid_handles), stream, ctypes.byref(h)))
    return h


def pf_batch_set_tiles_per_block(batch, tiles_per_block):
    _check(B.load().pf_batch_set_tiles_per_block(batch, int(tiles_per_block)))


def pf_batch_set_tiling(batch, tiles_per_block, z_planes):
    _check(B.load().pf_batch_set_tiling(batch, int(tiles_per_block), int(z_planes)))


def _tune_dict(t):
    return {"tiles_per_block": [t.tiles_per_block[i] for i in range(t.n)],
            "z_planes": [t.z_planes[i] for i in range(t.n)], "ms": [t.ms[i] for i in range(t.n)],
            "chosen": t.chosen, "chosen_z": t.chosen_z}


def pf_batch_autotune(batch):
    t = B.pf_batch_tune()
    _check(B.load().pf_batch_autotune(batch, ctypes.byref(t)))
    return _tune_dict(t)


def pf_batch_get_tune(batch):
    t = B.pf_batch_tune()
    _check(B.load().pf_batch_get_tune(batch, ctypes.byref(t)))
    return _tune_dict(t)


def pf_batch_nonlinear_solve(batch, sizes, opts=None, outs=None, allow=()):
    """sizes: [(n_nodes, n_species)] per grid; outs: per-grid output dicts as for pf_nonlinear_solve (or None).
    Returns [(out, report)] in batch order."""
    res = (B.pf_result * len(sizes))()
    outs = outs if outs is not None else [None] * len(sizes)
    outs = [_result_for(res[i], n, ns, outs[i]) for i, (n, ns) in enumerate(sizes)]
    st = B.load().pf_batch_nonlinear_solve(batch, ctypes.byref(opts) if opts is not None else None, res)
    _check(st, allow)
    return [(outs[i], _report(res[i])) for i in range(len(sizes))]


def pf_batch_destroy(batch):
    if batch is not None and batch.value:
        _check(B.load().pf_batch_destroy(batch))


def pf_destroy_grid(grid):
    if grid is not None and grid.value:
        _check(B.load().pf_destroy_grid(grid))


def pf_profile_enable(grid, on=True):
    _check(B.load().pf_profile_enable(grid, 1 if on else 0))


def pf_profile_get(grid):
    """{'launches': n, '<kind>': (count, ms), ...} for the grid's kernel launches."""
    p = B.pf_profile()
    _check(B.load().pf_profile_get(grid, ctypes.byref(p)))
    out = {"launches": p.launches}
    for k, name in enumerate(B.PROF_NAMES):
        out[name] = (p.count[k], p.ms[k])
    return out


def pf_fermi_noalloc(phi_V, solvent, species, C_M, S=None, Gamma=None, T_K=298.15, warm_start=False,
                     cuda_stream=None, allow=()):
    """The pointwise Fermi/steric step on caller-owned CUDA tensors without any device allocation (see
    include/pf_gb300.h): phi_V (float64, volts), solvent (uint8) -> C_M (float64, species-major), S, Gamma;
    warm_start starts each node's root search from the previous call's ln Gamma there."""
    n = phi_V.numel()
    sp = (B.pf_species * len(species))()
    for i, s_ in enumerate(species):
        sp[i].z, sp[i].radius_A, sp[i].bulk_M = int(s_.z), float(s_.radius_A), float(s_.bulk_M)
    ptr = lambda a: ctypes.c_void_p(a.data_ptr()) if a is not None else None  # noqa: E731
    stream = _torch_stream() if cuda_stream is None else ctypes.c_void_p(cuda_stream)
    st = B.load().pf_fermi_noalloc(n, ptr(phi_V), ptr(solvent), len(species), sp, float(T_K), int(bool(warm_start)),
                                   ptr(C_M), ptr(S), ptr(Gamma), stream)
    return _check(st, allow)


def pf_last_error():
    return B.last_error()


def pf_server_create(hbm_budget_bytes, max_slots):
    h = ctypes.c_void_p()
    _check(B.load().pf_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
    return h


def pf_set_potential(grid, phi_V):
    """Sets the grid's potential (volts; numpy host array or CUDA tensor) as the start of a warm-started solve."""
    p, m = _ptr(phi_V, np.float64)
    _check(B.load().pf_set_potential(grid, p, m))


def make_request(prob, opts=None, phi0_V=None):
    """A pf_request for a problem of the workloads module (keeps its arrays alive on the object); phi0_V: an
    optional starting potential (host array, volts)."""
    q = B.pf_request()
    g = prob.grid
    q.nx, q.ny, q.nz, q.h_A = g.nx, g.ny, g.nz, g.h
    for a in range(3):
        q.origin_A[a] = g.origin[a]
    co = coeffs_of(prob)
    q.coeffs = co.c
    q.opts = opts if opts is not None else nl_opts()
    q._keep = co
    if phi0_V is not None:
        q._phi0 = np.ascontiguousarray(phi0_V, dtype=np.float64)
        q.phi0_V = q._phi0.ctypes.data
    return q


def pf_submit(server, request):
    t = ctypes.c_uint64()
    _check(B.load().pf_submit(server, ctypes.byref(request), ctypes.byref(t)))
    return t.value


def pf_done(server, ticket):
    """True when the ticket has finished (its result stays for pf_poll)."""
    done = ctypes.c_int(0)
    _check(B.load().pf_poll(server, ticket, None, ctypes.byref(done)), allow=(PF_PENDING,))
    return bool(done.value)


def pf_poll(server, ticket, n_nodes, n_species, allow=(), out=None):
    """(done, outputs-or-None, report-or-None) for a ticket; outputs are numpy arrays (those of `out`, a dict
    with phi_V, C_M, S and Gamma, when given)."""
    if out is None:
        out = {"phi_V": np.zeros(n_nodes), "C_M": np.zeros(n_species * n_nodes), "S": np.zeros(n_nodes),
               "Gamma": np.zeros(n_nodes)}
    res = B.pf_result()
    for k in out:
        setattr(res, k, out[k].ctypes.data)
    res.mem = PF_MEM_HOST
    done = ctypes.c_int(0)
    st = B.load().pf_poll(server, ticket, ctypes.byref(res), ctypes.byref(done))
    if not done.value:
        _check(st, allow=(PF_PENDING,))
        return False, None, None
    _check(st, allow)
    return True, out, {"status": res.status, "outer_iters": res.outer_iters, "lin_iters_total": res.lin_iters_total,
                       "delta": res.delta, "time_ms": res.time_ms}


def pf_server_destroy(server):
    if server is not None and server.value:
        _check(B.load().pf_server_destroy(server))


# ---------------------------------------------------------------- convenience wrappers
class Batch:
    """Owns one pf_batch over a list of Grid objects (which it keeps alive)."""

    def __init__(self, grids, cuda_stream=None, tiles_per_block=0):
        self.grids = list(grids)
        self.handle = pf_batch_create([g.handle for g in self.grids], cuda_stream)
        if tiles_per_block:
            pf_batch_set_tiles_per_block(self.handle, tiles_per_block)

    def autotune(self):
        return pf_batch_autotune(self.handle)

    def tune(self):
        return pf_batch_get_tune(self.handle)

    def set_tiles_per_block(self, tiles_per_block):
        pf_batch_set_tiles_per_block(self.handle, tiles_per_block)

    def set_tiling(self, tiles_per_block, z_planes):
        pf_batch_set_tiling(self.handle, tiles_per_block, z_planes)

    def nonlinear_solve(self, opts=None, outs=None, allow=()):
        return pf_batch_nonlinear_solve(self.handle, [(g.n, g.n_species) for g in self.grids], opts, outs, allow)

    def stats(self):
        st = B.pf_batch_stats()
        _check(B.load().pf_batch_get_stats(self.handle, ctypes.byref(st)))
        return {"ticks": st.ticks, "wall_ms": st.wall_ms, "device_ms": st.device_ms}

    def close(self):
        pf_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None:
                self.close()
        except Exception:
            pass


class Grid:
    """Owns one pf_grid handle."""

    def __init__(self, nx, ny, nz, h_A, origin_A, cuda_stream=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self.n_species = 0
        self.handle = pf_create_grid(nx, ny, nz, h_A, origin_A, cuda_stream)

    @classmethod
    def for_problem(cls, prob, cuda_stream=None):
        g = prob.grid
        grid = cls(g.nx, g.ny, g.nz, g.h, g.origin, cuda_stream)
        grid.set_problem(prob)
        return grid

    def set_problem(self, prob):
        self._coeffs = coeffs_of(prob)
        self.n_species = len(prob.species)
        pf_set_coeffs(self.handle, self._coeffs)

    def set_coeffs(self, eps, solvent, charges, phi_lo_V, phi_hi_V, species, eps_s, lc_A, T_K=298.15):
        self._coeffs = _Coeffs(eps, solvent, charges, phi_lo_V, phi_hi_V, species, eps_s, lc_A, T_K)
        self.n_species = len(species)
        pf_set_coeffs(self.handle, self._coeffs)

    def set_kappa(self, kappa):
        pf_set_kappa(self.handle, kappa)

    def set_filter(self, fixed=None, phi_V=None):
        pf_set_filter(self.handle, fixed, phi_V)

    def set_filter_sites(self, *args, **kw):
        return pf_set_filter_sites(self.handle, *args, **kw)

    def set_charge_mode(self, mode):
        return pf_set_charge_mode(self.handle, mode)

    def get_decomposition(self, G_V=None, b_if=None):
        pf_get_decomposition(self.handle, G_V, b_if)

    def linear_solve(self, op, b, x, opts=None, allow=(), method="bicgstab"):
        return pf_linear_solve(self.handle, op, b, x, opts, allow, method)

    def nonlinear_solve(self, opts=None, out=None, allow=()):
        return pf_nonlinear_solve(self.handle, self.n, self.n_species, opts, out, allow)

    def set_potential(self, phi_V):
        pf_set_potential(self.handle, phi_V)

    def profile(self, on=True):
        pf_profile_enable(self.handle, on)

    def profile_get(self):
        return pf_profile_get(self.handle)

    def close(self):
        pf_destroy_grid(self.handle)
        self.handle = None

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None:
                self.close()
        except Exception:
            pass
