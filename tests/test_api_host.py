"""The Python binding's host-side marshalling (no device): option structs from the library's defaults, argument
type checks before any call reaches the library, and the error type."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def api():
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api as A
    return A


def test_option_structs(api):
    o = api.solve_opts(max_iter=123, tol=1e-7, norm=api.PF_NORM_ABSINF, precision=api.PF_MIXED, inner_tol=0.2)
    assert (o.max_iter, o.tol, o.norm, o.precision, o.inner_tol) == (123, 1e-7, api.PF_NORM_ABSINF, api.PF_MIXED, 0.2)
    n = api.nl_opts(omega=0.4, tol_outer=1e-5, max_outer=77, accel_depth=3, lin_forcing=0.5, tol=1e-8)
    assert (n.omega, n.tol_outer, n.max_outer, n.accel_depth, n.lin_forcing, n.lin.tol) == (0.4, 1e-5, 77, 3, 0.5, 1e-8)
    assert n.warm_start == 0
    # the library's defaults: the paper's relaxation and tolerances, extrapolated starting vectors, BiCGSTAB
    d = api.nl_opts()
    assert (d.omega, d.tol_outer, d.accel_depth, d.lin_forcing, d.predict) == (0.3, 1e-9, 0, 0.0, 2)
    assert (d.lin.method, d.lin.precision, d.lin.inner_tol) == (api.PF_BICGSTAB, api.PF_FP64, 0.1)
    assert api.nl_opts(predict=0).predict == 0


def test_arrays_are_checked_before_the_library_is_called(api):
    with pytest.raises(TypeError):
        api.pf_linear_solve(None, api.PF_OP_POISSON, np.zeros(8, np.float32), np.zeros(8))
    with pytest.raises(TypeError):
        api.pf_linear_solve(None, api.PF_OP_POISSON, np.zeros((4, 2))[:, 0], np.zeros(4))  # not contiguous
    with pytest.raises(ValueError):
        api.pf_linear_solve(None, api.PF_OP_POISSON, np.zeros(4), np.zeros(4), method="gmres")
    with pytest.raises(TypeError):
        api.pf_set_filter(None, np.zeros(4, np.int32), np.zeros(4))


def test_library_errors_raise_with_the_status_and_message(api):
    with pytest.raises(api.PFError) as e:
        api.pf_linear_solve(None, api.PF_OP_POISSON, np.zeros(4), np.zeros(4))
    assert e.value.status == 1 and "required" in str(e.value)
    assert api.pf_grid_bytes(33, 33, 33) > 0
