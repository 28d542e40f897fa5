"""Error paths through the C ABI on the GPU: every failure is a status code,
made on the host or by the solver's own checks; nothing faults the device."""
import numpy as np
import pytest

import sem_inputs as si
from gpu_common import H, T, ctx_for, dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_inverted_element_is_rejected():
    dev()
    from paper_2104_05829_gb300 import SemError, _lib
    mesh = si.box_mesh(2, 3, perm_seed=0)
    x = mesh["x"].copy()
    x[0] = x[0][:, :, ::-1]
    with pytest.raises(SemError) as ei:
        ctx_for(dict(mesh, x=x))
    assert ei.value.code == _lib.SEM_EMESH


def test_not_converged_reports_and_keeps_iterate():
    dev()
    from paper_2104_05829_gb300 import _lib
    mesh = si.box_mesh(3, 5, warp=0.1)
    ctx = ctx_for(mesh)
    _, f = si.manufactured(mesh)
    x, info = ctx.solve(T(f), tol=1e-14, maxit=3, raise_on_error=False)
    assert info["status"] == _lib.SEM_ENOTCONV
    assert info["iters"] == 3 and np.isfinite(info["relres"]) and info["relres"] > 1e-14
    assert np.all(np.isfinite(H(x)))


def test_nan_input_is_a_breakdown():
    dev()
    from paper_2104_05829_gb300 import _lib
    mesh = si.box_mesh(2, 3)
    ctx = ctx_for(mesh)
    f = np.ones(mesh["x"].size)
    f[5] = np.nan
    _, info = ctx.solve(T(f), tol=1e-8, maxit=10, raise_on_error=False)
    assert info["status"] in (_lib.SEM_EBREAKDOWN, _lib.SEM_ENOTCONV)
    assert info["status"] == _lib.SEM_EBREAKDOWN


def test_bad_arguments():
    dev()
    from paper_2104_05829_gb300 import SemError
    mesh = si.box_mesh(2, 2)
    ctx = ctx_for(mesh, prec_copies=0)
    u = T(np.zeros(mesh["x"].size))
    with pytest.raises(SemError):
        ctx.level_ax(5, u)                       # no such level
    with pytest.raises(SemError):
        ctx.level_ax(0, u.float(), prec="fp32")  # FP32 copy not built
    with pytest.raises(SemError):
        ctx.vcycle(u)                            # preconditioner not set up
    with pytest.raises(SemError):
        ctx.solve(u, h1_L=u, precond="pmg")      # pMG needs scalar coefficients
