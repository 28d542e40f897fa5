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


def test_device_waits_that_give_up_end_the_solve_with_a_breakdown():
    """Every device-side wait is bounded (sem_opts.spin_limit, SM clock cycles). With a limit of
    zero the pipelined coarse solve's waits on other blocks' exchange words give up at their
    first unanswered poll: the kernel ends, and the flexible-CG solve that launched it returns
    SEM_EBREAKDOWN instead of going on with stale coarse values. A solve that meets no
    unanswered poll is correct. A fresh context with the default limit then solves correctly."""
    dev()
    import oracle as O
    from gpu_common import global_from_L
    from paper_2104_05829_gb300 import _lib
    mesh = si.box_mesh((8, 7, 6), 7, warp=0.1, perm_seed=1, dirichlet=("x0",))
    b = si.gaussian_assembled_rhs(mesh, 0)
    bt = T(b)
    lev = O.level_from_mesh(mesh)
    bg = lev.mask(global_from_L(lev, b))

    def oracle_residual(x):
        xg = global_from_L(lev, H(x))
        return np.linalg.norm(bg - lev.apply(xg)) / np.linalg.norm(bg)

    ctx = ctx_for(mesh, spin_limit=0, coarse_mode="pipe")
    statuses = []
    for _ in range(3):
        x, info = ctx.solve(bt, tol=1e-8, maxit=100, precond="pmg", prec="fp64", rhs="assembled",
                            raise_on_error=False)
        statuses.append(info["status"])
        assert info["status"] in (_lib.SEM_OK, _lib.SEM_EBREAKDOWN), info
        if info["status"] == _lib.SEM_OK:
            assert oracle_residual(x) < 2e-8
        else:
            assert "breakdown" in _lib.load().sem_last_error_detail().decode()
    print("statuses with a zero wait limit:", statuses)
    assert _lib.SEM_EBREAKDOWN in statuses
    ctx.close()
    good = ctx_for(mesh, coarse_mode="pipe")
    x, info = good.solve(bt, tol=1e-8, maxit=100, precond="pmg", prec="fp64", rhs="assembled")
    assert info["relres"] <= 1e-8 and oracle_residual(x) < 2e-8


def test_bulk_copy_wait_that_gives_up_writes_nan_and_leaves_the_context_usable():
    """The FP32 operator stages a block's u and factors by bulk copies on an mbarrier; with a
    wait limit of zero a block whose copies have not landed at its first look writes NaN to its
    elements (after waiting, with the default limit, for the copies to land). Every element's
    output is then either exact or all NaN, and a context with the default limit is exact.
    The 24^3 box's FP32 factors (198 MB) exceed the L2, so most copies come from HBM and
    cannot have landed at the first look."""
    dev()
    import oracle as O
    from gpu_common import relmax
    mesh = si.box_mesh(24, 7, warp=0.1, perm_seed=2)
    lev = O.level_from_mesh(mesh)
    u = si.uniform_field(mesh, 0)
    ref = O.ax_local(u, lev.G, lev.B, lev.D, 1.0, 0.5).reshape(mesh["E"], -1)
    ctx = ctx_for(mesh, spin_limit=0, prec_copies=1)
    w = H(ctx.level_ax(0, T(u, torch.float32), h1=1.0, h2=0.5, prec="fp32", assemble=False)).reshape(mesh["E"], -1)
    bad = np.isnan(w)
    whole = bad.all(axis=1)
    assert np.array_equal(bad.any(axis=1), whole)          # NaN comes in whole elements
    if (~whole).any():
        assert relmax(w[~whole], ref[~whole]) < 2e-6
    print(f"elements whose wait gave up: {int(whole.sum())} of {mesh['E']}")
    assert whole.any()      # a zero limit looks once: copies from HBM have not landed by then
    ctx.close()
    good = ctx_for(mesh, prec_copies=1)
    w = H(good.level_ax(0, T(u, torch.float32), h1=1.0, h2=0.5, prec="fp32", assemble=False))
    assert relmax(w, ref.ravel()) < 2e-6
