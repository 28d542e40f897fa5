"""sem_dot_static: the dot product for callers that cannot allocate device memory.

It keeps its scratch in a static device array instead of memory from
cudaMalloc. Checked through the C ABI against sem_dot (the context-based
entry point) on two calls in a row, within the 1e-12 relative tolerance the
FP64 tests use (relative to sum |a_l b_l|, since the two reductions add in
different orders). This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import sem_inputs as si
from gpu_common import T, ctx_for, dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _owner_mask(maps, n):
    return ((maps["label"] == np.arange(n)) & (maps["dmask"] == 0)).astype(np.uint8)


def test_dot_static_matches_sem_dot_on_two_calls():
    dev()
    from paper_2104_05829_gb300 import _lib
    lib = _lib.load()
    mesh = si.box_mesh((6, 5, 4), 7, warp=0.1, perm_seed=2, dirichlet=("x0", "z1"))
    ctx = ctx_for(mesh, prec_copies=0)
    n = mesh["x"].size
    own = T(_owner_mask(ctx.maps(0), n), torch.uint8)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    for seed in (0, 1):                                  # two calls in a row
        a = si.uniform_field(mesh, seed).ravel()
        b = si.uniform_field(mesh, seed + 10).ravel()
        at, bt = T(a), T(b)
        ref = ctx.dot(at, bt)
        rc = lib.sem_dot_static(at.data_ptr(), bt.data_ptr(), own.data_ptr(), n, out.data_ptr(), stream)
        assert rc == _lib.SEM_OK, lib.sem_last_error_detail().decode()
        torch.cuda.synchronize()
        m = _owner_mask(ctx.maps(0), n) == 1
        scale = float(np.sum(np.abs(a * b)[m]))
        assert abs(out.item() - ref) <= 1e-12 * scale, (seed, out.item(), ref)
        host = float(np.sum((a * b)[m]))                 # the same sum on the host
        assert abs(out.item() - host) <= 1e-12 * scale, (seed, out.item(), host)


# one tile (8192 elements per block) plus one element, three tiles exactly, and a length
# whose last block holds a single element after many full ones
@pytest.mark.parametrize("n", [8193, 3 * 8192, 37 * 8192 + 1])
def test_dot_static_without_mask_matches_the_host_sum(n):
    dev()
    from paper_2104_05829_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(n)
    a, b = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    at, bt = T(a), T(b)
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                                   # two calls in a row
        out.fill_(np.nan)
        rc = lib.sem_dot_static(at.data_ptr(), bt.data_ptr(), None, n, out.data_ptr(), stream)
        assert rc == _lib.SEM_OK, lib.sem_last_error_detail().decode()
        torch.cuda.synchronize()
        scale = float(np.sum(np.abs(a * b)))
        assert abs(out.item() - float(np.sum(a * b))) <= 1e-12 * scale
        assert abs(out.item() - torch.dot(at, bt).item()) <= 1e-12 * scale


def test_dot_static_empty_input_writes_zero():
    dev()
    from paper_2104_05829_gb300 import _lib
    lib = _lib.load()
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    rc = lib.sem_dot_static(x.data_ptr(), x.data_ptr(), None, 0, out.data_ptr(), None)
    assert rc == _lib.SEM_OK
    torch.cuda.synchronize()
    assert out.item() == 0.0


def test_dot_static_rejects_oversized_input_without_launching():
    dev()
    from paper_2104_05829_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.sem_dot_static(x.data_ptr(), x.data_ptr(), None, 67_108_865, out.data_ptr(), None)
    assert rc == _lib.SEM_EINVAL
    assert "capacity" in lib.sem_last_error_detail().decode()
