"""Shared helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def ctx_for(mesh, **opts):
    from paper_2104_05829_gb300 import SemContext
    return SemContext.from_mesh(mesh, **opts)


def T(a, dtype=None):
    """Host array -> flat CUDA tensor."""
    t = torch.tensor(np.ascontiguousarray(a).ravel(), device=dev())
    return t if dtype is None else t.to(dtype)


def H(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    """max|a-b| / max|b|: the norm-wise relative error used throughout the parity tests."""
    b = np.asarray(b)
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


def global_from_L(level, vL):
    """Unique-node vector from a continuous L-vector (average of the copies)."""
    return O.q_scatter(np.ravel(vL) / level.maps["mult"], level.node, level.n_G)


def bf16_rne(v):
    """Round float64 values to bfloat16 (round-to-nearest-even) and return the 16-bit codes."""
    v = np.asarray(v, dtype=np.float64)
    m, ex = np.frexp(v)                           # v = m 2^ex, 0.5 <= |m| < 1
    ulp = np.ldexp(1.0, ex - 8)                   # 8 significant bits
    q = np.rint(v / ulp) * ulp                    # rint rounds half to even
    f = q.astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16), q
