"""The allocation-free guard (gf_true_residual_noalloc) against the grid-based one.

gf_true_residual_noalloc serves callers that cannot allocate device memory (work
recorded into a CUDA graph or under stream capture, fixed memory budgets): its
scratch is a static array inside the library. It must return the same acceptance
residual as gf_true_residual. This file is collected last on purpose and works both
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth
from oracle import gf_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the tolerance the FP64 guard parity tests use (relative)
RTOL = 1e-10


@pytest.fixture(scope="module")
def gf():
    from paper_2607_26382_b300 import build
    build.build()
    import paper_2607_26382_b300 as gf
    return gf


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("dims", [(24, 12, 8), (96, 48, 48)])
def test_noalloc_guard_matches_grid_guard_twice(gf, dims):
    nx, ny, nz = dims
    rho = _dev(synth.smoothed_gaussian_density(nx, ny, nz, 3))
    m_ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    f = torch.zeros(m_ndof, dtype=torch.float64, device="cuda")
    g = gf.create_grid(nx, ny, nz, levels=2 if nx == 24 else 5)
    g.cantilever_load(f)
    g.set_density(rho, 3.0)
    g.set_floor(1e-4)
    eta = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    # two calls in a row on different inputs: the shared scratch keeps the first
    # call's contents, which must not leak into the second
    for seed, scale in ((1, 1e-2), (2, 3.0)):
        u = _dev(synth.random_vector(m_ndof, seed) * scale)
        ref = g.true_residual(f, u)
        gf.true_residual_noalloc(nx, ny, nz, rho, 3.0, 1e-4, f, u, eta)
        torch.cuda.synchronize()
        got = float(eta.item())
        assert abs(got - ref) <= RTOL * ref, (got, ref)
    g.close()


def test_noalloc_guard_rejects_oversize_grid(gf):
    nx, ny, nz = 128, 64, 64            # 1,622,400 DOFs > 1,048,576
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rho = torch.zeros(nx * ny * nz, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GFError) as e:
        gf.true_residual_noalloc(nx, ny, nz, rho, 3.0, 1e-3, x, x, eta)
    assert e.value.code == -1 and "1048576" in str(e.value)
