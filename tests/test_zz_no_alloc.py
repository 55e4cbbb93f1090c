"""The allocation-free denoising step (d4orm_denoise_step_noalloc).

It serves callers that cannot call cudaMalloc (a real-time control loop, or
a host that owns all device memory through its own pool): the step's
scratch sits in a fixed array of the library's device image.  This checks,
through the C ABI, that two calls in a row give what the allocating entry
point d4orm_denoise_step gives on the same inputs, and that sizes beyond the
stated maximum are refused before anything is launched.  Both entry points
launch the same kernels with the same split of the weighted sum, so their
outputs are compared bit for bit.

The file is named to be collected last, so a failure here does not stop a
-x run before the other tests; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

import scenarios
from helpers import gpu_params, small_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return torch


@pytest.fixture(scope="module")
def g(torch):
    from helpers import build_library
    build_library()
    import paper_2503_12204_gb300 as g
    return g


def _inputs(torch, inst, seed):
    rng = np.random.default_rng(seed)
    ub = torch.as_tensor(scenarios.random_controls(rng, inst, 0.5), dtype=torch.float32, device="cuda")
    du = torch.as_tensor(scenarios.random_deformation(rng, inst, 0.3), dtype=torch.float32, device="cuda")
    return ub, du


@pytest.mark.parametrize("dyn,n,T,N", [(1, 16, 40, 3000), (2, 5, 23, 700)])
def test_noalloc_matches_allocating_step_twice(torch, g, dyn, n, T, N):
    inst = small_instance(dyn, n, T, N, seed=21, K=30)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    for call, (it, i, seed) in enumerate([(0, 30, 1), (2, 7, 2)]):   # two calls in a row
        ub, du = _inputs(torch, inst, seed)
        ref_out, ref_fit = torch.zeros_like(du), torch.zeros(N, device="cuda")
        g.d4orm_denoise_step(prob.handle, p, it, i, ub, du, ref_out, ref_fit)
        out, fit = torch.full_like(du, float("nan")), torch.full((N,), float("nan"), device="cuda")
        g.d4orm_denoise_step_noalloc(prob.handle, p, it, i, ub, du, out, fit)
        torch.cuda.synchronize()
        # the same kernels with the same launch shapes and reduction split:
        # identical bits, not merely within the oracle tolerance
        assert torch.equal(fit, ref_fit), call
        assert torch.equal(out, ref_out), call


def test_noalloc_without_fitness_output(torch, g):
    inst = small_instance(0, 4, 30, 512, seed=3, K=20)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    ub, du = _inputs(torch, inst, 5)
    ref = torch.zeros_like(du)
    g.d4orm_denoise_step(prob.handle, p, 1, 20, ub, du, ref)
    for _ in range(2):
        out = torch.zeros_like(du)
        g.d4orm_denoise_step_noalloc(prob.handle, p, 1, 20, ub, du, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_oversize(torch, g):
    inst = small_instance(0, 2, 8, 16)
    prob = g.Problem(inst)
    p = gpu_params(g, inst, N=g.NOALLOC_MAX_SAMPLES + 1)
    a = torch.zeros((8, 2, 2), device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_denoise_step_noalloc(prob.handle, p, 0, 1, a, a, b)
    assert ei.value.status == 2
