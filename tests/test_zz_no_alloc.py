"""rcf_apply_noalloc, the entry point for callers that cannot let the library allocate
device memory (their GPU memory is held by their own pooling allocator, or their
service loop forbids allocation after start-up).  It must give what rcf_apply gives,
within the tolerances used elsewhere (FP64 1e-12, FP32 2e-6 relative), on repeated
calls that share its one fixed scratch array.  This file is collected last."""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    pr = Pair((5, 3, 2), (10.0, 6.0, 4.0), 5, natoms=3)
    yield pr
    pr.close()


@pytest.mark.parametrize("form", [0, 1, 2], ids=["H", "DinvH", "HDinv"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_noalloc_matches_apply_twice(pair, form, prec):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    tol = 1e-12 if prec == R.RCF_FP64 else 2e-6
    dt = torch.complex128 if prec == R.RCF_FP64 else torch.complex64
    for call, seed in enumerate((31, 32)):
        X = workloads.complex_normal(seed + 10 * form, (pair.N, 7))
        Xd = to_dev(X, dt)
        Y_ref = torch.zeros_like(Xd)
        Y_new = torch.full_like(Xd, complex(3.0, -1.0))
        R.rcf_apply(pair.g.ctx, pair.g.op, form, Xd, Y_ref, prec)
        R.rcf_apply_noalloc(pair.g.ctx, pair.g.op, form, Xd, Y_new, prec)
        assert rel(to_host(Y_new), to_host(Y_ref)) < tol, (call, form, prec)


def test_noalloc_rejects_sizes_beyond_its_scratch(pair):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    nvec = 16384 // 3 + 1          # 3 atoms: natoms * nvec just above the capacity
    Xd = torch.zeros((nvec, pair.N), dtype=torch.complex64, device="cuda")
    Yd = torch.zeros_like(Xd)
    with pytest.raises(R.RcfError) as e:
        R.rcf_apply_noalloc(pair.g.ctx, pair.g.op, 2, Xd, Yd, R.RCF_FP32)
    assert e.value.status == R.RCF_EINVAL
    assert "capacity" in str(e.value)


def test_noalloc_allocates_nothing_on_a_fresh_context(pair):
    """The promise itself: on a context and operator that have never run rcf_apply, the
    allocation-free product leaves the context's scratch memory at zero bytes, and still
    agrees with rcf_apply (which then allocates its scratch)."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.problem import GPUProblem
    g = GPUProblem(pair.w, params=pair.params)
    try:
        g.set_potential(pair.V, pair.B)
        assert R.rcf_workspace_bytes(g.ctx) == 0
        X = to_dev(workloads.complex_normal(77, (pair.N, 5)))
        Y1 = torch.zeros_like(X)
        for _ in range(2):
            R.rcf_apply_noalloc(g.ctx, g.op, 0, X, Y1, R.RCF_FP64)
        torch.cuda.synchronize()
        assert R.rcf_workspace_bytes(g.ctx) == 0
        Y2 = torch.zeros_like(X)
        R.rcf_apply(g.ctx, g.op, 0, X, Y2, R.RCF_FP64)
        assert R.rcf_workspace_bytes(g.ctx) > 0          # rcf_apply keeps its coefficients in scratch
        assert rel(to_host(Y1), to_host(Y2)) < 1e-12
    finally:
        g.close()
