"""rcf_filter_host: the filter with X and Y in host memory, band blocks streamed through
device slots with copies overlapping the filtering.  Its output must equal the device
filter's bit for bit (same kernels, same order), for pinned and pageable host memory,
ragged last blocks and strided host layouts."""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pr():
    w = workloads.workload("cfg1")
    p = Pair(w.ncell, w.side, w.p, natoms=w.natoms, seed=w.seed)
    X = workloads.complex_normal(w.seed + 300, (p.N, 32))
    p.Xd = to_dev(X / np.linalg.norm(X, axis=0))
    p.lam = np.linspace(-1.0, 0.4, 32)
    p.bounds = (-1.2, 0.5, 60.0)
    yield p
    p.close()


@pytest.mark.parametrize("mode,prec", [(1, 2), (1, 1), (0, 0), (1, 3), (1, 4)],
                         ids=["rchfsi-fp32df", "rchfsi-fp32", "chfsi-fp64", "rchfsi-fp16", "rchfsi-bf16"])
@pytest.mark.parametrize("block", [0, 12, 32])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_filter_equals_device_filter(pr, mode, prec, block, pinned):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Yd = torch.empty_like(pr.Xd)
    R.rcf_filter(pr.g.ctx, pr.g.op, pr.Xd, pr.lam, 10, pr.bounds, mode, prec, block, Yd)
    Xh = torch.empty(pr.Xd.shape, dtype=torch.complex128, pin_memory=pinned)
    Xh.copy_(pr.Xd)
    Yh = torch.full(pr.Xd.shape, 3.0, dtype=torch.complex128, pin_memory=pinned)
    R.rcf_filter_host(pr.g.ctx, pr.g.op, Xh, pr.lam, 10, pr.bounds, mode, prec, block, Yh)
    assert torch.equal(Yh, Yd.cpu())


def test_host_filter_strided_and_invalid(pr):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Yd = torch.empty_like(pr.Xd)
    R.rcf_filter(pr.g.ctx, pr.g.op, pr.Xd, pr.lam, 10, pr.bounds, 1, 2, 12, Yd)
    big = torch.zeros((32, pr.N + 6), dtype=torch.complex128, pin_memory=True)
    big[:, :pr.N] = pr.Xd.cpu()
    Yb = torch.full((32, pr.N + 10), 7.0, dtype=torch.complex128, pin_memory=True)
    R.rcf_filter_host(pr.g.ctx, pr.g.op, big[:, :pr.N], pr.lam, 10, pr.bounds, 1, 2, 12, Yb[:, :pr.N])
    assert torch.equal(Yb[:, :pr.N], Yd.cpu())
    assert torch.all(Yb[:, pr.N:] == 7.0)                      # nothing written past the rows
    with pytest.raises(R.RcfError):
        R.rcf_filter_host(pr.g.ctx, pr.g.op, big[:, :pr.N], pr.lam, 10, pr.bounds, 1, 2, 12, big[:, :pr.N])
    with pytest.raises(TypeError):
        R.rcf_filter_host(pr.g.ctx, pr.g.op, pr.Xd, pr.lam, 10, pr.bounds, 1, 2, 12, Yb[:, :pr.N])
    R.rcf_filter_host(pr.g.ctx, pr.g.op, big[:0, :pr.N], pr.lam[:0], 10, pr.bounds, 1, 2, 12, Yb[:0, :pr.N])
