"""Double-float residual (rcf_residual_df, the residual of RCF_FP32_DF) against the FP64 oracle.

R = H X - M X diag(lambda) is evaluated on the GPU as pairs of floats with exact products and
error-free sums.  Each entry of Rh + Rl must lie within 2^-40 (9.1e-13) of the oracle's R,
relative to the sum of the magnitudes of the terms at that entry, S_i = (|H| |X| + M |lambda|
|X|)_i.  Worst case of the compensated sums: per term, the two rounded cross-product FMAs, the
dropped lo*lo product and the two splits cost at most 1.5 2^-45 of |c x|; each addition into
the low word rounds by at most 2^-24 of a low word bounded by 1.5 2^-22 S; with n <= 4 P + 16
terms (P <= 6) that totals below 2^-40 S.  The oracle's FP64 error (n 2^-53 S) is negligible.
Rh must be the FP32 rounding of R: within one FP32 ulp of fl32(R) everywhere and equal to it
except where R lies within that error of a rounding boundary (here: at least 99.9 % of the
entries).
"""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, to_dev

pytestmark = pytest.mark.gpu

MESHES = [
    ((7, 3, 2), (7.0, 4.5, 3.0), 3, {}),                            # ragged tiles
    ((4, 4, 4), 8.0, 4, {}),
    ((5, 3, 2), (10.0, 6.0, 4.0), 5, {}),                           # Gx = 25 > 20
    ((4, 3, 2), (8.0, 6.0, 4.0), 6, {}),
    ((1, 2, 3), (2.0, 4.0, 6.0), 2, {}),                            # a node is its own x image
    ((9, 2, 1), (9.0, 2.0, 1.0), 1, {}),
    ((4, 4, 4), 8.0, 4, dict(with_b=False, with_proj=False)),       # no B, no projectors
]


@pytest.fixture(scope="module", params=MESHES, ids=lambda m: f"n{m[0]}-p{m[2]}" + ("-plain" if m[3] else ""))
def pair(request):
    n, L, p, kw = request.param
    pr = Pair(n, L, p, natoms=2, **kw)
    yield pr
    pr.close()


def magnitude_bound(H, X, lam):
    """(|H| |X| + M |lambda| |X|) entrywise, with |H| the entrywise modulus of every term."""
    A = abs(H.Hloc) @ np.abs(X)
    for pr in H.projectors:
        r = pr["rows"]
        A[r] += np.abs(pr["P"]) @ (np.abs(pr["Delta"]) @ (np.abs(pr["P"]).T @ np.abs(X[r])))
    return A + H.Mdiag[:, None] * np.abs(X) * np.abs(lam)[None, :]


def _run(pair, X, lam, ld_pad=0):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    nv = X.shape[1]
    Xd = to_dev(X)
    Rh = torch.zeros((nv, H.N + ld_pad), dtype=torch.complex64, device="cuda")
    Rl = torch.zeros_like(Rh)
    R.rcf_residual_df(pair.g.ctx, pair.g.op, Xd, lam, Rh[:, :H.N], Rl[:, :H.N])
    rh = Rh[:, :H.N].cpu().numpy().T
    rl = Rl[:, :H.N].cpu().numpy().T
    if ld_pad:
        assert torch.all(Rh[:, H.N:] == 0) and torch.all(Rl[:, H.N:] == 0)
    return rh, rl


def _check(H, X, lam, rh, rl, exact_frac=0.999):
    """Rh + Rl within 2^-40 A of R; Rh within one FP32 ulp plus that error of fl32(R), and
    (where R is not much smaller than A) equal to fl32(R) for a fraction exact_frac."""
    ref = H.apply(X) - H.Mdiag[:, None] * X * lam[None, :]
    A = magnitude_bound(H, X, lam)
    got = rh.astype(np.complex128) + rl.astype(np.complex128)
    for part in (np.real, np.imag):
        err = np.abs(part(got) - part(ref))
        assert np.all(err <= 2.0 ** -40 * A + 1e-300), float(np.max(err / A))
        f32 = part(ref).astype(np.float32)
        h = part(rh)
        assert np.all(np.abs(h.astype(np.float64) - f32) <= np.spacing(np.abs(f32)) + 2.0 ** -40 * A)
        if exact_frac is not None:
            assert np.mean(h == f32) >= exact_frac


def test_residual_df_matches_oracle(pair):
    H = pair.H
    X = workloads.complex_normal(6, (H.N, 5))
    lam = np.array([-0.3, 0.1, 0.5, 2.0, -1.7])
    rh, rl = _run(pair, X, lam)
    _check(H, X, lam, rh, rl)


def test_residual_df_near_eigenvectors(pair):
    """Columns close to eigenvectors (smooth, strongly cancelling R): the bound is relative to
    the magnitudes of the terms, not to R itself."""
    H = pair.H
    if H.N > 3000:
        pytest.skip("dense eigensolve only on the small meshes")
    import scipy.linalg as sla
    w, V = sla.eigh(H.dense(), np.diag(H.Mdiag))
    X = V[:, :4] + 1e-7 * workloads.complex_normal(8, (H.N, 4))
    lam = w[:4]
    rh, rl = _run(pair, X, lam, ld_pad=6)
    # R is ~1e-7 of the terms here, so its FP32 ulp can be below the double-float error
    _check(H, X, lam, rh, rl, exact_frac=None)


def test_residual_df_strided_and_empty(pair):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    X = workloads.complex_normal(9, (H.N, 3))
    lam = np.array([0.2, -0.4, 1.1])
    big = torch.zeros((3, H.N + 4), dtype=torch.complex128, device="cuda")
    big[:, :H.N] = to_dev(X)
    Rh = torch.zeros((3, H.N), dtype=torch.complex64, device="cuda")
    R.rcf_residual_df(pair.g.ctx, pair.g.op, big[:, :H.N], lam, Rh)          # Rl omitted
    ref = H.apply(X) - H.Mdiag[:, None] * X * lam[None, :]
    assert np.max(np.abs(Rh.cpu().numpy().T - ref)) <= 2 ** -23 * np.max(np.abs(ref))
    R.rcf_residual_df(pair.g.ctx, pair.g.op, big[:0, :H.N], lam[:0], Rh[:0])  # no vectors: no-op


def test_residual_df_adjacent_buffers_accepted_overlap_rejected(pair):
    """X (complex128) directly after Rh (complex64) in one allocation is legal; X overlapping
    Rh is rejected."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    nv = 2
    X = workloads.complex_normal(10, (H.N, nv))
    lam = np.array([0.3, -0.2])
    nb_r, nb_x = nv * H.N * 8, nv * H.N * 16
    buf = torch.zeros(nb_r + nb_x, dtype=torch.uint8, device="cuda")
    Rh = buf[:nb_r].view(torch.complex64).view(nv, H.N)
    Xd = buf[nb_r:].view(torch.complex128).view(nv, H.N)
    Xd.copy_(to_dev(X))
    R.rcf_residual_df(pair.g.ctx, pair.g.op, Xd, lam, Rh)
    ref = H.apply(X) - H.Mdiag[:, None] * X * lam[None, :]
    assert np.max(np.abs(Rh.cpu().numpy().T - ref)) <= 2 ** -23 * np.max(np.abs(ref))
    Rbad = buf[nb_r - 8 * H.N:2 * nb_r - 8 * H.N].view(torch.complex64).view(nv, H.N)   # ends inside X
    with pytest.raises(R.RcfError) as e:
        R.rcf_residual_df(pair.g.ctx, pair.g.op, Xd, lam, Rbad)
    assert e.value.status == R.RCF_EINVAL
