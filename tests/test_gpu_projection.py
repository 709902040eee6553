"""The tensor-core projections the search decides on stay inside the error
bound the decisions assume, with margin: |p - q^T r| <= c ||q|| ||r||."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build
    _build.build()
    F.load()
    return F


@pytest.mark.parametrize("d,D,L", [(128, 256, 3), (64, 64, 4), (30, 5, 3), (960, 64, 2), (96, 128, 2)])
def test_projection_error_within_bound(F, d, D, L):
    X, Q = W.small_mixture(600, 300, d, 32, 0.25, 95 + d)
    ix = F.Index(X, L, D, 0.5, seed=40 + d)
    P = F.fpp_debug_projections(ix.handle, Q).astype(np.float64)
    R = O.gaussian_rotations(40 + d, L, D, d).astype(np.float64).reshape(-1, d)
    Q64 = Q.astype(np.float64)
    exact = Q64 @ R.T
    c = F.fpp_projection_error_bound(ix.handle)
    bound = c * np.linalg.norm(Q64, axis=1)[:, None] * np.linalg.norm(R, axis=1)[None, :]
    err = np.abs(P - exact)
    ratio = float((err / bound).max())
    assert ratio < 0.25, f"max error / bound = {ratio}"
    # and the split path is far more accurate than plain BF16 would be
    assert float(err.max()) < 1e-4 * np.abs(exact).max()


@pytest.mark.parametrize("d,D,L", [(128, 256, 2), (30, 5, 3)])
def test_projection_error_within_bound_fp32_vectors(F, d, D, L):
    # random vectors off the BF16 grid take the six-product split
    X, Q = W.small_mixture(600, 300, d, 32, 0.25, 195 + d)
    R = np.random.default_rng(7 + d).standard_normal((L, 2, D, d)).astype(np.float32)
    ix = F.Index(X, L, D, 0.5, R=R)
    assert ix.info()["r_pieces"] == 3
    P = F.fpp_debug_projections(ix.handle, Q).astype(np.float64)
    R64 = R.astype(np.float64).reshape(-1, d)
    Q64 = Q.astype(np.float64)
    exact = Q64 @ R64.T
    c = F.fpp_projection_error_bound(ix.handle)
    bound = c * np.linalg.norm(Q64, axis=1)[:, None] * np.linalg.norm(R64, axis=1)[None, :]
    assert float((np.abs(P - exact) / bound).max()) < 0.25
    # the seeded vectors are on the BF16 grid: three products
    assert F.Index(X, L, D, 0.5, seed=1).info()["r_pieces"] == 1


def test_projection_table_range(F):
    X, Q = W.small_mixture(500, 20, 64, 16, 0.25, 99)
    ix = F.Index(X, 6, 32, 0.5, seed=3)
    full = F.fpp_debug_projections(ix.handle, Q)
    part = F.fpp_debug_projections(ix.handle, Q, 2, 5)
    assert np.array_equal(part, full[:, 2 * 2 * 32: 5 * 2 * 32])


def test_bounded_wait_runs_out_and_the_context_stays_usable(F):
    # 2 L D = 128 projections of 100 queries: one 128 x 256 tile, one CTA.
    # With the host's test hook that CTA never loads its first K chunk, so
    # the tensor-core warp's wait runs out after about 10 ms; the CTA drains
    # what it issued, frees its tensor memory and the call reports
    # FPP_ETIMEOUT.  The next calls run normally on the same context.
    X, Q = W.small_mixture(2000, 100, 64, 16, 0.25, 501)
    ix = F.Index(X, 1, 64, 0.5, seed=5)
    ref = F.fpp_debug_projections(ix.handle, Q)
    gi, gs = ix.search(Q, 10, 2)
    F.fpp_debug_wait_test(1, 20_000_000)
    try:
        with pytest.raises(F.FppError) as e:
            F.fpp_debug_projections(ix.handle, Q)
        assert e.value.status == F.FPP_ETIMEOUT and "bounded wait" in str(e.value)
    finally:
        F.fpp_debug_wait_test(0, 0)
    assert np.array_equal(F.fpp_debug_projections(ix.handle, Q), ref)
    gi2, gs2 = ix.search(Q, 10, 2)
    assert np.array_equal(gi2, gi) and np.array_equal(gs2, gs)
    with pytest.raises(F.FppError) as e:
        F.fpp_debug_wait_test(2, 0)
    assert e.value.status == F.FPP_EINVAL
