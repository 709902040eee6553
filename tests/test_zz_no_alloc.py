"""fpp_bruteforce_static: exact search that allocates nothing inside libfpp.

It serves callers that cannot allocate device memory when they search (their
framework already holds the GPU's memory, or cudaMalloc's implicit
synchronisation is too costly for them).  Its results must match those of
fpp_bruteforce, which allocates its scratch, within the tolerance used by the
other parity tests, and the FP64 brute force of the CPU oracle.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
RTOL = 1e-5


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build
    _build.build()
    F.load()
    return F


def _same(F, Xd, Qd, k):
    ref_i, ref_s = F.fpp_bruteforce(Xd, Qd, k)
    got_i, got_s = F.fpp_bruteforce_static(Xd, Qd, k)
    torch.cuda.synchronize()
    ri, rs = ref_i.cpu().numpy(), ref_s.cpu().numpy()
    gi, gs = got_i.cpu().numpy(), got_s.cpu().numpy()
    assert np.array_equal(gi, ri)
    fin = np.isfinite(rs)
    assert np.array_equal(np.isfinite(gs), fin)
    assert np.allclose(gs[fin], rs[fin], rtol=RTOL, atol=1e-6)


def test_static_scratch_matches_allocating_path_on_consecutive_calls(F):
    X, Q = W.small_mixture(50000, 64, 64, 128, 0.25, 90)
    _same(F, torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 10)
    # second call in a row: other sizes (ragged n, larger k); the array still
    # holds the first call's contents
    X2, Q2 = W.small_mixture(30001, 77, 32, 64, 0.3, 91)
    _same(F, torch.from_numpy(X2).cuda(), torch.from_numpy(Q2).cuda(), 17)


def test_static_scratch_matches_oracle_brute_force(F):
    import oracle as O
    X, Q = W.small_mixture(20001, 50, 32, 96, 0.25, 94)
    gi, gs = F.fpp_bruteforce_static(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 10)
    torch.cuda.synchronize()
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    oi, osc, flags = O.brute_force(X, Q, 10)
    compared = 0
    for i in range(len(Q)):
        if flags[i]:      # FP64 near-tie at the k-th place: either order is right
            continue
        assert np.array_equal(gi[i], oi[i]), i
        assert np.allclose(gs[i], osc[i], rtol=RTOL, atol=1e-6), i
        compared += 1
    print(f"static brute force vs oracle: {compared} compared, {len(Q) - compared} near-tie skipped")
    assert compared >= 0.9 * len(Q)


def test_static_scratch_many_query_chunks(F):
    # n = 1M leaves room for 8 queries per pass of the 32 MiB array
    X, Q = W.small_mixture(1_000_000, 40, 16, 256, 0.25, 92)
    _same(F, torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 5)


def test_static_scratch_rejects_what_it_cannot_serve(F):
    X, Q = W.small_mixture(1000, 4, 16, 8, 0.2, 93)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with pytest.raises(F.FppError) as e:   # host memory
        F.fpp_bruteforce_static(torch.from_numpy(X), torch.from_numpy(Q), 5,
                                ids=torch.empty((4, 5), dtype=torch.int64),
                                scores=torch.empty((4, 5)))
    assert e.value.status == F.FPP_EINVAL
    big = torch.zeros((8_400_000, 4), device="cuda")
    with pytest.raises(F.FppError) as e:   # more scores than the array holds
        F.fpp_bruteforce_static(big, Qd[:, :4].contiguous(), 5)
    assert e.value.status == F.FPP_EINVAL and "static scratch" in str(e.value)
