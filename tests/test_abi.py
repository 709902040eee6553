"""The C-ABI library builds, loads, exports every declared symbol, and its
host-only entry points agree with the oracle.  No GPU needed."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2206_01382_gb300 as F
from paper_2206_01382_gb300 import _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return F.load()


def test_every_declared_symbol_is_exported(lib):
    names = F.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_struct_sizes_match_header(lib):
    # the C side fills these with defaults; a layout mismatch would corrupt them
    p = F.fpp_default_params()
    assert (p.L, p.D, p.iprobes, p.kappa, p.precision) == (10, 64, 1, 0, 0)
    assert p.alpha == 0.1 and p.R is None and p.stream is None
    o = F.fpp_search_opts()
    lib.fpp_default_search_opts(ctypes.byref(o))
    assert (o.k, o.probes, o.k_max, o.table_begin, o.table_end) == (10, 1, 0, 0, 0)
    assert ctypes.sizeof(F.fpp_params) == 80
    assert ctypes.sizeof(F.fpp_search_opts) == 64
    assert ctypes.sizeof(F.fpp_search_stats) == 96
    assert ctypes.sizeof(F.fpp_server_cfg) == 32
    assert ctypes.sizeof(F.fpp_server_stats) == 80


@pytest.mark.parametrize("seed,L,D,d", [(2000, 10, 64, 64), (7, 3, 5, 13), (2001, 4, 256, 128)])
def test_rotations_byte_equal_to_oracle(lib, seed, L, D, d):
    R = F.fpp_rotations(seed, L, D, d)
    Ro = O.gaussian_rotations(seed, L, D, d)
    assert np.array_equal(R.view(np.uint32), Ro.view(np.uint32))


def test_keep_count_matches_oracle(lib):
    for alpha in (0.1, 0.2, 0.05, 0.3, 1.0, 0.01):
        for kappa in (0, 20):
            for ip in (1, 3):
                B = np.array([0, 1, 2, 3, 9, 10, 11, 19, 20, 21, 99, 100, 101, 1000, 12345])
                want = O.keep_count(B, alpha, ip, kappa)
                got = [F.fpp_keep_count(int(b), alpha, ip, kappa) for b in B]
                assert got == want.tolist()


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    X = np.zeros((10, 4), np.float32)
    for kw in (dict(L=0, D=4, alpha=0.1), dict(L=2, D=0, alpha=0.1),
               dict(L=2, D=2000, alpha=0.1), dict(L=2, D=4, alpha=0.0),
               dict(L=2, D=4, alpha=1.5), dict(L=2, D=4, alpha=0.1, kappa=-1),
               dict(L=2, D=4, alpha=0.1, precision=3),
               dict(L=2, D=4, alpha=0.1, precision=F.FPP_BF16, rerank_k=257),
               dict(L=2, D=4, alpha=0.1, precision=F.FPP_BF16, rerank_k=-1)):
        with pytest.raises(F.FppError) as e:
            F.fpp_build(X, **kw)
        assert e.value.status == F.FPP_EINVAL
    with pytest.raises(F.FppError) as e:
        F.fpp_build(np.zeros((0, 4), np.float32), 2, 4, 0.1)
    assert e.value.status == F.FPP_EINVAL
    st = lib.fpp_search(None, None, 1, 10, 1, None, None)
    assert st == F.FPP_EINVAL
    assert b"NULL" in lib.fpp_last_error()
    lib.fpp_free(None)   # NULL-safe
    assert lib.fpp_set_candidate_budget(None, 1 << 20) == F.FPP_EINVAL
    assert b"NULL" in lib.fpp_last_error()


def test_launch_count_starts_at_zero_without_work(lib):
    assert F.fpp_launch_count() >= 0
