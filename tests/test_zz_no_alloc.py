"""psf_norm1_noalloc: the exact 1-norm computed in the library's static
scratch region, without allocating, called through the C ABI.

It must give what psf_norm1 gives and what the CPU oracle's exact 1-norm
gives (the test tolerance is bitwise equality: all three round the exact
column sums correctly), on two calls in a row, whether this file runs alone
in a fresh process or after every other test, and it must take no memory
from the device's memory pool, from which the library's other entry points
allocate.  The file name sorts last so that the latter is the default order.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic as syn
from gpu_helpers import dev

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")
from paper_2208_05683_gb300 import _abi  # noqa: E402


def c_norm1(fn, M):
    out = ctypes.c_double()
    ms = M._struct()
    rc = fn(ctypes.byref(ms), None, ctypes.byref(out))
    return rc, out.value


def wide_range_csr(n, per_row, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        rows.append(np.sort(rng.choice(n, size=per_row, replace=False)))
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(col.size) * 10.0 ** rng.uniform(-40, 40, col.size)
    return rp, col, val


CASES = {
    "wide_range": lambda: wide_range_csr(3000, 9, 5),
    "lap2d_128": lambda: syn.laplacian_2d(128),
    "banded_max_n": lambda: syn.banded_random(_abi.PSF_NORM1_NOALLOC_MAX_N, 5, 0, 2.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_norm_equals_norm1_and_oracle_twice(case):
    rp, col, val = CASES[case]()
    expect = oracle.norm1(oracle.CSR(len(rp) - 1, rp, col, val))
    M = dev((rp, col, val))
    L = psf.lib()
    rc, ref = c_norm1(L.psf_norm1, M)
    assert rc == _abi.PSF_OK
    assert ref == expect
    for _ in range(2):
        rc, got = c_norm1(L.psf_norm1_noalloc, M)
        assert rc == _abi.PSF_OK, L.psf_last_error()
        assert abs(got - expect) <= 1e-12 * abs(expect)
        assert got == expect


# The library allocates its device memory with cudaMallocAsync from the
# device's default memory pool.  The pool's in-use high-water mark, reset
# before a call, shows whether the call took any memory from it, even memory
# it gave back before returning.
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8  # CUmemPool_attribute


def _default_pool():
    import torch
    cu = ctypes.CDLL("libcuda.so.1")
    d = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(d), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), d) == 0
    return cu, pool


def _pool_attr(cu, pool, attr):
    v = ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def _pool_high_after(cu, pool, call):
    import torch
    torch.cuda.synchronize()
    cur = _pool_attr(cu, pool, _USED_MEM_CURRENT)
    zero = ctypes.c_uint64(0)
    assert cu.cuMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0
    call()
    torch.cuda.synchronize()
    return cur, _pool_attr(cu, pool, _USED_MEM_HIGH), _pool_attr(cu, pool, _USED_MEM_CURRENT)


def test_noalloc_takes_no_pool_memory():
    M = dev(syn.laplacian_2d(96))
    L = psf.lib()
    cu, pool = _default_pool()
    assert c_norm1(L.psf_norm1_noalloc, M)[0] == _abi.PSF_OK  # set-up done
    # control: the allocating entry point raises the high-water mark
    cur, high, after = _pool_high_after(cu, pool, lambda: c_norm1(L.psf_norm1, M))
    assert high > cur
    # two calls in a row take nothing
    def twice():
        for _ in range(2):
            rc, got = c_norm1(L.psf_norm1_noalloc, M)
            assert rc == _abi.PSF_OK and got == 4.0
    cur, high, after = _pool_high_after(cu, pool, twice)
    assert high <= cur and after == cur


def test_noalloc_limits_and_bad_input():
    L = psf.lib()
    # one column past the static limit: rejected on the host, nothing runs
    n = _abi.PSF_NORM1_NOALLOC_MAX_N + 1
    big = dev((np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n)))
    rc, _ = c_norm1(L.psf_norm1_noalloc, big)
    assert rc == _abi.PSF_ETOOBIG
    assert b"static scratch limit" in L.psf_last_error()
    # a column outside the matrix is reported, not used
    bad = dev((np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([7], np.int32), np.array([1.0])))
    rc, _ = c_norm1(L.psf_norm1_noalloc, bad)
    assert rc == _abi.PSF_EINVAL
    # the region is reusable afterwards, and an empty matrix needs no launch
    M = dev(syn.laplacian_1d(500))
    assert psf.norm1_noalloc(M) == psf.norm1(M) == 2.0
    empty = dev((np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)))
    assert psf.norm1_noalloc(empty) == 0.0
