"""Helpers shared by the GPU parity tests."""
import numpy as np

from oracle import CSR


def dev(csr_or_triple, device="cuda"):
    import paper_2208_05683_gb300 as psf
    if isinstance(csr_or_triple, CSR):
        t = (csr_or_triple.rowptr, csr_or_triple.col, csr_or_triple.val)
    else:
        t = csr_or_triple
    return psf.DeviceCSR.from_host(*t, device=device)


def ocsr(triple):
    rp, col, val = triple
    return CSR(len(rp) - 1, np.asarray(rp, np.int32), np.asarray(col, np.int32), np.asarray(val, np.float64))


def assert_csr_bitwise(gpu_csr, ref: CSR, what=""):
    rp, col, val = gpu_csr.to_host()
    assert rp.shape == ref.rowptr.shape, what
    if not np.array_equal(rp, ref.rowptr):
        bad = np.nonzero(np.diff(rp) != np.diff(ref.rowptr))[0]
        raise AssertionError(f"{what}: row lengths differ in {len(bad)} rows, first {bad[:5]}")
    assert np.array_equal(col, ref.col), f"{what}: columns differ"
    same = val.view(np.int64) == ref.val.view(np.int64)
    if not same.all():
        i = np.nonzero(~same)[0]
        rel = np.max(np.abs(val[i] - ref.val[i]) / np.abs(ref.val[i]))
        raise AssertionError(f"{what}: {len(i)} values differ (max rel {rel:.3e}), first at {i[:5]}")


def rel_fro(gpu_csr, ref: CSR) -> float:
    import scipy.sparse as sp
    rp, col, val = gpu_csr.to_host()
    G = sp.csr_matrix((val, col, rp), shape=(ref.n, ref.n))
    R = ref.to_scipy()
    return float(sp.linalg.norm(G - R) / sp.linalg.norm(R))
