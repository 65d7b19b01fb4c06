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


def check_same(got, ref, what=""):
    info = got.info
    p = ref.plan
    assert (info["N"], info["q"], info["b"], info["g"]) == (p.N, p.q, p.b, p.g), what
    zsub = [ref.norms[1] ** i for i in range(11)]  # z_i = ||Z||^i (submultiplicative)
    assert info["z"] in (ref.norms[:11], p.z[:11], zsub), what
    assert_csr_bitwise(got.csr, ref.F, what)
    if ref.F.nnz:
        assert rel_fro(got.csr, ref.F) <= 1e-12
    # per-step Algorithm 1 decisions (S_0 and the g = 1 add are kind "add")
    gsteps = [s for s in got.steps if s["kind"] != "add"]
    osteps = [s for s in ref.steps if not (s.kind == "giant" and s.threshold == 0.0 and s.iters == 0
                                           and p.g == 1 and s.index == 1)]
    assert len(gsteps) == len(osteps), what
    for g, o in zip(gsteps, osteps):
        assert g["nnz_pre"] == o.nnz_pre and g["nnz_post"] == o.nnz_post, (what, g, o)
        if o.threshold > 0:
            assert g["eps_f"] == o.eps_f and g["iters"] == o.iters and g["dropped"] == o.c, (what, g, o)
