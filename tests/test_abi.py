"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol the header declares, validates host arguments, and its host planner
matches the oracle's planner bit for bit."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import synthetic as syn
from oracle import CSR, planner, power_norms

import paper_2208_05683_gb300 as psf
from paper_2208_05683_gb300 import _abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "psf.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PSF_API\s+(?:int|const char\*)\s+(psf_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = psf.lib()
    names = declared_functions()
    assert len(names) >= 15
    assert sorted(_abi.EXPORTS) == names
    for name in names:
        assert hasattr(L, name), name
    assert L.psf_version() >= 1


def test_library_exports_nothing_else():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", psf._build.LIB], capture_output=True,
                         text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if l.split() and l.split()[1] in "TDB"]
    assert sorted(s for s in syms if s.startswith("psf_")) == declared_functions()


def test_series_create_rejects_bad_arguments():
    with pytest.raises(psf.PsfError) as e:
        psf.Series([1.0, 1.0], tol=0.0)
    assert e.value.code == _abi.PSF_EINVAL
    with pytest.raises(psf.PsfError):
        psf.Series([1.0, float("nan")], tol=1e-12)
    with pytest.raises(psf.PsfError):
        psf.Series([1.0], tol=1e-12, s=_abi.PSF_MAX_Q + 1)
    with pytest.raises(psf.PsfError):
        psf.Series([], tol=1e-12)
    s = psf.Series(syn.coeffs("exp"), 1e-12, e_r=0.2, maxit=50)
    with pytest.raises(psf.PsfError):
        _abi.check(psf.lib().psf_series_set_param(s._h, 99, 1.0))
    with pytest.raises(psf.PsfError):
        _abi.check(psf.lib().psf_series_set_param(s._h, _abi.PSF_PARAM_ER, -1.0))
    # product kernel: 0 auto .. 4 one row per block of four warps
    for k in (0.0, 1.0, 2.0, 3.0, 4.0):
        _abi.check(psf.lib().psf_series_set_param(s._h, _abi.PSF_PARAM_KERNEL, k))
    for bad in (-1.0, 2.5, 5.0):
        with pytest.raises(psf.PsfError):
            _abi.check(psf.lib().psf_series_set_param(s._h, _abi.PSF_PARAM_KERNEL, bad))
    psf.Series(syn.coeffs("exp"), 1e-12, kernel="cta")


def _same(a, b):
    return a == b or (math.isinf(a) and math.isinf(b))


@pytest.mark.parametrize("kind", ["exp", "cos", "cosh", "sinh"])
@pytest.mark.parametrize("tol", [1e-8, 1e-12, 1e-14])
@pytest.mark.parametrize("mat", ["lap1d", "lap2d", "banded"])
def test_host_planner_matches_oracle_bitwise(kind, tol, mat):
    if mat == "lap1d":
        Z = CSR(64, *syn.laplacian_1d(64))
    elif mat == "lap2d":
        Z = CSR(256, *syn.laplacian_2d(16))
    else:
        Z = CSR(200, *syn.banded_random(200, 3, 5, 3.0))
    norms = power_norms(Z)
    a = syn.coeffs(kind)
    ref = planner.plan(a, tol, norms)
    got = psf.plan(a, tol, norms)
    assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g)
    assert got["products"] == planner.mult_count(ref.N)
    assert got["trunc"] == ref.trunc and got["budget"] == ref.budget
    assert got["z"] == ref.z[:11]
    assert set(got["zeta"]) == set(ref.zeta) and set(got["sigma"]) == set(ref.sigma)
    for k in ref.zeta:
        assert _same(got["zeta"][k], ref.zeta[k]), k
    for j in ref.sigma:
        assert _same(got["sigma"][j], ref.sigma[j]), j


@pytest.mark.parametrize("N", range(2, 40))
def test_host_planner_poly_and_override(N):
    norms = [1.0] + [1.7 ** i for i in range(1, 11)]
    a = [1.0 / math.factorial(i) for i in range(N)]
    for s in (0, 2, 3):
        ref = planner.plan(a, 1e-10, norms, poly=True, s=s)
        got = psf.plan(a, 1e-10, norms, poly=True, s=s)
        assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g)
        for k in ref.zeta:
            assert _same(got["zeta"][k], ref.zeta[k])
        for j in ref.sigma:
            assert _same(got["sigma"][j], ref.sigma[j])
    ref = planner.plan(a, 1e-10, norms, poly=True, submult=True)
    got = psf.plan(a, 1e-10, norms, poly=True, submult=True)
    assert got["z"] == ref.z[:11]


@pytest.mark.parametrize("seed", range(12))
def test_host_planner_random_sweep_bitwise(seed):
    # seeded random coefficient sets (decaying, flat, with zeros and sign
    # changes), power-norm sequences that are not submultiplicative in
    # general (and those of zero and nilpotent matrices), tolerances
    # 1e-15..1e-5, series and polynomial mode, SUBMULT and the s override:
    # the C++ planner gives the oracle's plan bit for bit, and both report
    # "not converged" for the same inputs
    rng = np.random.default_rng(1000 + seed)
    for case in range(40):
        m = int(rng.integers(1, 130))
        if rng.uniform() < 0.5:
            r = rng.uniform(0.2, 6.0)
            a = [r ** i / math.factorial(i) for i in range(m)]
        else:
            a = list(rng.standard_normal(m) * 10.0 ** rng.uniform(-12, 0, m))
        for i in range(m):
            if rng.uniform() < 0.15:
                a[i] = 0.0
            elif rng.uniform() < 0.3:
                a[i] = -a[i]
        # the zero matrix, or a nilpotent one (powers vanish from some i on)
        z1 = 0.0 if rng.uniform() < 0.05 else rng.uniform(0.05, 6.0)
        cut = int(rng.integers(2, 11)) if rng.uniform() < 0.15 else 11
        norms = [1.0, z1]
        for i in range(2, 11):
            norms.append(0.0 if i >= cut else norms[-1] * z1 * rng.uniform(0.2, 1.0))
        tol = 10.0 ** rng.uniform(-15, -5)
        poly = rng.uniform() < 0.25
        submult = rng.uniform() < 0.25
        s = int(rng.integers(1, _abi.PSF_MAX_Q + 1)) if rng.uniform() < 0.2 else 0
        what = f"seed {seed} case {case}: m={m} tol={tol:.3e} poly={poly} submult={submult} s={s}"
        try:
            ref = planner.plan(a, tol, norms, poly=poly, s=s, submult=submult)
        except ValueError:
            with pytest.raises(psf.PsfError) as e:
                psf.plan(a, tol, norms, poly=poly, submult=submult, s=s)
            assert e.value.code == _abi.PSF_ENOTCONV, what
            continue
        bare = psf.plan(a, tol, norms, poly=poly, submult=submult, s=s, thresholds=False)
        assert (bare["N"], bare["q"], bare["b"], bare["g"]) == (ref.N, ref.q, ref.b, ref.g), what
        assert bare["trunc"] == ref.trunc and _same(bare["budget"], ref.budget), what
        assert bare["z"] == ref.z[:11], what
        if ref.q > _abi.PSF_MAX_Q + 1 or ref.b > _abi.PSF_MAX_Q + 2:
            # thresholds past the header's arrays of PSF_MAX_Q + 2 entries
            with pytest.raises(psf.PsfError) as e:
                psf.plan(a, tol, norms, poly=poly, submult=submult, s=s)
            assert e.value.code == _abi.PSF_ETOOBIG, what
            continue
        got = psf.plan(a, tol, norms, poly=poly, submult=submult, s=s)
        assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g), what
        assert set(got["zeta"]) == set(ref.zeta) and set(got["sigma"]) == set(ref.sigma), what
        for k in ref.zeta:
            assert _same(got["zeta"][k], ref.zeta[k]), (what, k)
        for j in ref.sigma:
            assert _same(got["sigma"][j], ref.sigma[j]), (what, j)


@pytest.mark.parametrize("seed", range(6))
def test_host_planner_square_random_sweep_bitwise(seed):
    # PSF_Z_SQUARE on seeded random series of one parity: the plan of g in
    # W = Z^2 (z of W = z_{2i} of Z, tol / z_1 for an odd series) is the
    # oracle's bit for bit, with the same "not converged" cases
    rng = np.random.default_rng(2000 + seed)
    for case in range(40):
        m = int(rng.integers(2, 130))
        odd = bool(rng.uniform() < 0.5)
        r = rng.uniform(0.2, 5.0)
        a = [0.0] * m
        for i in range(int(odd), m, 2):
            a[i] = (-1.0) ** (i // 2) * r ** i / math.factorial(i) if rng.uniform() < 0.9 else 0.0
        if not any(a):
            continue
        z1 = rng.uniform(0.05, 6.0)
        norms = [1.0, z1]
        for i in range(2, 11):
            norms.append(norms[-1] * z1 * rng.uniform(0.2, 1.0))
        tol = 10.0 ** rng.uniform(-15, -5)
        poly = rng.uniform() < 0.25
        submult = rng.uniform() < 0.25
        what = f"seed {seed} case {case}: m={m} odd={odd} tol={tol:.3e} poly={poly} submult={submult}"
        c, o = planner.split_even_odd(a)
        assert o == odd, what
        tol_g = tol / norms[1] if odd else tol
        try:
            ref = planner.plan(c, tol_g, norms, poly=poly, submult=submult, stride=2)
        except ValueError:
            with pytest.raises(psf.PsfError) as e:
                psf.plan(a, tol, norms, poly=poly, submult=submult, square=True)
            assert e.value.code == _abi.PSF_ENOTCONV, what
            continue
        got = psf.plan(a, tol, norms, poly=poly, submult=submult, square=True, thresholds=False)
        assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g), what
        assert got["products"] == planner.mult_count(ref.N) + 1 + int(odd), what
        assert got["trunc"] == ref.trunc and _same(got["budget"], ref.budget), what
        if ref.q <= _abi.PSF_MAX_Q + 1 and ref.b <= _abi.PSF_MAX_Q + 2:
            got = psf.plan(a, tol, norms, poly=poly, submult=submult, square=True)
            for k in ref.zeta:
                assert _same(got["zeta"][k], ref.zeta[k]), (what, k)
            for j in ref.sigma:
                assert _same(got["sigma"][j], ref.sigma[j]), (what, j)


def test_host_planner_not_converged():
    with pytest.raises(psf.PsfError) as e:
        psf.plan(syn.coeffs("exp", 6), 1e-12, [1.0] + [10.0 ** i for i in range(1, 11)])
    assert e.value.code == _abi.PSF_ENOTCONV


def test_tuning_keys_are_checked_on_the_host():
    old = psf.tune_get(_abi.PSF_TUNE_TABLE_CROSSOVER)
    try:
        psf.tune_set(_abi.PSF_TUNE_TABLE_CROSSOVER, 512.0)
        assert psf.tune_get(_abi.PSF_TUNE_TABLE_CROSSOVER) == 512.0
        with pytest.raises(psf.PsfError):
            psf.tune_set(_abi.PSF_TUNE_TABLE_CROSSOVER, -1.0)
        with pytest.raises(psf.PsfError):
            psf.tune_set(99, 1.0)
        with pytest.raises(psf.PsfError):
            psf.tune_get(99)
    finally:
        psf.tune_set(_abi.PSF_TUNE_TABLE_CROSSOVER, old)
    old = psf.tune_get(_abi.PSF_TUNE_ALG1_FAR_SHIFT)
    assert old == 6.0
    try:
        for v in (0.0, 1.0, 2047.0):
            psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, v)
            assert psf.tune_get(_abi.PSF_TUNE_ALG1_FAR_SHIFT) == v
        for bad in (-1.0, 2.5, 2048.0):
            with pytest.raises(psf.PsfError):
                psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, bad)
    finally:
        psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, old)
    old = psf.tune_get(_abi.PSF_TUNE_ROW_BITMAPS)
    assert old == 1.0
    try:
        for v in (0.0, 2.0, 1.0):
            psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, v)
            assert psf.tune_get(_abi.PSF_TUNE_ROW_BITMAPS) == v
        for bad in (-1.0, 0.5, 3.0):
            with pytest.raises(psf.PsfError):
                psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, bad)
    finally:
        psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, old)
    for key in (_abi.PSF_TUNE_BATCH_GRAPH, _abi.PSF_TUNE_BATCH_REUSE):
        old = psf.tune_get(key)
        assert old == 1.0
        try:
            psf.tune_set(key, 0.0)
            assert psf.tune_get(key) == 0.0
            with pytest.raises(psf.PsfError):
                psf.tune_set(key, 0.5)
        finally:
            psf.tune_set(key, old)


def test_estimate_flag_checked_on_the_host():
    # the estimator flag is known, and it excludes the submultiplicative bound
    s = psf.Series(syn.coeffs("exp"), 1e-12, estimate=True)
    assert s.flags & _abi.PSF_Z_ESTIMATE
    with pytest.raises(psf.PsfError) as e:
        psf.Series(syn.coeffs("exp"), 1e-12, submult=True, estimate=True)
    assert e.value.code == _abi.PSF_EINVAL


@pytest.mark.parametrize("kind", ["cos", "cosh", "sinh"])
@pytest.mark.parametrize("tol", [1e-8, 1e-12, 1e-14])
@pytest.mark.parametrize("mat", ["lap2d", "banded", "zero"])
def test_host_planner_square_matches_oracle_bitwise(kind, tol, mat):
    # PSF_Z_SQUARE: the plan of g in W = Z^2, with z_i of W = z_{2i} of Z and,
    # for an odd series, the tolerance divided by ||Z||_1
    if mat == "lap2d":
        norms = power_norms(CSR(256, *syn.laplacian_2d(16)))
    elif mat == "banded":
        norms = power_norms(CSR(200, *syn.banded_random(200, 3, 5, 3.0)))
    else:
        norms = [1.0] + [0.0] * 10
    a = syn.coeffs(kind)
    c, odd = planner.split_even_odd(a)
    tol_g = (tol / norms[1] if norms[1] != 0.0 else math.inf) if odd else tol
    ref = planner.plan(c, tol_g, norms, stride=2)
    got = psf.plan(a, tol, norms, square=True)
    assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g)
    assert got["products"] == planner.mult_count(ref.N) + 1 + int(odd)
    assert got["trunc"] == ref.trunc and _same(got["budget"], ref.budget)
    assert got["z"] == planner.z_sequence(norms, 11)[:11]
    assert set(got["zeta"]) == set(ref.zeta) and set(got["sigma"]) == set(ref.sigma)
    for k in ref.zeta:
        assert _same(got["zeta"][k], ref.zeta[k]), k
    for j in ref.sigma:
        assert _same(got["sigma"][j], ref.sigma[j]), j


@pytest.mark.parametrize("N", range(2, 30))
def test_host_planner_square_poly_and_submult(N):
    norms = [1.0] + [1.7 ** i for i in range(1, 11)]
    for odd in (False, True):
        a = [0.0] * N
        for i in range(int(odd), N, 2):
            a[i] = 1.0 / math.factorial(i)
        if not any(a):
            continue
        c, o = planner.split_even_odd(a)
        assert o == odd or not any(c)
        for submult in (False, True):
            tol_g = 1e-10 / norms[1] if o else 1e-10
            ref = planner.plan(c, tol_g, norms, poly=True, submult=submult, stride=2)
            got = psf.plan(a, 1e-10, norms, poly=True, submult=submult, square=True)
            assert (got["N"], got["q"], got["b"], got["g"]) == (ref.N, ref.q, ref.b, ref.g)
            assert got["budget"] == ref.budget
            for k in ref.zeta:
                assert _same(got["zeta"][k], ref.zeta[k])
            for j in ref.sigma:
                assert _same(got["sigma"][j], ref.sigma[j])


def test_square_flag_needs_one_parity():
    s = psf.Series(syn.coeffs("cos"), 1e-12, square=True)
    assert s.flags & _abi.PSF_Z_SQUARE
    psf.Series(syn.coeffs("sinh"), 1e-12, square=True, poly=True)
    for bad in (syn.coeffs("exp"), [1.0, 1.0]):
        with pytest.raises(psf.PsfError) as e:
            psf.Series(bad, 1e-12, square=True)
        assert e.value.code == _abi.PSF_EINVAL
        with pytest.raises(psf.PsfError) as e:
            psf.plan(bad, 1e-12, [1.0] + [2.0 ** i for i in range(1, 11)], square=True)
        assert e.value.code == _abi.PSF_EINVAL


def test_torch_sparse_csr_round_trip_on_the_host():
    # the binding's torch interop: a torch sparse CSR tensor in, the same
    # arrays (int32 / float64) out, and back to a torch tensor
    import torch
    rp, col, val = syn.laplacian_2d(6)
    t = torch.sparse_csr_tensor(torch.tensor(rp, dtype=torch.int64), torch.tensor(col, dtype=torch.int64),
                                torch.tensor(val, dtype=torch.float32), size=(36, 36))
    d = psf.DeviceCSR.from_torch(t)
    assert d.n == 36 and d.rowptr.dtype == torch.int32 and d.val.dtype == torch.float64
    assert np.array_equal(d.rowptr.numpy(), rp) and np.array_equal(d.col.numpy(), col)
    assert np.array_equal(d.val.numpy(), np.asarray(val, np.float32).astype(np.float64))
    back = d.to_torch()
    assert back.layout == torch.sparse_csr and tuple(back.shape) == (36, 36)
    assert torch.equal(back.to_dense(), t.to_dense().double())
    with pytest.raises(psf.PsfError):
        psf.DeviceCSR.from_torch(torch.zeros(3, 3))
    with pytest.raises(psf.PsfError):
        psf.DeviceCSR.from_torch(torch.zeros(3, 4).to_sparse_csr())


def test_c_caller_compiles_links_and_plans(tmp_path):
    # the header is plain C99 and the library serves a C caller (host-side
    # entry points only: no GPU is touched)
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    lib = psf._build.build()
    exe = str(tmp_path / "c_abi_check")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    os.path.join(here, "c_abi_check.c"), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok N=28 q=5 b=6 products=9"), out.stdout


def test_host_planner_rejects_bad_inputs():
    norms = [1.0] + [2.0 ** i for i in range(1, 11)]
    a = syn.coeffs("exp")
    for bad_a, bad_n, code in ((a[:5] + [float("nan")] + a[6:], norms, _abi.PSF_EINVAL),
                               (a, norms[:3] + [-1.0] + norms[4:], _abi.PSF_EINVAL),
                               (a, norms[:2] + [float("inf")] + norms[3:], _abi.PSF_EINVAL),
                               ([1e-30] * 100001, norms, _abi.PSF_ETOOBIG)):
        with pytest.raises(psf.PsfError) as e:
            psf.plan(bad_a, 1e-12, bad_n)
        assert e.value.code == code
    # SUBMULT reads only z_0 and z_1
    psf.plan(a, 1e-12, [1.0, 2.0] + [float("nan")] * 9, submult=True)


def test_product_filter_host_checks():
    # argument checks that precede any device work
    import ctypes
    L = psf.lib()
    out = ctypes.c_void_p()
    for thr, word in ((float("inf"), "threshold"), (float("nan"), "threshold"), (-1.0, "threshold")):
        rc = L.psf_product_filter(None, None, 0, None, None, thr, 0.1, 10, None, ctypes.byref(out))
        assert rc == _abi.PSF_EINVAL and word in L.psf_last_error().decode()
    rc = L.psf_product_filter(None, None, _abi.PSF_MAX_Q + 2, None, None, 0.0, 0.1, 10, None, ctypes.byref(out))
    assert rc == _abi.PSF_EINVAL and "nadd" in L.psf_last_error().decode()


def test_binding_constants_match_the_header():
    # every numeric #define of the header has the same value in the binding
    text = open(HEADER).read()
    defs = dict(re.findall(r"^#define (PSF_[A-Z0-9_]+) (\d+)u?\b", text, flags=re.M))
    assert len(defs) >= 25
    for name, value in defs.items():
        assert hasattr(_abi, name), name
        assert getattr(_abi, name) == int(value), name


def test_binding_struct_layouts_match_the_header(tmp_path):
    # the ctypes structures of the binding have the C structs' sizes and
    # field offsets (as the C compiler lays them out from the header)
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "c_abi_layout")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    os.path.join(here, "c_abi_layout.c"), "-o", exe], check=True, capture_output=True, text=True)
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {}
    for line in filter(None, lines):
        t, f, v = line.split()
        c[(t, f)] = int(v)
    pairs = {"psf_csr_t": _abi.CSRStruct, "psf_info_t": _abi.InfoStruct, "psf_step_info_t": _abi.StepStruct,
             "psf_server_config_t": _abi.ServerConfig, "psf_completion_t": _abi.Completion,
             "psf_server_stats_t": _abi.ServerStats, "psf_batch_tune_t": _abi.BatchTune}
    for t, S in pairs.items():
        assert ctypes.sizeof(S) == c[(t, "-")], t
        fields = [f for f, _ in S._fields_]
        assert {f for (tt, f) in c if tt == t and f != "-"} == set(fields), t
        for f in fields:
            assert getattr(S, f).offset == c[(t, f)], (t, f)
