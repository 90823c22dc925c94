"""CPU tests of the C ABI boundary: the library loads, exports every declared entry point, and its
host-side logic (BSR assembly, input validation) behaves as include/pfe.h states. No GPU compute."""
import os
import re

import numpy as np
import pytest

import glassgen
import oracle
import paper_1902_07041_gb300 as pfe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pfe_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1902_07041_gb300 import build

    build.build()
    return pfe.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pfe.EXPORTS)


def test_springs_to_bsr_matches_oracle_hessian(lib):
    g = glassgen.generate(80, 3)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    N = g.n_atoms
    assert rp[0] == 0 and rp[-1] == ci.size
    D = np.zeros((3 * N, 3 * N))
    for i in range(N):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        for q in range(rp[i], rp[i + 1]):
            D[3 * i:3 * i + 3, 3 * ci[q]:3 * ci[q] + 3] = vals[9 * q:9 * q + 9].reshape(3, 3)
    assert np.array_equal(D, D.T)
    s = np.repeat(1.0 / np.sqrt(g.mass), 3)
    H = oracle.csr_from_springs(g).dense()
    assert np.allclose(s[:, None] * D * s[None, :], H, rtol=0, atol=1e-15 * np.abs(H).max())


def test_springs_to_bsr_rejects_bad_bonds(lib):
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_springs_to_bsr(4, [0, 1], [1, 1], [1.0, 1.0], np.ones((2, 3)) / np.sqrt(3))
    assert e.value.status == pfe.PFE_E_ARG
    with pytest.raises(pfe.PfeError):
        pfe.pfe_springs_to_bsr(4, [0], [7], [1.0], np.ones((1, 3)))


def test_duplicate_bonds_are_summed(lib):
    r = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    rp, ci, v = pfe.pfe_springs_to_bsr(2, [0, 0], [1, 1], [1.0, 2.0], r)
    assert list(rp) == [0, 2, 4] and list(ci) == [0, 1, 0, 1]
    assert v[0] == 3.0 and v[9] == -3.0


def _tiny():
    g = glassgen.generate(20, 1)
    return g, pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)


def test_create_validates_inputs_on_host(lib):
    g, (rp, ci, vals) = _tiny()
    N = g.n_atoms
    bad = vals.copy()
    bad[9 * 1 + 1] += 1e-3  # breaks Delta_ij = Delta_ji^T
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_create(N, rp, ci, bad, g.mass)
    assert e.value.status == pfe.PFE_E_NOTSYM
    nanv = vals.copy()
    nanv[5] = np.nan
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_create(N, rp, ci, nanv, g.mass)
    assert e.value.status == pfe.PFE_E_ARG
    badc = ci.copy()
    badc[0] = N + 5
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_create(N, rp, badc, vals, g.mass)
    assert e.value.status == pfe.PFE_E_ARG
    m = g.mass.copy()
    m[3] = -1.0
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_create(N, rp, ci, vals, m)
    assert e.value.status == pfe.PFE_E_ARG
    # a row without its diagonal block
    rp2 = np.array([0, 1, 2], np.int32)
    ci2 = np.array([1, 0], np.int32)
    v2 = np.zeros(18)
    with pytest.raises(pfe.PfeError) as e:
        pfe.pfe_create(2, rp2, ci2, v2)
    assert e.value.status == pfe.PFE_E_ARG


def test_null_context_is_an_argument_error(lib):
    assert lib.pfe_set_param(None, pfe.PFE_P_TOL, 1e-8) == pfe.PFE_E_ARG
    assert lib.pfe_set_interval(None, 0.0, 1.0) == pfe.PFE_E_ARG
    assert lib.pfe_solve(None, None) == pfe.PFE_E_ARG
    assert lib.pfe_solve_begin(None) == pfe.PFE_E_ARG
    assert lib.pfe_solve_iterate(None, None) == pfe.PFE_E_ARG
    assert lib.pfe_solve_end(None, None) == pfe.PFE_E_ARG
    assert lib.pfe_get_stats(None, None) == pfe.PFE_E_ARG
    lib.pfe_destroy(None)


def test_fp64_probe_rejects_bad_arguments_before_any_launch(lib):
    import ctypes

    t = ctypes.c_double(0)
    assert lib.pfe_probe_fp64_fma(0, 1, None, 8, ctypes.byref(t)) == pfe.PFE_E_ARG
    assert lib.pfe_probe_fp64_fma(10, 0, None, 8, ctypes.byref(t)) == pfe.PFE_E_ARG
    assert lib.pfe_probe_fp64_fma(10, 1, None, None, ctypes.byref(t)) == pfe.PFE_E_ARG
    assert lib.pfe_probe_fp64_fma(10, 1, None, 8, None) == pfe.PFE_E_ARG


_RATES = {"0.1": 0.1, "sqrt(0.1)": 0.1 ** 0.5, "0.1^(1/4)": 0.1 ** 0.25}


def test_library_filter_design_reproduces_tables_1_3(lib, golden):
    """The library's own degree selection (host code of libpfe.so, no GPU): all 27 piecewise-quadratic
    and all 18 Dirac degrees that Tables 1-3 print."""
    pq = golden("degrees_tables_1_3.json")
    for case in pq["cases"]:
        for i, rname in enumerate(pq["rows_r"]):
            for j, kind in enumerate(pq["columns"]):
                m, _ = pfe.pfe_design_filter("pq", case["xi"], case["eta"], eps=case["eps"], r=_RATES[rname],
                                             damping=kind)
                assert m == case["degrees"][i][j], (case["table"], rname, kind, m)
    dr = golden("dirac_degrees_tables_1_3.json")
    for case in dr["cases"]:
        for i, phi in enumerate(dr["rows_phi"]):
            for j, kind in enumerate(dr["columns"]):
                m, _ = pfe.pfe_design_filter("dirac", case["xi"], case["eta"], phi=phi, damping=kind)
                assert m == case["degrees"][i][j], (case["table"], phi, kind, m)


@pytest.mark.parametrize("kind", ["none", "jackson", "lanczos"])
def test_library_filter_coefficients_match_oracle(lib, kind):
    """Coefficients of both filters at a fixed degree against the oracle's independent routines."""
    xi, eta, eps = -0.9, -0.885, 0.002
    m, c = pfe.pfe_design_filter("pq", xi, eta, eps=eps, r=0.3, damping=kind, degree=150)
    assert m == 150
    ref = oracle.filter_coeffs(xi, eta, eps, 150, kind)
    # the two sides evaluate the App. A integrals independently: agreement to ~1e-11 of the largest
    # coefficient (sin(l arccos x) at l = 150 amplifies rounding of arccos by ~l / sqrt(1 - x^2))
    assert np.allclose(c, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    m, c = pfe.pfe_design_filter("dirac", xi, eta, phi=0.8, damping=kind, degree=120)
    g = oracle.dirac_gamma(xi, eta, 120, kind)
    ref = oracle.dirac_coeffs(g, 120, kind)
    assert np.allclose(c, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    # the Dirac filter is balanced: equal values at the interval edges
    assert abs(oracle.series_value(c, xi) - oracle.series_value(c, eta)) <= 1e-10 * np.abs(c).sum()


def test_library_filter_design_rejects_bad_input(lib):
    with pytest.raises(pfe.PfeError):
        pfe.pfe_design_filter("pq", -0.8, -0.9, eps=0.01, r=0.3)  # xi > eta
    with pytest.raises(pfe.PfeError):
        pfe.pfe_design_filter("pq", -0.9, -0.8, eps=0.01, r=1.5)  # r outside (0, 1)
    with pytest.raises(pfe.PfeError):
        pfe.pfe_design_filter("dirac", -0.9, -0.8, phi=0.0)
    # explicit degrees share the automatic search's limit of 60000
    for deg in (60001, 2 ** 31 - 1):
        with pytest.raises(pfe.PfeError) as e:
            pfe.pfe_design_filter("pq", -0.9, -0.8, eps=0.01, r=0.3, degree=deg)
        assert e.value.status == pfe.PFE_E_ARG
    m, c = pfe.pfe_design_filter("pq", -0.9, -0.8, eps=0.01, r=0.3, degree=60000)
    assert m == 60000 and c.size == 60001


def test_missing_library_fails_loudly(tmp_path):
    """Without libpfe.so the binding raises: there is no CPU or eager fallback."""
    import subprocess
    import sys

    code = ("import paper_1902_07041_gb300 as p\n"
            "try:\n"
            f"    p.load({str(tmp_path / 'libpfe.so')!r})\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'not built' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stderr


def test_product_path_is_independent_of_the_oracle():
    """The library, its binding and its build share nothing with the oracle: no import of it, no
    include of its sources, no link against it, and nothing committed reads the scratch folder."""
    pkg = os.path.join(ROOT, "paper_1902_07041_gb300")
    bad = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|#\s*include\s*[<\"][^>\"]*oracle|liboracle|[\"'/]_work/", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not bad.search(src), os.path.join(dirpath, f)
    for f in os.listdir(os.path.join(ROOT, "include")):
        assert "oracle" not in open(os.path.join(ROOT, "include", f)).read().lower(), f
