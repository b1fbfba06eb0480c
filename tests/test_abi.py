"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/holstein.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^(?!typedef|#)[\w \t*]+?\b(\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hol_create", "hol_destroy", "hol_set_field", "fermion_matvec",
                     "cg_solve", "force"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2203_01291_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2203_01291_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(declared_functions())


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2203_01291_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_context_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2203_01291_gb300 as hg
    with pytest.raises(RuntimeError):
        hg.Context(L=4, Ltau=8)


@pytest.mark.parametrize("field,value", [("L", 3), ("L", 34), ("L", 2), ("L", 7), ("Ltau", 3),
                                         ("Ltau", 0), ("max_rhs", 0), ("max_rhs", 5000),
                                         ("dtau", 0.0), ("dtau", -0.1), ("kinetic", 2),
                                         ("kinetic", -1)])
def test_create_refuses_bad_parameters_before_touching_a_device(field, value):
    """hol_create validates the parameters on the host first: an unsupported
    shape or value is HOL_EINVAL with a message, whether or not a GPU exists."""
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    p = _abi.hol_params(8, 8, 0.1, 1.0, 0.0, 1.0, 1.0, 1, 0)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    rc = lib.hol_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == _abi.HOL_EINVAL
    assert not h.value
    assert lib.hol_last_error().decode()


def test_create_refuses_exact_propagator_with_huge_hopping_step():
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    p = _abi.hol_params(8, 8, 1.0, 5.0, 0.0, 1.0, 1.0, 1, _abi.HOL_KINETIC_EXACT)
    h = ctypes.c_void_p()
    assert lib.hol_create(ctypes.byref(p), ctypes.byref(h)) == _abi.HOL_EINVAL


def test_null_arguments_are_refused():
    """Every entry point taking a context refuses a null one with HOL_EINVAL."""
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    v = ctypes.c_void_p()
    assert lib.hol_set_field(None, None, None) == _abi.HOL_EINVAL
    assert lib.fermion_matvec(None, 0, 0, None, None, 1, None) == _abi.HOL_EINVAL
    assert lib.force(None, None, None, 1, None, 1, None, None) == _abi.HOL_EINVAL
    assert lib.hol_destroy(None) == _abi.HOL_OK
    lo, hi = ctypes.c_double(), ctypes.c_double()
    assert lib.hol_get_bounds(None, ctypes.byref(lo), ctypes.byref(hi), None) == _abi.HOL_EINVAL
    assert lib.hol_arnoldi_bounds(None, None, 20, 0.05, 0, None, None, None, None) == \
        _abi.HOL_EINVAL
    del v


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (12, 3), (20, 4), (32, 5)])
def test_host_hessenberg_eigenvalues_match_numpy(n, seed):
    """The host shifted-QR eigen-solver behind the Arnoldi bounds (no GPU):
    random upper Hessenberg matrices, including ones with complex pairs,
    against numpy's eigvals (matched as multisets)."""
    import numpy as np
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    rng = np.random.default_rng(seed)
    H = np.triu(rng.standard_normal((n, n)), -1)
    if n > 3:
        H[:3, :3] += np.eye(3) * 2.0                  # a well separated block too
    re = np.zeros(n)
    im = np.zeros(n)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    Hc = np.ascontiguousarray(H)
    assert lib.hol_hessenberg_eigenvalues(n, p(Hc), p(re), p(im)) == _abi.HOL_OK
    got = np.sort_complex(re + 1j * im)
    ref = np.sort_complex(np.linalg.eigvals(H))
    # match each reference eigenvalue to the nearest computed one
    for z in ref:
        assert np.min(np.abs(got - z)) < 1e-9 * max(1.0, np.abs(ref).max())
    assert abs(got.sum() - np.trace(H)) < 1e-9 * max(1.0, np.abs(H).sum())


def test_host_hessenberg_eigenvalues_refuses_a_full_matrix():
    import numpy as np
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    H = np.ones((4, 4))
    re = np.zeros(4)
    im = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    assert lib.hol_hessenberg_eigenvalues(4, p(H), p(re), p(im)) == _abi.HOL_EINVAL


@pytest.mark.parametrize("L", [4, 6, 8, 16, 32])
@pytest.mark.parametrize("dtau,t", [(0.1, 1.0), (0.1, 3.0), (0.2, -1.0), (1.0, 1.0)])
def test_host_exact_propagator_taps(L, dtau, t):
    """The taps of the exact kinetic propagator (no GPU): the first row of
    scipy's matrix exponential of dtau t times the ring adjacency, and the
    taps the FP64 / FP32 kernels drop are below 2^-60 / 2^-30 of e[0]."""
    import numpy as np
    import scipy.linalg
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    e = np.zeros(17)
    d64, d32 = ctypes.c_int(), ctypes.c_int()
    assert lib.hol_exact_taps(L, dtau, t, e.ctypes.data_as(ctypes.c_void_p), ctypes.byref(d64),
                              ctypes.byref(d32)) == _abi.HOL_OK
    A = np.zeros((L, L))
    for i in range(L):
        A[i, (i + 1) % L] = A[(i + 1) % L, i] = 1.0
    ref = scipy.linalg.expm(dtau * t * A)[0, : L // 2 + 1]
    assert np.abs(e[: L // 2 + 1] - ref).max() < 1e-14 * abs(ref[0])
    assert np.all(e[L // 2 + 1:] == 0.0)
    assert np.all(np.abs(ref[d64.value + 1:]) <= 2.0 ** -60 * abs(ref[0]) * 1.01)
    assert np.all(np.abs(ref[d32.value + 1:]) <= 2.0 ** -30 * abs(ref[0]) * 1.01)
    assert 0 <= d32.value <= d64.value <= L // 2


@pytest.mark.parametrize("kinetic", [0, 1])
def test_create_without_a_device_fails_cleanly(kinetic):
    """Valid parameters on a host without a GPU: HOL_ECUDA with a message and
    no context (the partly built context is released)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    p = _abi.hol_params(8, 8, 0.1, 1.0, 0.0, 1.0, 1.0, 2, kinetic)
    h = ctypes.c_void_p()
    assert lib.hol_create(ctypes.byref(p), ctypes.byref(h)) == _abi.HOL_ECUDA
    assert not h.value
    assert "device" in lib.hol_last_error().decode()


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++11")])
def test_header_is_plain_c_and_cxx(tmp_path, lang, std):
    """include/holstein.h is a C ABI: it compiles as C99 and as C++11 with all
    warnings as errors, and declares everything a caller needs (the types and
    every entry point) without CUDA or torch headers."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
    calls = "\n".join(f"    (void){name};" for name in declared_functions())
    src.write_text('#include "holstein.h"\nint main(void)\n{\n    hol_params p = {0};\n'
                   '    hol_cg_opts o = {0};\n    hol_md_opts m = {0};\n'
                   '    (void)p; (void)o; (void)m;\n' + calls + "\n    return 0;\n}\n")
    r = subprocess.run([cc, "-std=" + std, "-Wall", "-Wextra", "-Werror",
                        "-Wno-missing-field-initializers", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("case", ["dtau0", "t_nan", "mu_nan", "alpha_inf", "exact", "overlap",
                                  "overlap_tail", "oversize"])
def test_static_operator_refuses_bad_arguments_on_the_host(case):
    """fermion_matvec_static validates couplings, propagator, aliasing (by
    address range, not only equal pointers) and the static scratch limit on
    the host before it looks at a device; the fake device addresses below
    are never dereferenced."""
    from paper_2203_01291_gb300 import _abi
    lib = _abi.load()
    L, T, nr = 8, 8, 2
    p = _abi.hol_params(L, T, 0.1, 1.0, 0.2, 1.0, 1.0, 1, 0)
    nbytes = nr * L * L * T * 8
    x, v, out = 0x100000, 0x200000, 0x200000 + nbytes
    if case == "dtau0":
        p.dtau = 0.0
    elif case == "t_nan":
        p.t = float("nan")
    elif case == "mu_nan":
        p.mu = float("nan")
    elif case == "alpha_inf":
        p.alpha = float("inf")
    elif case == "exact":
        p.kinetic = _abi.HOL_KINETIC_EXACT
    elif case == "overlap":
        out = v + 16 * 64                 # inside v's range, different pointer
    elif case == "overlap_tail":
        out = v - nbytes + 16             # ends inside v's range
    elif case == "oversize":
        p.L, p.Ltau = 32, 400             # 409600 doubles per rhs: 3 rhs of M^T M exceed 2^20
        nr = 3
        out = 0x40000000                  # far from v: only the size is wrong
    rc = lib.fermion_matvec_static(ctypes.byref(p), ctypes.c_void_p(x), _abi.HOL_OP_MTM,
                                   ctypes.c_void_p(v), ctypes.c_void_p(out), nr, None)
    assert rc == _abi.HOL_EINVAL, case
    msg = lib.hol_last_error().decode()
    assert msg
    if case == "oversize":
        assert "scratch" in msg
    if case.startswith("overlap"):
        assert "overlap" in msg


def test_every_documented_launch_option_is_implemented_both_ways():
    """The launch options listed in include/holstein.h (hol_set_option) are
    exactly those hol_set_option and hol_get_option accept: a documented
    option the library does not know, or an accepted one the header does not
    describe, fails here."""
    header = open(os.path.join(ROOT, "include", "holstein.h")).read()
    a = header.index("Runtime launch options of a context")
    b = header.index("*/", a)
    documented = set(re.findall(r'^ \*   "([a-z0-9_]+)"', header[a:b], flags=re.M))
    src = open(os.path.join(ROOT, "paper_2203_01291_gb300", "csrc", "context.cu")).read()
    s0 = src.index("int hol_set_option(")
    g0 = src.index("int hol_get_option(")
    setter = set(re.findall(r'is\("([a-z0-9_]+)"\)', src[s0:g0]))
    getter = set(re.findall(r'is\("([a-z0-9_]+)"\)', src[g0:]))
    assert documented and documented == setter == getter, (documented ^ setter,
                                                           documented ^ getter)


def _prototypes():
    """name -> number of parameters of every function declared in include/."""
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^(?!typedef|#)[\w \t*]+?\b(\w+)\s*\(([^;{]*?)\)\s*;", src,
                             flags=re.M | re.S):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_and_definitions_match_the_header_prototypes():
    """Every function the header declares has a definition in csrc/ with
    extern "C" linkage and the ctypes prototype of the binding takes as many
    arguments as the header's declaration (an argument added to one side
    only fails here, without a GPU); no extern "C" definition is left out of
    the header."""
    from paper_2203_01291_gb300 import _abi
    protos = _prototypes()
    assert set(protos) == set(declared_functions())
    for name, n in protos.items():
        assert len(_abi.SIGNATURES[name][1]) == n, (name, n, len(_abi.SIGNATURES[name][1]))
    defined = set()
    csrc = os.path.join(ROOT, "paper_2203_01291_gb300", "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh")):
            defined |= set(re.findall(r'extern "C"[\w \t*]+?\b(\w+)\s*\(',
                                      open(os.path.join(csrc, f)).read()))
    assert defined == set(protos), (defined ^ set(protos))
