"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/sft.h declares; argument validation that happens
before any CUDA call is checked here (no compute)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sft_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    from paper_1407_8315_gb300 import sft
    return sft.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"sft_plan_create", "sft_exact", "sft_exact_host", "sft_plan_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    """The binding names exactly the entry points the header declares."""
    from paper_1407_8315_gb300 import sft
    assert set(sft.EXPORTS) == _declared()


def test_strerror(lib):
    from paper_1407_8315_gb300 import sft
    assert lib.sft_strerror(sft.SFT_OK) == b"SFT_OK"
    assert b"EINVAL" in lib.sft_strerror(sft.SFT_EINVAL)


def test_params_default(lib):
    from paper_1407_8315_gb300 import sft
    p = sft.sft_params_default(1 << 22, 4096, 512, "iter", "mixed")
    assert (p.N, p.K, p.d, p.a_max, p.max_iters) == (1 << 22, 4096, 512, 4, 4)
    assert p.zero_tol == 1e-6 and p.res_tol == 1e-6 and p.root_tol == 0.1
    p = sft.sft_params_default(1 << 16, 64, 256, "fixed", "fp64")
    assert p.zero_tol == 1e-10 and p.res_tol == 1e-9


@pytest.mark.parametrize("field,value,status", [
    ("N", 1000, 1), ("N", 4, 1), ("d", 3, 1), ("d", 1 << 23, 1), ("a_max", 9, 1),
    ("max_iters", 5, 1), ("mode", 7, 1), ("precision", 9, 1), ("reserved_", 1, 1),
])
def test_plan_create_rejects_before_touching_the_gpu(lib, field, value, status):
    from paper_1407_8315_gb300 import sft
    p = sft.sft_params_default(1 << 22, 4096, 512, "iter", "mixed")
    setattr(p, field, value)
    h = C.c_void_p()
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == status
    assert h.value is None


@pytest.mark.parametrize("r,d", [(17, 32), (9, 8), (-1, 32)])
def test_general_plan_rejects_bad_shift_counts(lib, r, d):
    """r random shifts must be 1..16 and no more than d (they are distinct)."""
    from paper_1407_8315_gb300 import sft
    p = sft.sft_params_default(1 << 20, 1024, d, "general", "mixed")
    assert p.a_max == 3 and p.n_cs_shifts == 9
    p.n_cs_shifts = r
    h = C.c_void_p()
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EINVAL


def test_unpruned_plan_defaults_and_limits(lib):
    """The CS model without pruning takes the general defaults (a_m = 3,
    r = 9) and a shared-memory table of d roots: d above 4096 is refused."""
    from paper_1407_8315_gb300 import sft
    p = sft.sft_params_default(1 << 20, 16, 8192, "general-unpruned", "mixed")
    assert p.mode == sft.SFT_GENERAL_UNPRUNED and p.a_max == 3 and p.n_cs_shifts == 9
    h = C.c_void_p()
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED
    p.n_cs_shifts = 17
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EINVAL


def test_more_than_four_aliases_only_on_the_exact_paths(lib):
    """a_max up to 8 is valid for the exact modes; the general modes keep
    a_max <= 4 (SFT_EUNSUPPORTED)."""
    from paper_1407_8315_gb300 import sft
    h = C.c_void_p()
    p = sft.sft_params_default(1 << 20, 1024, 32, "general", "mixed")
    p.a_max = 5
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED
    p = sft.sft_params_default(1 << 20, 1024, 256, "fixed", "mixed")
    p.a_max = 9
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EINVAL
    p.a_max = 6  # FIXED decodes from 2 a_max = 16 syndromes only at a_max = 8
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED


def test_more_than_four_levels_need_complex128_input(lib):
    """ITER above four levels (5..8 aliases among 2^l d candidates) is
    offered for complex128 input only: on complex64 input the input's
    rounding decides which borderline bins validate there, so the mixed form
    refuses it (SFT_EUNSUPPORTED); FIXED at a_max = 8 stays available."""
    from paper_1407_8315_gb300 import sft
    h = C.c_void_p()
    p = sft.sft_params_default(1 << 18, 1024, 256, "iter", "mixed")
    p.a_max, p.max_iters = 8, 8
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED
    assert "SFT_FP64" in lib.sft_last_cuda_error().decode()
    p.max_iters = 5
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED


def test_plan_create_rejects_too_many_bins(lib):
    """N/d = 2^27 bins is above the four-step FFT limit (2^26)."""
    from paper_1407_8315_gb300 import sft
    p = sft.sft_params_default(1 << 28, 4096, 2, "iter", "mixed")
    h = C.c_void_p()
    assert lib.sft_plan_create(C.byref(p), 1, C.byref(h)) == sft.SFT_EUNSUPPORTED


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.sft_plan_create(None, 1, C.byref(h)) == 1
    assert lib.sft_params_default(None, 8, 1, 1, 0, 0) == 1
    assert lib.sft_exact(None, 1, None, 0, None, None) == 1
    assert lib.sft_plan_workspace_bytes(None) == 0
    assert lib.sft_plan_set_quad_decoders(None, 1) == 1


def test_mlp_config_and_create_validation(lib):
    """The learned proposal's dimensions follow the general plan; bad shapes
    are rejected before any device memory is touched."""
    import ctypes as C
    from paper_1407_8315_gb300 import sft
    c = sft.sft_mlp_config()
    p = sft.sft_params_default(1 << 20, 1024, 32, "general", "mixed")
    assert lib.sft_mlp_config_for(C.byref(p), C.byref(c)) == sft.SFT_OK
    assert (c.n_in, c.n_hidden, c.n_sup, c.n_cls) == (30, 128, 32, 5)
    p.a_max, p.n_cs_shifts = 4, 12
    assert lib.sft_mlp_config_for(C.byref(p), C.byref(c)) == sft.SFT_OK
    assert (c.n_in, c.n_cls) == (40, 6)
    big = sft.sft_params_default(1 << 27, 1 << 16, 512, "general", "mixed")
    assert lib.sft_mlp_config_for(C.byref(big), C.byref(c)) == sft.SFT_EUNSUPPORTED
    ex = sft.sft_params_default(1 << 16, 64, 256, "iter", "mixed")
    assert lib.sft_mlp_config_for(C.byref(ex), C.byref(c)) == sft.SFT_EINVAL
    h = C.c_void_p()
    bad = sft.sft_mlp_config(30, 64, 32, 5, 0, 1e-3, 0.9, 0.999, 1e-8)
    assert lib.sft_mlp_create(C.byref(bad), C.byref(h)) == sft.SFT_EUNSUPPORTED
    bad = sft.sft_mlp_config(30, 128, 200, 5, 0, 1e-3, 0.9, 0.999, 1e-8)
    assert lib.sft_mlp_create(C.byref(bad), C.byref(h)) == sft.SFT_EINVAL
    bad = sft.sft_mlp_config(30, 128, 32, 5, 0, -1.0, 0.9, 0.999, 1e-8)
    assert lib.sft_mlp_create(C.byref(bad), C.byref(h)) == sft.SFT_EINVAL
    assert lib.sft_plan_attach_mlp(None, None) == sft.SFT_EINVAL


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built CUDA library the binding raises: there is no CPU
    fallback behind the product entry points."""
    import paper_1407_8315_gb300.sft as S
    from paper_1407_8315_gb300 import _build_lib
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(_build_lib, "LIB", "/nonexistent/libsft.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        S.load()


def test_product_code_never_reaches_the_oracle():
    """The library, its header and its binding neither include, import,
    call nor load anything of the oracle (test infrastructure only)."""
    import pathlib
    import re
    root = pathlib.Path(__file__).resolve().parents[1]
    pkg = root / "paper_1407_8315_gb300"
    bad = re.compile(r'#\s*include\s*[<"][^>"]*oracle|^\s*(import|from)\s+oracle\b|'
                     r'sfft_oracle|liboracle|\borc_[a-z0-9_]+\s*\(', re.M)
    files = [p for ext in ("*.py", "*.cu", "*.cuh", "*.h") for p in pkg.rglob(ext)]
    files += list((root / "include").glob("*.h"))
    assert files
    for f in files:
        m = bad.search(f.read_text())
        assert m is None, (str(f), m.group(0))


def test_device_math_check_validates_before_launching(lib):
    """Bad arguments are refused before any CUDA call; n = 0 is a no-op."""
    from paper_1407_8315_gb300 import sft
    assert lib.sft_device_math_check(None, -1, None, 0, None) == sft.SFT_EINVAL
    assert lib.sft_device_math_check(None, 4, None, 0, None) == sft.SFT_EINVAL
    assert lib.sft_device_math_check(None, 0, None, 3, None) == sft.SFT_EINVAL
    assert lib.sft_device_math_check(None, 0, None, 1, None) == sft.SFT_OK
