"""Host-side checks of the C-ABI library: it builds, loads and exports every
entry point that include/sw.h declares (no GPU call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsw():
    import paper_1801_07823_gb300 as sw
    if not os.path.exists(sw.LIB_PATH):
        from paper_1801_07823_gb300 import build
        build.build_library()
    return sw.lib()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sw_gauge_load", "sw_mg_setup", "sw_dslash", "sw_mg_solve", "sw_mg_solve_batch",
                 "sw_context_create", "sw_last_error", "sw_debug_maps"):
        assert name in syms


def test_library_exports_every_declared_symbol(libsw):
    for name in declared_symbols():
        assert hasattr(libsw, name), name


def test_stream_seed_matches_input_module(libsw):
    import paper_1801_07823_gb300 as sw
    import sw_inputs as si
    for lv, i in [(0, 0), (1, 3), (2, 31)]:
        assert sw.sw_stream_seed(42, lv, i) == si.stream_seed(42, lv, i)


def test_params_default_is_table_kcycle(libsw):
    import paper_1801_07823_gb300 as sw
    p = sw.sw_mg_params_default()
    assert (p.setup_maxiter, p.setup_tol, p.outer_restart, p.smoother_iters, p.omega) == \
        (250, 1e-4, 32, 2, 0.85)
    assert (p.inter_restart, p.inter_maxiter, p.inter_tol) == (8, 16, 0.2)
    assert (p.coarsest_maxiter, p.coarsest_tol) == (256, 0.2)


def test_binding_has_no_fallback(tmp_path, monkeypatch):
    import paper_1801_07823_gb300 as sw
    monkeypatch.setattr(sw, "_LIB", None)
    monkeypatch.setattr(sw, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        sw.lib()
