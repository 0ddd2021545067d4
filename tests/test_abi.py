"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/m2l.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "m2l.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(m2l_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l
    return m2l.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("m2l_precompute", "m2l_apply_level", "m2l_apply_level_adjoint", "m2l_apply_batch",
                     "m2l_ops_query", "m2l_ops_free", "m2l_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    from paper_1210_7292_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_precompute_rejects_bad_arguments_on_host(lib):
    from paper_1210_7292_gb300 import m2l
    for kt, ell, eps, width in [(0, 1, 0.0, 0.0), (0, 9, 0.0, 0.0), (7, 4, 0.0, 0.0), (0, 4, 1.5, 0.0),
                                (0, 4, -1.0, 0.0), (2, 4, 0.0, 0.0), (2, 4, 0.0, -1.0)]:
        for fn in (m2l.m2l_precompute, m2l.m2l_precompute_aca):
            with pytest.raises(m2l.M2LError) as ei:
                fn(kt, ell, eps, width)
            assert ei.value.status == m2l.M2L_EINVAL
        assert m2l.m2l_last_error()


def test_null_handles_rejected(lib):
    from paper_1210_7292_gb300 import m2l
    assert lib.m2l_ops_query(None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_plan_apply(None, None, None, 1, 0, None) == m2l.M2L_EINVAL
    assert lib.m2l_apply_level(None, None, None, None, 1, 0, None) == m2l.M2L_EINVAL
    assert lib.m2l_build_lists(-1, None, 0, None, None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_plan_classify(None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_ops_prepare(None, 1, None) == m2l.M2L_EINVAL
    assert lib.m2l_fmm_create(None, 0, None, 0, 3, -1.0, 2.0, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_fmm_evaluate(None, None, None, None, 1, None) == m2l.M2L_EINVAL
    assert lib.m2l_fmm_info(None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_sa_create(None, 1e-5, 0, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_sa_info(None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_sa_copy_factors(None, None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_sa_apply_level(None, None, None, None, 1, 0, None) == m2l.M2L_EINVAL
    lib.m2l_sa_free(None)
    assert lib.m2l_dfmm_build_lists(-1, 1.0, 2.0, 0, None, 0, None, None, None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_dfmm_plan_create(4, 1.0, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_dfmm_plan_info(None, None, None, None, None, None) == m2l.M2L_EINVAL
    assert lib.m2l_dfmm_plan_apply(None, None, None, 1, None) == m2l.M2L_EINVAL
    assert lib.m2l_dfmm_plan_prepare(None, 3, None) == m2l.M2L_EINVAL
    assert lib.m2l_dfmm_plan_sync(None, None) == m2l.M2L_EINVAL
    lib.m2l_dfmm_plan_free(None)
    assert lib.m2l_ops_aca_info(None, None, None) == m2l.M2L_EINVAL
    lib.m2l_fmm_free(None)
    lib.m2l_ops_free(None)
    lib.m2l_plan_free(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1210_7292_gb300 import m2l
    monkeypatch.setattr(m2l, "_lib", None)
    monkeypatch.setattr(m2l, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        m2l.lib()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1210_7292_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "m2l_oracle" not in text, f


def test_binding_rejects_vectors_on_another_device(monkeypatch):
    """Operators built on one device are never used with tensors, lists or a
    stream of another: the binding raises before it reaches the library (the
    library refuses the same call itself when the current device differs)."""
    from types import SimpleNamespace as NS

    from paper_1210_7292_gb300 import m2l

    def no_library():
        raise AssertionError("the library was called")
    monkeypatch.setattr(m2l, "lib", no_library)

    def tensor(dev, rows, cols=64):
        return NS(device=NS(index=dev), shape=(rows, cols))
    ops = NS(handle=None, ell=4, n3=64, device=0)

    def level(dev):
        return NS(struct=NS(ncells_src=8, ncells_tgt=8), tgt_ijk=tensor(dev, 8, 3), src_ijk=tensor(dev, 8, 3),
                  il_offsets=tensor(dev, 9, 1), il_sources=tensor(dev, 0, 1))
    for lv, mp, loc in ((level(1), tensor(0, 8), tensor(0, 8)), (level(0), tensor(1, 8), tensor(0, 8)),
                        (level(0), tensor(0, 8), tensor(1, 8))):
        for call in (lambda: m2l.m2l_apply_level(ops, lv, mp, loc, "fp32"),
                     lambda: m2l.m2l_apply_level_adjoint(ops, lv, loc, mp, "fp32"),
                     lambda: m2l.m2l_apply_level_noalloc(ops, lv, mp, loc)):
            with pytest.raises(ValueError, match="device"):
                call()
    with pytest.raises(ValueError, match="stream"):
        m2l._stream_ptr(NS(device=NS(index=1), cuda_stream=0), 0)
