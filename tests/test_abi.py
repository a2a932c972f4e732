"""The C ABI library builds, loads and exports every entry point that
include/fde.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_1706_06844_gb300 import fde

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fde_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    if not os.path.exists(fde.LIB_PATH):
        from paper_1706_06844_gb300 import build
        build.build()
    lib = ctypes.CDLL(fde.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert set(names) <= set(fde.SIGNATURES)


def test_param_struct_layout_matches_header():
    # fde_params field order in the header and in the binding
    src = open(os.path.join(ROOT, "include", "fde.h")).read()
    body = src[src.index("typedef struct fde_params"):src.index("} fde_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:double|int)\s+([^;]+);", body)
    names = [f.strip() for grp in fields for f in grp.split(",")]
    assert names == [f[0] for f in fde.fde_params._fields_]


def test_argument_errors_without_gpu():
    # fde_create validates on the host before touching the device
    import pytest
    for kw in [dict(alpha=1.0), dict(beta=2.0), dict(qx=1), dict(n1=2), dict(restart=0),
               dict(omega=2.5), dict(rtol=0.0), dict(precond=9)]:
        with pytest.raises(fde.FDEError) as e:
            fde.fde_create(fde.params(**kw))
        assert e.value.code == fde.FDE_ERR_ARG, kw
    for kw in [dict(cycles=5), dict(cycles=-1), dict(relax=2), dict(solver=2), dict(warm=3),
               dict(solver=1, precond=0)]:
        with pytest.raises(fde.FDEError) as e:
            fde.fde_create(fde.params(**kw))
        assert e.value.code == fde.FDE_ERR_ARG, kw


def test_batch_argument_errors_without_gpu():
    # fde_batch_create rejects an empty batch before any CUDA call
    b = ctypes.c_void_p()
    assert fde.lib().fde_batch_create(None, 1, None, ctypes.byref(b)) == fde.FDE_ERR_ARG
    p = (fde.fde_params * 1)(fde.fde_default_params())
    assert fde.lib().fde_batch_create(p, 0, None, ctypes.byref(b)) == fde.FDE_ERR_ARG
    assert not b.value
    assert fde.fde_batch_size(None) == 0
    assert fde.fde_batch_status(None, 0) == fde.FDE_ERR_ARG
    assert fde.lib().fde_batch_step(None, None, None, None, None) == fde.FDE_ERR_ARG
    assert fde.lib().fde_wait_selftest(None, 0) == fde.FDE_ERR_ARG
