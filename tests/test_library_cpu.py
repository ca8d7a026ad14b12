"""No-GPU checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/subquad.h, and its host-only functions agree with
the oracle (the BLOSUM62 tables were typed independently on each side)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libmod():
    from paper_2602_17330_gb300 import _build, subquad

    _build.build()
    subquad.lib()
    return subquad


def declared_entry_points():
    names = []
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(subquad_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported_and_bound(libmod):
    names = declared_entry_points()
    assert len(names) >= 14
    handle = libmod.lib()
    for name in names:
        assert hasattr(handle, name), name
        assert name in libmod.SIGNATURES, f"binding lacks {name}"


def test_builtin_blosum62_matches_oracle_cell_by_cell(libmod, oracle_mod):
    lib_m = np.array(libmod.default_matrix(), dtype=np.int32).reshape(20, 20)
    assert (lib_m == oracle_mod.blosum62()).all()


def test_pack_stride_and_strerror(libmod):
    assert libmod.pack_stride(24) == 16
    assert libmod.pack_stride(30) == 32
    assert libmod.pack_stride(31) == 0
    for st in (0, -1, -2, -4, -5, -6):
        assert libmod.lib().subquad_strerror(st)
    assert libmod.lib().subquad_version() >= 100


def test_create_without_gpu_fails_cleanly(libmod):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes

    h = ctypes.c_void_p()
    st = libmod.lib().subquad_create(ctypes.byref(h), 0, None)
    assert st != 0 and not h.value


def test_default_edit_costs_match_oracle(libmod, oracle_mod):
    """The library derives its default edit costs from its own BLOSUM62 table;
    they must equal the oracle's, derived from the independently typed one."""
    lib_costs = np.array(libmod.default_edit_costs(), dtype=np.uint8).reshape(20, 20)
    assert (lib_costs == oracle_mod.default_edit_costs()).all()


def test_every_entry_point_has_a_context_method(libmod):
    """Each C entry point that runs on a context has a binding method (module
    level wrappers call ctx.<name without the prefix>)."""
    import inspect

    src = inspect.getsource(libmod)
    for name in libmod.SIGNATURES:
        wrapper = f"def {name}(ctx: Context"
        if wrapper in src:
            body = src[src.index(wrapper):].split("\n")[1]
            method = body.strip().split("ctx.")[1].split("(")[0]
            assert hasattr(libmod.Context, method), f"{name}: Context.{method} missing"
