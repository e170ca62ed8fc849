"""The C ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; the binding's constants match the header."""

import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ovs_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0704_3486_gb300 import build
    build.build()
    import paper_0704_3486_gb300 as ovs
    return ovs.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ovs_create_gauge", "ovs_set_mu", "ovs_deflate_setup", "ovs_sign_apply"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_0704_3486_gb300 as ovs
    assert sorted(ovs.EXPORTS) == sorted(n for n in _declared_functions())


def test_enum_values_match_header():
    import paper_0704_3486_gb300 as ovs
    text = open(os.path.join(ROOT, "include", "ovsign.h")).read()
    for code, name in ovs.STATUS.items():
        m = re.search(rf"\b{name}\s*=\s*(-?\d+)", text)
        assert m and int(m.group(1)) == code, name
    assert re.search(r"OVS_F64\s*=\s*0", text) and re.search(r"OVS_MIXED\s*=\s*1", text)
    assert ovs.F64 == 0 and ovs.MIXED == 1


def test_struct_layouts():
    import ctypes

    import paper_0704_3486_gb300 as ovs
    assert ctypes.sizeof(ovs.ApplyOpts) == 24
    assert ctypes.sizeof(ovs.ApplyInfo) == 32


def test_version_and_error_without_gpu(lib):
    assert b"sm_103a" in lib.ovs_version()
    assert isinstance(lib.ovs_last_error(), bytes)


def test_host_argument_checks_without_gpu(lib):
    """Argument errors are reported before any CUDA call."""
    import ctypes

    import paper_0704_3486_gb300 as ovs
    h = ctypes.c_void_p()
    bad = (ctypes.c_int32 * 4)(4, 4, 1, 4)
    assert lib.ovs_create_gauge(bad, 1, 0.5, 0, ctypes.byref(h)) == -1
    assert b"below 2" in lib.ovs_last_error()
    assert lib.ovs_set_mu(None, 0.1, -1.5) == -1
    assert lib.ovs_sign_apply(None, None, None, 1, None, None, None) == -1
    with pytest.raises(ovs.OvsError):
        ovs._check(-1)


def test_stencil_shapes_and_trace_classes_match_header():
    """The binding's shape list is the header's candidate order (the order of
    the times ovs_stencil_tuning returns), and its trace classes are the
    header's OVS_PROF_* values in order."""
    import paper_0704_3486_gb300 as ovs
    text = open(os.path.join(ROOT, "include", "ovsign.h")).read()
    block = text[text.index("The 18 candidates are"):text.index("The first stencil launch")]
    shapes = [tuple(int(v) for v in m) for m in re.findall(r"\((\d+),(\d+),(\d+)\)", block)]
    assert shapes == ovs.STENCIL_SHAPES and len(shapes) == 18
    kernels = open(os.path.join(ROOT, "paper_0704_3486_gb300", "csrc", "kernels.h")).read()
    table = kernels[kernels.index("kStencilShapes[kNumStencilShapes] = {"):]
    table = table[:table.index("};")]
    assert [tuple(int(v) for v in m) for m in re.findall(r"\{(\d+), (\d+), (\d+)\}", table)] == shapes
    classes = re.findall(r"OVS_PROF_([A-Z]+)\s*=\s*(\d+)", text)
    named = {int(v): n.lower() for n, v in classes if n != "NCLASS"}
    assert [named[i] for i in range(len(named))] == ovs.PROF_CLASSES


def test_solve_struct_layouts_and_flags():
    import ctypes
    import re

    import paper_0704_3486_gb300 as ovs
    assert ctypes.sizeof(ovs.SolveOpts) == 16
    assert ctypes.sizeof(ovs.SolveInfo) == 24
    text = open(os.path.join(ROOT, "include", "ovsign.h")).read()
    m = re.search(r"#define\s+OVS_APPLY_HARMONIC\s+(\d+)", text)
    assert m and int(m.group(1)) == ovs.APPLY_HARMONIC
    m = re.search(r"#define\s+OVS_APPLY_SKIP_AHEAD\s+(\d+)", text)
    assert m and int(m.group(1)) == ovs.APPLY_SKIP_AHEAD
