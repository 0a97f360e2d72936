"""The C-ABI library builds, loads, exports every entry point of
include/cams.h, and refuses bad arguments without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cams.h")
LIB = os.path.join(ROOT, "paper_1705_05783_gb300", "_lib", "libcams.so")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(cams_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1705_05783_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1705_05783_gb300 import cams
    assert sorted(cams.EXPORTS) == _declared()
    for n in cams.EXPORTS:
        assert callable(getattr(cams, n))


def test_struct_layouts_match_header(tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's
    offsetof for include/cams.h."""
    import subprocess
    from paper_1705_05783_gb300 import cams
    structs = [cams.cams_grid, cams.cams_fluid, cams.cams_bc, cams.cams_options, cams.cams_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cams.h"', 'int main(void){']
    for s in structs:
        lines.append(f'printf("{s.__name__} %zu\\n", sizeof({s.__name__}));')
        for name, _ in s._fields_:
            lines.append(f'printf("{s.__name__}.{name} %zu\\n", offsetof({s.__name__}, {name}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for s in structs:
        assert int(out[s.__name__]) == ctypes.sizeof(s), s.__name__
        for name, _ in s._fields_:
            assert int(out[f"{s.__name__}.{name}"]) == getattr(s, name).offset, (s.__name__, name)


def test_setup_rejects_bad_arguments_before_touching_the_gpu():
    from paper_1705_05783_gb300 import cams
    g = cams.cams_grid(10, 10, 1, 0.1, 0.1, 0.1)
    f = cams.cams_fluid(0, 0.1, 1.0, 1.0, 0.1)
    k = np.ones(100)
    for bad in ((3, 5, 1), (5, 5, 2), (1, 5, 1)):      # not dividing / inactive z / b < 2
        o = cams.make_options(bad)
        with pytest.raises(cams.CamsError) as e:
            cams.cams_setup(g, f, o, k)
        assert e.value.code == cams.CAMS_EINVAL
    o = cams.make_options((5, 5, 1), basis=7)
    with pytest.raises(cams.CamsError) as e:
        cams.cams_setup(g, f, o, k)
    assert e.value.code == cams.CAMS_EINVAL
    assert "basis" in cams.cams_last_error()
    o = cams.make_options((5, 5, 1))
    o.cf = 2
    with pytest.raises(cams.CamsError) as e:
        cams.cams_setup(g, f, o, k)
    assert e.value.code == cams.CAMS_EINVAL
    assert "cf" in cams.cams_last_error()


def test_ensemble_and_network_entry_points_reject_bad_arguments_without_a_gpu():
    """Argument checks of the ensemble, surrogate and network entry points
    come before any CUDA call."""
    import ctypes as C
    from paper_1705_05783_gb300 import cams
    lib = cams._lib
    assert lib.cams_ensemble_solve(-1, None, None, None, None, None, None, None, 0) == cams.CAMS_EINVAL
    assert lib.cams_ensemble_solve(0, None, None, None, None, None, None, None, 0) == cams.CAMS_OK
    assert lib.cams_ensemble_solve(2, None, None, None, None, None, None, None, 0) == cams.CAMS_EINVAL
    assert lib.cams_set_surrogate(None, None, 0.5) == cams.CAMS_EINVAL
    n = C.c_int(7)
    assert lib.cams_surrogate_data(None, 0, None, None, None, C.byref(n)) == cams.CAMS_EINVAL
    assert lib.cams_net_conv_forward(1, 0, 1, 1, None, None, None, 0, None, None) == cams.CAMS_EINVAL
    assert lib.cams_net_conv_backward(0, 4, 1, 1, None, None, None, None, None, None, None,
                                      None) == cams.CAMS_EINVAL
    assert lib.cams_net_mse(0, None, None, None, 1.0, None, None, None, None) == cams.CAMS_EINVAL
    assert lib.cams_net_energy(1, 1, 8, 12, None, None, None, None, 1.0, None, None, None,
                               None) == cams.CAMS_EINVAL
    assert lib.cams_net_adam(10, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 0,
                             None) == cams.CAMS_EINVAL
    assert "Adam" in cams.cams_last_error()


def test_binding_constants_match_header():
    """Every #define CAMS_* integer constant of include/cams.h that the
    binding mirrors has the header's value, and the quantity, status and
    precision constants are all mirrored."""
    from paper_1705_05783_gb300 import cams
    txt = open(HEADER).read()
    defs = dict(re.findall(r"^#define\s+(CAMS_\w+)\s+(-?\d+)", txt, re.M))
    assert len(defs) > 20
    for name, val in defs.items():
        if hasattr(cams, name):
            assert getattr(cams, name) == int(val), name
    for name in defs:
        if name.startswith(("CAMS_Q_", "CAMS_PREC_", "CAMS_E", "CAMS_OK", "CAMS_HOST", "CAMS_DEVICE")):
            assert hasattr(cams, name), name
    # the profile classes, in the header's order
    assert len(cams.PROF_CLASSES) == int(defs["CAMS_PROF_CLASSES"])
    for k, name in enumerate(cams.PROF_CLASSES):
        assert int(defs["CAMS_PROF_" + name.upper()]) == k, name


def test_variant_options_are_checked_before_the_gpu():
    from paper_1705_05783_gb300 import cams
    g = cams.cams_grid(10, 10, 1, 0.1, 0.1, 0.1)
    f = cams.cams_fluid(0, 0.1, 1.0, 1.0, 0.1)
    k = np.ones(100)
    o = cams.make_options((5, 5, 1), jacobian=3)
    with pytest.raises(cams.CamsError) as e:
        cams.cams_setup(g, f, o, k)
    assert e.value.code == cams.CAMS_EINVAL and "jacobian" in cams.cams_last_error()
