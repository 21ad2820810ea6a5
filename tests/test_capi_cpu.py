"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/fic.h declares; host-side helpers.  No compute calls (no GPU
here)."""
import ctypes as C

import numpy as np

from paper_1501_04140_gb300 import build, fic


def test_library_exports_every_declared_function():
    build.build()
    lib = fic.load()
    names = fic.header_functions()
    assert "fic_encode" in names and "fic_match_level" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function also has a binding with the same name
    assert set(names) <= set(fic._SIGS), set(names) - set(fic._SIGS)


def test_struct_layouts_match_header(tmp_path):
    # the binding's structs have the sizes a C compiler gives the header's
    import os
    import subprocess
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "fic.h"\nint main(void) { printf("%zu %zu %zu\\n", '
                   'sizeof(fic_transform), sizeof(fic_params), sizeof(fic_level_stats)); return 0; }\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", hdr, str(src), "-o", str(exe)], check=True)
    c_sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                              check=True).stdout.split()]
    assert c_sizes == [C.sizeof(fic.fic_transform), C.sizeof(fic.fic_params),
                       C.sizeof(fic.fic_level_stats)]
    assert C.sizeof(fic.fic_transform) == 88 == fic.TRANSFORM_DTYPE.itemsize


def test_status_strings_and_defaults():
    fic.load()
    assert fic.status_string(fic.FIC_OK) == "FIC_OK"
    assert "invalid" in fic.status_string(fic.FIC_EINVAL)
    p = fic.default_params()
    assert (p.n_levels, p.range_size0, p.domain_step, p.rms_threshold) == (4, 16, 2, 8.0)
    assert p.s_mode == fic.FIC_S_PREDEFINED and p.precision == fic.FIC_PREC_TENSOR


def test_no_device_fails_loudly():
    """Without a GPU fic_create reports an error; nothing falls back to CPU."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fic.FicError):
        fic.Context(0)


def test_image_descriptor_host_and_pitch():
    a = np.zeros((32, 48), np.uint8)
    d, keep = fic.make_image(a)
    assert (d.width, d.height, d.pitch, d.host) == (48, 32, 48, 1)


def test_binding_constants_match_header():
    """Every FIC_* constant the binding defines has the value include/fic.h
    gives it (status codes, modes, pool fields, the static decoder's limits)."""
    import re
    txt = open(fic.HEADER).read()
    defs = dict(re.findall(r"#define (FIC_[A-Z0-9_]+) \(?([-0-9 *()]+?)\)?\s*(?:/\*|\n)", txt))
    checked = 0
    for name, expr in defs.items():
        if hasattr(fic, name):
            assert getattr(fic, name) == eval(expr, {}), name
            checked += 1
    assert checked >= 15
    assert fic.FIC_DECODE_STATIC_MAX_PIXELS == 1024 * 1024
