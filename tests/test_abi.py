"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry
point declared in include/fem3.h (no compute call is made here)."""
import ctypes
import os
import re

from paper_1811_03339_gb300 import _build_lib, fem3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fem3.h")).read()
    return sorted(set(re.findall(r"^(?:int|void)\s+\*?(fem3_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol():
    path = _build_lib.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(fem3.SYMBOLS) == declared


def test_binding_loads():
    lib = fem3.load_library()
    buf = ctypes.create_string_buffer(64)
    assert lib.fem3_last_error(buf, 64) == 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1811_03339_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "fem3_oracle" not in src, f


def test_options_struct_matches_header():
    """The binding's fem3_options mirror has the header's fields, in order and type."""
    import ctypes as C
    import re
    from paper_1811_03339_gb300 import fem3
    hdr = open(os.path.join(ROOT, "include", "fem3.h")).read()
    body = hdr[hdr.index("typedef struct fem3_options {"):hdr.index("} fem3_options;")]
    fields = re.findall(r"^\s*(double|int32_t)\s+(\w+);", body, re.M)
    ctype = {"double": C.c_double, "int32_t": C.c_int32}
    assert [(n, ctype[t]) for t, n in fields] == list(fem3.Options._fields_)
