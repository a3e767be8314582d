"""The Python binding's ctypes structures and enum tables against the C
header: a small C program compiled against include/atm3.h prints every
struct's size and field offsets and every enum constant, and the binding
must agree field by field (a mismatch would silently corrupt arguments at
the boundary).  CPU only."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (C type, binding class name, fields in declaration order)
STRUCTS = [
    ("atm_params", "Params", ["box", "rc", "nu", "lj_eps", "lj_sigma", "dt", "lj_shift", "device",
                              "cuda_stream"]),
    ("atm_result", "Result", ["e2", "e3", "w2", "w3", "ekin", "n_cand3", "n_int3", "n_cand2",
                              "n_int2"]),
    ("atm_tuning", "Tuning", ["persistent", "nwarps", "ms_per_eval", "nclass", "cut"]),
    ("atm_profile", "Profile", ["ms_cells", "ms_lj", "ms_atm", "ms_md", "n_launches",
                                "n_atm_launches"]),
]
ENUMS = {
    "TRAVERSALS": {"3c01": "ATM_3C01", "3c18": "ATM_3C18", "3c08": "ATM_3C08", "3cw": "ATM_3CW",
                   "3c08a": "ATM_3C08A"},
    "TRUNCATIONS": {"pair": "ATM_TRUNC_PAIR", "product": "ATM_TRUNC_PRODUCT"},
    "PRECISIONS": {"fp64": "ATM_FP64", "fp32c": "ATM_FP32C", "surrogate": "ATM_SURROGATE"},
}
STATUS_NAMES = ["ATM_OK", "ATM_E_INVALID", "ATM_E_BOX_TOO_SMALL", "ATM_E_CUDA", "ATM_E_TIMEOUT",
                "ATM_E_NONFINITE", "ATM_E_STATE", "ATM_E_CAPACITY", "ATM_E_RANGE"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "atm3.h"', "int main(void) {"]
    for ctype, _, fields in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (ctype, ctype))
        for f in fields:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (ctype, f, ctype, f))
    for names in list(ENUMS.values()) + [dict(enumerate(STATUS_NAMES))]:
        for c in names.values():
            lines.append('printf("%s %%d\\n", (int)%s);' % (c, c))
    lines.append('printf("ATM3_ABI_VERSION %d\\n", ATM3_ABI_VERSION);')
    lines.append("return 0; }")
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    vals = {}
    for line in out.splitlines():
        parts = line.split()
        vals[parts[0] if len(parts) == 2 else parts[0] + " " + parts[1]] = int(parts[-1])
    return vals


def test_structs_match_the_header(c_layout):
    from paper_2510_21230_gb300 import atm3
    for ctype, cls, fields in STRUCTS:
        S = getattr(atm3, cls)
        assert [f for f, _ in S._fields_] == fields, cls
        assert ctypes.sizeof(S) == c_layout[ctype + " size"], ctype
        for f in fields:
            assert getattr(S, f).offset == c_layout["%s.%s" % (ctype, f)], (ctype, f)


def test_enum_tables_match_the_header(c_layout):
    from paper_2510_21230_gb300 import atm3
    for table, names in ENUMS.items():
        py = getattr(atm3, table)
        assert set(py) == set(names), table
        for key, cname in names.items():
            assert py[key] == c_layout[cname], (table, key)
    assert sorted(atm3.STATUS) == [c_layout[c] for c in STATUS_NAMES]
    assert atm3.ABI_VERSION == c_layout["ATM3_ABI_VERSION"]
