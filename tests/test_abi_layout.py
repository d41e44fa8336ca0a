"""The binding's view of the C ABI matches include/rankfhe.h (no GPU needed): the
parameter struct's fields in declaration order, and every RK_ constant the binding
restates (layouts, masks, key kinds, tie flags, options, serving operations)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header():
    with open(os.path.join(ROOT, "include", "rankfhe.h")) as f:
        return f.read()


def _params_fields(text):
    body = re.search(r"typedef struct \{(.*?)\} rk_params;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"uint32_t\s+([a-z0-9_]+)\s*;", body)


def _defines(text):
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define RK_([A-Z0-9_]+)\s+(\d+)u?\b", text)}


def test_params_struct_matches_the_header():
    from paper_2412_15126_gb300 import build
    build.build()
    from paper_2412_15126_gb300 import rankfhe
    fields = _params_fields(_header())
    assert fields == [name for name, _ in rankfhe.Params._fields_]
    assert all(t is ctypes.c_uint32 for _, t in rankfhe.Params._fields_)
    assert ctypes.sizeof(rankfhe.Params) == 4 * len(fields)
    assert "prime_form" in fields


def test_binding_constants_match_the_header():
    from paper_2412_15126_gb300 import build
    build.build()
    from paper_2412_15126_gb300 import rankfhe
    defs = _defines(_header())
    checked = 0
    for name, value in defs.items():
        if hasattr(rankfhe, name):
            assert getattr(rankfhe, name) == value, name
            checked += 1
    # every option, mask, tie flag and serving operation the header defines is restated
    for prefix in ("OPT_", "MASK_", "TIES_", "OP_", "LAYOUT_", "KEY_"):
        for name in defs:
            if name.startswith(prefix):
                assert hasattr(rankfhe, name), name
    assert checked >= 30
