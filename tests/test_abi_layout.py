"""The binding's view of the C ABI matches include/rankfhe.h, and the library's host
code agrees with the oracle (no GPU needed): the parameter struct's fields in
declaration order, every RK_ constant the binding restates (layouts, masks, key kinds,
tie flags, options, serving operations), and the prime chain and canonical scales the
library derives from a parameter set."""
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


def _sets():
    """Every parameter set the tests and the benchmark build contexts from."""
    from tests import helpers
    import bench
    out = []
    for name, cfg in helpers.CONFIGS.items():
        log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, _, _ = cfg
        out.append((name, (log_n, n_limbs, alpha, dsize, log_scale, log_q0, log_sp, helpers.PRIME_FORM.get(name, 0))))
    for name in ("WORKLOAD", "SMALL_WORKLOAD", "ORDER_WORKLOAD", "RING17", "SERVE_RANK", "SERVE_SORT"):
        W = getattr(bench, name)
        out.append((name, (W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                           W["log_special"], W.get("prime_form", 0))))
    return out


def test_library_chain_matches_the_oracle_on_the_host():
    """The library's own prime chain and canonical scales (rk_params_chain, host code,
    no device) equal the oracle's, word for word and double for double, for every
    parameter set used here, both prime forms included."""
    from paper_2412_15126_gb300 import build
    build.build()
    from paper_2412_15126_gb300 import rankfhe
    from oracle import ckks
    for name, (log_n, n_limbs, alpha, dsize, log_scale, log_q0, log_sp, form) in _sets():
        q, sc = rankfhe.params_chain(log_n, n_limbs, alpha, dsize, log_scale, log_q0, log_sp, form)
        P = ckks.gen_params(log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, form)
        assert q == list(P.q) + list(P.p), name
        assert sc == list(P.scales), name


def test_library_chain_rejects_what_a_context_rejects():
    import pytest
    from paper_2412_15126_gb300 import build
    build.build()
    from paper_2412_15126_gb300 import rankfhe
    with pytest.raises(rankfhe.RkError):
        rankfhe.params_chain(16, 28, 3, 3, 30, prime_form=1)     # k 2^32 + 1 primes need scales >= 2^34
    with pytest.raises(rankfhe.RkError):
        rankfhe.params_chain(16, 60, 3, 3, 45)                  # more than 16 digits
