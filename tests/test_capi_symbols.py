"""The C-ABI library builds, loads and exports every function include/exa.h declares (no GPU needed)."""
import ctypes
import os
import re

from paper_1908_06936_gb300 import build as exa_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(exa_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["exa_loglik", "exa_loglik_grad", "exa_loglik_batched", "exa_ctx_create", "exa_ctx_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = exa_build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    import paper_1908_06936_gb300 as exa

    missing = [n for n in declared_functions() if not callable(getattr(exa, n, None))]
    assert not missing, missing


def test_setters_reject_a_null_context():
    # host-side argument checks: every option setter returns EXA_ERR_ARG for a NULL context
    # without touching the device
    import paper_1908_06936_gb300 as exa

    calls = [
        lambda: exa.exa_ctx_set_mixed_band(0, 1),
        lambda: exa.exa_ctx_set_lookahead(0, 16),
        lambda: exa.exa_ctx_set_panel_fusion(0, 1),
        lambda: exa.exa_ctx_set_tc_pairs(0, 1),
        lambda: exa.exa_ctx_set_far_tile_margin(0, 16),
        lambda: exa.exa_ctx_set_model(0, 0.0, 0, 0.0),
    ]
    for call in calls:
        assert call() == exa.EXA_ERR_ARG


def header_enum(name):
    src = open(os.path.join(ROOT, "include", "exa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\}\s*" + name + ";", src).group(1)
    return {k: int(v) for k, v in re.findall(r"(EXA_\w+)\s*=\s*(\d+)", body)}


def test_binding_enums_match_the_header():
    # the precision and status codes the binding passes are the header's, and the precision
    # codes are the boundary's: FP64 0, FP32 1, BF16x3 2, TF32x3 3
    import paper_1908_06936_gb300 as exa

    prec = header_enum("exa_prec")
    assert prec == {"EXA_FP64": 0, "EXA_MIXED_FP32": 1, "EXA_MIXED_BF16X3": 2, "EXA_MIXED_TF32X3": 3}
    for k, v in list(prec.items()) + list(header_enum("exa_status").items()) + list(header_enum("exa_gemm_kind").items()):
        assert getattr(exa, k) == v, k


def header_prototypes():
    """{name: (return type, [parameter types])} of every function include/exa.h declares."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(exa_\w+)\s*\(([^;{)]*)\)\s*;", src):
            ps = []
            for p in params.split(","):
                p = " ".join(p.split())
                if not p or p == "void":
                    continue
                if "[" in p:  # an array parameter is a pointer
                    ps.append("*")
                    continue
                ps.append(re.sub(r"\s*\b\w+$", "", p) if re.search(r"[\w\*]\s+\w+$|\*\s*\w+$", p) else p)
            out[name] = (" ".join(ret.split()), ps)
    return out


def _c_kind(t):
    """(kind, bytes) of a C type as the header spells it; kind is 'ptr', 'int', 'float' or None (void)."""
    t = t.replace("const", "").strip()
    if "*" in t:
        return ("ptr", ctypes.sizeof(ctypes.c_void_p))
    table = {"void": (None, 0), "int": ("int", 4), "int32_t": ("int", 4), "int64_t": ("int", 8),
             "long long": ("int", 8), "size_t": ("int", 8), "double": ("float", 8), "float": ("float", 4),
             "exa_status": ("int", 4), "exa_prec": ("int", 4), "exa_gemm_kind": ("int", 4)}
    assert t in table, "type not mapped: %r" % t
    return table[t]


def _ctypes_kind(ct):
    if ct is None:
        return (None, 0)
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ct, ctypes._Pointer):
        return ("ptr", ctypes.sizeof(ctypes.c_void_p))
    if ct in (ctypes.c_double, ctypes.c_float):
        return ("float", ctypes.sizeof(ct))
    return ("int", ctypes.sizeof(ct))


def test_binding_signatures_match_the_header():
    # every argument the binding marshals has the kind and width the prototype declares, in order,
    # and the return types agree: a wrong width or a dropped argument would corrupt the call
    import paper_1908_06936_gb300 as exa

    L = exa.lib()
    protos = header_prototypes()
    assert len(protos) == len(declared_functions())
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        want = [_c_kind(p) for p in params]
        got = [_ctypes_kind(a) for a in f.argtypes]
        assert got == want, (name, params, f.argtypes)
        assert _ctypes_kind(f.restype) == _c_kind(ret), (name, ret, f.restype)
