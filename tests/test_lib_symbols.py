"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/amg_gnn.h declares; the Python binding covers them all.
No compute call is made here (no GPU on this side)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "amg_gnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:void|int|long long|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("amg_setup", "amg_load_hierarchy", "gnn_predict_coeffs", "amg_solve", "amg_loss_grad",
                 "gcin_trainer_forward", "gcin_trainer_backward", "amg_residual_norm_noalloc"):
        assert must in names
    assert len(names) >= 30


def test_library_exports_every_declared_symbol():
    from paper_2606_19251_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2606_19251_gb300 as P
    assert sorted(P.api.exported_symbols()) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(P, n)), n


def test_missing_cuda_is_loud():
    # creating a context without a usable GPU reports a CUDA error instead of
    # silently computing on the CPU
    import torch
    import paper_2606_19251_gb300 as P
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.AmgError) as e:
        P.amg_create()
    assert e.value.code == P.AMG_ERR_CUDA


def _header_text():
    src = open(os.path.join(ROOT, "include", "amg_gnn.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def test_binding_constants_match_the_header():
    # every numeric #define the binding mirrors has the header's value
    import paper_2606_19251_gb300 as P
    defines = dict((m.group(1), int(m.group(2)))
                   for m in re.finditer(r"^\s*#define\s+(AMG_\w+)\s+(-?\d+)\s*$", _header_text(), flags=re.M))
    mirrored = [k for k in defines if hasattr(P, k)]
    assert len(mirrored) >= 20, mirrored
    for k in mirrored:
        assert getattr(P, k) == defines[k], k
    for k in ("AMG_SPLIT_SECOND_PASS", "AMG_SPLIT_RS_BLOCKS", "AMG_GNN_BF16", "AMG_FP32_IN_FP64"):
        assert k in mirrored, k


def test_binding_structs_match_the_header():
    # field names, order and C types of amg_options and amg_csr
    import ctypes as C
    from paper_2606_19251_gb300 import api
    ctype = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong}
    src = _header_text()
    m = re.search(r"typedef struct \{([^}]*)\}\s*amg_options;", src)
    fields = re.findall(r"(int|double|long long)\s+(\w+)\s*;", m.group(1))
    assert [n for _, n in fields] == [f[0] for f in api.amg_options._fields_]
    for (t, n), (bn, bt) in zip(fields, api.amg_options._fields_):
        assert bt == ctype[t], n
    m = re.search(r"typedef struct \{([^}]*)\}\s*amg_csr;", src)
    names = re.findall(r"(\w+)\s*;", m.group(1))
    assert names == [f[0] for f in api.amg_csr._fields_]
