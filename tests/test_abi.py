"""The C-ABI library builds, loads and exports every symbol include/amg.h declares.

Runs without a GPU: only host-only entry points are called.
"""
import ctypes
import json
import os
import re

import pytest

from paper_2303_02352_gb300 import amg, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(amg_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return amg.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_follow_listing1(lib):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_settings.json")))
    p = amg.params_default()
    L = gold["listing1"]
    assert p.aggr_steps == L["aggrsweeps"] + 1
    assert p.max_levels == L["max_levels"]
    assert (p.pre_sweeps, p.post_sweeps, p.coarse_sweeps) == (L["prerelax_sweeps"], L["postrelax_sweeps"],
                                                               L["relaxnumber_coarse"])
    assert p.precision == amg.FP64 and p.use_graph == 1


def test_setup_rejects_null_arguments_without_a_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.amg_setup(None, None, None, ctypes.byref(h)) == amg.ERR_INVALID_ARG
    bad = amg.amg_csr(0, 0, None, None, None)
    assert lib.amg_setup(ctypes.byref(bad), None, None, ctypes.byref(h)) == amg.ERR_INVALID_ARG
    assert lib.amg_setup(ctypes.byref(bad), None, None, None) == amg.ERR_INVALID_ARG
    assert isinstance(lib.amg_last_error(None), bytes)
    lib.amg_destroy(None)


def test_structs_match_header_layout(lib):
    src = open(os.path.join(ROOT, "include", "amg.h")).read()
    body = re.findall(r"typedef struct \{([^{}]*?)\} amg_params;", src, re.S)[0]
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert tuple(fields) == amg.PARAM_FIELDS


def test_binding_rejects_non_square_sparse_tensor_before_any_gpu_call():
    import torch
    from paper_2303_02352_gb300 import amg
    A = torch.sparse_csr_tensor(torch.tensor([0, 1, 2]), torch.tensor([0, 1]),
                                torch.tensor([1.0, 1.0], dtype=torch.float64), size=(2, 3))
    with pytest.raises(ValueError, match="square"):
        amg.setup(A)
