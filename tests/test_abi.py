"""The C-ABI library builds, loads and exports every entry point that
include/dspg.h declares (no GPU needed; no compute call is made)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "dspg.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dspg_[a-z_A-Z]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("dspg_build", "dspg_apply_batch", "dspg_read_C", "dspg_destroy", "dspg_last_error"):
        assert name in syms


def test_library_loads_and_exports_all_declared_symbols():
    import paper_2202_08808_gb300 as pkg
    lib = pkg.load()
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in dspg.h but not exported"
    # the exported list of the binding covers the header too
    assert set(declared_symbols()) == set(pkg.EXPORTED)
    raw = ctypes.CDLL(pkg.library_path())
    for name in declared_symbols():
        getattr(raw, name)


def test_library_is_built_for_sm103a():
    from paper_2202_08808_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_last_error_without_handle_is_callable():
    import paper_2202_08808_gb300 as pkg
    lib = pkg.load()
    assert isinstance(lib.dspg_last_error(None), bytes)


def _struct_fields(name):
    with open(os.path.join(ROOT, "include", "dspg.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split(None, 2)[2]
        for n in names.split(","):
            fields.append(n.strip().lstrip("*").strip())
    return fields


def test_binding_structs_mirror_the_header():
    """ctypes mirrors must list the header's fields in order (a missing field
    makes the library write past the Python-side struct)."""
    from paper_2202_08808_gb300 import dspg as b
    assert [f for f, _ in b._Stats._fields_] == _struct_fields("dspg_batch_stats")
    assert [f for f, _ in b._Opt._fields_] == _struct_fields("dspg_options")
    assert [f for f, _ in b._Csr._fields_] == _struct_fields("dspg_csr")
    assert [f for f, _ in b._Upd._fields_] == _struct_fields("dspg_updates")
    assert [f for f, _ in b._Tuning._fields_] == _struct_fields("dspg_tuning")
    assert [f for f, _ in b._Form._fields_] == _struct_fields("dspg_form")


def test_tuning_candidates_start_with_the_defaults_and_stay_in_range():
    """The autotuner's list (host data, no GPU call): the first candidate is
    the documented default, and every candidate keeps each hash table at or
    above the bound (the ranges that make any tuning give the same C)."""
    import paper_2202_08808_gb300 as pkg
    cands = pkg.tuning_candidates()
    assert len(cands) >= 8
    assert cands[0] == dict(merge_k=8, merge_ub=64, lanes_min=8, table_shift=0, warp_max=1024, cta_max=16384,
                            sort_max=64)
    for c in cands:
        assert 0 <= c["merge_k"] <= 8 and 0 <= c["merge_ub"] <= 64
        assert c["lanes_min"] in (8, 16, 32) and c["table_shift"] in (0, 1)
        assert 0 <= c["warp_max"] <= 1024 and 0 <= c["cta_max"] <= 16384
        assert 0 <= c["sort_max"] <= 256
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)


def test_host_result_arrays():
    """Arrays the binding reads results into: the asked length and dtype
    (page-locked when a GPU is there, plain numpy memory otherwise)."""
    import numpy as np
    from paper_2202_08808_gb300 import dspg as b
    for dt in (np.int64, np.int32, np.float64):
        a = b._host_empty(7, dt)
        assert a.shape == (7,) and a.dtype == np.dtype(dt)
    assert b._host_empty(0, np.int32).shape == (0,)
