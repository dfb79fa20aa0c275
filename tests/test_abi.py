"""The C-ABI library builds, loads and exports every declared symbol; host-side
validation answers without touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import snp_synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "snp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(snp_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol(built_library):
    lib = ctypes.CDLL(built_library)
    names = header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(built_library):
    import paper_1104_1824_gb300 as snp
    assert sorted(snp.EXPORTS) == header_functions()
    for name in header_functions():
        assert callable(getattr(snp, name)), name


def test_binding_declares_every_argument_list(built_library):
    """Every entry point has its argument types declared: without them ctypes
    passes a Python int as a 32-bit C int, which truncates a pointer."""
    import paper_1104_1824_gb300 as snp
    lib = snp.load_library(built_library)
    for name in snp.EXPORTS:
        assert getattr(lib, name).argtypes is not None, name


def test_abi_version_and_defaults(built_library):
    import paper_1104_1824_gb300 as snp
    assert snp.snp_abi_version() == 1
    o = snp.snp_explore_opts_init()
    assert (o.depth, o.transition, o.frontier_cap, o.candidate_budget, o.max_expand_value, o.record_parents,
            o.chunk) == (1, snp.SNP_T_SPARSE_I32, 0, 0, -1, 0, 0)


def test_struct_layouts_match_the_c_header(built_library, tmp_path):
    """ctypes layouts of the binding against sizeof/offsetof from the C compiler."""
    import subprocess
    import paper_1104_1824_gb300 as snp
    structs = {"snp_system_desc": snp.snp_system_desc, "snp_explore_opts": snp.snp_explore_opts,
               "snp_depth_info": snp.snp_depth_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "snp.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


def _desc_args(s):
    return [s.m, s.rule_neuron, s.rule_i, s.rule_j, s.M, s.c0]


@pytest.mark.parametrize("case", ["m0", "neuron_order", "neg_c0", "own_entry", "offdiag", "neg_i", "too_many_rules",
                                  "m_too_big"])
def test_invalid_systems_are_refused_before_any_device_work(built_library, case):
    import paper_1104_1824_gb300 as snp
    s = snp_synth.paper_example()
    m, rn, ri, rj, M, c0 = [np.array(x, copy=True) if not isinstance(x, int) else x for x in _desc_args(s)]
    if case == "m0":
        m = 0
    elif case == "neuron_order":
        rn = rn[::-1].copy()
    elif case == "neg_c0":
        c0[1] = -1
    elif case == "own_entry":
        M[0, 0] = 0
    elif case == "offdiag":
        M[2, 2] = -1
    elif case == "neg_i":
        ri[0] = -1
    elif case == "too_many_rules":
        rn = np.zeros(33, dtype=np.int32)
        ri = np.ones(33, dtype=np.int32)
        rj = np.ones(33, dtype=np.int32)
        M = np.tile(np.array([[-1, 1, 1]], dtype=np.int32), (33, 1))
    elif case == "m_too_big":
        m = 1025
    with pytest.raises(snp.SnpError) as ei:
        snp.snp_load_system(m, rn, ri, rj, M, c0)
    assert ei.value.code == snp.SNP_E_INVALID
    assert snp.snp_last_error()


def test_missing_library_fails_loudly(tmp_path):
    import paper_1104_1824_gb300 as snp
    with pytest.raises(ImportError):
        snp._lib_saved = snp._lib
        try:
            snp._lib = None
            snp.load_library(str(tmp_path / "nope.so"))
        finally:
            snp._lib = snp._lib_saved
