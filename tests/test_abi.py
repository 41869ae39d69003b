"""The C ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no GPU calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//.*", "", src)
        for m in re.finditer(r"\b((?:sim|srv)_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sim_create", "sim_apply_circuit", "sim_probabilities", "sim_expectation", "sim_top_k"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = built_lib
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_symbols_are_c_linkage(built_lib):
    from paper_2604_12256_gb300 import svsim as S
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in declared_functions():
        assert n in exported, n


def test_errors_without_gpu_are_reported(built_lib):
    from paper_2604_12256_gb300 import svsim as S
    import torch
    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    with pytest.raises(S.SimError) as e:
        S.Sim(10, S.SIM_C64)
    assert e.value.code in (S.SIM_ECUDA, S.SIM_ENOMEM)


def test_fault_injection_arguments(built_lib):
    from paper_2604_12256_gb300 import svsim as S
    lib = built_lib
    assert lib.sim_fault_inject(99, 0, 1) == S.SIM_EINVAL
    assert lib.sim_fault_inject(S.SIM_FAULT_ALLOC, 0, -1) == S.SIM_EINVAL
    assert lib.sim_fault_inject(S.SIM_FAULT_ALLOC, -1, 1) == S.SIM_EINVAL
    assert lib.sim_fault_inject(S.SIM_FAULT_ALLOC, 0, 0) == S.SIM_OK
    assert lib.sim_fault_inject(S.SIM_FAULT_LAUNCH, 0, 0) == S.SIM_OK
