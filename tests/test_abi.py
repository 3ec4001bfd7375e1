"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/lbm.h declares; the ctypes mirrors have the C layouts."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_00907_gb300 import build as B
from paper_2506_00907_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_[a-z_0-9]+)", out))
    declared = declared_functions()
    assert len(declared) >= 18
    missing = [f for f in declared if f not in exported]
    assert not missing, missing


def test_library_loads_and_binds_without_gpu(libpath):
    L = lbm.lib()
    for f in declared_functions():
        assert getattr(L, f) is not None
    # a pure host call: the error string of a NULL context
    assert isinstance(L.lbm_last_error(None), bytes)


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "lbm.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(lbm_link), sizeof(lbm_case),'
                   ' sizeof(lbm_config), offsetof(lbm_link, d), offsetof(lbm_case, rho0));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == lbm.LINK_DTYPE.itemsize == 64
    assert vals[1] == ctypes.sizeof(lbm.lbm_case)
    assert vals[2] == ctypes.sizeof(lbm.lbm_config)
    assert vals[3] == lbm.LINK_DTYPE.fields["d"][1]
    assert vals[4] == lbm.lbm_case.rho0.offset


def test_create_without_gpu_fails_loudly():
    """On a machine without a GPU the solver raises instead of falling back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    case = lbm.make_case((4, 4, 1), 0.8)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(lbm.LBM_D2Q9, lbm.LBM_FP32, lbm.LBM_FLOW, [case], None, 0)


def test_wall_kind_values_agree_with_the_header():
    """The link-kind and field values are part of the link interface: the
    header's enum, the binding's constants and the oracle's constants (which
    shares no code with the product) must name the same numbers."""
    import oracle as O
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef enum \{(.*?)\} lbm_wall_kind;", text, flags=re.S).group(1)
    header = {name: int(v) for name, v in re.findall(r"(LBM_W_[A-Z0-9_]+)\s*=\s*(\d+)", body)}
    assert header == {k: getattr(lbm, k) for k in header}
    oracle_names = {"LBM_W_VELOCITY": O.VELOCITY, "LBM_W_GIVEN": O.GIVEN, "LBM_W_FLUX": O.FLUX,
                    "LBM_W_NEUMANN_BFL": O.NEUMANN_BFL, "LBM_W_VELOCITY_EQ15": O.VELOCITY_EQ15,
                    "LBM_W_FLUX_SIMPLIFIED": O.FLUX_SIMPLIFIED, "LBM_W_PRESSURE": O.PRESSURE,
                    "LBM_W_REACTION": O.REACTION}
    assert set(oracle_names) == set(header)
    for k, v in oracle_names.items():
        assert header[k] == v, k
    # concentration species fields: the header's macro, the binding and the oracle
    for k in range(3):
        assert lbm.field_species(k) == O.species_field(k) == (1 if k == 0 else 4 + k)
