"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/lbrbc.h declares; the
ctypes parameter struct matches the header's layout; argument validation
fails loudly with a message."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbrbc.h")).read()
    return sorted(set(re.findall(r"\b(lbrbc_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_10794_gb300 import _build, lbrbc

    _build.build()
    return lbrbc.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lbrbc_create" in names and "lbrbc_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2306_10794_gb300 import lbrbc

    for n in _declared():
        assert n in lbrbc.EXPORTED or n.startswith("lbrbc_") and hasattr(lbrbc, n), n


def test_params_struct_layout(tmp_path):
    # the ctypes mirror has the offsets gcc gives the C declaration
    import subprocess

    from paper_2306_10794_gb300 import lbrbc

    P = lbrbc.lbrbc_params
    src = tmp_path / "off.c"
    fields = [f[0] for f in P._fields_]
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbrbc.h"\nint main(void){\n' +
                   "".join('printf("%%zu\\n", offsetof(lbrbc_params, %s));\n' % f for f in fields) +
                   'printf("%zu\\n", sizeof(lbrbc_params)); return 0;}\n')
    exe = tmp_path / "off"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got[:-1] == [getattr(P, f).offset for f in fields]
    assert got[-1] == ctypes.sizeof(P)
    txt = open(os.path.join(ROOT, "include", "lbrbc.h")).read()
    body = txt[txt.index("typedef struct {\n    int dim;"):txt.index("} lbrbc_params;")]
    decl = re.findall(r"^\s*(int|double)\s+([^;]+);", body, re.M)
    names = []
    for _, group in decl:
        for part in group.split(","):
            part = part.split("/*")[0].strip()
            names.append(re.sub(r"\[.*\]", "", part).strip())
    assert names == [f[0] for f in P._fields_]


def test_invalid_arguments_fail_loudly(lib):
    from paper_2306_10794_gb300 import lbrbc

    mask = np.zeros((4, 4, 4), np.uint8)
    for bad in (dict(tau_solute=0.5), dict(rest_fraction=1.0), dict(k_r=-1.0), dict(dim=4),
                dict(flow_q=9), dict(bc=("periodic", "open", "periodic"))):
        p = dict(nx=4, ny=4, nz=4)
        p.update(bad)
        with pytest.raises(lbrbc.LbrbcError) as ei:
            lbrbc.lbrbc_create(lbrbc.make_params(p), mask)
        assert ei.value.status in (lbrbc.LBRBC_ERR_ARG,), str(ei.value)
        assert len(str(ei.value)) > 20


def test_no_cpu_fallback_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2306_10794_gb300 import lbrbc

    with pytest.raises(lbrbc.LbrbcError) as ei:
        lbrbc.Sim(dict(nx=4, ny=4, nz=4), np.zeros((4, 4, 4), np.uint8))
    assert ei.value.status == lbrbc.LBRBC_ERR_CUDA
