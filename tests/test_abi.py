"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function that
include/*.h declares; the Python binding mirrors the parameter struct exactly (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(fas_\w+|ns_\w+|fasb_\w+|gg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2510_11152_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "fas_create" in names and "fas_solve" in names and "fas_heat_run" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib):
    import paper_2510_11152_gb300 as fas
    fas.load()
    for n in _declared():
        assert hasattr(fas, n), "binding lacks %s" % n


def test_default_params_roundtrip(lib):
    import paper_2510_11152_gb300 as fas
    p = fas.fas_default_params()
    assert (p.dim, p.nu1, p.nu2, p.kmax, p.coarsest, p.tol_relative, p.precision) == (2, 2, 2, 20, 4, 1, 0)
    assert p.tol == 1e-10 and p.kappa is None and p.kappa_const == 1.0
    # the ctypes mirror has the C struct's size and field offsets (checked with the C compiler)
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in fas.fas_params._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"fas.h\"\nint main(void){printf(\"%zu\", sizeof(fas_params));"
    src += "".join('printf(" %%zu", offsetof(fas_params, %s));' % f for f in fields) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(fas.fas_params)
    for f, off in zip(fields, out[1:]):
        assert getattr(fas.fas_params, f).offset == int(off), f


def test_create_rejects_bad_sizes_without_gpu(lib):
    import paper_2510_11152_gb300 as fas
    p = fas.make_params((48, 64), 1.0 / 64)
    with pytest.raises(fas.FasError) as e:
        fas.fas_create(p, stream=0)
    assert e.value.status == fas.FAS_EINVAL
    assert "power of two" in fas.fas_last_error()
