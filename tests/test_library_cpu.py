"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/gbstencil.h.  Host-only logic is checked here;
nothing launches a kernel."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2404_02218_gb300 import native as N
from oracle.weights import central_weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gbstencil.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*(?:\s+|\s*\*\s*)([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in {"if", "for", "while", "return", "sizeof"}))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("stencil_create", "stencil_set_field", "stencil_run", "stencil_get_field",
                 "stencil_destroy", "stencil_reduce_f64", "stencil_set_source", "stencil_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = N.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", N.lib_path()], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)


def test_library_is_built_for_sm103a():
    from paper_2404_02218_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(N.lib_path())


@pytest.mark.parametrize("so", [2, 4, 8, 12])
def test_product_weights_match_exact_rationals(so):
    w = N.stencil_fd_weights(so)
    ref = [float(x) for x in central_weights(so)]
    assert w == pytest.approx(ref, rel=4e-16, abs=1e-16)


def test_bad_space_order_is_einval():
    with pytest.raises(N.GbstError) as e:
        N.stencil_fd_weights(3)
    assert e.value.status == N.GBST_EINVAL
    assert "space_order" in N.last_error()


def test_version():
    assert N.gbst_version() >= 10000
