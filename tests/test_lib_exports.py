"""CPU checks of the C-ABI library: it loads, and it exports every entry
point that include/pdcloth.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdcloth.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_19272_gb300 import build
    return build.build()


def test_header_declares_api():
    names = declared()
    for must in ("pdc_create", "pdc_step", "pdc_get_positions", "pdc_get_stats", "pdc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pdc_[a-z_0-9]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2403_19272_gb300 import pdcloth
    L = pdcloth.lib()  # loads the .so (no CUDA call happens at load)
    for n in declared():
        assert n in pdcloth.SIGNATURES, n
        assert hasattr(L, n)


def test_struct_layouts_match_header(libpath):
    """pdc_default_params only writes host memory: check a few fields land
    where the header puts them."""
    from paper_2403_19272_gb300 import pdcloth
    p = pdcloth.pdc_default_params()
    assert abs(p.dt - 1 / 200) < 1e-15
    assert p.gravity[2] == -9.8
    assert p.samples_vt == 3 and p.samples_ee == 4
    assert p.a_max == 20 and p.collisions == 1 and p.seed == 12345
