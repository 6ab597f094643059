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
    # dependent launches on, residual forwarding off (8 iterations when enabled)
    assert p.launch_overlap == 1 and p.rf_toi == 0.0 and p.rf_iters == 8
    assert p.tensor_cores == 1 and p.bp_reuse == 0.0
    # LG loops as graphs; fixed partial-CCD patterns, one line-search fraction, no autotuning
    assert p.loop_control == 1 and p.pccd_adaptive == 0 and p.pccd_max_axis == 64
    assert p.instance_line_search == 0 and p.autotune == 0 and p.graph_unroll == 1 and p.loop_ahead == 1 and p.cheb_source == -1 and p.residual_patch == 1


def test_binding_structs_have_the_header_layout(tmp_path):
    """Every field of the ctypes structures sits at the offset (and every
    structure has the size) that a C compiler gives the header's struct."""
    import ctypes
    from paper_2403_19272_gb300 import pdcloth
    structs = [pdcloth.pdc_mesh_desc, pdcloth.pdc_material, pdcloth.pdc_params, pdcloth.pdc_stats,
               pdcloth.pdc_kernel_time, pdcloth.pdc_tuning]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pdcloth.h"', "int main(void) {"]
    for S in structs:
        t = S.__name__
        lines.append(f'printf("{t} %zu\\n", sizeof({t}));')
        for f, _ in S._fields_:
            lines.append(f'printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    try:
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no C compiler")
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for S in structs:
        t = S.__name__
        assert int(got[t]) == ctypes.sizeof(S), t
        for f, _ in S._fields_:
            assert int(got[f"{t}.{f}"]) == getattr(S, f).offset, (t, f)
