"""The C-ABI library loads, exports every entry point include/edgb.h declares,
and the Python structures match the C layout (CPU only: no compute calls)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

import paper_2105_06806_gb300 as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "edgb.h")


def _built():
    if not os.path.exists(E.LIB_PATH):
        from paper_2105_06806_gb300 import _build
        _build.build()
    return E.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ed_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    L = _built()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(E.EXPORTED) == names


def test_status_strings_without_gpu():
    L = _built()
    assert L.ed_status_string(0) == b"ok"
    assert L.ed_status_string(-6) == b"Lanczos not converged"
    assert E.kernel_launches() >= 0


STRUCTS = {
    "ed_model": ["norb", "nbath", "U", "Ust", "Jh", "Jx", "Jp", "e_imp", "e_bath", "v_bath"],
    "ed_sector_info": ["ns", "dim_up", "dim", "device_bytes", "blocked_stride", "blocked_dim"],
    "ed_lanczos_opts": ["precision", "max_iter", "tol", "seed", "polish_steps", "want_vector",
                        "basis_mib"],
    "ed_lanczos_result": ["e0", "residual_estimate", "iterations", "matvecs", "matvecs_fp64"],
    "ed_gf_info": ["weight_hole", "steps_particle", "steps_hole"],
    "ed_solve_opts": ["lanczos", "gf_steps", "nmats", "beta", "gf_precision"],
    "ed_solve_result": ["ground", "t_build_s", "t_gf_s", "gf_chains", "gf_product_bytes"],
    "ed_server_opts": ["slots", "device_mem_budget", "queue_capacity"],
    "ed_request": ["model", "nup", "ndw", "opts"],
    "ed_result": ["status", "e0", "ground", "norb", "nmats", "t_submit_s", "t_done_s"],
    "ed_phonon": ["w0", "g", "nph", "reserved"],
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed for the layout probe")
def test_struct_layout_matches_c(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "edgb.h"', 'int main(void){']
    for s, fields in STRUCTS.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        s, f, v = line.split()
        cls = getattr(E, s)
        if f == "size":
            assert C.sizeof(cls) == int(v), s
        else:
            assert getattr(cls, f).offset == int(v), (s, f)


def test_psi_dtype_is_checked_before_the_call():
    """A ground state of the wrong type or device is refused by the binding
    before any pointer reaches the library (no GPU needed)."""
    torch = pytest.importorskip("torch")
    import paper_2105_06806_gb300 as ed
    for prec in ("fp64", "fp32_polish", "fp32"):
        with pytest.raises(ValueError):
            ed._psi_ptr(torch.zeros(4, dtype=torch.float64), prec)   # host tensor
