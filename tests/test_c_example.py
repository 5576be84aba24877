"""The C ABI from plain C: the header compiles as strict C99, and the example program
(paper_2607_03413_gb300/examples/cw_solve.c: load vector, loose solve, host checkpoint, resumed
solve, nodal error against the manufactured solution, assembled apply) builds against libcwfem.so
and, on a GPU, runs to its own checks."""
import glob
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXAMPLE = os.path.join(ROOT, "paper_2607_03413_gb300", "examples", "cw_solve.c")


def _gcc():
    return shutil.which("gcc") or pytest.skip("no gcc")


def _cuda_dirs():
    from paper_2607_03413_gb300 import build
    home = os.path.dirname(os.path.dirname(os.path.realpath(build._nvcc())))
    libs = [d for d in [os.path.join(home, "lib64")] + glob.glob(os.path.join(home, "targets", "*", "lib"))
            if os.path.exists(os.path.join(d, "libcudart.so"))]
    if not libs:
        pytest.skip("no libcudart.so next to nvcc")
    return os.path.join(home, "include"), libs[0]


def build_example(tmp_path):
    from paper_2607_03413_gb300 import build
    lib = build.build()
    inc, cudalib = _cuda_dirs()
    exe = str(tmp_path / "cw_solve")
    libdir = os.path.dirname(lib)
    subprocess.run([_gcc(), "-std=c11", "-O2", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-I", inc, EXAMPLE, "-L", libdir, "-lcwfem",
                    "-L", cudalib, "-lcudart", "-lm", f"-Wl,-rpath,{libdir}", "-o", exe], check=True)
    return exe


def test_header_is_strict_c99(tmp_path):
    src = tmp_path / "hdr.c"
    src.write_text('#include "cwfem.h"\n'
                   "int main(void) { cw_cg_stats s = {0, 0, 0.0, 0.0, 0.0}; (void)s;\n"
                   "  return cw_status_string(CW_OK) == 0; }\n")
    subprocess.run([_gcc(), "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True)


def test_c_example_builds(tmp_path):
    assert os.access(build_example(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_example_solves(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = build_example(tmp_path)
    out = subprocess.run([exe, "12", "3"], capture_output=True, text=True, timeout=600)
    print(out.stdout, out.stderr)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok")
