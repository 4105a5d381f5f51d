"""include/ctm.h is a plain C header and libctm.so is callable from C (gcc, no GPU needed)."""
import os
import subprocess

import numpy as np

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_header_compiles_as_c_and_library_links_from_c(tmp_path):
    import __graft_entry__ as g
    g.build()
    from paper_2512_14414_gb300 import _lib
    libdir = os.path.dirname(_lib.LIB_PATH)
    exe = tmp_path / "c_abi_check"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", os.path.join(HERE, "c_abi_check.c"), "-o", str(exe),
                    "-L" + libdir, "-l:libctm.so", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    expect = sum(int(np.prod(s)) for site in W.env_shapes(1, 1, 2, 2, 4) for s in site)
    assert out.stdout.split() == ["ok", str(expect)]
