"""Host-side index maps of the strided GEMM, checked against direct row-major offsets (no GPU)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_group_maps_reproduce_row_major_offsets(tmp_path):
    exe = tmp_path / "stride_map_check"
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(HERE, "stride_map_check.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
