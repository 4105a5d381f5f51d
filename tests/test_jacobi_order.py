"""The block-cyclic Jacobi schedule covers every column pair once per sweep (host check, no GPU)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_block_cyclic_schedule_rotates_every_pair_once_per_sweep(tmp_path):
    exe = tmp_path / "jacobi_order_check"
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(HERE, "jacobi_order_check.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
