"""The library's own bijection code (paper_1704_03767_gb300/csrc/bijection.cuh), both the FP32-root
variant the kernels use and the FP64-root variant the host uses, checked exhaustively on the CPU
against row-major enumeration of the upper triangle (Sec. 4.1 numbering)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_bijection_exhaustive(tmp_path):
    exe = tmp_path / "bijection_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I",
                           os.path.join(ROOT, "paper_1704_03767_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "bijection_check.cpp"),
                           "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout
