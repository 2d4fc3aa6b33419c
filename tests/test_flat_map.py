"""The factorization's host block map (csrc/flat_map.h, an open-addressing
hash map) against std::unordered_map on random operation sequences: the C++
check in tests/cpp is compiled with the host compiler and run."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_flat_map_agrees_with_std_unordered_map(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "flat_map_test")
    src = os.path.join(HERE, "cpp", "flat_map_test.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
