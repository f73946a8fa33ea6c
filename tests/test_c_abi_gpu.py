"""libdm driven from plain C (tests/c/abi_driver.c): caller-owned device buffers from
cudaMalloc, build, updates through dm_update_tf and dm_update_tf_host, full recomputes, and
a batched precompute and batched update of three volumes; every PDM plane and map equals
the oracle's (its C source is compiled into the driver)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def test_c_driver_matches_oracle(tmp_path):
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import _abi as A
    libdir = os.path.dirname(A.LIB_PATH)
    cuda = _cuda_home()
    exe = str(tmp_path / "abi_driver")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           os.path.join(ROOT, "tests", "c", "abi_driver.c"),
           os.path.join(ROOT, "oracle", "dm_oracle.c"),
           "-L", libdir, "-ldm", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-o", exe]
    subprocess.check_call(cmd)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi driver: OK" in r.stdout
