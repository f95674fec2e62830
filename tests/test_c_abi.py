"""The C ABI from a plain C program (gcc, no Python or torch in the loop): the
argument checks and the memory contract on the host, and a short run with
device memory the program allocates itself on a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(tlbm.library_path())
    out = str(tmp_path_factory.mktemp("c_abi") / "abi_c")
    cmd = ["gcc", "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "abi_c.c"), "-o", out, "-L", lib_dir,
           "-ltlbm", "-L", os.path.join(CUDA, "lib64"), "-lcudart", f"-Wl,-rpath,{lib_dir}",
           f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_c_program_host_checks(exe):
    r = subprocess.run([exe, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.gpu
def test_c_program_gpu_run(exe, tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([exe, "gpu", str(tmp_path / "c.ckpt")], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
