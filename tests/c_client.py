"""Builds tests/c_abi_client.c (a plain C99 user of include/mppi.h) against
the in-tree library."""
import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2407_09812_gb300")


def build_client(out_dir: str) -> str:
    from paper_2407_09812_gb300 import build as B
    B.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    assert cc, "a C compiler is needed for the C-ABI client"
    exe = os.path.join(out_dir, "c_abi_client")
    cmd = [cc, "-std=c99", "-O1", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-L", PKG, "-lmppi_gb300", f"-Wl,-rpath,{PKG}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe
