"""The C ABI used from C: tests/c/abi_host.c includes both headers, is
compiled as strict C11 by gcc, linked against liblbs.so and run without a
GPU (host-side entry points only)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdir():
    from paper_2502_00920_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2502_00920_gb300")


def test_headers_compile_link_and_run_as_c(libdir, tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "abi_host")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_host.c"),
                        "-L", libdir, "-llbs", f"-Wl,-rpath,{libdir}", "-lm", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
