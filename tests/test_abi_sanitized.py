"""The C-ABI library's host code under AddressSanitizer and UndefinedBehaviorSanitizer (CPU only).

The library is rebuilt with the host compiler's sanitizers (device code as PTX only: no kernel
runs without a GPU) and the argument-checking tests of test_abi.py run against it: every
entry point's validation of sizes, pointers and bounds must pass without an out-of-bounds
access, use after free, leak of a partly built handle's host memory or undefined behaviour.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PLUGIN = """
import paper_2204_12346_gb300.build as b
b.LIB = {lib!r}
b.up_to_date = lambda: True
b.build = lambda *a, **k: b.LIB
"""


def test_argument_checks_are_clean_under_sanitizers(tmp_path):
    from paper_2204_12346_gb300 import build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    asan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    nvcc = build.nvcc()
    arch = ["-gencode", "arch=compute_103a,code=compute_103a"]
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"]

    def compile_one(src):
        obj = str(tmp_path / (os.path.basename(src)[:-3] + ".o"))
        r = subprocess.run([nvcc, *arch, "-O0", "-std=c++17", "-Xcompiler", "-fPIC", *san, "--expt-relaxed-constexpr",
                            "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, build._sources()))
    lib = str(tmp_path / "libsird_pso.so")
    r = subprocess.run([nvcc, *arch, "-shared", "-cudart", "static", *san, "-o", lib, *objs], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    (tmp_path / "sanitized_library.py").write_text(PLUGIN.format(lib=lib))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]), LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0", UBSAN_OPTIONS="print_stacktrace=1")
    # -s: the sanitizers' reports go to stderr, which pytest then leaves alone
    run = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_abi.py"), "-q", "-s",
                          "-p", "sanitized_library", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=900)
    out = run.stdout[-4000:] + run.stderr[-4000:]
    assert run.returncode == 0, out
    assert "runtime error" not in out and "AddressSanitizer" not in out, out
