"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer and
driven through every entry point of oracle/lgref.h (oracle/sanitize_check.c)
on small graphs of several shapes and option sets, with leak detection on:
no invalid access, no undefined behaviour, no leak, and the solves reach
their residuals. CPU only."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAGS = ["-std=c11", "-O1", "-g", "-Wall", "-Wextra", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def test_oracle_under_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    probe = tmp_path / "probe.c"
    probe.write_text("int main(void) { return 0; }\n")
    if subprocess.run([gcc, *FLAGS, "-o", str(tmp_path / "probe"), str(probe)], capture_output=True).returncode:
        pytest.skip("gcc without the sanitizer runtimes")
    exe = tmp_path / "sanitize_check"
    subprocess.run([gcc, *FLAGS, "-o", str(exe), os.path.join(ROOT, "oracle", "lgref.c"),
                    os.path.join(ROOT, "oracle", "sanitize_check.c"), "-lm"], check=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "all oracle checks passed" in r.stdout
