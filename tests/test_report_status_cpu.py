"""How a timed-out bounded device wait reaches the caller, checked on the host.

The tensor-core kernels give up a bounded mbarrier wait by setting the instance's error
word in its device scalars; the reconstruction copies the scalars back and maps them to
report.status and the call's status (csrc/scalars.h).  A host-only C++ program presets the
error word (and a non-finite loss) and checks the mapping: DMCR_ETIMEOUT for the instance
and for a single-instance call, per-instance statuses for the batched call.  No GPU wait is
made to run out."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_preset_error_word_reports_timeout(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "report_probe")
    subprocess.check_call([cxx, "-std=c++17", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2103_09686_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "report_probe.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "timeout instance status: 5 (want 5)" in out.stdout
