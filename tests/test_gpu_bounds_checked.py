"""The bounds-checked library (libfse_checked.so, FSE_BOUNDS_CHECK) over every
kernel path (tests/bounds_workloads.py): no index leaves its buffer (fse_sync
reports none), and the outputs equal the normal library's bit for bit, so the
checks change nothing but the checking.  Each library runs in a process of
its own (the binding picks one per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCRIPT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bounds_workloads.py")


def _run(checked):
    env = dict(os.environ)
    env["FSE_BOUNDS_CHECK"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return dict(ln.split() for ln in lines)


def test_checked_library_finds_no_violation_and_matches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plain = _run(False)
    checked = _run(True)
    assert plain.pop("library") == "libfse.so"
    assert checked.pop("library") == "libfse_checked.so"
    print("workloads:", sorted(plain))
    assert len(plain) == 12
    assert checked == plain
