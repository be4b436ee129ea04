"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every entry point include/fse.h declares; the ctypes mirror has
the header's struct layout; configuration errors are reported as statuses."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2204_14193_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fse.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:fse_status|const char \*|void|size_t)\s*\*?\s*(fse_\w+)\s*\(",
                                 src, re.M)))


def test_library_exports_every_declared_symbol():
    lib = P._load()
    names = declared_functions()
    assert {"fse_create", "fse_extrapolate_batch", "fse_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_checked_library_exports_every_declared_symbol():
    """The bounds-checked build (FSE_BOUNDS_CHECK) offers the same interface."""
    from paper_2204_14193_gb300 import _build
    P._load()   # builds both libraries if needed
    lib = ctypes.CDLL(_build.LIB_CHECKED)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_ctypes_structs_match_header_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "fse.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(fse_class), sizeof(fse_config), sizeof(fse_block),
         offsetof(fse_config, init), offsetof(fse_config, flags), offsetof(fse_class, iters));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(P.fse_class), ctypes.sizeof(P.fse_config), ctypes.sizeof(P.fse_block),
            P.fse_config.init.offset, P.fse_config.flags.offset, P.fse_class.iters.offset]
    assert got == want


@pytest.mark.parametrize("bad,status", [
    (dict(fft=48), 1), (dict(fft=128), 2), (dict(block=40), 1), (dict(border=0), 1),
    (dict(border=30), 1), (dict(rho=0.0), 1), (dict(rho=1.5), 1), (dict(gamma=0.0), 1),
    (dict(gamma=2.0), 1), (dict(iters=-1), 1), (dict(iters=5000), 1), (dict(frames=2), 1),
    (dict(frames=5), 2), (dict(frames=3), 2)])
def test_config_validation_statuses(bad, status):
    cls = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=10)
    cls.update(bad)
    with pytest.raises(P.FseError) as ei:
        P.fse_create(P.make_config([cls]))
    assert ei.value.status == status
    assert len(P.fse_last_error(None)) > 0


def test_null_handle_is_rejected():
    st = P._load().fse_extrapolate_batch(None, None, 0, 1, 1, 1, 1, None, None, 0, None, None, None)
    assert st == 1
    P.fse_destroy(None)


@pytest.mark.parametrize("n_classes,init_iters,status", [(2, 10, 2), (1, -1, 1), (1, 5000, 1)])
def test_learned_config_validation(n_classes, init_iters, status):
    cls = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=10)
    with pytest.raises(P.FseError) as ei:
        P.fse_create(P.make_config([cls] * n_classes, init="learned", init_iters=init_iters))
    assert ei.value.status == status


@pytest.mark.parametrize("kw,status", [(dict(ordered=True, reuse_weight=0.0), 1), (dict(ordered=True, reuse_weight=1.5), 1),
                                       (dict(ordered=True, n=2), 2), (dict(ordered=True, init="learned"), 2),
                                       (dict(ordered=True, fft=16), 2)])
def test_ordered_config_validation(kw, status):
    cls = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=10)
    n = kw.pop("n", 1)
    if "fft" in kw:
        cls = dict(block=4, border=6, fft=kw.pop("fft"), rho=0.8, gamma=0.5, iters=10)
    with pytest.raises(P.FseError) as ei:
        P.fse_create(P.make_config([cls] * n, **kw))
    assert ei.value.status == status


@pytest.mark.parametrize("kw,status", [(dict(fft=32), 2), (dict(frames=3), 2), (dict(ordered=True), 2),
                                       (dict(bits=0x10), 1)])
def test_fixed_w_config_validation(kw, status):
    """Reduced-precision residual storage: image classes of fft 64 only, not
    with ordered concealment; unknown flag bits are rejected."""
    cls = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=10)
    if "fft" in kw:
        cls = dict(block=8, border=12, fft=kw.pop("fft"), rho=0.8, gamma=0.5, iters=10)
    if "frames" in kw:
        cls = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=10, frames=kw.pop("frames"))
    bits = kw.pop("bits", 0)
    cfg = P.make_config([cls], fixed_w=True, **kw)
    cfg.flags |= bits
    with pytest.raises(P.FseError) as ei:
        P.fse_create(cfg)
    assert ei.value.status == status
    hdr = open(HEADER).read()
    assert re.search(r"#define FSE_FLAG_FIXED_W (\d+)u", hdr).group(1) == str(P.FSE_FLAG_FIXED_W)
    assert re.search(r"#define FSE_FIXED_W_FROM (\d+)", hdr).group(1) == str(P.FSE_FIXED_W_FROM)


def test_tuning_api_argument_errors():
    lib = P._load()
    assert lib.fse_set_tuning(None, 0) == 1
    assert lib.fse_get_tuning(None, None, None) == 1
    assert (P.FSE_TUNE_SYNC, P.FSE_TUNE_ASYNC, P.FSE_TUNE_OFF) == (0, 1, 2)
    hdr = open(HEADER).read()
    for name, v in (("FSE_TUNE_SYNC", 0), ("FSE_TUNE_ASYNC", 1), ("FSE_TUNE_OFF", 2)):
        assert re.search(rf"#define {name} (\d+)", hdr).group(1) == str(v)
