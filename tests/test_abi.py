"""The C ABI library loads and exports every symbol include/ctd.h declares (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "ctd.h")).read()
    return sorted(set(re.findall(r"^CTD_API\s+[a-z_ ]+\*?\s*(ctd_[A-Za-z_0-9]+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_03608_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ctd_static", "ctd_dynamic_step", "ctd_error"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ctd_[A-Za-z_0-9]+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_1710_03608_gb300 import ctd
    assert sorted(ctd.EXPORTED) == declared()
    L = ctd.load()
    assert ctd.version().startswith("ctd-gb300")
    for n in declared():
        assert hasattr(L, n)


def test_no_compute_without_gpu_raises_cleanly(lib):
    """Without a GPU a call fails with a status, not a crash or a CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1710_03608_gb300 import ctd, synth
    x = synth.tiny()
    X = ctd.Coo.from_synth(x, device=False)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_static(X, 1, 5, 1e-6, 0, 0, stream=0)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ctd.h"

static void* my_alloc(size_t bytes, void* stream) { (void)bytes; (void)stream; return NULL; }
static void my_release(void* p, void* stream) { (void)p; (void)stream; }

int main(void) {
  const char* v = ctd_version();
  if (!v || strncmp(v, "ctd-gb300", 9) != 0) return 2;
  /* an invalid argument is rejected before any device work */
  ctd_factors* F = NULL;
  if (ctd_static(NULL, 1, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F) != CTD_EINVAL || F) return 3;
  if (!ctd_last_error() || !ctd_last_error()[0]) return 4;
  int32_t i[1] = {0}, j[1] = {0}, k[1] = {0}, val[1] = {1};
  ctd_coo3 X = {{1, 1, 1}, 1, i, j, k, val, CTD_MEM_HOST};
  if (ctd_static(&X, 4, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F) != CTD_EINVAL || F) return 5;
  /* the allocator hook takes both functions or neither */
  if (ctd_set_allocator(my_alloc, NULL) != CTD_EINVAL) return 6;
  if (ctd_set_allocator(NULL, my_release) != CTD_EINVAL) return 7;
  if (ctd_set_allocator(my_alloc, my_release) != CTD_OK) return 8;
  if (ctd_set_allocator(NULL, NULL) != CTD_OK) return 9;
  size_t held = 1;
  if (ctd_allocated_bytes(&held) != CTD_OK || held != 0) return 10;
  if (ctd_allocated_bytes(NULL) != CTD_EINVAL) return 11;
  /* launch-shape knobs: known keys, ranges, -1 restores the default */
  int64_t t = 0;
  if (ctd_get_tuning("copy_blocks_per_sm", &t) != CTD_OK || t != 8) return 12;
  if (ctd_set_tuning("copy_blocks_per_sm", 3) != CTD_OK) return 13;
  if (ctd_get_tuning("copy_blocks_per_sm", &t) != CTD_OK || t != 3) return 14;
  if (ctd_set_tuning("copy_blocks_per_sm", 0) != CTD_EINVAL) return 15;
  if (ctd_set_tuning("cfill_dense_kb", 221) != CTD_EINVAL) return 16;
  if (ctd_set_tuning("no_such_knob", 1) != CTD_EINVAL) return 17;
  if (ctd_set_tuning(NULL, 1) != CTD_EINVAL) return 18;
  if (ctd_set_tuning("copy_blocks_per_sm", -1) != CTD_OK) return 19;
  if (ctd_get_tuning("copy_blocks_per_sm", &t) != CTD_OK || t != 8) return 20;
  if (ctd_get_tuning("qform_hot_kb", NULL) != CTD_EINVAL) return 21;
  printf("%s\n", v);
  return 0;
}
"""


def test_plain_c_caller(lib, tmp_path):
    """The header is plain C99 and a C program links the library and calls
    it (no GPU work: the version and argument checks)."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir,
                        "-lctd", "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ctd-gb300")


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises on first use: there is
    no fallback path that computes anything."""
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1710_03608_gb300 import ctd\n"
            "try:\n"
            "    ctd.load(%r)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % (ROOT, str(tmp_path / "libctd.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "not built" in r.stdout, (r.stdout, r.stderr)


def test_host_coo_must_be_contiguous_int32():
    import numpy as np
    from paper_1710_03608_gb300 import ctd
    a = np.zeros(4, np.int32)
    with pytest.raises(TypeError):
        ctd.Coo((2, 2, 1), a, a, a, np.zeros(4, np.int64))
    with pytest.raises(TypeError):
        ctd.Coo((2, 2, 1), a, a, a, np.zeros(8, np.int32)[::2])
    X = ctd.Coo((2, 2, 1), a, a, a, a)
    assert X.desc.memory == ctd.CTD_MEM_HOST and X.desc.nnz == 4
