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


C_ARGS_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ctd.h"

/* every entry point rejects a NULL or out-of-range argument with CTD_EINVAL
   and a message, before it touches the device; returns the failing check */
static int bad(ctd_status rc) { return rc != CTD_EINVAL || !ctd_last_error()[0]; }

int main(void) {
  int32_t i[1] = {0}, j[1] = {0}, k[1] = {0}, val[1] = {1};
  ctd_coo3 X = {{1, 1, 1}, 1, i, j, k, val, CTD_MEM_HOST};
  ctd_coo3 Xdev = {{1, 1, 1}, 1, i, j, k, val, CTD_MEM_DEVICE};
  ctd_factors* F = NULL;
  int64_t dims2[2] = {4, 4}, zero2[2] = {0, 4}, t = 0, draws[4], uniq[4], n = 0;
  int64_t s1[1] = {4};
  uint64_t seed1[1] = {0};
  double ms[3], e = 0.0, rs = 1.0;
  int nu = 0, st = 0;
  char buf[8];
  ctd_server* S = NULL;
  ctd_sizes sz;
  /* CTD-S */
  if (bad(ctd_static(&X, 1, 10, 1e-6, 0, CTD_FP64, 0, NULL, NULL))) return 1;
  if (bad(ctd_static(&X, 1, 0, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 2;
  if (bad(ctd_static(&X, 1, 8193, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 3;
  if (bad(ctd_static(&X, 1, 10, 1.0, 0, CTD_FP64, 0, NULL, &F)) || F) return 4;
  if (bad(ctd_static(&X, 1, 10, -0.5, 0, CTD_FP64, 0, NULL, &F)) || F) return 5;
  if (bad(ctd_static(&X, 1, 10, 1e-6, 0, 7, 0, NULL, &F)) || F) return 6;
  /* N-way */
  ctd_coon Xn;
  memset(&Xn, 0, sizeof Xn);
  if (bad(ctd_static_nway(NULL, 1, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F))) return 10;
  Xn.order = 0;
  if (bad(ctd_static_nway(&Xn, 1, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 11;
  Xn.order = CTD_MAX_ORDER + 1;
  if (bad(ctd_static_nway(&Xn, 1, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 12;
  Xn.order = 4;
  if (bad(ctd_static_nway(&Xn, 5, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 13;
  Xn.val_type = 9;
  if (bad(ctd_static_nway(&Xn, 2, 10, 1e-6, 0, CTD_FP64, 0, NULL, &F)) || F) return 14;
  /* batched: no tensors is a no-op, a negative count is refused */
  if (ctd_static_batched(0, NULL, 1, NULL, NULL, 1e-6, CTD_FP64, 0, 0, NULL, NULL) != CTD_OK)
    return 20;
  if (bad(ctd_static_batched(-1, &X, 1, s1, seed1, 1e-6, CTD_FP64, 0, 0, NULL, &F))) return 21;
  if (bad(ctd_static_batched(1, &X, 1, NULL, seed1, 1e-6, CTD_FP64, 0, 0, NULL, &F))) return 22;
  /* CTD-D */
  if (bad(ctd_dynamic_create(NULL, 1, CTD_FP64, 0, 0, 0, &F))) return 30;
  if (bad(ctd_dynamic_create(dims2, 3, CTD_FP64, 0, 0, 0, &F))) return 31;
  if (bad(ctd_dynamic_create(zero2, 1, CTD_FP64, 0, 0, 0, &F))) return 32;
  if (bad(ctd_dynamic_create(dims2, 1, 5, 0, 0, 0, &F))) return 33;
  if (bad(ctd_dynamic_step(NULL, &X, 10, 1e-6, NULL))) return 34;
  if (bad(ctd_dynamic_from_static(NULL, 0, 0, NULL, &F))) return 35;
  if (bad(ctd_get_step(NULL, 0, NULL, NULL))) return 36;
  if (bad(ctd_get_M(NULL, 0, NULL))) return 37;
  /* serving */
  if (bad(ctd_server_create(1, dims2, 1, CTD_FP64, 0, 10, 1e-6, 1, 0.5, NULL))) return 40;
  if (bad(ctd_server_create(0, dims2, 1, CTD_FP64, 0, 10, 1e-6, 1, 0.5, &S)) || S) return 41;
  if (bad(ctd_server_create(1, dims2, 1, CTD_FP64, 0, 0, 1e-6, 1, 0.5, &S)) || S) return 42;
  if (bad(ctd_server_create(1, dims2, 1, CTD_FP64, 0, 8193, 1e-6, 1, 0.5, &S)) || S) return 43;
  if (bad(ctd_server_create(1, dims2, 1, CTD_FP64, 0, 10, 1.5, 1, 0.5, &S)) || S) return 44;
  if (bad(ctd_server_submit(NULL, 0, &X, &t))) return 45;
  if (bad(ctd_server_wait(NULL, -1))) return 46;
  if (bad(ctd_server_result(NULL, 0, &st, ms))) return 47;
  if (bad(ctd_server_state(NULL, 0, &F))) return 48;
  ctd_server_free(NULL);
  /* getters on no factors */
  if (bad(ctd_error(NULL, &e))) return 50;
  if (bad(ctd_get_sizes(NULL, &sz))) return 51;
  if (bad(ctd_get_samples(NULL, draws, uniq))) return 52;
  if (bad(ctd_get_fibers(NULL, draws, NULL))) return 53;
  if (bad(ctd_get_R(NULL, draws, i, val))) return 54;
  if (bad(ctd_get_U(NULL, &e))) return 55;
  if (bad(ctd_get_R_f64(NULL, draws, i, &e))) return 56;
  if (bad(ctd_get_C_columns(NULL, 1, draws, &e))) return 57;
  if (bad(ctd_get_C(NULL, draws, i, &e))) return 58;
  if (bad(ctd_get_column_dist(NULL, NULL, NULL))) return 59;
  if (bad(ctd_ddos_candidates(NULL, 4, draws, &n, &e))) return 60;
  ctd_free(NULL);
  /* the allocation-free draws: device memory only, alpha and s in range */
  if (bad(ctd_sample_noalloc(NULL, 1, 4, 0, draws, uniq, &nu, NULL))) return 70;
  if (bad(ctd_sample_noalloc(&X, 1, 4, 0, draws, uniq, &nu, NULL))) return 71;
  if (bad(ctd_sample_noalloc(&Xdev, 4, 4, 0, draws, uniq, &nu, NULL))) return 72;
  if (bad(ctd_sample_noalloc(&Xdev, 1, 0, 0, draws, uniq, &nu, NULL))) return 73;
  if (bad(ctd_sample_noalloc(&Xdev, 1, 8193, 0, draws, uniq, &nu, NULL))) return 74;
  /* diagnostics and self-tests */
  if (bad(ctd_profile_report(NULL, 8))) return 80;
  if (bad(ctd_profile_report(buf, 0))) return 81;
  if (bad(ctd_selftest_rsqrt(&rs, -1, &e, &e))) return 82;
  if (bad(ctd_selftest_rsqrt(NULL, 1, &e, &e))) return 83;
  if (ctd_selftest_rsqrt(NULL, 0, NULL, NULL) != CTD_OK) return 84;
  printf("ok\n");
  return 0;
}
"""


def test_plain_c_argument_checks(lib, tmp_path):
    """Every entry point of the header refuses a NULL or out-of-range argument
    with CTD_EINVAL and a message, from plain C, before any device work
    (runs without a GPU)."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "args.c"
    src.write_text(C_ARGS_PROGRAM)
    exe = tmp_path / "args"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir,
                        "-lctd", "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, ("failing check", r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "ok"


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
