"""CPU-side checks of the C ABI: the library builds and exports every entry
point that include/fams.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fams.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fams_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fams_setup", "fams_solve", "fams_flux", "fams_destroy", "fams_setup_batch",
              "fams_solve_batch", "fams_sizes", "fams_query", "fams_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1705_05784_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"no CUDA toolkit: {e}")
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    lib.fams_strerror.restype = ctypes.c_char_p
    assert lib.fams_strerror(-3) == b"iteration did not reach the tolerance"


def test_binding_loads_and_reports_missing_gpu_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1705_05784_gb300 import fams, inputs
    with pytest.raises(fams.FamsError) as e:
        fams.Context(inputs.config_2d_small())
    assert e.value.status == fams.ECUDA


def test_argument_checks_need_no_gpu():
    """Null and empty arguments are rejected before any CUDA call."""
    from paper_1705_05784_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"no CUDA toolkit: {e}")
    lib = ctypes.CDLL(path)
    ctx = ctypes.c_void_p()
    assert lib.fams_setup_batch(0, None, None, None, None, ctypes.byref(ctx)) == -1   # FAMS_EINVAL
    assert lib.fams_setup(None, None, None, None, ctypes.byref(ctx)) == -1
    assert lib.fams_solve(None, None, None, ctypes.c_double(1e-8), None) == -1
    assert lib.fams_flux(None, 0, None, None, None) == -1
    assert lib.fams_update(None, None) == -1


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "fams.h"

int main(void) {
  fams_grid g;
  fams_opts o;
  fams_ctx* ctx = 0;
  memset(&g, 0, sizeof g);
  memset(&o, 0, sizeof o);
  /* argument checks answer before any CUDA call */
  if (fams_setup_batch(0, &g, 0, 0, &o, &ctx) != FAMS_EINVAL) return 1;
  if (fams_solve(0, 0, 0, 1e-8, 0) != FAMS_EINVAL) return 2;
  if (strcmp(fams_strerror(FAMS_ENOCONV), "iteration did not reach the tolerance") != 0) return 3;
  printf("%s\n", fams_last_error());
  return 0;
}
"""


def test_header_compiles_as_c_and_links(tmp_path):
    """A plain C99 client: the header compiles without C++, every call links
    against the library, and the argument checks answer without a GPU."""
    import shutil
    import subprocess
    from paper_1705_05784_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    try:
        lib = build.build()
    except RuntimeError as e:
        pytest.skip(f"no CUDA toolkit: {e}")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lfams", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
