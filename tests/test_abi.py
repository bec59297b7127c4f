"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
include/ppcg.h declares; the Python binding's structs match the header's layout.  CPU only:
no compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ppcg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ppcg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2105_06176_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ppcg_create", "ppcg_solve", "ppcg_batch_solve", "ppcg_destroy", "ppcg_server_create",
              "ppcg_submit", "ppcg_poll", "ppcg_server_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(ppcg_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    lib = ctypes.CDLL(libpath)
    for f in declared_functions():
        assert hasattr(lib, f), f
    import paper_2105_06176_b300 as pp
    assert set(pp.EXPORTED_SYMBOLS) == set(declared_functions())
    o = pp.Opts()
    lib.ppcg_opts_default(ctypes.byref(o))     # host-only call
    assert o.precision == pp.FP64 and o.norm == pp.NORM_REL_R and o.inner_tol == 1e-2
    assert o.epoch_iters == 256 and o.cluster_max_rows == 16384
    assert o.gap_theta == 1e-6 and o.gap_fall == 100 and o.cluster_ctas == 8
    # host-only argument checks: no CUDA call is made before they fail
    info = pp.Info()
    assert lib.ppcg_last_info(None, ctypes.byref(info)) == pp.ERR_ARG
    lib.ppcg_last_error.restype = ctypes.c_char_p
    assert b"ppcg_last_info" in lib.ppcg_last_error()
    assert lib.ppcg_plan_info(None, ctypes.byref(pp.Plan())) == pp.ERR_ARG


def test_struct_layouts_match_header(tmp_path):
    """Compile a tiny C program against include/ppcg.h and compare sizeof/offsetof with ctypes."""
    import paper_2105_06176_b300 as pp
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "ppcg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ppcg_opts), offsetof(ppcg_opts, inner_tol),
         offsetof(ppcg_opts, spin_limit_ns), offsetof(ppcg_opts, epoch_iters), sizeof(ppcg_info));
  printf("%zu %zu\n", offsetof(ppcg_info, rel_res_recursive), offsetof(ppcg_info, bnorm));
  printf("%zu %zu %zu\n", offsetof(ppcg_opts, gap_theta), offsetof(ppcg_opts, gap_fall),
         offsetof(ppcg_opts, cluster_ctas));
  printf("%zu %zu %zu\n", sizeof(ppcg_plan), offsetof(ppcg_plan, slots), offsetof(ppcg_plan, bytes_per_iter));
  return 0;
}''')
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(prog), "-o", str(exe)],
                   check=True)
    a, b, c, d = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:4]
    so, oi, osp, oe, si = map(int, a.split())
    orr, ob = map(int, b.split())
    og, of, occ = map(int, c.split())
    assert og == pp.Opts.gap_theta.offset and of == pp.Opts.gap_fall.offset
    assert occ == pp.Opts.cluster_ctas.offset
    sp_, osl, obp = map(int, d.split())
    assert sp_ == ctypes.sizeof(pp.Plan) and osl == pp.Plan.slots.offset and obp == pp.Plan.bytes_per_iter.offset
    assert so == ctypes.sizeof(pp.Opts) and oi == pp.Opts.inner_tol.offset
    assert osp == pp.Opts.spin_limit_ns.offset and oe == pp.Opts.epoch_iters.offset
    assert si == ctypes.sizeof(pp.Info) and orr == pp.Info.rel_res_recursive.offset
    assert ob == pp.Info.bnorm.offset


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    """The product path raises when the compiled library is absent (no CPU fallback)."""
    import importlib
    import paper_2105_06176_b300 as pp
    monkeypatch.setattr(pp._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pp, "_lib", None)
    with pytest.raises(RuntimeError):
        pp.lib(build_if_missing=False)
    importlib.reload(pp)
