"""The C ABI library loads without a GPU, exports every function that
include/gamblet.h and include/gamblet3d.h declare, and the ctypes structures
match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gamblet.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in ("gamblet.h", "gamblet3d.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1503_03467_gb300 import build
    build.build()
    from paper_1503_03467_gb300 import native
    return native


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"GAMBLET_API\s+[\w\s\*]+?\b(gamblet\w*?_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gamblet_setup", "gamblet_solve", "gamblet_grad", "gamblet_destroy",
                     "gamblet3d_setup", "gamblet3d_solve", "gamblet3d_get_operator"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(gamblet\w*?_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding knows each of them
    assert set(declared_functions()) <= set(lib.SIGNATURES)


def test_struct_layouts_match_header(lib):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gamblet.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(gamblet_csr), sizeof(gamblet_opts), sizeof(gamblet_info),
         sizeof(gamblet_kernel_stat));
  printf("%zu %zu %zu %zu\n", offsetof(gamblet_opts, stream), offsetof(gamblet_info, rel_residual),
         offsetof(gamblet_csr, val), offsetof(gamblet_opts, autotune));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        l1, l2 = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    sizes = [int(x) for x in l1.split()]
    offs = [int(x) for x in l2.split()]
    assert sizes == [ctypes.sizeof(lib.Csr), ctypes.sizeof(lib.Opts), ctypes.sizeof(lib.Info),
                     ctypes.sizeof(lib.KernelStat)]
    assert offs == [lib.Opts.stream.offset, lib.Info.rel_residual.offset, lib.Csr.val.offset,
                    lib.Opts.autotune.offset]


def test_host_only_calls(lib):
    o = lib.gamblet_default_opts()
    assert o.rho == 3.0 and o.precision == lib.FP64 and o.refine_max_iter == 50
    assert o.autotune == 1 and o.galerkin_variant == -1 and o.patch_gather == -1
    assert lib.gamblet_status_string(lib.ERR_NOT_SPD).startswith("matrix not")
    assert lib.gamblet_device_bytes(0) == 0
    assert lib.gamblet_kernel_stats(0) == []
    lib.gamblet_destroy(0)  # NULL is ignored
    with pytest.raises(lib.GambletError):
        lib.gamblet_level_size(0, 1)


def test_noalloc_source_calls_no_allocator():
    """The allocation-free objective's translation unit, comments removed,
    names no device or host allocation routine (its scratch is a fixed
    file-scope device array)."""
    import re
    src = open(os.path.join(ROOT, "paper_1503_03467_gb300", "csrc", "noalloc.cu")).read()
    code = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    for name in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaMemPool", "cudaHostAlloc",
                 "malloc(", "new ", "torch", "at::"):
        assert name not in code, name
    assert re.search(r"static __device__ __align__\(256\) double g_objective_scratch\[", code)
