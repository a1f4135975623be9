"""CPU checks of the C ABI: libgs.so builds, loads and exports every symbol
include/gs.h declares, and the ctypes mirror matches the C layouts. No
compute call is made (no GPU here)."""
import ctypes
import os
import subprocess

import pytest

from paper_2607_15951_gb300 import _native as N
from paper_2607_15951_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def test_every_declared_symbol_exported(lib):
    names = N.declared_symbols(HEADER)
    assert "gs_render" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the ctypes table covers exactly the header
    assert sorted(N.SIGNATURES) == names


def test_header_is_c99_and_layouts_match(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "gs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gs_record), sizeof(gs_camera), sizeof(gs_gaussians),
         sizeof(gs_options), sizeof(gs_framebuffer), sizeof(gs_render_stats));
  printf("%zu %zu %zu %zu\n", offsetof(gs_record, depth), offsetof(gs_record, radius),
         offsetof(gs_camera, near_z), offsetof(gs_gaussians, sh_degree));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                           str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = list(map(int, out[:6]))
    offs = list(map(int, out[6:]))
    assert sizes == [ctypes.sizeof(N.gs_record), ctypes.sizeof(N.gs_camera),
                     ctypes.sizeof(N.gs_gaussians), ctypes.sizeof(N.gs_options),
                     ctypes.sizeof(N.gs_framebuffer), ctypes.sizeof(N.gs_render_stats)]
    assert offs == [N.gs_record.depth.offset, N.gs_record.radius.offset,
                    N.gs_camera.near_z.offset, N.gs_gaussians.sh_degree.offset]
    assert sizes[0] == 48


def test_default_options(lib):
    o = N.gs_options()
    lib.gs_default_options(ctypes.byref(o))
    assert (o.tile_w, o.tile_h, o.record_dtype) == (16, 16, 0)
    assert list(o.bg) == [0.0, 0.0, 0.0]


def test_null_context_rejected(lib):
    # Host-side argument checks run before any CUDA call.
    assert lib.gs_render(None, None, None, None, None, None) == N.GS_ERR_INVALID_ARG
    assert lib.gs_sync_status(None, None) == N.GS_ERR_INVALID_ARG
    assert lib.gs_workspace_bytes(None) == 0
    assert lib.gs_create(None, 0) == N.GS_ERR_INVALID_ARG


def test_kernels_built_for_sm103a_only():
    # The build passes exactly one -gencode, for sm_103a.
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_plain_c_program_links_and_calls_the_library(lib, tmp_path):
    """A C99 program (no Python, no torch) links against libgs.so and calls
    it: default options, argument checks, and a context that is created where
    a device exists and refused with a status (not a crash) where none does."""
    src = tmp_path / "use_gs.c"
    src.write_text(r'''
#include <stdio.h>
#include "gs.h"
int main(void) {
  gs_options o;
  gs_default_options(&o);
  if (o.tile_w != 16 || o.tile_h != 16 || o.record_dtype != GS_RECORD_F32) return 1;
  if (gs_render(NULL, NULL, NULL, NULL, NULL, NULL) != GS_ERR_INVALID_ARG) return 2;
  gs_context *ctx = NULL;
  gs_status st = gs_create(&ctx, 0);
  if (st == GS_OK) {
    if (!ctx) return 3;
    gs_destroy(ctx);
  } else if (ctx != NULL) {
    return 4;
  }
  printf("%d\n", (int)st);
  return 0;
}
''')
    exe = tmp_path / "use_gs"
    libdir = os.path.dirname(B.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src),
                           "-L", libdir, "-l:" + os.path.basename(B.LIB), "-Wl,-rpath," + libdir,
                           "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    # GS_OK where device 0 exists, GS_ERR_INVALID_ARG where it does not.
    assert int(r.stdout.split()[0]) in (N.GS_OK, N.GS_ERR_INVALID_ARG)
