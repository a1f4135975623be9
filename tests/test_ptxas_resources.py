"""Register and spill guard for the kernels of one frame (compiler output of
`nvcc -Xptxas -v`; no GPU needed). The frame's kernels must not spill, and
the blend keeps the register allocation its launch bounds were chosen for
(8x4 warp blocks: more than 46 registers, which measured 4 % slower; 8x8
blocks: at most 56, for 36 resident warps per SM)."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

import pytest

from paper_2607_15951_gb300 import build as B

pytestmark = pytest.mark.slow

FRAME_KERNELS = {
    # mangled-name fragment: (source, registers allowed (lo, hi))
    "19project_list_kernelILi3E": ("gs_project.cu", (1, 64)),
    "18list_gather_kernel": ("gs_project.cu", (1, 255)),
    "16emit_sort_kernelItE": ("gs_project.cu", (1, 80)),
    "17entry_scan_kernel": ("gs_project.cu", (1, 255)),
    "15onesweep_kernelImLi8ELi2E": ("gs_sort.cu", (1, 128)),
    "15onesweep_kernelItLi16ELi2E": ("gs_sort.cu", (1, 128)),
    "19ranges_tiles_kernelItE": ("gs_bin.cu", (1, 255)),
    "19blend_culled_kernelILi16ELi16ELi8ELi4E": ("gs_blend.cu", (47, 64)),
    "19blend_culled_kernelILi16ELi16ELi8ELi8E": ("gs_blend.cu", (1, 56)),
}


def _resources(src: str, tmp: str) -> dict:
    nvcc = B._nvcc()
    cmd = [nvcc, *B.ARCH, *B.FLAGS, "-Xptxas", "-v", "-c", os.path.join(B.CSRC, src),
           "-o", os.path.join(tmp, src + ".o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)' for 'sm_103a'", line)
        if m:
            name = m.group(1)
            out[name] = {}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[name]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out[name]["regs"] = int(m.group(1))
    return out


@pytest.fixture(scope="module")
def resources(tmp_path_factory):
    try:
        B._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    tmp = str(tmp_path_factory.mktemp("ptxas"))
    srcs = sorted({s for s, _ in FRAME_KERNELS.values()})
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        parts = list(ex.map(lambda s: _resources(s, tmp), srcs))
    shutil.rmtree(tmp, ignore_errors=True)
    merged = {}
    for p in parts:
        merged.update(p)
    return merged


@pytest.mark.parametrize("frag", sorted(FRAME_KERNELS))
def test_frame_kernel_resources(resources, frag):
    hits = {k: v for k, v in resources.items() if frag in k}
    assert hits, f"no kernel matching {frag}"
    lo, hi = FRAME_KERNELS[frag][1]
    for name, r in hits.items():
        assert r.get("spill", 0) == 0, (name, r)
        assert lo <= r["regs"] <= hi, (name, r)
