"""Failure detection on the device: every wait of one thread block on another
(the decoupled look-backs of the key-count scan and of the radix sort) gives
up after a time limit and reports GS_ERR_TIMEOUT instead of hanging.

The self-test entry point starts the wait with partition 0 never taken, so
every block waits on a status word that nothing sets. The test checks that
the status comes back within a bounded time and that the same context then
renders correctly (the CUDA context is unharmed)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

from parity_util import RGB_TOL, T_TOL, compare_image  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind", [0, 1], ids=["scan", "onesweep"])
def test_bounded_wait_times_out_and_context_survives(ctx, oracle_mod, kind):
    for _ in range(2):  # twice in a row: the error word is cleared between runs
        t0 = time.perf_counter()
        st = gs.gs_selftest_bounded_wait(ctx, kind, 20_000_000)  # 20 ms limit
        dt = time.perf_counter() - t0
        assert st == N.GS_ERR_TIMEOUT, N.STATUS_NAMES.get(st, st)
        assert dt < 5.0
    gs.gs_sync_status(ctx)
    scene = scenes.uniform_box(3000, 11)
    cam = scenes.pinhole(160, 120)
    out = gs.render(ctx, gs.scene_to_device(scene), scene.sh_degree, cam)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    _, _, img = oracle_mod.render(scene, cam)
    st = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
    st.pop("keep")
    assert st["max_rgb_err"] <= RGB_TOL, st
    assert st["max_T_err"] <= T_TOL, st


def test_bounded_wait_rejects_bad_arguments(ctx):
    assert gs.gs_selftest_bounded_wait(ctx, 2, 20_000_000) == N.GS_ERR_INVALID_ARG
    assert gs.gs_selftest_bounded_wait(ctx, 0, 10) == N.GS_ERR_INVALID_ARG
    assert gs.gs_selftest_bounded_wait(ctx, 0, 10 ** 10) == N.GS_ERR_INVALID_ARG
