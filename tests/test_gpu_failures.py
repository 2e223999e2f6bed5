"""Failure detection without a GPU fault: allocation failures injected on the
host at every allocation of a call (each returns AW_ENOMEM and frees what the
call had allocated), and the library's bounded device waits run against a
condition that never becomes true (each returns AW_ETIMEOUT, and the context
keeps working afterwards)."""
import math
import time

import numpy as np
import pytest
import torch

from paper_2206_15117_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _small():
    ob = sy.small_observation(n_ant=8, radius_m=80.0, n_t=6, freq=(1.3e9, 1.4e9), npa=2)
    N = 64
    kw = dict(N=N, dl=math.radians(3.0) / N, OS=4, W=7.0, npol=4, nw=2, w_max=ob.w_max, supports=[8, 10],
              pa=list(ob.pa_centres), fbin_freqs=list(ob.fbin_freqs), dish_d=12.0, d_xy=0.01j, d_yx=-0.01j)
    return ob, kw


def _sweep(make):
    """Run make() once to count its device allocations, then once per
    allocation with that allocation failing; every failure must be AW_ENOMEM
    and leave the live-buffer count where it was."""
    from paper_2206_15117_gb300 import aw
    live0, calls0 = aw.aw_debug_alloc_stats()
    obj = make()
    live1, calls1 = aw.aw_debug_alloc_stats()
    n = calls1 - calls0
    assert n > 0 and live1 > live0
    del obj
    assert aw.aw_debug_alloc_stats()[0] == live0
    try:
        for k in range(n):
            aw.aw_debug_fail_alloc(k)
            with pytest.raises(aw.AWError) as ei:
                make()
            assert ei.value.code == aw.AW_ENOMEM, (k, str(ei.value))
            assert aw.aw_debug_alloc_stats()[0] == live0, k
    finally:
        aw.aw_debug_fail_alloc(-1)
    obj = make()            # disarmed: works again
    del obj
    assert aw.aw_debug_alloc_stats()[0] == live0
    return n


def test_injected_allocation_failures_in_kernel_synthesis(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = _small()
    n = _sweep(lambda: aw.aw_make_kernels(ctx, **kw))
    assert n >= 4


def test_injected_allocation_failures_in_plan_creation(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = _small()
    ks = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob)
    n = _sweep(lambda: aw.aw_plan_create(ctx, vd, ks))
    assert n >= 8


def test_injected_allocation_failures_in_surrogate_creation(ctx):
    from paper_2206_15117_gb300 import aw
    _sweep(lambda: aw.aw_surrogate_create(ctx, npol=4, width=32, n_hidden=4, omega0=30.0, seed=2))


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_give_up_and_the_context_stays_usable(ctx, which):
    from paper_2206_15117_gb300 import aw
    t0 = time.perf_counter()
    rc = aw.aw_debug_wait_timeout(ctx, which)
    dt = time.perf_counter() - t0
    assert rc == aw.AW_ETIMEOUT, rc
    assert dt < 60.0, dt
    # the context and the device keep working: a full-pol grid pass after the timeout
    ob, kw = _small()
    ks = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, ks)
    grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
    st = aw.aw_grid(ctx, plan, ks, torch.as_tensor(sy.random_vis(ob.nvis, 4, seed=3), device="cuda"), None, grid,
                    want_stats=True)
    assert st.n_gridded == aw.aw_plan_query(plan).nvalid > 0
    assert torch.isfinite(torch.view_as_real(grid)).all()
    assert aw.aw_debug_wait_timeout(ctx, 2) == aw.AW_EINVAL
