"""The time-out path of the persistent march, without faulting or hanging the GPU.

Every wait of the persistent march for work is bounded.  am_test_stall_next_march hands out
cell ids that no block ever publishes, with a short wait limit, so the blocks that take those
tickets must give up, set the time-out status and return: am_march reports AM_ERR_TIMEOUT
within about the limit, refuses to march again until am_reset, and afterwards the same
context meshes a net exactly as the oracle does."""
import ctypes as C
import time

import numpy as np
import pytest

from synth import sphere_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))


def test_ticket_wait_times_out_then_the_context_recovers(oracle_mod):
    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300 import native as nt
    mlp = sphere_net(seed=21, width=32, depth=4)
    with am.Mesher(max_cells=1 << 16, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, ORIGIN, X_RAY)
        assert m.lib.am_test_stall_next_march(m.ctx, 4096, 20.0) == nt.AM_OK
        t0 = time.perf_counter()
        st = m.lib.am_march(m.ctx, C.byref(nt.am_march_opts()))       # persistent schedule
        dt = time.perf_counter() - t0
        assert st == nt.AM_ERR_TIMEOUT, m.lib.am_last_error(m.ctx)
        assert dt < 2.0, f"gave up after {dt:.2f} s, not after the 20 ms limit"
        # no mesh from a march that timed out, and no further march before am_reset
        assert m.lib.am_march(m.ctx, C.byref(nt.am_march_opts())) == nt.AM_ERR_STATE
        with pytest.raises(am.AMError):
            m.get_mesh(nid)
        m.reset()
        m.seed(nid, ORIGIN, X_RAY)
        m.march()
        mesh = m.get_mesh(nid)
    net, ref = oracle_mod.mesh_from_rays(mlp, ORIGIN, X_RAY)
    parity.compare(ref, mesh, mlp.N, rtol=1e-9)


def test_stall_hook_refuses_the_level_schedule_and_bad_arguments():
    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300 import native as nt
    mlp = sphere_net(seed=21, width=32, depth=4)
    with am.Mesher(max_cells=1 << 16, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        assert m.lib.am_test_stall_next_march(m.ctx, 0, 20.0) == nt.AM_ERR_INVALID_ARG
        assert m.lib.am_test_stall_next_march(m.ctx, 16, 0.0) == nt.AM_ERR_INVALID_ARG
        assert m.lib.am_test_stall_next_march(m.ctx, (1 << 16) + 1, 20.0) == nt.AM_ERR_INVALID_ARG
        m.seed(nid, ORIGIN, X_RAY)
        assert m.lib.am_test_stall_next_march(m.ctx, 16, 20.0) == nt.AM_OK
        op = nt.am_march_opts(schedule=nt.AM_SCHED_LEVELS)
        assert m.lib.am_march(m.ctx, C.byref(op)) == nt.AM_ERR_INVALID_ARG
        # the refused march consumed the hook: the next one runs normally
        m.march(schedule="levels")
        assert m.stats()["faces"] > 0
