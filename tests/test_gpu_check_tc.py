"""The dense all-constraint check on the tcgen05 tensor cores (am_tuning.check_kernel = 1): every
row of a cell tested at every vertex of its clipped polygon (Eq. 10), each 128-row tile of rows
times the vertices as one product of exact BF16 parts, then a certified sign test with FP64 close
calls.  The sliced level march with it must give the same mesh as with the check in the warp
(faces, edge cycles, vertex identities) and the oracle's mesh: on the 3-[64]x4-1 net face by
face, on the whole 3-[256]x8-1 mesh through the oracle's whole-mesh digest.  Needs a GPU."""
import json
import os

import numpy as np
import pytest

from synth import proposal_target_net, sphere_net
from tests import meshcheck, parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])
ORIGIN = np.zeros((1, 3))
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "whole_mesh_oracle.json")


def _march_both(mlp, candidates, ctx, **kw):
    import paper_2106_10031_gb300 as am
    out = {}
    with am.Mesher(**ctx) as m:
        nid = m.load_mlp(mlp)
        if candidates == "learned":
            m.proposal_init(7 + mlp.L, 64, mlp.N, max_batch=1024, seed=3)
        for ck in (0, 1):
            m.set_tuning(check_kernel=ck)
            m.reset()
            m.seed(nid, ORIGIN, X_RAY)
            rc = m.march(precision="sliced", candidates=candidates, **kw)
            assert rc == 0
            out[ck] = (m.get_mesh(nid), m.stats())
    return out


@pytest.mark.parametrize("candidates", ["nearest", "learned"])
def test_tc_check_sphere_net_equals_warp_check_and_oracle(oracle_mod, candidates):
    mlp = sphere_net()
    res = _march_both(mlp, candidates, dict(max_cells=1 << 17, max_neurons=256, max_width=64))
    (m0, s0), (m1, s1) = res[0], res[1]
    f0, f1 = parity.gpu_faces(m0), parity.gpu_faces(m1)
    assert set(f0) == set(f1)
    assert all(f0[k][0] == f1[k][0] for k in f0)
    worst = max(float(np.abs(f0[k][1] - f1[k][1]).max()) for k in f0)
    print(f"\nsphere {candidates}: {len(f1)} faces; warp check {s0['ms_clip']:.1f} ms clip, tensor-core check "
          f"{s1['ms_clip']:.1f} ms; fallbacks {s0['clip_fallbacks']} / {s1['clip_fallbacks']}; close calls "
          f"{s0['close_calls']} / {s1['close_calls']}; max vertex difference {worst:.1e}")
    assert worst < 1e-9                      # cells with violated rows are cut in by another kernel
    assert s1["degenerate"] == 0
    _, ref = oracle_mod.mesh_from_rays(mlp, ORIGIN, X_RAY)
    parity.compare(ref, m1, mlp.N, rtol=1e-9)


def test_tc_check_whole_target_net_is_the_oracles(oracle_mod):
    mlp = proposal_target_net()
    res = _march_both(mlp, "nearest", dict(max_cells=1 << 22, max_neurons=2048, max_width=256))
    (m0, s0), (m1, s1) = res[0], res[1]
    print(f"\n3-[256]x8-1: {s1['faces']} faces; march {s0['ms_march']:.0f} ms (warp check) vs {s1['ms_march']:.0f} ms "
          f"(tensor-core check), clip {s0['ms_clip']:.0f} vs {s1['ms_clip']:.0f} ms; fallbacks {s0['clip_fallbacks']} "
          f"/ {s1['clip_fallbacks']}")
    d0, d1 = meshcheck.digest(m0, mlp.N), meshcheck.digest(m1, mlp.N)
    for k in ("faces", "corners", "vertices", "open_faces", "euler", "keys0", "keys1", "cycles"):
        assert d0[k] == d1[k], (k, d0[k], d1[k])
    assert d1["open_faces"] == 0 and d1["euler"] == 2
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            g = [x for x in json.load(f)["meshes"] if x["name"] == "learned_target_256x8"]
        if g:
            for k in ("faces", "corners", "vertices", "open_faces", "euler", "keys0", "keys1", "cycles"):
                assert d1[k] == g[0]["digest"][k], (k, d1[k], g[0]["digest"][k])
    net = oracle_mod.OracleNet(mlp)
    parity.compare_sampled(oracle_mod, net, m1, mlp.N, 300, 1e-9, 1.5)
