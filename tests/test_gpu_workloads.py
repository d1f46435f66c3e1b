"""The DeepSDF-shaped decoder (latent + skip-concat) in every precision on the first 60000
cells of its march, sampled faces re-solved by the oracle.  (The whole meshes of the large
workloads, the 64-net batch included, are in test_gpu_fullsize.py.)"""
import numpy as np
import pytest

from synth import decoder_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])


@pytest.mark.parametrize("precision", ["mixed", "fp64", "sliced"])
def test_full_decoder_sampled(oracle_mod, precision):
    # (3 + 256 latent) -> 512 x 8 -> 1, skip-concat of [x; z] at hidden layer 4 (N = 4096):
    # the first 60000 cells of the march, every sampled face re-solved by the oracle
    import paper_2106_10031_gb300 as am
    nt = decoder_net()
    with am.Mesher(max_cells=1 << 20, max_neurons=4096, max_width=512) as m:
        nid = m.load_mlp(nt)
        m.seed(nid, np.zeros((1, 3)), X_RAY)
        st = m.march(precision=precision, max_cells=60000)
        mesh = m.get_mesh(nid)
        stats = m.stats()
    print(f"decoder {precision}: {mesh.n_faces} faces of the first {stats['cells']} cells, "
          f"{stats['ms_march']:.1f} ms, refined {stats['refined_cells']}, close calls {stats['close_calls']}, "
          f"fixups {stats['fixups']}")
    assert st == 7 and mesh.n_faces >= 59000
    net = oracle_mod.OracleNet(nt)
    parity.compare_sampled(oracle_mod, net, mesh, nt.N, 24, 1e-5 if precision == "mixed" else 1e-9, 1.5)
