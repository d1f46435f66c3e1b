"""The larger workloads on the GPU: 64 nets marched together in one launch, and the
DeepSDF-shaped decoder (latent + skip-concat) at full size.  Parity with the oracle on every
face where the oracle finishes in seconds, on sampled faces otherwise, plus completeness by
the closure invariants."""
import numpy as np
import pytest

from synth import batch_nets, decoder_net
from tests import parity

pytestmark = pytest.mark.gpu
X_RAY = np.array([[1.0, 0.0, 0.0]])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_of_nets_in_one_march(oracle_mod, precision):
    # the nets of the 64-net batch with width <= 64 (21 nets, widths 32/64, depths 4/6/8,
    # sigma 0.02..0.1, about 1.5e6 cells together), marched in one persistent launch
    import paper_2106_10031_gb300 as am
    nets = [n for n in batch_nets() if n.widths[0] <= 64]
    box = 2.0
    with am.Mesher(max_cells=1 << 22, max_neurons=512, max_width=64) as m:
        ids = [m.load_mlp(n) for n in nets]
        for i in ids:
            m.seed(i, np.zeros((1, 3)), X_RAY, R=2.0)
        m.march(box=box, precision=precision)
        meshes = [m.get_mesh(i) for i in ids]
        st = m.stats()
    assert st["cell_launches"] == 1                # every net in one persistent launch
    sizes = [mm.n_faces for mm in meshes]
    print(f"batch {precision}: {sum(sizes)} faces over {len(nets)} nets (min {min(sizes)}, max {max(sizes)}), "
          f"{st['ms_march']:.1f} ms march, refined {st['refined_cells']}, close calls {st['close_calls']}")
    assert min(sizes) > 0
    small = np.argsort([n.N * s for n, s in zip(nets, sizes)])[:6]
    for i, (nt, mesh) in enumerate(zip(nets, meshes)):
        parity.closure(mesh, nt.N)
        net = oracle_mod.OracleNet(nt)
        if i in small:
            seeds = oracle_mod.seed_cells(net, np.zeros((1, 3)), X_RAY, R=2.0)
            ref = oracle_mod.march(net, seeds, box=box)
            parity.compare(ref, mesh, nt.N, rtol=1e-9 if precision == "fp64" else 1e-5)
        else:
            parity.compare_sampled(oracle_mod, net, mesh, nt.N, 8, 1e-9 if precision == "fp64" else 1e-5, box)


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
