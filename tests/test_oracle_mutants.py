"""The oracle's pins must catch plausible mistakes.  Each case compiles a copy of the oracle's
C source with one planted mistake (in a temporary directory, on the CPU) and checks that
the pin that guards that part of the method fails for it, while the unmodified oracle passes."""
import os
import subprocess

import numpy as np
import pytest

from synth import decoder_net, octahedron, polytope_max_of_planes, tiny_net
from tests import pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "am_oracle.c")

MUTANTS = {
    "compose_drops_bias": ("Z[k * 4 + c] = acc + (c == 3 ? net.b[l][k] : 0.0);", "Z[k * 4 + c] = acc;"),
    "compose_ignores_mask": ("H[k * 4 + c] = s[row0 + k] ? Z[k * 4 + c] : 0.0;", "H[k * 4 + c] = Z[k * 4 + c];"),
    "aF_uses_unmasked_rows": ("acc += net.w_out[k] * H[k * 4 + c];", "acc += net.w_out[k] * Z[k * 4 + c];"),
    "skip_concat_misplaced": ("if (l == net.skip) memcpy(In + 4 * net.n[l - 1], X0, sizeof(double) * 4 * net.in_dim);",
                              "if (l == net.skip) memcpy(In + 4, X0, sizeof(double) * 4 * net.in_dim);"),
    "cell_sign_flipped": ("double sg = 1.0 - 2.0 * (double)s[k];", "double sg = 2.0 * (double)s[k] - 1.0;"),
    "tie_gives_one": ("s[k] = pre[k] > 0.0 ? 1 : 0;", "s[k] = pre[k] >= 0.0 ? 1 : 0;"),
    "pivot_keeps_previous_plane": ("if (u == t || u == tprev) continue;", "if (u == t) continue;"),
    "box_rows_wrong_sign": ("r[3] = -B;", "r[3] = B;"),
    "validity_skips_last_row": ("for (k = 0; k < M; ++k) {\n        const double *r = C + (size_t)k * 4;\n        double d;",
                                "for (k = 0; k < M - 7; ++k) {\n        const double *r = C + (size_t)k * 4;\n        double d;"),
    "trace_steps_uphill": ("x[i] = x[i] - eta * F * aF[i];", "x[i] = x[i] + eta * F * aF[i];"),
    "trace_drops_F": ("x[i] = x[i] - eta * F * aF[i];", "x[i] = x[i] - eta * aF[i];"),
}


def _build(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    return str(so)


def _pins_pass(O, lib):
    """A compact run of the pins: forward/compose/clip/mesh on small nets.  True if all hold."""
    try:
        for mlp in (tiny_net((6, 5, 4), 12), decoder_net(width=12, depth=4, latent_dim=4, skip_layer=3, seed=5)):
            net = O.OracleNet(mlp, lib=lib)
            rng = np.random.default_rng(0)
            for _ in range(4):
                s = rng.integers(0, 2, mlp.N).astype(np.uint8)
                A, aF = net.compose(s)
                A2, aF2 = pins.masked_affine_maps(mlp, s)
                if not (np.allclose(A, A2, atol=1e-10) and np.allclose(aF, aF2, atol=1e-10)):
                    return False
        o = O.OracleNet(octahedron(), lib=lib)
        if o.state(np.zeros(3)).tolist() != [0, 0, 0, 1, 1, 1]:
            return False
        ray = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])
        mlp = polytope_max_of_planes()
        area_ref, vol_ref, _ = pins.polytope_facets(mlp.meta["normals"], mlp.meta["offset"])
        net = O.OracleNet(mlp, lib=lib)
        for n in mlp.meta["normals"][:3]:
            # one sphere-tracing step, eta = 1/2, from 2 n_i where F = 3/2 and grad F = n_i
            rc, x, F, g, t = net.sphere_trace(2.0 * n, 0.5, 1, 0.0)
            if rc != 0 or np.abs(x - 1.25 * n).max() > 1e-12:
                return False
        net, mesh = O.mesh_from_rays(mlp, np.zeros((1, 3)), ray, lib=lib)
        if mesh.failed or not mesh.faces:
            return False
        xyz, faces, _ = mesh.assemble()
        if abs(pins.signed_volume(xyz, faces) - vol_ref) > 1e-9:
            return False
        if abs(sum(f.area() for f in mesh.faces) - area_ref.sum()) > 1e-9:
            return False
        mlp = tiny_net((8, 8), 11)
        brute = pins.enumerate_faces(mlp, O.DEFAULT_BOX)
        net = O.OracleNet(mlp, lib=lib)
        mesh = O.march(net, list(brute.items()))
        if mesh.failed or set(f.key for f in mesh.faces) != set(brute):
            return False
        for f in mesh.faces:
            C, aF = net.cell_rows(O.key_to_state(f.key, net.N))
            V3 = pins.halfspace_polygon(C, aF, f.verts.mean(0), O.DEFAULT_BOX)
            if len(V3) != len(f.verts):
                return False
            for v in f.verts:
                if np.min(np.linalg.norm(V3 - v, axis=1)) > 1e-8:
                    return False
        return True
    except (AssertionError, ValueError, np.linalg.LinAlgError, RuntimeError, Exception):
        return False


@pytest.mark.slow
def test_unmodified_oracle_passes(oracle_mod):
    assert _pins_pass(oracle_mod, oracle_mod.load_library())


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle_mod, tmp_path, name):
    lib = oracle_mod.load_library(_build(tmp_path, name))
    assert not _pins_pass(oracle_mod, lib)
