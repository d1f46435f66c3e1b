"""The binding checks every array's shape before it reaches the C side (which trusts the sizes
it is given).  The real Mesher methods run against a stub library that records the calls; CPU
only."""
import ctypes as C

import numpy as np
import pytest

from synth import (batch_nets, decoder_net, leaky, octahedron, polytope_max_of_planes, proposal_target_net,
                   pooled_net, proposal_train_nets, residual_net, sibling, sphere_net, tiny_net)


class _Stub:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            return 0
        return f


@pytest.fixture
def mesher():
    from paper_2106_10031_gb300 import mesher as M
    m = object.__new__(M.Mesher)
    m.lib, m.ctx, m.nets, m.device = _Stub(), C.c_void_p(), [], 0
    return m


@pytest.mark.parametrize("make", [
    lambda: decoder_net(width=24, depth=6, latent_dim=9, skip_layer=3, seed=7, sigma=0.05),
    lambda: decoder_net(), sphere_net, polytope_max_of_planes, lambda: tiny_net((6, 5, 4), 12), octahedron,
    proposal_target_net, lambda: batch_nets()[0], lambda: batch_nets()[63],
    lambda: sibling(sphere_net(), seed=99), lambda: sibling(leaky(sphere_net(), 0.1), seed=3),
    lambda: leaky(tiny_net((6, 5, 4), 12), -0.25), lambda: proposal_train_nets()[31],
    lambda: residual_net(seed=40, width=12, depth=6), lambda: leaky(residual_net(seed=32, width=24, depth=6), 0.1),
    lambda: pooled_net(seed=62, count=4, width=8, depth=3), lambda: pooled_net(),
])
def test_every_workload_net_passes(mesher, make):
    mesher.load_mlp(make())
    assert mesher.lib.calls == ["am_load_mlp"]


def test_malformed_nets_never_reach_the_library(mesher):
    import copy
    base = tiny_net((6, 5, 4), 12)
    bad_fan = copy.deepcopy(base)
    bad_fan.weights[1] = np.zeros((5, 7))
    bad_bias = copy.deepcopy(base)
    bad_bias.biases[2] = np.zeros(3)
    bad_out = copy.deepcopy(base)
    bad_out.w_out = np.zeros(5)
    bad_skip = copy.deepcopy(base)
    bad_skip.skip_layer = 9
    bad_sc_src = copy.deepcopy(base)
    bad_sc_src.shortcuts = {2: (2, None)}                  # not an earlier layer
    bad_sc_id = copy.deepcopy(base)
    bad_sc_id.shortcuts = {3: (1, None)}                   # identity from 6 units into 4
    bad_sc_S = copy.deepcopy(base)
    bad_sc_S.shortcuts = {3: (1, np.zeros((4, 5)))}        # S must be 4 x 6
    bad_heads = copy.deepcopy(base)
    bad_heads.heads = [(np.zeros(4), 0.0), (np.zeros(5), 0.0)]   # a head must read the 4 last units
    one_head = copy.deepcopy(base)
    one_head.heads = [(np.zeros(4), 0.0)]                   # pooling needs two heads or more
    for mlp in (bad_fan, bad_bias, bad_out, bad_skip, bad_sc_src, bad_sc_id, bad_sc_S, bad_heads, one_head):
        with pytest.raises(ValueError):
            mesher.load_mlp(mlp)
    assert mesher.lib.calls == []


def test_point_arrays_are_checked(mesher):
    for o, d in ((np.zeros((2, 3)), np.zeros((1, 3))), (np.zeros((2, 2)), np.zeros((2, 2))),
                 (np.zeros((0, 3)), np.zeros((0, 3)))):
        with pytest.raises(ValueError):
            mesher.seed(0, o, d)
    with pytest.raises(ValueError):
        mesher.seed_sphere_trace(0, np.zeros((4, 2)))
    with pytest.raises(ValueError):
        mesher.seed_pairs(0, np.zeros(5), 3)
    with pytest.raises(ValueError):
        mesher.seed_pairs(0, np.zeros((5, 3)), 0)
    assert mesher.lib.calls == []
    mesher.seed(0, np.zeros(3), [1.0, 0.0, 0.0])        # a single ray as flat 3-vectors
    mesher.seed_sphere_trace(0, [[0.1, 0.2, 0.3]])
    mesher.seed_pairs(0, np.zeros((5, 3)), 2)
    assert mesher.lib.calls == ["am_seed", "am_seed_sphere_trace", "am_seed_pairs"]


def test_key_arrays_are_checked():
    from paper_2106_10031_gb300 import mesher as M
    assert M._key_array(np.zeros((5, 2), dtype=np.uint64), 128).shape == (5, 2)
    assert M._key_array(np.zeros((0, 1), dtype=np.uint64), 16).shape == (0, 1)
    for bad, N in ((np.zeros((5, 1)), 128), (np.zeros(5), 16), (np.zeros((5, 3)), 128)):
        with pytest.raises(ValueError):
            M._key_array(bad, N)


def test_proposal_tensors_are_checked(mesher):
    # no CUDA here: every host tensor must be refused before a pointer reaches the library
    import torch
    mesher.prop_shape = (15, 32, 64)
    X, Y = torch.zeros((8, 15)), torch.zeros((8, 64))
    for call in (lambda: mesher.proposal_forward(X), lambda: mesher.proposal_grad(X, Y),
                 lambda: mesher.proposal_train(X, Y, 4, 2, 1e-3)):
        with pytest.raises(ValueError):
            call()
    assert mesher.lib.calls == []
    del mesher.prop_shape
    with pytest.raises(ValueError):
        mesher.proposal_forward(X)
