"""Seeded synthetic inputs (ReLU MLP implicit surfaces and seed rays).

This package only *builds* networks and rays from seeds.  It holds none of
the meshing arithmetic, so that both the CPU oracle and the CUDA path can
consume the same inputs without sharing any code of the method itself.
"""
from .nets import (  # noqa: F401
    MLP,
    octahedron,
    polytope_max_of_planes,
    fibonacci_normals,
    geometric_init,
    sibling,
    sphere_net,
    decoder_net,
    batch_nets,
    proposal_target_net,
    proposal_train_nets,
    tiny_net,
    leaky,
    residual_net,
    pooled_net,
    seed_rays,
    trigger_points,
)
