"""ctypes binding of the C ABI in include/analytic_marching.h (argument marshalling only).

Every step of analytic marching runs in the CUDA library; this module only declares the
entry points with the same names and converts numpy arrays to pointers.  Loading fails
loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libam_gb300.so")

# am_status
AM_OK = 0
AM_ERR_INVALID_ARG = 1
AM_ERR_CUDA = 2
AM_ERR_CAPACITY = 3
AM_ERR_TIMEOUT = 4
AM_ERR_NO_SEED_CELL = 5
AM_ERR_DEGENERATE = 6
AM_INCOMPLETE = 7
AM_ERR_STATE = 8
STATUS_NAMES = {0: "AM_OK", 1: "AM_ERR_INVALID_ARG", 2: "AM_ERR_CUDA", 3: "AM_ERR_CAPACITY",
                4: "AM_ERR_TIMEOUT", 5: "AM_ERR_NO_SEED_CELL", 6: "AM_ERR_DEGENERATE",
                7: "AM_INCOMPLETE", 8: "AM_ERR_STATE"}

AM_PREC_FP64 = 0
AM_PREC_MIXED = 1
AM_PREC_TENSOR = 2
AM_PREC_SLICED = 3
AM_SCHED_PERSISTENT = 0
AM_SCHED_LEVELS = 1
AM_CAND_NEAREST = 0
AM_CAND_LEARNED = 1
AM_CAND_NONE = 2


class am_ctx_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("max_cells", C.c_int64),
                ("hash_slots", C.c_int64), ("max_face_verts", C.c_int), ("max_neurons", C.c_int),
                ("max_width", C.c_int)]


class am_mlp_desc(C.Structure):
    _fields_ = [("latent_dim", C.c_int), ("latent", C.POINTER(C.c_double)), ("n_hidden", C.c_int),
                ("width", C.POINTER(C.c_int)), ("W", C.POINTER(C.POINTER(C.c_double))),
                ("b", C.POINTER(C.POINTER(C.c_double))), ("skip_layer", C.c_int),
                ("w_out", C.POINTER(C.c_double)), ("b_out", C.c_double), ("slope", C.c_double),
                ("shortcut_src", C.POINTER(C.c_int)), ("shortcut_S", C.POINTER(C.POINTER(C.c_double))),
                ("n_heads", C.c_int), ("w_heads", C.POINTER(C.c_double)), ("b_heads", C.POINTER(C.c_double))]


class am_march_opts(C.Structure):
    _fields_ = [("box", C.c_double), ("delta", C.c_double), ("precision", C.c_int),
                ("max_cells", C.c_int64), ("candidates", C.c_int), ("schedule", C.c_int),
                ("grid_blocks", C.c_int)]


class am_tuning(C.Structure):
    _fields_ = [("compose_tile_cells", C.c_int), ("rank1_period", C.c_int), ("clip_kernel", C.c_int),
                ("check_kernel", C.c_int)]


class am_tune_point(C.Structure):
    _fields_ = [("compose_tile_cells", C.c_int), ("ms", C.c_float)]


class am_march_point(C.Structure):
    _fields_ = [("precision", C.c_int), ("schedule", C.c_int), ("ms", C.c_float)]


class am_stats_t(C.Structure):
    _fields_ = [("cells", C.c_int64), ("faces", C.c_int64), ("empty_faces", C.c_int64),
                ("vertices", C.c_int64), ("corners", C.c_int64), ("degenerate", C.c_int64),
                ("open_faces", C.c_int64), ("refined_cells", C.c_int64), ("levels", C.c_int64),
                ("ms_march", C.c_double), ("ms_assemble", C.c_double), ("ms_cell_kernels", C.c_double),
                ("cell_launches", C.c_int64), ("kernel_launches", C.c_int64), ("close_calls", C.c_int64),
                ("fixups", C.c_int64), ("cuts", C.c_int64), ("phase_cycles", C.c_int64 * 10),
                ("ms_compose", C.c_double), ("ms_clip", C.c_double), ("ms_proposal", C.c_double),
                ("clip_fallbacks", C.c_int64), ("tensor_macs", C.c_int64)]


class am_mesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_faces", C.c_int64), ("n_corners", C.c_int64),
                ("key_words", C.c_int), ("n_open_faces", C.c_int64),
                ("xyz", C.POINTER(C.c_double)), ("face_offsets", C.POINTER(C.c_int64)),
                ("face_vertices", C.POINTER(C.c_int32)), ("edge_planes", C.POINTER(C.c_int32)),
                ("face_keys", C.POINTER(C.c_uint64))]


# (name, restype, argtypes) of every entry point declared in include/analytic_marching.h
ENTRY_POINTS = [
    ("am_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(am_ctx_opts)]),
    ("am_destroy", None, [C.c_void_p]),
    ("am_last_error", C.c_char_p, [C.c_void_p]),
    ("am_load_mlp", C.c_int, [C.c_void_p, C.POINTER(am_mlp_desc), C.POINTER(C.c_int)]),
    ("am_reset", C.c_int, [C.c_void_p]),
    ("am_release_nets", C.c_int, [C.c_void_p]),
    ("am_seed", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                          C.c_double, C.POINTER(C.c_int)]),
    ("am_march", C.c_int, [C.c_void_p, C.POINTER(am_march_opts)]),
    ("am_get_mesh", C.c_int, [C.c_void_p, C.c_int, C.POINTER(am_mesh)]),
    ("am_get_stats", C.c_int, [C.c_void_p, C.POINTER(am_stats_t)]),
    ("am_get_mesh_device", C.c_int, [C.c_void_p, C.c_int, C.POINTER(am_mesh)]),
    ("am_seed_sphere_trace", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double,
                                        C.POINTER(C.c_int), C.c_void_p]),
    ("am_mesh_canonicalize", C.c_int, [C.POINTER(am_mesh)]),
    ("am_mesh_triangulate", C.c_int, [C.POINTER(am_mesh), C.c_void_p, C.POINTER(C.c_int64)]),
    ("am_seed_pairs", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.c_void_p]),
    ("am_compose", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    ("am_compose_neighbors", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                       C.c_void_p]),
    ("am_set_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("am_autotune_compose", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_int, C.c_void_p]),
    ("am_get_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("am_autotune_march", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int64,
                                    C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("am_proposal_samples", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("am_proposal_init", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64]),
    ("am_proposal_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    ("am_proposal_set_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    ("am_proposal_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("am_proposal_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int64,
                                   C.c_void_p]),
    ("am_proposal_train", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_float,
                                    C.c_void_p]),
    ("am_test_stall_next_march", C.c_int, [C.c_void_p, C.c_int64, C.c_double]),
    ("am_assign_vertices_noalloc", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                             C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
]

_lib = None


def load(path: str | None = None):
    """Load libam_gb300.so (built by paper_2106_10031_gb300.build) and declare its entry points."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_2106_10031_gb300.build.build())")
    lib = C.CDLL(p)
    for name, res, args in ENTRY_POINTS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib
