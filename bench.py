"""Benchmark: analytic faces per second of analytic marching on one GB300.

One step = the whole hot path on one mesh: forget the previous cells, trigger the seed
cell by bisection on the device, march every analytic cell (compose, clip, emit, hash
march) and assemble the mesh.  The workload is the 3-[64]x4-1 geometric-init SDF net
(seed 2, every parameter perturbed by N(0, 0.05^2)) with one seed ray along +x, clipped
to the box [-1.5, 1.5]^3 (43,780 faces).  The headline is mixed precision with the learned
constraint proposal (trained before timing on the plain method's mesh of a nearby checkpoint
of the net); the comparison legs time the plain FP64 method (every cutting row clipped), the
nearest-row candidates and the other precision.  Inputs (the net, the proposal) are resident
in HBM when the timed region starts; the e2e leg repeats the step through the C ABI from
pinned host buffers (net upload, seed ray, mesh download) inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                  [--candidates learned|nearest|none] [--impl reference]

Multi-GPU: each rank meshes its own copy of the workload (replicas, no collective on the
data path); the job's value is the faces of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "analytic faces/sec on 1 GB300 (oracle-exact mesh); mixed+learned vs plain FP64"
UNIT = "faces/s"
WORKLOAD = "3-[64]x4-1 geometric-init SDF MLP (seed 2, sigma 0.05), 1 seed ray +x, box 1.5"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12     # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (derived)
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12   # 128 FFMA/clk/SM x 152 SMs x 2.07 GHz (derived)


def _measured_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0                              # fallback figure for a GB300


BF16_PEAK_TFLOPS = _measured_bf16_peak()


def _measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0                              # fallback figure for a GB300


HBM_PEAK_GBS = _measured_hbm_peak()


# DRAM bytes of one march_persistent_kernel launch (double-float + learned candidates, bench
# workload) from the committed ncu capture, valid while the kernel source is the one captured
TRAFFIC_CAPTURE = {"sha256_prefix": "46d62118611829ca", "precision": "mixed", "candidates": "learned",
                   "bytes": 2.973440e6 + 0.518912e6}


def captured_traffic(precision, candidates):
    import hashlib
    src = os.path.join(ROOT, "paper_2106_10031_gb300", "csrc", "am_march.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    c = TRAFFIC_CAPTURE
    if h == c["sha256_prefix"] and (precision, candidates) == (c["precision"], c["candidates"]):
        return c["bytes"]
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--schedule", default="persistent", choices=["persistent", "levels"])
    p.add_argument("--candidates", default="learned", choices=["nearest", "learned", "none"])
    p.add_argument("--no-compare", action="store_true", help="skip the comparison legs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--learned-only", action="store_true",
                   help="run only the 3-[256]x8-1 learned-proposal leg and print its JSON")
    p.add_argument("--decoder-only", action="store_true",
                   help="run only the decoder march leg (FP64 vs sliced tensor-core compose) and print its JSON")
    p.add_argument("--batch-only", action="store_true",
                   help="run only the 64-net batch leg (nets sharded over the ranks) and print its JSON")
    p.add_argument("--triggers-only", action="store_true",
                   help="run only the customised-trigger leg (sphere tracing, random pairs) and print its JSON")
    p.add_argument("--compose-only", action="store_true",
                   help="run only the compose benchmark (am_compose on the decoder) and print its JSON")
    return p.parse_args()


def workload():
    from synth import sphere_net
    return sphere_net(seed=2, width=64, depth=4, sigma=0.05), np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])


# ------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)


class Dist:
    def __init__(self, n_gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def allreduce(self, x: float, op: str) -> float:
        if not self.pg:
            return x
        import torch
        dev = f"cuda:{self.local}" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# algorithmic work of the cell kernel


def algorithmic_work(mlp, mesh) -> dict:
    """Work the cell kernel must do per mesh, from the mesh's cell keys.

    macs: masked multiply-adds of the compose (Cor. 1), per cell sum over l >= 2 of
    n_l x |active(l-1)| row-column products for 4 columns, plus a_F over |active(L)|;
    checks: (row, vertex) sign tests of the certification, (N + 6) x |face| per cell.
    FP64 path: 2 flops per multiply-add and per check term (4-term dot products).
    Learned candidates add the proposal's forward pass, 2 (I H + H H + H N) FP32 flops per cell.
    Mixed path: one double-float multiply-add is 15 FP32 flops (TwoProd + TwoSum + 2 cross
    FMAs) per column, 63 per row-column product with the error-bound FMA; one check is 22 FP32
    flops (dot product, magnitude and bound)."""
    widths = mlp.widths
    N = mlp.N
    keys = mesh.face_keys
    bits = np.unpackbits(keys.view(np.uint8), axis=1, bitorder="little")[:, :N].astype(np.int64)
    r = np.cumsum([0] + widths)
    rc = np.zeros(len(keys), dtype=np.int64)
    for l in range(1, len(widths)):
        rc += widths[l] * bits[:, r[l - 1]:r[l]].sum(1)
    rc += bits[:, r[-2]:r[-1]].sum(1)
    checks = (N + 6) * np.diff(mesh.face_offsets)
    I, H = 7 + len(widths), 256
    prop = 2 * (I * H + H * H + H * N) * len(keys)          # the learned proposal's forward per cell
    return {"row_col_products": int(rc.sum()), "checks": int(checks.sum()), "proposal_fp32_flops": int(prop),
            "fp64_flops": int(8 * rc.sum() + 8 * checks.sum()),
            "df_fp32_flops": int(63 * rc.sum() + 22 * checks.sum())}


# ------------------------------------------------------------------------------------------


def cpu_baseline(mlp, o, d, budget_s=12.0):
    """The oracle as it stands on this host, on a bounded prefix of the same march
    (breadth-first order, at most budget_s of single-thread CPU time): timed single-threaded,
    then on every host core (oracle/parallel.py: the same per-cell arithmetic, each
    breadth-first level solved by a pool of spawned processes; the mesh is the serial one).
    `value` is the all-core figure; if the pool cannot run, the single-thread one."""
    from oracle import oracle as O
    O.build()
    net = O.OracleNet(mlp)
    seeds = O.seed_cells(net, o, d)
    probe = 500
    t0 = time.perf_counter()
    O.march(net, seeds, max_cells=probe)
    per = (time.perf_counter() - t0) / probe
    n = max(probe, min(60000, int(budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    mesh = O.march(net, seeds, max_cells=n)
    dt = time.perf_counter() - t0
    faces = len(mesh.faces)
    single = {"value": faces / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"first {n} cells of the breadth-first march ({faces} faces) in {dt:.1f} s, "
                        f"single thread (plain C per cell + Python loop)"}
    try:
        from oracle.parallel import LevelMarcher
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        with LevelMarcher(mlp, workers=cores, timeout=120.0) as lm:
            t0 = time.perf_counter()
            pm = lm.march(seeds, max_cells=n)
            dtp = time.perf_counter() - t0
        if len(pm.faces) != faces:
            raise RuntimeError("the all-core march differs from the serial one")
        return {"value": faces / dtp, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"first {n} cells of the breadth-first march ({faces} faces) in {dtp:.1f} s on {cores} "
                          f"processes, one breadth-first level at a time (per cell: plain C + Python)",
                "single_thread": single}, mesh
    except Exception as e:                          # noqa: BLE001 -- the single-thread figure stands
        single["all_cores_unavailable"] = f"{type(e).__name__}: {e}"
        return single, mesh


def oracle_agreement(ref, mesh):
    """The headline mesh against the oracle's mesh of the CPU-baseline run: every oracle face
    must be a GPU face with the same edge cycle; vertex error relative to max(1, |v|)."""
    from tests import parity
    got = parity.gpu_faces(mesh)
    errs, cycles, missing = [], 0, 0
    for f in ref.faces:
        g = got.get(f.key)
        if g is None:
            missing += 1
            continue
        if f.edges != g[0]:
            cycles += 1
            continue
        errs.append(np.linalg.norm(f.verts - g[1], axis=1) / np.maximum(1.0, np.linalg.norm(f.verts, axis=1)))
    e = np.concatenate(errs) if errs else np.zeros(1)
    return {"oracle_faces": len(ref.faces), "gpu_faces": len(got), "missing_in_gpu": missing,
            "edge_cycles_differing": cycles, "max_rel_vertex_err": float(e.max()),
            "p99_rel_vertex_err": float(np.quantile(e, 0.99)),
            "whole_mesh_identical": missing == 0 and cycles == 0 and len(ref.faces) == len(got)}


def run_reference(args, dist):
    """The oracle as it stands, as the reference arm, on every host core: each step is the
    whole breadth-first march of the workload, one level at a time in a pool of spawned
    processes (oracle/parallel.py; the mesh is the serial march's).  If the pool cannot run,
    each step is the first 3000 cells of the serial march, single-threaded."""
    if dist.rank != 0:
        return 0
    mlp, o, d = workload()
    from oracle import oracle as O
    O.build()
    net = O.OracleNet(mlp)
    seeds = O.seed_cells(net, o, d)
    lm, cores = None, 1
    try:
        from oracle.parallel import LevelMarcher
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        lm = LevelMarcher(mlp, workers=cores, timeout=120.0)
    except Exception:                               # noqa: BLE001 -- single-thread fallback below
        lm, cores = None, 1
    try:
        if lm is not None:
            def step():
                return lm.march(seeds)
            sample = f"each step: the whole breadth-first march on {cores} processes, one level at a time"
        else:
            def step():
                return O.march(net, seeds, max_cells=3000)
            sample = "each step: first 3000 cells of the breadth-first march, single thread"
        for _ in range(max(0, args.warmup)):
            step()
        t0 = time.perf_counter()
        faces = 0
        for _ in range(args.steps):
            faces += len(step().faces)
        dt = time.perf_counter() - t0
    finally:
        if lm is not None:
            lm.close()
    v = faces / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def e2e_leg(mlp, o, d, steps, device, stream_ptr, precision, candidates, prop=None):
    """Same step through the C ABI with host buffers: upload the net from pinned memory,
    seed from a pinned host ray, march, copy the mesh back into pinned host buffers.  A
    learned proposal (prop = (params, (n_in, hidden, n_out))) is loaded once, untimed."""
    import torch

    from paper_2106_10031_gb300 import native as nt
    lib = nt.load()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()  # noqa: E731
    Wp = [pin(w) for w in mlp.weights]
    bp = [pin(b) for b in mlp.biases]
    wo = pin(mlp.w_out)
    ray_o, ray_d = pin(o), pin(d)
    L = mlp.L
    dp = lambda t: C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double))  # noqa: E731
    desc = nt.am_mlp_desc(latent_dim=0, latent=None, n_hidden=L, width=(C.c_int * L)(*mlp.widths),
                          W=(C.POINTER(C.c_double) * L)(*[dp(w) for w in Wp]),
                          b=(C.POINTER(C.c_double) * L)(*[dp(b) for b in bp]), skip_layer=0,
                          w_out=dp(wo), b_out=float(mlp.b_out))
    ctx = C.c_void_p()
    opts = nt.am_ctx_opts(device=device, stream=stream_ptr, max_cells=1 << 17, hash_slots=0, max_face_verts=32,
                          max_neurons=256, max_width=64)
    assert lib.am_create(C.byref(ctx), C.byref(opts)) == 0, lib.am_last_error(ctx)
    cand = {"nearest": nt.AM_CAND_NEAREST, "learned": nt.AM_CAND_LEARNED, "none": nt.AM_CAND_NONE}[candidates]
    if cand == nt.AM_CAND_LEARNED:
        params, (n_in, hidden, n_out) = prop
        assert lib.am_proposal_init(ctx, n_in, hidden, n_out, 1024, 0) == 0
        assert lib.am_proposal_set_params(ctx, params.ctypes.data_as(C.c_void_p), len(params)) == 0
    mo = nt.am_march_opts(box=1.5, delta=1e-10, precision=precision, max_cells=0, candidates=cand)
    bufs = None
    h2d = sum(w.numel() * 8 for w in Wp + bp) + wo.numel() * 8 + 48
    d2h = 0

    def step():
        nonlocal bufs, d2h
        assert lib.am_release_nets(ctx) == 0
        nid = C.c_int()
        assert lib.am_load_mlp(ctx, C.byref(desc), C.byref(nid)) == 0
        ns = C.c_int()
        assert lib.am_seed(ctx, nid, dp(ray_o), dp(ray_d), 1, 2.0, C.byref(ns)) == 0
        assert lib.am_march(ctx, C.byref(mo)) == 0, lib.am_last_error(ctx)
        m = nt.am_mesh()
        assert lib.am_get_mesh(ctx, nid, C.byref(m)) == 0
        if bufs is None:
            bufs = {"xyz": torch.empty(3 * m.n_vertices + 3, dtype=torch.float64).pin_memory(),
                    "off": torch.empty(m.n_faces + 1, dtype=torch.int64).pin_memory(),
                    "fv": torch.empty(m.n_corners + 1, dtype=torch.int32).pin_memory(),
                    "fe": torch.empty(m.n_corners + 1, dtype=torch.int32).pin_memory(),
                    "keys": torch.empty(m.n_faces * m.key_words + 1, dtype=torch.int64).pin_memory()}
            d2h = (3 * m.n_vertices * 8 + (m.n_faces + 1) * 8 + 2 * m.n_corners * 4 + m.n_faces * m.key_words * 8)
        m.xyz = C.cast(C.c_void_p(bufs["xyz"].data_ptr()), C.POINTER(C.c_double))
        m.face_offsets = C.cast(C.c_void_p(bufs["off"].data_ptr()), C.POINTER(C.c_int64))
        m.face_vertices = C.cast(C.c_void_p(bufs["fv"].data_ptr()), C.POINTER(C.c_int32))
        m.edge_planes = C.cast(C.c_void_p(bufs["fe"].data_ptr()), C.POINTER(C.c_int32))
        m.face_keys = C.cast(C.c_void_p(bufs["keys"].data_ptr()), C.POINTER(C.c_uint64))
        assert lib.am_get_mesh(ctx, nid, C.byref(m)) == 0
        return m.n_faces

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    faces = 0
    for _ in range(steps):
        faces += step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    lib.am_destroy(ctx)
    return {"value": faces / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt / steps * 1e3}


def measure(m, nid, o, d, steps, precision, schedule, flush, stream, candidates="nearest"):
    """K timed steps; L2 flushed before each (outside the events).  Returns totals."""
    import torch

    def step():
        m.reset()
        m.seed(nid, o, d)
        m.march(precision=precision, schedule=schedule, candidates=candidates)

    total_ms, cell_ms, launches, cell_launches = 0.0, 0.0, 0, 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        st = m.stats()
        cell_ms += st["ms_cell_kernels"]
        cell_launches += st["cell_launches"]
        launches += st["kernel_launches"]
    return {"total_ms": total_ms, "cell_ms": cell_ms, "launches": launches, "cell_launches": cell_launches,
            "stats": m.stats()}


def compose_leg(dev, n_cells=4000, reps=5):
    """The compose step alone (am_compose) on the decoder-shaped net, (3 + 256) -> [512] x 8 -> 1
    with skip-concat at layer 4, for the patterns of the first n_cells cells of its march, in the
    four precisions.  Dense work per cell: 8 n_l n_{l-1} flops over the hidden layers (4 columns
    of the cell's affine maps, Cor. 1); the split-BF16 path issues 4 m16n8k16 MMAs per 16 x 16
    weight tile, the sliced path 36 digit-plane products per layer (the tile shape picked by the
    autotuner on these patterns)."""
    import ctypes as C

    import torch

    import paper_2106_10031_gb300 as am
    from synth import decoder_net
    mlp = decoder_net()
    out = {"workload": f"decoder (3+256)-[512]x8-1, skip at 4; patterns of the first {n_cells} cells"}
    with am.Mesher(device=dev, max_cells=1 << 16, max_neurons=4096, max_width=512) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
        m.march(max_cells=n_cells)
        keys = m.get_mesh(nid).face_keys
        N, n = mlp.N, keys.shape[0]
        k = torch.as_tensor(np.ascontiguousarray(keys).view(np.int64), device=f"cuda:{dev}")
        rows = torch.empty((n, N + 1, 4), dtype=torch.float64, device=f"cuda:{dev}")
        err = torch.empty((n, N + 1), dtype=torch.float32, device=f"cuda:{dev}")
        w = mlp.widths
        dense = n * sum(8 * w[l] * w[l - 1] for l in range(1, mlp.L))
        issued = n * sum(4 * 2 * 16 * 16 * 8 * ((w[l] + 15) // 16) * ((w[l - 1] + 15) // 16) for l in range(1, mlp.L))
        out["autotune"] = m.autotune_compose(nid, keys=keys, reps=3)      # picks the sliced tile shape
        for name, code in (("fp64", 0), ("mixed", 1), ("tensor", 2), ("sliced", 3)):
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc = m.lib.am_compose(m.ctx, nid, C.c_void_p(k.data_ptr()), n, code, C.c_void_p(rows.data_ptr()),
                                      C.c_void_p(err.data_ptr()))
                ts.append(time.perf_counter() - t0)
                assert rc == 0, m.lib.am_last_error(m.ctx)
            dt = statistics.median(ts)
            out[name] = {"cells_per_s": n / dt, "ms": dt * 1e3, "dense_tflops": dense / dt / 1e12}
        t = out["tensor"]
        t["issued_tflops"] = issued / (t["ms"] / 1e3) / 1e12
        t["roofline"] = {"bound": "tensor", "achieved": t["issued_tflops"], "peak": BF16_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": t["issued_tflops"] / BF16_PEAK_TFLOPS,
                         "peak_source": "measured cuBLAS bf16 burst"}
        out["tensor_speedup_vs_fp64"] = out["fp64"]["ms"] / t["ms"]
        sl = out["sliced"]
        # 36 plane products per layer for each real cell's 4 columns (rows padded to the 128-row
        # tile and K to 64; the tile's padding columns are not counted)
        sl["issued_tflops"] = 36 * 2 * 4 * n * sum(-(-w[l] // 128) * 128 * (-(-w[l - 1] // 64) * 64)
                                                   for l in range(1, mlp.L)) / (sl["ms"] / 1e3) / 1e12
        sl["roofline"] = {"bound": "tensor", "achieved": sl["issued_tflops"], "peak": BF16_PEAK_TFLOPS,
                          "unit": "TFLOP/s", "frac": sl["issued_tflops"] / BF16_PEAK_TFLOPS,
                          "peak_source": "measured cuBLAS bf16 burst", "scope": "whole am_compose call"}
        out["sliced_speedup_vs_fp64"] = out["fp64"]["ms"] / sl["ms"]
    return out


def decoder_leg(dev, n_cells=60000, reps=2):
    """The decoder-shaped workload, (3 + 256) -> [512] x 8 -> 1 with skip-concat of [x; z] at
    hidden layer 4 (N = 4096), one seed ray along +x: the first n_cells cells of its march
    (the whole mesh exceeds 4e6 cells), timed by am_march's CUDA events, seeding outside.
    Plain FP64 (compose and clip in one persistent kernel) against the sliced path (the compose
    of each level's cells on the tensor cores into device memory as FP32 pairs, then the clip
    reading those rows with certified FP32 sign tests, FP64 for the close calls).  Rooflines of the two sliced kernels: the compose's issued tensor flops (36
    digit-plane products per layer) and the clip's algorithmic bytes (its rows, (N + 1) x 32 B
    per cell, plus the key and the face record) over their own device time."""
    import paper_2106_10031_gb300 as am
    from synth import decoder_net
    mlp = decoder_net()
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    out = {"workload": f"decoder (3+256)-[512]x8-1, skip at 4, seed 3; first {n_cells} cells of the march"}
    with am.Mesher(device=dev, max_cells=1 << 17, max_neurons=4096, max_width=512) as m:
        nid = m.load_mlp(mlp)
        out["autotune"] = m.autotune_compose(nid, n=512, reps=3)      # batches of a breadth-first level
        for prec in ("fp64", "sliced"):
            runs = []
            for _ in range(reps + 1):                   # the first run warms up
                m.reset()
                m.seed(nid, o, d)
                m.march(precision=prec, max_cells=n_cells)
                runs.append(m.stats())
            st = min(runs[1:], key=lambda x: x["ms_march"])
            out[prec] = {"faces": st["faces"], "ms": st["ms_march"], "faces_per_s": st["faces"] / (st["ms_march"] / 1e3),
                         "levels": st["levels"], "launches": st["kernel_launches"], "degenerate": st["degenerate"]}
            if prec == "sliced":
                w, cells = mlp.widths, st["cells"]
                issued = 36 * 2 * 4 * cells * sum(-(-w[l] // 128) * 128 * (-(-w[l - 1] // 64) * 64)
                                                  for l in range(1, mlp.L))
                ach = issued / (st["ms_compose"] / 1e3) / 1e12
                out[prec]["ms_compose"], out[prec]["ms_clip"] = st["ms_compose"], st["ms_clip"]
                out[prec]["compose_roofline"] = {"kernel": "oz_gemm_kernel + oz_prep_kernel", "bound": "tensor",
                                                 "achieved": ach, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                                                 "frac": ach / BF16_PEAK_TFLOPS}
                kw = (mlp.N + 63) // 64
                clip_bytes = cells * ((mlp.N + 1) * 32 + 8 * kw + 32 * (24 + 4) + 64)
                gbs = clip_bytes / (st["ms_clip"] / 1e3) / 1e9
                out[prec]["clip_roofline"] = {"kernel": "march_range_kernel<double-float> (rows from HBM)", "bound": "hbm",
                                              "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                              "frac": gbs / HBM_PEAK_GBS, "bytes_per_cell": clip_bytes / cells}
        out["sliced_speedup_vs_fp64"] = out["sliced"]["faces_per_s"] / out["fp64"]["faces_per_s"]
        out["march_autotune"] = m.autotune_march(nid, o, d, max_cells=n_cells, reps=1)
    return out


def learned_leg(dev, n_cells=60000, reps=2):
    """The learned-proposal workload: 3 -> [256] x 8 -> 1 (geometric init, sigma 0.05, seed 5;
    N = 2048) with a proposal 15 -> 256 -> 256 -> 2048 (BF16 operands, FP32 accumulation),
    trained before timing on the plain method's mesh of a nearby checkpoint of the net (first
    n_cells cells).  The first n_cells cells of the net's own march, one seed ray along +x,
    timed by am_march's CUDA events: the plain FP64 method (every cutting row clipped) against
    mixed precision (compose on the tensor cores, certified clip) with learned candidates, and
    the other candidate rules for context.  Every configuration's mesh is exact: the all-row
    check corrects any face the candidates got wrong."""
    import paper_2106_10031_gb300 as am
    from synth import proposal_target_net, sibling
    mlp = proposal_target_net()
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    out = {"workload": f"3-[256]x8-1 geometric init (seed 5, sigma 0.05), proposal 15-256-256-2048; "
                       f"first {n_cells} cells of the march"}
    with am.Mesher(device=dev, max_cells=1 << 17, max_neurons=2048, max_width=256) as m:
        sid = m.load_mlp(sibling(mlp, seed=99))
        m.seed(sid, o, d)
        m.march(precision="fp64", candidates="none", max_cells=n_cells)
        X, Y = m.proposal_samples(sid, max_samples=120000)
        m.proposal_init(7 + mlp.L, 256, mlp.N, max_batch=1024, seed=0)
        t0 = time.perf_counter()
        losses = m.proposal_train(X, Y, batch=1024, steps=3000, lr=2e-3)
        out["training"] = {"samples": int(X.shape[0]), "steps": 3000, "train_s": time.perf_counter() - t0,
                           "loss_first": float(losses[:5].mean()), "loss_last": float(losses[-50:].mean())}
        del X, Y
        m.reset()
        m.release_nets()
        nid = m.load_mlp(mlp)
        out["autotune"] = m.autotune_compose(nid, n=512, reps=3)      # batches of a breadth-first level
        for name, prec, cand in (("plain_fp64", "fp64", "none"), ("fp64_learned", "fp64", "learned"),
                                 ("sliced_learned", "sliced", "learned"), ("fp64_nearest", "fp64", "nearest"),
                                 ("sliced_nearest", "sliced", "nearest")):
            runs = []
            for _ in range(reps + 1):                   # the first run warms up
                m.reset()
                m.seed(nid, o, d)
                m.march(precision=prec, candidates=cand, max_cells=n_cells)
                runs.append(m.stats())
            st = min(runs[1:], key=lambda x: x["ms_march"])
            out[name] = {"faces": st["faces"], "ms": st["ms_march"], "faces_per_s": st["faces"] / (st["ms_march"] / 1e3),
                         "cuts_per_cell": st["cuts"] / max(1, st["cells"]),
                         "corrected_frac": st["fixups"] / max(1, st["cells"]), "degenerate": st["degenerate"]}
        base = out["plain_fp64"]["faces_per_s"]
        for k in ("fp64_learned", "sliced_learned", "fp64_nearest", "sliced_nearest"):
            out[k]["speedup_vs_plain_fp64"] = out[k]["faces_per_s"] / base
        out["march_autotune"] = m.autotune_march(nid, o, d, max_cells=n_cells, reps=1, candidates="learned")
    return out


def trigger_leg(dev, n_starts=1024, n_samples=4096, reps=5):
    """The customised triggers (Sec. 4.3) on the headline 3-[64]x4-1 net, with the paper's
    1024 initial points: sphere tracing from n_starts points uniform in [-1.4, 1.4]^3 (eta 1,
    at most 64 steps, eps 1e-12) and the random-pair dichotomy on n_samples points uniform in
    [-1.5, 1.5]^3 (up to 1024 pairs).  Each call is timed whole on the host clock (copy of the
    points in, the trigger kernels, the dichotomy, the push of the seed cells, the copy of the
    seed points out), best of `reps` after one warm-up; the oracle's time for the same call on
    a 64-point sample is reported beside it.  Afterwards the march from all traced seeds."""
    import paper_2106_10031_gb300 as am
    from synth import trigger_points
    mlp, _, _ = workload()
    starts = trigger_points(n_starts, seed=4, box=1.4)
    samples = trigger_points(n_samples, seed=7, box=1.5)
    out = {"workload": f"{mlp.name}: {n_starts} sphere-tracing starts, {n_samples} samples for up to 1024 pairs"}
    with am.Mesher(device=dev, max_cells=1 << 18, max_neurons=max(64, mlp.N), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        for name, call in (("sphere_trace", lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12)),
                           ("pairs", lambda: m.seed_pairs(nid, samples, 1024))):
            times, res = [], None
            for _ in range(reps + 1):                   # the first call warms up
                m.reset()
                t0 = time.perf_counter()
                res = call()
                times.append(time.perf_counter() - t0)
            best = min(times[1:])
            pts = res[-1]
            n_in = n_starts if name == "sphere_trace" else n_samples
            out[name] = {"ms": best * 1e3, "points_per_s": n_in / best, "seeds": int(np.sum(~np.isnan(pts[:, 0]))),
                         "new_cells": int(res[-2] if name == "pairs" else res[0])}
        # parallel marching from many seeds (Sec. 4.2): the same mesh, a shallower breadth-first
        # walk; the depth is counted by the level schedule, the persistent one gives the time
        seedings = {"traced_seeds": lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12),
                    "one_seed": lambda: m.seed(nid, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))}
        out["march_by_seeding"] = {"precision": "fp64", "candidates": "nearest"}
        for sched in ("persistent", "levels"):         # warm-up: first launches of both schedules
            m.reset()
            seedings["one_seed"]()
            m.march(schedule=sched)
        for name, seed in seedings.items():
            row = {}
            for sched in ("persistent", "levels"):
                m.reset()
                seed()
                m.march(schedule=sched)
                st = m.stats()
                row[sched] = {"faces": st["faces"], "ms_march": st["ms_march"], "levels": st["levels"]}
            out["march_by_seeding"][name] = row
    out["cpu_baseline"] = trigger_cpu_baseline(mlp, starts[:64], samples[:256])
    return out


def shard_nets(n_nets: int, rank: int, world: int) -> list:
    """Indices of the nets a rank meshes: round robin over the net index.  The nets are
    independent problems, so the ranks exchange nothing on the data path; the round robin
    spreads the batch's mix of small and large nets."""
    return list(range(rank, n_nets, world))


def batch_leg(dist, max_cells=2_000_000, precision="mixed", reps=1, box=2.0):
    """The 64-net batch: batch_nets(master_seed=4) (widths 32-256, depths 4-8, sigma in
    [0.02, 0.1]), one seed ray along +x per net, box [-2, 2]^3 (some of the deeper nets reach
    past 1.5), all of a rank's nets in one persistent launch, the first max_cells cells of the
    job (split evenly over the ranks).  Sharded by
    net (shard_nets); value = all ranks' faces / the slowest rank's march time, by am_march's
    CUDA events; strong scaling (the total work is fixed)."""
    import paper_2106_10031_gb300 as am
    from synth import batch_nets
    nets = batch_nets()
    mine = [nets[i] for i in shard_nets(len(nets), dist.rank, dist.world)]
    cells = max_cells // dist.world
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    with am.Mesher(device=dist.local, max_cells=cells + 4096, max_neurons=max(n.N for n in mine),
                   max_width=max(max(n.widths) for n in mine)) as m:
        ids = [m.load_mlp(n) for n in mine]
        runs, unseeded = [], 0
        for _ in range(reps + 1):                   # the first run warms up
            m.reset()
            unseeded = 0
            for i in ids:
                try:
                    m.seed(i, o, d)
                except am.AMError:
                    unseeded += 1
            dist.barrier()
            m.march(box=box, precision=precision, max_cells=cells)
            runs.append(m.stats())
        st = min(runs[1:], key=lambda x: x["ms_march"])
    faces = dist.allreduce(float(st["faces"]), "sum")
    ms = dist.allreduce(float(st["ms_march"]), "max")
    return {"workload": f"64 nets of batch_nets(master_seed=4), box {box}, first {max_cells} cells of the job, "
                        f"{precision}",
            "n_gpus": dist.world, "scaling": "strong", "sharding": "nets round robin over the ranks, no exchange",
            "faces": int(faces), "ms": ms, "faces_per_s": faces / (ms / 1e3),
            "rank0": {"nets": len(mine), "unseeded_nets": unseeded, "cells": int(st["cells"]),
                      "faces": int(st["faces"]), "ms": float(st["ms_march"])}}


def trigger_cpu_baseline(mlp, starts, samples):
    """The oracle's triggers as they stand, single-threaded, on a sample of the trigger leg's
    points: sphere tracing from `starts`, random pairs (up to 64) from `samples`."""
    from oracle import oracle as orc
    net = orc.OracleNet(mlp)
    t0 = time.perf_counter()
    orc.seed_sphere_trace(net, starts, eta=1.0, max_steps=64, eps=1e-12)
    t_tr = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.seed_pairs(net, samples, 64)
    t_pr = time.perf_counter() - t0
    return {"kind": "oracle", "cores": 1, "sample": f"{len(starts)} starts / {len(samples)} samples",
            "sphere_trace_points_per_s": len(starts) / t_tr, "pairs_points_per_s": len(samples) / t_pr}


def train_proposal(m, mlp, o, d):
    """The learned proposal for the workload: trained on the plain method's mesh (full clip,
    FP64) of a nearby checkpoint of the net (every weight moved by N(0, 0.005^2)), outside
    every timed region.  Leaves the context holding the workload net only."""
    from synth import sibling
    m.reset()
    m.release_nets()
    sid = m.load_mlp(sibling(mlp, seed=99))
    m.seed(sid, o, d)
    m.march(precision="fp64", candidates="none")
    X, Y = m.proposal_samples(sid)
    m.proposal_init(7 + mlp.L, 256, mlp.N, max_batch=1024, seed=0)
    t0 = time.perf_counter()
    losses = m.proposal_train(X, Y, batch=1024, steps=3000, lr=2e-3)
    train_s = time.perf_counter() - t0
    m.reset()
    m.release_nets()
    nid = m.load_mlp(mlp)
    return nid, {"samples": int(X.shape[0]), "steps": 3000, "batch": 1024, "train_s": train_s,
                 "loss_first": float(losses[:5].mean()), "loss_last": float(losses[-50:].mean())}


def leg(m, nid, o, d, steps, precision, schedule, flush, stream, candidates, dist, all_faces):
    measure(m, nid, o, d, 2, precision, schedule, flush, stream, candidates)
    p = measure(m, nid, o, d, steps, precision, schedule, flush, stream, candidates)
    p_ms = dist.allreduce(p["total_ms"], "max")
    st = p["stats"]
    return {"value": all_faces / (p_ms / 1e3), "unit": UNIT, "ms_per_step": p_ms / steps,
            "precision": precision, "candidates": candidates,
            "cuts_per_cell": st["cuts"] / max(1, st["cells"]), "corrected_frac": st["fixups"] / max(1, st["cells"]),
            "_cell_ms": p["cell_ms"], "_cell_launches": p["cell_launches"]}


def run_ours(args, dist):
    import torch

    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300 import native as nt
    mlp, o, d = workload()
    base, ref_mesh = None, None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        base, ref_mesh = cpu_baseline(mlp, o, d)          # before any GPU work
    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    precision = nt.AM_PREC_FP64 if args.precision == "fp64" else nt.AM_PREC_MIXED
    m = am.Mesher(device=dev, max_cells=1 << 17, max_neurons=256, max_width=64, stream=stream.cuda_stream)
    nid = m.load_mlp(mlp)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")   # > 129 MB L2
    warm = max(args.warmup, 3)
    train = None
    if args.candidates == "learned" or not args.no_compare:
        nid, train = train_proposal(m, mlp, o, d)
    measure(m, nid, o, d, warm, args.precision, args.schedule, flush, stream, args.candidates)
    mesh = m.get_mesh(nid)
    faces_per_step = mesh.n_faces
    work = algorithmic_work(mlp, mesh)
    torch.cuda.synchronize()
    dist.barrier()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed steps
        r = measure(m, nid, o, d, args.steps, args.precision, args.schedule, flush, stream, args.candidates)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    dist.barrier()
    agreement = oracle_agreement(ref_mesh, m.get_mesh(nid)) if ref_mesh is not None else None
    max_ms = dist.allreduce(r["total_ms"], "max")
    all_faces = dist.allreduce(float(faces_per_step * args.steps), "sum")
    value = all_faces / (max_ms / 1e3)
    legs = None
    if not args.no_compare:
        legs = {}
        for name, prec, cand in (("plain_fp64", "fp64", "none"), ("fp64_nearest", "fp64", "nearest"),
                                 ("mixed_nearest", "mixed", "nearest"), ("fp64_learned", "fp64", "learned"),
                                 ("mixed_learned", "mixed", "learned")):
            if (prec, cand) == (args.precision, args.candidates):
                continue
            g = leg(m, nid, o, d, args.steps, prec, args.schedule, flush, stream, cand, dist, all_faces)
            if prec == "fp64":
                pk = g["_cell_ms"] / max(1, g["_cell_launches"])
                p_ach = work["fp64_flops"] / max(1, g["_cell_launches"] / args.steps) / (pk / 1e3) / 1e12
                g["roofline"] = {"kernel": "march_persistent_kernel<FP64>", "bound": "alu", "achieved": p_ach,
                                 "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": p_ach / FP64_PEAK_TFLOPS,
                                 "counts": "compose + checks FP64 flops only"}
            g.pop("_cell_ms"), g.pop("_cell_launches")
            g["headline_speedup"] = value / g["value"]
            legs[name] = g
        legs["proposal_training"] = train
        legs["compose"] = compose_leg(dev)
        legs["decoder"] = decoder_leg(dev)
        legs["learned_256x8"] = learned_leg(dev)
    e2e = None
    if not args.no_e2e:
        prop = (m.proposal_params(), m.prop_shape) if args.candidates == "learned" else None
        e2e = e2e_leg(mlp, o, d, args.steps, dev, stream.cuda_stream, precision, args.candidates, prop)
        e2e_ms = dist.allreduce(e2e.pop("ms_per_step") * args.steps, "max")
        e2e["value"] = dist.allreduce(float(faces_per_step * args.steps), "sum") / (e2e_ms / 1e3)
    m.close()
    if dist.rank != 0:
        return 0
    per_launch_ms = r["cell_ms"] / max(1, r["cell_launches"])
    launches_per_step = max(1, r["cell_launches"] / args.steps)
    st = r["stats"]
    if args.precision == "fp64":
        flops, peak, kname = work["fp64_flops"], FP64_PEAK_TFLOPS, "march_persistent_kernel<FP64>"
        psrc = "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (probe: 1.19 TFLOP/s at 1995 MHz)"
    else:
        flops, peak, kname = work["df_fp32_flops"], FP32_PEAK_TFLOPS, "march_persistent_kernel<double-float>"
        if args.candidates == "learned":
            flops += work["proposal_fp32_flops"]
        psrc = "derived: 128 FP32 FMA/clk/SM x 152 SMs x 2.07 GHz (probe: 69.4 TFLOP/s at 1995 MHz)"
    if args.schedule == "levels":
        kname = kname.replace("persistent", "range")
    achieved = flops / launches_per_step / (per_launch_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": warm, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32x2+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "faces_per_step": faces_per_step, "precision": args.precision,
                   "candidates": args.candidates, "schedule": args.schedule,
                   "parallelism": f"replicas x{dist.world}",
                   "l2": "flushed before every step (256 MiB write)"},
        "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": captured_traffic(args.precision, args.candidates), "flops_per_launch": flops / launches_per_step,
                     "launch_ms": per_launch_ms, "kernel_share_of_step": r["cell_ms"] / max(r["total_ms"], 1e-9),
                     "peak_source": psrc},
        "legs": legs,
        "exactness": {"refined_cells": st["refined_cells"], "close_calls": st["close_calls"],
                      "fixups": st["fixups"], "cuts_per_cell": st["cuts"] / max(1, st["cells"]),
                      "degenerate": st["degenerate"], "vs_oracle": agreement},
        "cpu_baseline": base,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": int(r["launches"]),
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        if args.compose_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "compose", **compose_leg(dist.local)}))
            return 0
        if args.decoder_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "decoder", **decoder_leg(dist.local)}))
            return 0
        if args.batch_only:
            out = batch_leg(dist, precision=args.precision)
            if dist.rank == 0:
                print(json.dumps({"leg": "batch64", **out}))
            return 0
        if args.triggers_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "triggers", **trigger_leg(dist.local)}))
            return 0
        if args.learned_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "learned_256x8", **learned_leg(dist.local)}))
            return 0
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
