#!/usr/bin/env python3
"""Throughput of the entropy-split SBP-SAT solver on one GB300.

Workload (default): 2D isentropic vortex + 1e-3 uniform noise (seed 2) on the
periodic [0,10]^2 square, 128 x 128 quads cut into 32,768 curved triangles
(sinusoidal warp, amplitude 0.05), degree p = 3 diagonal-E SBP operator
(18 nodes), entropy-split volume term + EC SATs + matrix interface
dissipation, float64.  A step is one relaxation RK4 step (four residual
evaluations, the stage entropy productions, the relaxation root solve and the
update).  The metric counts node-DOF residual evaluations per second:
4 * n_e * n_p per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl esplit|reference]

Prints one JSON line on rank 0.  N > 1 runs independent replicas (the
solver does not shard), launched by torch.distributed.run.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "DOF-residual evals/s vs Hadamard form, FP64 & FP32, % roofline; 1 GB300"
UNIT = "DOF-residual evals/s"
FP64_PEAK_NOMINAL = 1.25e12            # GB300 nominal FP64 1.25 TFLOP/s (context; the roofline uses the measured rate)
# DRAM bytes (read + write) per launch from one ncu capture of the unchanged
# kernel; keyed by (kernel, p, precision, N)
NCU_TRAFFIC = {("split_volume", 3, "fp64", 128): 229.391e6}
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
# precision settings timed per scheme (the Hadamard forms have one float32 setting,
# plain float32 two-point fluxes) and the error bound each is tested to
SPLIT_PRECS = ("fp64", "fp32_bulk", "fp32")
HAD_PRECS = ("fp64", "fp32")
ERROR_BOUND = {"split_fp64": 1e-12, "split_fp32_bulk": 1e-11, "split_fp32": 1e-5, "hadamard_fp64": 1e-12,
               "hadamard_fp32": 1e-3, "hadamard_ir_fp64": 1e-12, "hadamard_ir_fp32": 1e-3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="esplit", choices=["esplit", "reference"])
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_bulk", "fp32"])
    ap.add_argument("--no-sweep", action="store_true", help="skip the residual-only sweep over p / scheme / precision")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-tgv", action="store_true", help="skip the 3D Taylor-Green (196,608 tets) measurement")
    ap.add_argument("--no-quadrants", action="store_true", help="skip the 2D quadrant Riemann problem (hybrid)")
    ap.add_argument("--quadrants-full", action="store_true", help="run the quadrant problem to t = 0.25")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 128-triangle step latency and the adjoint (residual / step VJP) timings")
    ap.add_argument("--no-tet-sweep", action="store_true",
                    help="skip the residual-only sweep on the 3D vortex tetrahedra, p = 1..4")
    ap.add_argument("--tet-n", type=int, default=16, help="cubes per direction of the 3D vortex sweep mesh")
    ap.add_argument("--tgv-n", type=int, default=32,
                    help="cubes per direction of the Taylor-Green mesh (6 N^3 tetrahedra; 32 is the workload, "
                         "smaller meshes serve profiling captures)")
    return ap.parse_args()


def workload(p, N):
    from esplit_inputs import tri_operator, periodic_tri_mesh, states
    op = tri_operator(p)
    mesh = periodic_tri_mesh(op, N, 10.0, 0.05)
    u0 = states.add_uniform_noise(states.isentropic_vortex(mesh), 1e-3, 2)
    dt = states.cfl_timestep(mesh, u0, 0.1)
    return op, mesh, u0, dt


def workload_name(p, N, precision):
    return (f"2D isentropic vortex + 1e-3 noise, {N}x{N} quads -> {2 * N * N} curved triangles (warp 0.05), "
            f"p={p} diagonal-E SBP, entropy split + EC SAT + matrix dissipation, {precision}, relaxation RK4 step")


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# algorithmic work per launch
# ---------------------------------------------------------------------------------------------
def algorithmic_flops(group, n_e, n_p, d, n_pairs):
    nc = d + 2
    if group == "split_volume":
        contraction = 2 * d * 2 * n_p * n_p * nc          # 2d applications of n_p x n_p to n_p x nc
        pointwise = n_p * (30 + 43 * d)                    # primitives, W, fluxes, A~_i D_i w, products
        return n_e * (contraction + pointwise)
    if group == "hadamard_volume":
        pairs = n_p * (n_p - 1) // 2
        return n_e * pairs * (60 + 2 * d)
    if group == "face":
        return n_pairs * 400
    return None


def algorithmic_bytes(group, n_e, n_p, d, n_pairs):
    nc = d + 2
    if group == "split_volume":
        n_slot = 2 * n_pairs // n_e
        # D_i operators, u in, r out, J, and at the facet slots nu and the facet contributions
        return n_e * (8 * d * n_p * n_p + 8 * n_p * (2 * nc + 1) + 8 * n_slot * (nc + d))
    if group == "face":
        return n_pairs * (2 * 8 * nc + 2 * 8 * nc + 8 * d + 8 + 16)
    return None


def algorithmic_bytes_f32_volume(n_e, n_p, d, n_pairs):
    """Bytes the float32-path volume kernel must move per launch: the float32
    D_i (unpadded), u in and r out (float64), the float32 1/(H J) and the
    float32 facet contributions at the element's facet slots."""
    nc = d + 2
    n_slot = 2 * n_pairs // n_e
    return n_e * (4 * d * n_p * n_p + 2 * 8 * n_p * nc + 4 * n_p + 4 * n_slot * nc)


def hbm_peak_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def f32_volume_roofline(prof, n_e, n_p, d, n_pairs):
    """HBM roofline of the float32-path volume kernel from the profiled groups
    of a timed region (the float32 path's volume launches are the split group)."""
    if prof.get("split_volume", (0, 0))[1] == 0:
        return None
    ms = prof["split_volume"][0] / prof["split_volume"][1]
    by = algorithmic_bytes_f32_volume(n_e, n_p, d, n_pairs)
    peak, src = hbm_peak_gbs()
    ach = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": None, "kernel": "split_volume_f32", "avg_launch_ms": ms,
            "launches": prof["split_volume"][1], "algorithmic_bytes": by, "peak_source": src}


# ---------------------------------------------------------------------------------------------
def dist_setup(gpus, backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measure_fp64_peak(es, device):
    """Arithmetic throughput of this GPU (the library's calibration kernels),
    with the SM clock sampled while they run: float64 FMA chains (the roofline
    peak), the float64 tensor-core MMA, both interleaved, float32 FMA chains,
    and the float64 divide and the library's log and exp, each as a cost in
    float64 FMAs."""
    names = ((0, "dfma"), (1, "dmma"), (2, "dfma_and_dmma"), (3, "ffma"), (4, "ddiv"), (5, "dlog"), (6, "dexp"),
             (7, "dlog_cuda"), (8, "dexp_cuda"), (9, "cvt_round_trip"), (10, "bf16_mma_sync"))
    out = {}
    with ClockSampler(device) as clk:
        for mode, name in names:
            best = 0.0
            t_end = time.perf_counter() + (1.0 if mode == 0 else 0.3)   # so that the sampler sees them
            while time.perf_counter() < t_end:
                rc, f, ms = es.capi.esplit_measure_fp64(device, mode)
                if rc != 0:
                    return None
                best = max(best, f)
            out[name] = best
    c = clk.summary()
    mhz = c["sm_mhz"]
    dfma_per_s = out["dfma"] / 2.0
    per_clk = {k: (v / 2.0 / (SM_COUNT * mhz * 1e6) if mhz else None) for k, v in out.items() if k in
               ("dfma", "dmma", "dfma_and_dmma", "ffma")}
    cost = {k: dfma_per_s / out[k] for k in ("ddiv", "dlog", "dexp", "dlog_cuda", "dexp_cuda", "cvt_round_trip")}
    cost["ffma"] = dfma_per_s / (out["ffma"] / 2.0)
    return {"tflops": out["dfma"] / 1e12, "sm_mhz": mhz, "dfma_per_clk_per_sm": per_clk["dfma"],
            "bf16_mma_sync_tflops": out["bf16_mma_sync"] / 1e12,
            "fma_per_clk_per_sm": per_clk, "cost_in_dfma": cost, "rates": out, "reasons": c["reasons"],
            "how": "esplit_measure_fp64: independent chains (8 per thread, 2048 threads per SM) of float64 FMA, "
                   "float64 MMA m8n8k4, both interleaved, float32 FMA, float64 divide, the library's and CUDA's "
                   "log and exp, a float64-float32-float64 round trip, the warp-level bf16 MMA; best launch "
                   "each, SM clock sampled meanwhile"}


def vs_hadamard(es, device, flush, p, N):
    """The metric's comparison at the headline mesh: residual-only time of
    the entropy split against the Hadamard form with the Sjogreen-Yee flux and
    against the Sec. 6 comparator (Hadamard form, Ismail-Roe flux), all with
    their matrix interface dissipation, float64 and float32 settings, and the
    error bound each setting is tested to (tests/test_gpu_parity.py,
    tests/test_gpu_ismail_roe.py)."""
    op, mesh, u0, dt = workload(p, N)
    stream = torch.cuda.current_stream(device)
    s = es.Solver(op, mesh, es.Params(dissipation=True), device=device)
    ud = s.to_device(u0)
    r = s.empty()
    ms = {}
    for scheme, precs in (("split", SPLIT_PRECS), ("hadamard", HAD_PRECS), ("hadamard_ir", HAD_PRECS)):
        for prec in precs:
            s.set_params(es.Params(dissipation=True, scheme=scheme, precision=prec))
            for _ in range(3):
                s.residual(ud, r)
            ms[f"{scheme}_{prec}"] = statistics.median(_timed(lambda: s.residual(ud, r), stream, flush, 10))
    s.close()
    out = {"mesh": f"{2 * N * N} triangles, p={p}", "residual_ms": {k: round(v, 4) for k, v in ms.items()},
           "error_bound": ERROR_BOUND,
           "split_over_ir_fp64": ms["hadamard_ir_fp64"] / ms["split_fp64"],
           "split_over_sy_fp64": ms["hadamard_fp64"] / ms["split_fp64"],
           "split_fp32_over_ir_fp64": ms["hadamard_ir_fp64"] / ms["split_fp32"],
           "split_fp32_over_ir_fp32": ms["hadamard_ir_fp32"] / ms["split_fp32"],
           "equal_accuracy": "split fp32 (bound 1e-5) against the Hadamard forms in fp64; their fp32 setting is "
                             "plain float32 (bound 1e-3): context, not equal accuracy"}
    return out


def fp32_step_run(es, device, flush, p, N, steps=10):
    """The same relaxation RK4 step with float32 residuals (precision fp32:
    fluxes, two-point fluxes, dissipation and contractions in float32 on
    float64-referenced variations; entropy, root solve and update float64),
    timed like the headline step."""
    op, mesh, u0, dt = workload(p, N)
    s = es.Solver(op, mesh, es.Params(dissipation=True, precision="fp32"), device=device)
    u = s.to_device(u0)
    for _ in range(3):
        s.rrk_step(u, dt)
    stream = torch.cuda.current_stream(device)
    ts = _timed(lambda: s.rrk_step(u, dt), stream, flush, steps)
    # kernel groups of as many steps again, with the library's per-group events
    s.profile(True)
    s.profile_read()
    _timed(lambda: s.rrk_step(u, dt), stream, flush, steps)
    prof = {g: v for g, v in s.profile_read().items() if v[1] > 0}
    s.profile(False)
    s.close()
    ms = sum(ts) / len(ts)
    return {"value": 4 * mesh.n_e * op.n_p / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "residual_error_bound": 1e-5,
            "volume_roofline": f32_volume_roofline(prof, mesh.n_e, op.n_p, op.d, solver_pairs(mesh, op)),
            "kernel_ms_per_step": {g: v[0] / steps for g, v in prof.items()},
            "note": "precision fp32 on the headline workload; L2 flushed between steps"}


def cpu_baseline(op, mesh, u0, budget_s=12.0):
    """The FP64 oracle (as it stands) on the host cores: full-mesh residual
    evaluations (split + EC SAT + dissipation) until the time budget is spent."""
    from oracle import residual as R
    from oracle.physics import Params as OP
    R.residual(u0, op, mesh, OP(), dissipation=True, elems=np.arange(min(64, mesh.n_e)))  # warm the vmap path
    n, t0 = 0, time.perf_counter()
    while True:
        R.residual(u0, op, mesh, OP(), dissipation=True)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 8:
            break
    return {"value": n * mesh.n_e * op.n_p / el, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{n} full-mesh residual evaluations ({mesh.n_e} elements, p={op.p}, split + EC SAT + "
                      f"dissipation, FP64) in {el:.1f} s; RK stage combination and relaxation root solve excluded"}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import residual as R
    from oracle.physics import Params as OP
    op, mesh, u0, dt = workload(args.p, args.N)
    R.residual(u0, op, mesh, OP(), dissipation=True, elems=np.arange(min(64, mesh.n_e)))
    for _ in range(args.warmup):
        R.residual(u0, op, mesh, OP(), dissipation=True)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        R.residual(u0, op, mesh, OP(), dissipation=True)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * mesh.n_e * op.n_p / tot
    cores = torch.get_num_threads()
    sample = (f"one full-mesh oracle residual per step ({mesh.n_e} elements, p={args.p}, split + EC SAT + "
              f"dissipation, FP64; RK stages and root solve excluded)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.p, args.N, "fp64"), "n_e": mesh.n_e, "p": args.p,
                       "n_p": op.n_p},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def residual_sweep(es, device, flush):
    """Residual-only throughput (no RK / root solve) of the split and Hadamard
    forms (Sjogreen-Yee flux), and of the Sec. 6 comparator, the Hadamard
    form with the Ismail-Roe flux, all with their matrix interface
    dissipation, FP64 and FP32-bulk, p = 1..4, on the same 32,768-triangle
    mesh."""
    out = {}
    stream = torch.cuda.current_stream(device)
    for p in (1, 2, 3, 4):
        op, mesh, u0, dt = workload(p, 128)
        s = es.Solver(op, mesh, es.Params(dissipation=True), device=device)
        ud = s.to_device(u0)
        r = s.empty()
        for scheme in ("split", "hadamard", "hadamard_ir"):
            for prec in (SPLIT_PRECS if scheme == "split" else HAD_PRECS):
                s.set_params(es.Params(dissipation=True, scheme=scheme, precision=prec))
                for _ in range(3):
                    s.residual(ud, r)
                ts = []
                for k in range(10):
                    flush.fill_(float(k))
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    s.residual(ud, r)
                    b.record(stream)
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                ms = statistics.median(ts)
                out[f"p{p}_{scheme}_{prec}"] = {"ms": ms, "dof_per_s": mesh.n_e * op.n_p / (ms * 1e-3)}
        s.close()
    return out


def tet_sweep(es, device, flush, n_cubes=16):
    """Residual-only throughput on the 3D isentropic vortex of Sec. 7.3
    (domain [-10, 10]^3, N^3 cubes x 6 curved tetrahedra, p = 1..4 diagonal-E
    tetrahedron operators; degree 1 on affine elements): the split form
    against the Hadamard form with the Sjogreen-Yee flux and against the
    Sec. 6 comparator (Hadamard form, Ismail-Roe flux), all with matrix
    interface dissipation, FP64 and FP32-bulk; and the Navier-Stokes residual
    (BO viscous terms) of the split form against the comparator's, FP64.
    Secs. 7.3 and 7.5 compare the same schemes on 750 tetrahedra, serially."""
    from esplit_inputs import tet_operator, states
    from esplit_inputs.mesh import periodic_tet_mesh, vortex3d_warp
    out = {"n_e": 6 * n_cubes ** 3}
    stream = torch.cuda.current_stream(device)
    for p in (1, 2, 3, 4):
        op = tet_operator(p)
        mesh = periodic_tet_mesh(op, n_cubes, 20.0, origin=-10.0, warp=vortex3d_warp)
        u0 = states.add_uniform_noise(states.isentropic_vortex_3d(mesh), 1e-3, 2)
        s = es.Solver(op, mesh, es.Params(dissipation=True), device=device)
        ud = s.to_device(u0)
        r = s.empty()
        for scheme in ("split", "hadamard", "hadamard_ir"):
            for prec in (SPLIT_PRECS if scheme == "split" else HAD_PRECS):
                s.set_params(es.Params(dissipation=True, scheme=scheme, precision=prec))
                for _ in range(3):
                    s.residual(ud, r)
                ms = statistics.median(_timed(lambda: s.residual(ud, r), stream, flush, 10))
                out[f"p{p}_{scheme}_{prec}"] = {"ms": ms, "dof_per_s": mesh.n_e * op.n_p / (ms * 1e-3)}
        # Navier-Stokes residual (BO viscous terms with heat flux, mu = 1/1600,
        # as in the Taylor-Green comparison of Sec. 7.5), FP64
        for scheme in ("split", "hadamard_ir"):
            s.set_params(es.Params(dissipation=True, scheme=scheme, viscous=True, mu=1.0 / 1600.0))
            for _ in range(3):
                s.residual(ud, r)
            ms = statistics.median(_timed(lambda: s.residual(ud, r), stream, flush, 10))
            out[f"p{p}_{scheme}_ns_fp64"] = {"ms": ms, "dof_per_s": mesh.n_e * op.n_p / (ms * 1e-3)}
        out[f"p{p}_n_p"] = op.n_p
        s.close()
        del s, ud, r, mesh
        torch.cuda.empty_cache()
    return out


def _timed(fn, stream, flush, n):
    ts = []
    for k in range(n):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def taylor_green_run(es, device, flush, steps=5, n_cubes=32):
    """Compressible Navier-Stokes Taylor-Green vortex (Re 1600, Ma 0.1, Pr
    0.71, heat flux on) on [0, 2 pi]^3: 32^3 cubes x 6 = 196,608 curved
    tetrahedra by default (n_cubes^3 x 6 otherwise; warp 0.02), p = 2 (25
    nodes); entropy split + EC SATs + BO
    viscous SATs + matrix dissipation; relaxation RK4 steps in FP64 and in
    FP32-bulk (entropy, production and root solve in FP64 in both), plus
    residual-only split vs Hadamard times on the same state."""
    from esplit_inputs import tet_operator, states
    from esplit_inputs.mesh import periodic_tet_mesh
    t0 = time.perf_counter()
    op = tet_operator(2)
    mesh = periodic_tet_mesh(op, n_cubes, 2 * np.pi, 0.02)
    u0 = states.taylor_green(mesh)
    dt = states.cfl_timestep(mesh, u0, 0.1)
    host_s = time.perf_counter() - t0
    mu = 1.0 / 1600.0
    stream = torch.cuda.current_stream(device)
    dof = mesh.n_e * op.n_p
    out = {"workload": f"3D Taylor-Green vortex, Re 1600, Ma 0.1, {n_cubes}^3 x 6 = {mesh.n_e:,} curved tets, p=2 "
                       "(25 nodes), entropy split + EC SAT + BO viscous SAT + matrix dissipation, relaxation RK4",
           "n_e": mesh.n_e, "n_p": op.n_p, "dof": dof, "dt": dt, "host_setup_s": host_s}
    s = es.Solver(op, mesh, es.Params(mu=mu, viscous=True, dissipation=True), device=device)
    r = s.empty()
    for prec in ("fp64", "fp32_bulk"):   # viscous terms: the float32 setting is FP32-bulk
        s.set_params(es.Params(mu=mu, viscous=True, dissipation=True, precision=prec))
        u = s.to_device(u0)
        for _ in range(2):
            s.rrk_step(u, dt)
        torch.cuda.synchronize()
        s.profile(True)
        s.profile_read()
        gs, est = [], []

        def step():
            g, info = s.rrk_step(u, dt)
            gs.append(g)
            est.append(info.estimate)
        ts = _timed(step, stream, flush, steps)
        prof = s.profile_read()
        s.profile(False)
        ms = statistics.median(ts)
        out[f"rrk_{prec}"] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "dof_residual_per_s": 4 * dof / (ms * 1e-3),
                              "g_range": [min(gs), max(gs)], "estimate_max": max(est), "status": s.status(),
                              "kernel_ms": {g: v[0] / steps for g, v in prof.items() if v[1] > 0}}
        for scheme in ("split", "hadamard"):
            s.set_params(es.Params(mu=mu, viscous=True, dissipation=True, precision=prec, scheme=scheme))
            ud = s.to_device(u0)
            for _ in range(2):
                s.residual(ud, r)
            ms = statistics.median(_timed(lambda: s.residual(ud, r), stream, flush, 5))
            out[f"residual_{scheme}_{prec}"] = {"ms": ms, "dof_per_s": dof / (ms * 1e-3)}
    s.close()
    return out


def small_and_adjoint_run(es, device, flush):
    """Config 1 (8 x 8 quads -> 128 curved triangles, p = 2, vortex, EC split,
    relaxation RK4 at CFL 0.1 for 20 steps: launch-latency bound) and config 4
    (32,768 curved triangles, p = 3, vortex + 1e-3 noise, FP64: reverse mode of
    the residual and of one relaxation step with dissipation, per call)."""
    from esplit_inputs import tri_operator, periodic_tri_mesh, states
    stream = torch.cuda.current_stream(device)
    out = {}
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 8, 10.0, 0.05)
    u0 = states.isentropic_vortex(m)
    dt = states.cfl_timestep(m, u0, 0.1)
    s = es.Solver(op, m, es.Params(), device=device)
    u = s.to_device(u0)
    for _ in range(3):
        s.rrk_step(u, dt)
    u = s.to_device(u0)
    ts = _timed(lambda: s.rrk_step(u, dt), stream, flush, 20)
    out["config1_rrk"] = {"ms_per_step": statistics.median(ts), "steps_per_s": 1e3 / statistics.median(ts),
                          "n_e": m.n_e, "steps": 20, "launch": "one host-driven step per call"}
    # the 20 steps as one batch of graph-launched steps (no host round trip
    # between steps); recorded by the first, untimed batch
    u = s.to_device(u0)
    s.rrk_steps(u, dt, 20)
    u = s.to_device(u0)
    ms = _timed(lambda: s.rrk_steps(u, dt, 20), stream, flush, 5)
    out["config1_rrk_graph"] = {"ms_per_step": statistics.median(ms) / 20, "steps_per_s": 20e3 / statistics.median(ms),
                                "n_e": m.n_e, "steps": 20,
                                "launch": "esplit_rrk_steps: 20 steps per call, each step one CUDA graph launch"}
    s.close()
    op, m, u0, dt = workload(3, 128)
    s = es.Solver(op, m, es.Params(dissipation=True), device=device)
    ud = s.to_device(u0)
    cot = s.to_device(np.random.default_rng(4).normal(size=u0.shape))
    g = s.empty()
    for _ in range(3):
        s.residual_vjp(ud, cot, g)
    ms_vjp = statistics.median(_timed(lambda: s.residual_vjp(ud, cot, g), stream, flush, 10))
    r = s.empty()
    ms_res = statistics.median(_timed(lambda: s.residual(ud, r), stream, flush, 10))
    for _ in range(2):
        s.rrk_step_vjp(ud, dt, cot)
    ms_step_vjp = statistics.median(_timed(lambda: s.rrk_step_vjp(ud, dt, cot), stream, flush, 5))
    dof = m.n_e * op.n_p
    out["config4_adjoint"] = {"residual_vjp_ms": ms_vjp, "residual_ms": ms_res, "vjp_over_residual": ms_vjp / ms_res,
                              "rrk_step_vjp_ms": ms_step_vjp, "dof": dof,
                              "note": "the step reverse recomputes the step from its checkpoint, then runs four "
                                      "residual VJPs and the implicit-function term of g"}
    s.close()
    return out


def quadrant_run(es, device, flush, t_final=None, steps=20):
    """2D Riemann-type problem: periodic [0, 1]^2, 256 x 256 quads -> 131,072
    affine triangles, p = 2, four constant quadrant states (seed 5, pressure
    ratio <= 10), hybrid scheme (on-device detector, threshold 1.1, re-run
    before every step) + matrix dissipation, relaxation RK4 at CFL 0.1:
    `steps` timed steps, or every step up to t_final when given.  Reports
    DOF-residual evals/s, the sign of every stage's entropy production, and
    whether positivity held (the library's sticky status, not NaN)."""
    from esplit_inputs import tri_operator, periodic_tri_mesh, states
    op = tri_operator(2)
    mesh = periodic_tri_mesh(op, 256, 1.0, 0.0)
    u0 = states.quadrant_states(mesh, 5)
    dt = states.cfl_timestep(mesh, u0, 0.1)
    stream = torch.cuda.current_stream(device)
    dof = mesh.n_e * op.n_p
    s = es.Solver(op, mesh, es.Params(scheme="hybrid", dissipation=True), device=device)
    u = s.to_device(u0)
    for _ in range(3):                      # warm-up on a copy
        uw = u.clone()
        s.detect_hybrid(uw, 1.1)
        s.rrk_step(uw, dt)
    torch.cuda.synchronize()
    t, n, max_rate, gs, flagged, status, ok = 0.0, 0, -np.inf, [], [], 0, True
    ms = []
    while (t_final is None and n < steps) or (t_final is not None and t < t_final - 1e-14):
        if n % 50 == 0:
            flush.fill_(float(n))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        try:
            nf = s.detect_hybrid(u, 1.1)
            g, info = s.rrk_step(u, dt)
        except es.EsplitError as ex:
            ok, status = False, ex.code
            break
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        t += g * dt
        n += 1
        gs.append(g)
        flagged.append(nf)
        max_rate = max(max_rate, max(info.stage_rate))
    tot = sum(ms) * 1e-3
    s.close()
    return {"workload": "2D quadrant Riemann problem, 256x256 quads -> 131,072 triangles, p=2, hybrid (device "
                        "detector, threshold 1.1, re-detected every step) + matrix dissipation, relaxation RK4, CFL 0.1",
            "n_e": mesh.n_e, "n_p": op.n_p, "dof": dof, "dt": dt, "steps": n, "t_reached": t,
            "ms_per_step": 1e3 * tot / max(n, 1), "steps_per_s": n / tot if tot else None,
            "dof_residual_per_s": 4 * dof * n / tot if tot else None,
            "flagged_elements": [min(flagged), max(flagged)] if flagged else None,
            "g_range": [min(gs), max(gs)] if gs else None, "max_stage_entropy_rate": max_rate,
            "stage_rates_nonpositive": bool(max_rate <= 0.0), "positivity_held": ok, "status": status,
            "timing": "detector + step per CUDA-event pair; L2 flushed every 50 steps"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_setup(args.gpus, "nccl")
    torch.cuda.set_device(local)
    device = local
    import paper_2305_07181_gb300 as es
    op, mesh, u0, dt = workload(args.p, args.N)
    solver = es.Solver(op, mesh, es.Params(dissipation=True, precision=args.precision), device=device)
    stream = torch.cuda.current_stream(device)
    u = solver.to_device(u0)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=f"cuda:{device}")  # 256 MB > L2
    n_p, n_e, d = op.n_p, mesh.n_e, op.d
    dof = n_e * n_p
    for _ in range(args.warmup):
        solver.rrk_step(u, dt)
    torch.cuda.synchronize()
    # ---------------- timed region (device state, per-step CUDA events, L2 flushed between steps)
    solver.profile(True)
    solver.profile_read()
    launches0 = solver.launch_count()
    step_ms = []
    gs = []
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(device) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g, _ = solver.rrk_step(u, dt)
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            gs.append(g)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier(ws)
    launches = solver.launch_count() - launches0
    prof = solver.profile_read()
    solver.profile(False)
    tot_s = max_over_ranks(sum(step_ms) * 1e-3, ws, device)
    value = ws * args.steps * 4 * dof / tot_s

    # ---------------- dominant kernel roofline (live event timing of the timed region)
    groups = {g: v for g, v in prof.items() if v[1] > 0}
    dom = max(groups, key=lambda g: groups[g][0])
    dom_ms = groups[dom][0] / groups[dom][1]
    per_launch_units = n_e if dom in ("split_volume", "hadamard_volume") else solver_pairs(mesh, op)
    fl = algorithmic_flops(dom, n_e, n_p, d, solver_pairs(mesh, op))
    fp64_peak = measure_fp64_peak(es, device)
    peak_tf = fp64_peak["tflops"] if fp64_peak else FP64_PEAK_NOMINAL / 1e12
    roofline = None
    if args.precision == "fp32" and d <= 2:
        roofline = f32_volume_roofline(groups, n_e, n_p, d, solver_pairs(mesh, op))
    elif fl is not None:
        achieved = fl / (dom_ms * 1e-3) / 1e12
        peak = peak_tf if args.precision == "fp64" else None
        src = (f"measured: float64 FMA chains {fp64_peak['tflops']:.3f} TFLOP/s = "
               f"{fp64_peak['dfma_per_clk_per_sm']:.2f} DFMA/clk/SM at {fp64_peak['sm_mhz']:.0f} MHz "
               f"(nominal 1.259 = 2 DFMA/clk/SM at 2070 MHz); FP64 pipe, not the bf16 tensor peak"
               if fp64_peak and fp64_peak.get("dfma_per_clk_per_sm") else
               "nominal FP64 1.25 TFLOP/s (the float64 FMA measurement failed)")
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": (achieved / peak) if peak else None,
                    "traffic": NCU_TRAFFIC.get((dom, args.p, args.precision, args.N)), "kernel": dom,
                    "avg_launch_ms": dom_ms, "launches": groups[dom][1], "units_per_launch": per_launch_units,
                    "peak_source": src}
    # every kernel group with an algorithmic flop count, against the same FP64 peak
    roofline_by_kernel = {}
    for g, (ms_tot, nl) in groups.items():
        fg = algorithmic_flops(g, n_e, n_p, d, solver_pairs(mesh, op))
        if fg is None:
            continue
        ms = ms_tot / nl
        ach = fg / (ms * 1e-3) / 1e12
        roofline_by_kernel[g] = {"avg_launch_ms": ms, "launches": nl, "achieved_tflops": ach,
                                 "frac_fp64_peak": ach / peak_tf if args.precision == "fp64" else None}
    # ---------------- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    u_host = torch.empty(u0.shape, dtype=torch.float64, pin_memory=True)
    u_host.copy_(torch.as_tensor(u0))
    uh = u_host.numpy()
    for _ in range(2):
        solver.rrk_step_host(uh, dt)
    e2e_tot = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        solver.rrk_step_host(uh, dt)          # H2D copy, step, D2H copy, stream sync
        e2e_tot += time.perf_counter() - t_a
    e2e_tot = max_over_ranks(e2e_tot, ws, device)
    nbytes = u0.size * 8
    e2e = {"value": ws * args.steps * 4 * dof / e2e_tot, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    vs_had = vs_hadamard(es, device, flush, args.p, args.N) if rank == 0 else None
    fp32_step = fp32_step_run(es, device, flush, args.p, args.N) if rank == 0 and args.precision == "fp64" else None
    extras = {"kernel_ms_timed_region": {g: {"ms_total": v[0], "launches": v[1]} for g, v in groups.items()},
              "roofline_by_kernel": roofline_by_kernel, "fp64_peak": fp64_peak,
              "g_range": [min(gs), max(gs)], "wall_s_timed": t_wall, "dt": dt}
    if rank == 0 and not args.no_sweep:
        extras["residual_sweep"] = residual_sweep(es, device, flush)
    if rank == 0 and not args.no_tet_sweep:
        extras["tet_sweep"] = tet_sweep(es, device, flush, n_cubes=args.tet_n)
    if rank == 0 and not args.no_tgv:
        extras["taylor_green"] = taylor_green_run(es, device, flush, n_cubes=args.tgv_n)
    if rank == 0 and not args.no_quadrants:
        extras["quadrants"] = quadrant_run(es, device, flush, t_final=0.25 if args.quadrants_full else None)
    if rank == 0 and not args.no_small:
        extras.update(small_and_adjoint_run(es, device, flush))
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(op, mesh, u0)
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.p, args.N, args.precision), "n_e": n_e, "p": args.p,
                       "n_p": n_p, "dof": dof, "residuals_per_step": 4, "dt": dt,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "vs_hadamard": vs_had, "fp32_step": fp32_step, "extras": extras}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def solver_pairs(mesh, op):
    return mesh.n_e * op.n_fac * op.n_f // 2


if __name__ == "__main__":
    sys.exit(main())
