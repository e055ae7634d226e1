"""Benchmark of the MG-PCG hot path on one GB300.

Workload (default): the plain FP64 MG-PCG at 192^3 (7,077,888 rows, 4 levels
192/96/48/24, b = A*ones, x0 = 0, one symmetric colour-ordered Gauss-Seidel
smoother application before and after each coarse correction, 50 CG
iterations).  One step = one whole solve.  The metric is HPCG-rule GFLOP/s
(flops counted by the HPCG rule below, not the flops executed) plus the mixed
vs FP64 time to a 1e-9 relative residual.

HPCG flop rule per CG iteration: 2 nnz_0 (SpMV) + 6 n_0 (3 dots) + 6 n_0
(3 vector updates) + sum over non-coarsest levels (8 nnz_l for the pre- and
post-smoother, each a forward and a backward sweep of 2 flops per nonzero,
+ 2 nnz_l for the residual + 2 n_{l+1} for restriction and refinement)
+ 4 nnz_coarsest.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = NZ = 192  # default grid; --grid changes it for profiling runs
LEVELS = 4
ITERS = 50
HBM_FALLBACK_GBS = 6800.0
L2_BYTES = 135528448
# the metric both arms report (the GPU solve, and --impl reference: the CPU oracle)
METRIC = "HPCG-rule GFLOP/s + HBM GB/s at 192^3; mixed vs FP64 time to 1e-9 residual"
# FP64-pipe warp instructions of one FP64 CG iteration per finest-level row at
# 192^3, from one ncu count of an iteration's kernels
# (sm__inst_executed_pipe_fp64.sum, profiles/fp64_instructions_per_iteration.md).
FP64_WARP_INSTR_PER_ROW_ITER = 0.2065


def bench_config(world=1):
    """The workload, the same for both arms."""
    return {"workload": "FP64 MG-PCG %dx%dx%d, %d levels, 1 pre + 1 post symmetric RBGS, %d CG iterations per step, "
                        "b=A*ones, x0=0" % (NX, NY, NZ, LEVELS, ITERS),
            "grid": [NX, NY, NZ], "levels": LEVELS, "cg_iters_per_step": ITERS,
            "l2": "working set (6 level-0 vectors = 340 MB) exceeds L2 (135.5 MB); no flush",
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def level_sizes(nx, ny, nz, levels):
    out = []
    for l in range(levels):
        a, b, c = nx >> l, ny >> l, nz >> l
        out.append((a * b * c, (3 * a - 2) * (3 * b - 2) * (3 * c - 2)))
    return out


def hpcg_flops_per_iter(nx, ny, nz, levels):
    sz = level_sizes(nx, ny, nz, levels)
    n0, nnz0 = sz[0]
    f = 2 * nnz0 + 6 * n0 + 6 * n0
    for l in range(levels - 1):
        f += 8 * sz[l][1] + 2 * sz[l][1] + 2 * sz[l + 1][0]
    f += 4 * sz[-1][1]
    return f


def algorithmic_bytes_per_iter(nx, ny, nz, levels, precision="fp64", kappa=False):
    """Bytes one CG iteration must move at least, per row of each level, with
    every vector touched once per pass (FP64 unless noted):
      finest level: SpMV 16 (x read, y written; + 8 for kappa), CG vector
        passes 88 (x, p, r, Ap -> x, r: 48; r, z, p -> p with r.z: 40);
      each level but the coarsest: two symmetric smoother applications of 48
        (r once, z read and written once per sweep direction), the residual
        with restriction 9, refinement 2; the coarsest level one application.
    precision "mixed": the preconditioner's vectors are FP32 (24, 4.5 and 1;
    + 4 per application with kappa for the FP32 inverse diagonal) and the CG
    passes read the FP32 z and write an FP32 copy of r (84)."""
    sz = level_sizes(nx, ny, nz, levels)
    n0 = sz[0][0]
    f = 4 if precision == "mixed" else 8
    sweep = 6 * f + (4 if (kappa and precision == "mixed") else (8 if kappa else 0))
    b = (16 + (8 if kappa else 0)) * n0 + (84 if precision == "mixed" else 88) * n0
    for l in range(levels):
        n = sz[l][0]
        if l < levels - 1:
            b += 2 * sweep * n + (9 * f / 8) * n + (2 * f / 8) * n
        else:
            b += sweep * n
    return b


def whole_solve_roofline(bytes_total, ms, peak):
    gbs = bytes_total / (ms * 1e-3) / 1e9
    return {"bytes": bytes_total, "ms": ms, "gbs": gbs, "frac": gbs / peak}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_ranks(world, backend="nccl"):
    """One process per GPU, rendezvous from MASTER_ADDR/MASTER_PORT.  The
    replicas exchange nothing on the data path: the process group carries only
    the barriers around the timed region and the max-over-ranks of the times."""
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)


def rank_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(values, world, device="cpu"):
    """Each value's maximum over the ranks: the slowest replica sets the job's time."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def whole_job_gflops(world, flops_per_step, ms_per_step):
    """Whole-job throughput: every replica did flops_per_step in ms_per_step
    (the max over ranks)."""
    return world * flops_per_step / (ms_per_step * 1e-3) / 1e9


def time_breakdown(prob, b):
    """Per-level time of one CG iteration, as the paper's Figs. 4-7 (smoother
    vs restriction/refinement per level, MG vs CG): kernels launched one by one
    with CUDA events between kernel groups (hpcg_profile_iteration)."""
    r = prob.profile_iteration(b)
    tot = r["total_ms"]
    mg = sum(r["smoother_ms"]) + sum(r["restriction_ms"]) + sum(r["refinement_ms"]) + r["persistent_coarse_ms"] \
        + r["convert_ms"]
    r["share"] = {"mg": mg / tot, "cg": 1 - mg / tot, "smoother": sum(r["smoother_ms"]) / tot,
                  "smoother_per_level": [v / tot for v in r["smoother_ms"]],
                  "transfer_per_level": [(a + c) / tot for a, c in zip(r["restriction_ms"], r["refinement_ms"])]}
    return r


def fp64_probe(dev):
    """FP64 FMA issue rate of this GPU (hpcg_probe_fp64_rate: 8 blocks of 256
    threads per SM, 8 independent FMA chains per thread)."""
    import ctypes
    import torch
    from paper_2304_08232_gb300 import _lib
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 8 * sms, 2000
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    ms, fma = ctypes.c_double(), ctypes.c_double()
    rc = _lib.load().hpcg_probe_fp64_rate(blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ms), ctypes.byref(fma),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError("hpcg_probe_fp64_rate failed: %d" % rc)
    lanes = fma.value / (ms.value * 1e-3)
    return {"sms": sms, "ms": ms.value, "lane_fma_per_s": lanes, "warp_instr_per_s": lanes / 32, "tflops": 2 * lanes / 1e12}


def persistent_first(prob):
    import ctypes
    from paper_2304_08232_gb300 import _lib
    v = ctypes.c_int()
    _lib.load().hpcg_persistent_levels(prob.h, ctypes.byref(v))
    return v.value


def tuned_shapes(prob):
    """Launch shapes the library's autotuner picked, per level:
    [row lines, row planes, colour-line lines, colour-line planes]."""
    import ctypes
    import torch
    from paper_2304_08232_gb300 import _lib
    lib = _lib.load()
    buf = (ctypes.c_int * (4 * prob.levels))()
    rc = lib.hpcg_autotune(prob.h, buf, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError("hpcg_autotune failed: %d" % rc)
    return [list(buf[4 * l:4 * l + 4]) for l in range(prob.levels)]


# ---------------------------------------------------------------------------
def oracle_lib(parallel):
    """(library, threads, how): the oracle's OpenMP build on every host core
    (one parallel loop per colour step and per SpMV, the parallelisation of the
    reference code the paper compares with; the same bits as the plain build),
    or the plain single-threaded build."""
    import oracle.oracle as om
    if parallel:
        try:
            lib = om.load_omp()
            return lib, int(lib.orc_threads()), "OpenMP build (rows of each colour step and SpMV in parallel, dots sequential)"
        except Exception as e:  # noqa: BLE001 - no OpenMP in the host compiler
            return om._load(), 1, "single-threaded build (OpenMP build failed: %s)" % str(e)[:80]
    return om._load(), 1, "single-threaded build"


def cpu_baseline(steps_iters=None, nx=None, ny=None, nz=None, parallel=True):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    `steps_iters` MG-PCG iterations at full size after building its CRS
    hierarchy (build time excluded)."""
    from oracle import OracleProblem
    nx, ny, nz = nx or NX, ny or NY, nz or NZ
    lib, threads, how = oracle_lib(parallel)
    if steps_iters is None:  # about 5-10 s of CPU work either way
        steps_iters = 24 if threads > 1 else 3
    t0 = time.perf_counter()
    o = OracleProblem(nx, ny, nz, levels=LEVELS, lib=lib)
    b = o.rhs()
    t1 = time.perf_counter()
    o.pcg(b, max_iters=steps_iters, tol=0.0)
    t2 = time.perf_counter()
    fl = hpcg_flops_per_iter(nx, ny, nz, LEVELS) * steps_iters
    return {"value": fl / (t2 - t1) / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": "%d MG-PCG iterations at %dx%dx%d, %s; CRS build %.1f s excluded" % (steps_iters, nx, ny, nz, how, t1 - t0),
            "seconds": round(t2 - t1, 3)}


def other_forms(dev, stream):
    """Timings of the batched and differentiable forms (one run each)."""
    import torch
    from hpcg_inputs import differentiable_inputs, multi_rhs, normal, uneven_batch_dims
    from paper_2304_08232_gb300 import HpcgBatch, HpcgProblem, hpcg_solve

    def timed(fn):
        fn()  # warm-up: graph capture, autotuning
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    res = {}
    # (a) 32 right-hand sides ~ N(0,1) (seed 2) on 128^3, to 1e-8
    n = 128 ** 3
    g = HpcgProblem(128, 128, 128, levels=4, max_rhs=32, device=dev)
    B = torch.as_tensor(multi_rhs(n, 32, seed=2), device=dev)
    ms, (X, sts) = timed(lambda: g.pcg_solve_multi(B, max_iters=1000, tol=1e-8))
    its = [s_.iters for s_ in sts]
    fl = hpcg_flops_per_iter(128, 128, 128, 4) * sum(its)
    peak = measured_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS)
    res["multi_rhs_32x128^3"] = {"ms": ms, "iters_max": max(its), "iters_sum": sum(its),
                                 "converged": all(s_.converged for s_ in sts), "hpcg_gflops": fl / (ms * 1e-3) / 1e9,
                                 "whole_solve_roofline": whole_solve_roofline(
                                     algorithmic_bytes_per_iter(128, 128, 128, 4) * sum(its), ms, peak)}
    del g, B, X
    # (b) 64 grids with edges from {32,48,64,80,96} (seed 3), 4 levels, to 1e-8
    dims = [tuple(int(v) for v in d) for d in uneven_batch_dims(64, seed=3)]
    bat = HpcgBatch(dims, levels=4, device=dev)
    bb = torch.as_tensor(normal(bat.n, 3), device=dev)
    ms, (xb, sts) = timed(lambda: bat.pcg_solve(bb, max_iters=1000, tol=1e-8))
    fl = sum(hpcg_flops_per_iter(*d, 4) * s_.iters for d, s_ in zip(dims, sts))
    by = sum(algorithmic_bytes_per_iter(*d, 4) * s_.iters for d, s_ in zip(dims, sts))
    res["batch_64_uneven_grids"] = {"ms": ms, "rows": bat.n, "iters_max": max(s_.iters for s_ in sts),
                                    "converged": all(s_.converged for s_ in sts), "hpcg_gflops": fl / (ms * 1e-3) / 1e9,
                                    "whole_solve_roofline": whole_solve_roofline(by, ms, peak)}
    del bat, bb, xb
    # (c) differentiable solve at 96^3: forward + adjoint backward, FP64 outer, FP32 M
    n = 96 ** 3
    kappa, b, xt = differentiable_inputs(n, seed=4)
    g = HpcgProblem(96, 96, 96, levels=4, precision="mixed", device=dev)
    kt = torch.as_tensor(kappa, device=dev).requires_grad_(True)
    bt = torch.as_tensor(b, device=dev).requires_grad_(True)
    xtt = torch.as_tensor(xt, device=dev)

    def fwd_bwd():
        kt.grad = None
        bt.grad = None
        x = hpcg_solve(bt, kt, g, max_iters=1000, tol=1e-10)
        loss = 0.5 * ((x - xtt) ** 2).sum()
        loss.backward()
        return loss

    ms, loss = timed(fwd_bwd)
    itf, itb = g.last_forward_stats.iters, g.last_backward_stats.iters
    # forward and adjoint solves (mixed, kappa), + the gradient pass (lambda, x read, grad written)
    by = algorithmic_bytes_per_iter(96, 96, 96, 4, "mixed", kappa=True) * (itf + itb) + 24 * n
    res["differentiable_96^3"] = {"ms_forward_backward": ms, "loss": float(loss), "tol": 1e-10,
                                  "iters_forward": itf, "iters_backward": itb,
                                  "whole_solve_roofline": whole_solve_roofline(by, ms, peak)}
    return res


def ell_study(b, x_ref, dev, stream):
    """The operator materialised as a sliced-ELL matrix (FP64 values, int32
    columns, 27 slots per row in slices of 32), rows grouped by colour
    (P^T A P, Section III-A) or in natural order: the same 50-iteration FP64
    solve as the headline, the level-0 SpMV kernel against its algorithmic
    bytes, and one level-0 smoother application (16 colour phases)."""
    import torch
    from paper_2304_08232_gb300 import HpcgEll
    peak = measured_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS)
    n = NX * NY * NZ

    def ev_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for name, sorted_, bf16 in [("colour_sorted", True, False), ("natural_order", False, False),
                                ("colour_sorted_bf16_values", True, True)]:
        e = HpcgEll(NX, NY, NZ, levels=LEVELS, colour_sorted=sorted_, bf16_values=bf16, device=dev)
        slot_b = (2 if bf16 else 8) + 4  # value + column
        rows, slices, _ = e.level_info(0)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        solve_ms = ev_ms(lambda: e.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x), 2)
        err = float((x - 1.0).abs().max())
        xs = e.to_stored(b)
        ys = torch.empty_like(xs)
        sp_ms = ev_ms(lambda: e.spmv(xs, out=ys), 10)
        # algorithmic bytes of one SpMV: every slot (8- or 2-byte value + 4-byte
        # column, padding slots included) once, x once, y once
        sp_bytes = slices * 27 * 32 * slot_b + 16 * rows
        zs = torch.zeros_like(xs)
        sm_ms = ev_ms(lambda: e.rbgs(xs, zs), 5)
        # one symmetric application: 16 colour phases; algorithmic bytes of a
        # phase: the slots of its eighth of the rows, r and z of those rows
        # (z read and written), and the z of the other seven colours its rows
        # neighbour, once (the same count for both layouts: a masked phase in
        # natural order drags in slots of rows of other colours as well)
        sm_bytes = 16 * (slices * 27 * 32 * slot_b / 8 + 8 * 3 * rows / 8 + 8 * 7 * rows / 8)
        out[name] = {"ms_per_step": solve_ms, "max_abs_err_vs_ones": err,
                     "max_abs_diff_x_vs_matrix_free": float((x - x_ref).abs().max()),
                     "matrix_bytes": e.nbytes(), "spmv_ms": sp_ms, "spmv_bytes": sp_bytes,
                     "spmv_gbs": sp_bytes / (sp_ms * 1e-3) / 1e9, "spmv_hbm_frac_of_measured": sp_bytes / (sp_ms * 1e-3) / 1e9 / peak,
                     "smoother_ms": sm_ms, "smoother_bytes": sm_bytes,
                     "smoother_hbm_frac_of_measured": sm_bytes / (sm_ms * 1e-3) / 1e9 / peak, "hpcg_gflops": hpcg_flops_per_iter(NX, NY, NZ, LEVELS) * ITERS / (solve_ms * 1e-3) / 1e9}
        del e, x, xs, ys, zs
        torch.cuda.synchronize()
    out["sorted_vs_natural_smoother_speedup"] = out["natural_order"]["smoother_ms"] / out["colour_sorted"]["smoother_ms"]
    # the same solve with the grid split into two z-slabs (own rows, halo
    # planes, colour-aware halo exchange), both slabs on this GPU
    from paper_2304_08232_gb300 import HpcgSplit
    sp = HpcgSplit(NX, NY, NZ, levels=LEVELS, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    v0, k0 = sp.exchange_count()
    sp.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x)
    v1, k1 = sp.exchange_count()
    solve_ms = ev_ms(lambda: sp.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x), 2)
    halo0 = sp.info(0, 0)["halo"] + sp.info(0, 1)["halo"]
    out["two_subdomains"] = {"ms_per_step": solve_ms, "max_abs_err_vs_ones": float((x - 1.0).abs().max()),
                             "max_abs_diff_x_vs_matrix_free": float((x - x_ref).abs().max()),
                             "halo_values_per_cg_iter": (v1 - v0) / ITERS, "exchange_steps_per_cg_iter": (k1 - k0) / ITERS,
                             "finest_halo_values": halo0,
                             "vs_colour_sorted_whole_grid": solve_ms / out["colour_sorted"]["ms_per_step"]}
    del sp, x
    torch.cuda.synchronize()
    return out


def hpcg_checks(prob, dev, stream):
    """The benchmark flow around the solver that HPCG runs (Sections II-A, III-A): the
    symmetry test of A and of the preconditioner M, |x'Ay - y'Ax| and
    |x'My - y'Mx| for random x, y in units of eps ||x|| ||y|| ||A||_inf
    (||A||_inf = 52; for M the bound 1/26 of a Jacobi step stands in), and a
    smoother study: time and iterations to 1e-9 of the symmetric smoother with
    one and two sweeps and of the forward-only ablation (b = A x_true,
    x_true ~ U[-1,1], seed 1)."""
    import torch
    from hpcg_inputs import mixed_precision_xtrue, normal
    from paper_2304_08232_gb300 import HpcgProblem
    n = NX * NY * NZ
    eps = 2.0 ** -52
    x = torch.as_tensor(normal(n, 41), device=dev)
    y = torch.as_tensor(normal(n, 42), device=dev)
    nx_, ny_ = float(torch.linalg.norm(x)), float(torch.linalg.norm(y))
    dA = abs(float(torch.dot(x, prob.spmv(y))) - float(torch.dot(y, prob.spmv(x))))
    dM = abs(float(torch.dot(x, prob.mg_vcycle(y))) - float(torch.dot(y, prob.mg_vcycle(x))))
    sym = {"A_departure_eps": dA / (eps * nx_ * ny_ * 52.0), "M_departure_eps": dM / (eps * nx_ * ny_ / 26.0)}
    xt = torch.as_tensor(mixed_precision_xtrue(n, seed=1), device=dev)
    bt = prob.spmv(xt)
    study = {}
    for name, kw in [("symmetric_1_sweep", {}), ("symmetric_2_sweeps", {"pre_sweeps": 2, "post_sweeps": 2}),
                     ("forward_only_1_sweep", {"symmetric": False})]:
        p = HpcgProblem(NX, NY, NZ, levels=LEVELS, device=dev, **kw)
        xs, st = p.pcg_solve(bt, max_iters=400, tol=1e-9)  # warm-up, graph capture
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs, st = p.pcg_solve(bt, max_iters=400, tol=1e-9)
        e1.record(stream)
        torch.cuda.synchronize()
        study[name] = {"ms": e0.elapsed_time(e1), "iters": st.iters, "converged": st.converged,
                       "err_vs_xtrue": float((xs - xt).abs().max() / xt.abs().max())}
        del p, xs
    return {"symmetry": sym, "smoother_study_to_1e-9": study}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import OracleProblem
    lib, threads, how = oracle_lib(True)
    o = OracleProblem(NX, NY, NZ, levels=LEVELS, lib=lib)
    b = o.rhs()
    for _ in range(args.warmup):
        o.pcg(b, max_iters=1, tol=0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.pcg(b, max_iters=1, tol=0.0)
    dt = time.perf_counter() - t0
    fl = hpcg_flops_per_iter(NX, NY, NZ, LEVELS) * args.steps
    val = fl / dt / 1e9
    sample = "1 MG-PCG iteration of the %dx%dx%d workload per step (the rate is per iteration, as the GPU arm's), %s" % (
        NX, NY, NZ, how)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (HPCG generates its own operator; b = A*ones)", "config": bench_config(1),
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": val, "unit": "GFLOP/s"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_ranks(world, "nccl")
    from hpcg_inputs import mixed_precision_xtrue
    from paper_2304_08232_gb300 import HpcgProblem, launch_count

    dev = torch.device("cuda", local)
    n = NX * NY * NZ
    prob = HpcgProblem(NX, NY, NZ, levels=LEVELS, precision=args.precision, device=dev)
    if args.shapes:
        prob.set_launch_shapes(json.loads(args.shapes))
    b = prob.get_rhs()
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        x.zero_()
        prob.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x)

    for _ in range(max(args.warmup, 3) if args.warmup >= 0 else 3):
        step()
    torch.cuda.synchronize()

    def barrier():
        rank_barrier(world)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    # an event after every step: the mean over the K steps is the value, the
    # per-step times give the spread (the paper averages 10 repetitions)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = launch_count() - l0
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms = evs[0].elapsed_time(evs[-1]) / args.steps
    clocks = sampler.stop()
    ms, ms_min = max_over_ranks([ms, min(step_ms)], world, dev)

    flops_iter = hpcg_flops_per_iter(NX, NY, NZ, LEVELS)
    value = whole_job_gflops(world, flops_iter * ITERS, ms)
    # correctness of the timed solve: exact solution is ones
    err_ones = float((x - 1.0).abs().max().item())

    if args.profile_iters > 0:
        # one solve of that many iterations inside cudaProfilerStart/Stop, for
        # ncu --profile-from-start off (per-iteration kernel counters)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        x.zero_()
        prob.pcg_solve(b, max_iters=args.profile_iters, tol=0.0, out=x)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": "HPCG-rule GFLOP/s (quick profiling run)", "value": value, "unit": "GFLOP/s",
                              "ms_per_step": ms, "grid": [NX, NY, NZ], "gpu_launches": launches,
                              "max_abs_err_vs_ones": err_ones,
                              "shapes": json.loads(args.shapes) if args.shapes else "autotuned"}), flush=True)
        return 0

    # --- dominant kernel: the block-floating-point colour-pair kernel
    # k_gs_lines_bfp on the finest level, as the FP64 solve runs it: CUDA
    # events on the launching stream bracket every kernel group of one CG
    # iteration (hpcg_profile_iteration); the finest level's pre- and
    # post-smoother are 14 launches of it (7 runs each: [0,1] [2,3] [4,5]
    # [6,7,6] [5,4] [3,2] [1,0]); the median of 5 iterations.
    shapes = tuned_shapes(prob)
    peaks, peak_kind = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    l0_ms = sorted(prob.profile_iteration(b)["smoother_ms"][0] for _ in range(5))[2]
    launches_l0 = 7 * 2
    k_ms = l0_ms / launches_l0
    # Algorithmic bytes (the method's, per row of the finest level and V-cycle):
    # two symmetric smoother applications of 48 (r once, z read and written
    # once per sweep direction), the residual with restriction 9, the
    # refinement 2: 107 n over the 14 launches that carry them (restriction
    # and refinement are fused into the smoother's runs).  The kernel itself
    # moves more: every colour-pair run streams all of z to read its class's
    # neighbours (12 n per full run, 158 n per V-cycle: traffic_model), which
    # ncu's DRAM bytes confirm (traffic).
    bytes_launch = 107 * n / launches_l0
    achieved_gbs = bytes_launch / (k_ms * 1e-3) / 1e9
    # DRAM bytes (read + write) per finest-level launch, averaged over the 14
    # launches of one V-cycle, from an ncu capture at 192^3
    # (profiles/k_gs_lines_bfp_192cubed.md)
    traffic = 61.75e6 if (NX, NY, NZ) == (192, 192, 192) else None
    roofline = {"bound": "hbm", "kernel": "k_gs_lines_bfp<3> (finest level, colour-pair runs of the V-cycle)",
                "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                "peak_basis": "%s copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" % peak_kind,
                "bytes_algorithmic_per_launch": bytes_launch, "traffic": traffic,
                "traffic_model_per_launch": 158 * n / launches_l0,
                "bytes_basis": "107 n per V-cycle (2 x 48 smoother + 9 restriction + 2 refinement) over the 14 finest-level "
                               "launches; the kernel's own model 158 n (12 n per run: all of z per colour pair)",
                "ms_per_launch": k_ms, "launches_timed": launches_l0,
                "timing": "CUDA events around the finest level's 14 smoother launches of one CG iteration, median of 5",
                "launch_shapes_per_level": shapes}
    # The FP64-storage colour kernel (k_gs_lines_fx: hpcg_rbgs, and the V-cycle
    # with block_fp = 0) for comparison: one symmetric sweep, 7 launches
    r = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.randn(n, dtype=torch.float64, device=dev)
    for _ in range(3):
        prob.rbgs(r, z, 0)
    reps = 20
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        prob.rbgs(r, z, 0)
    k1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = k0.elapsed_time(k1) / reps
    roofline["fp64_storage_kernel"] = {"kernel": "k_gs_lines_fx<3>", "ms_per_launch": sweep_ms / 7,
                                       "achieved_gbs": 12 * n / (sweep_ms / 7 * 1e-3) / 1e9,
                                       "fp64_instr_per_updated_row": 4}
    del r, z
    # the SpMV alone (y = A x, no partials): x and y together fit L2 at 192^3,
    # so L2 is flushed (a 256 MB write) before every timed launch; median of 10
    xs_ = torch.randn(n, dtype=torch.float64, device=dev)
    ys_ = torch.empty_like(xs_)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)
    for _ in range(3):
        prob.spmv(xs_, out=ys_)
    sp_times = []
    for _ in range(10):
        flush.zero_()
        k0.record(stream)
        prob.spmv(xs_, out=ys_)
        k1.record(stream)
        torch.cuda.synchronize()
        sp_times.append(k0.elapsed_time(k1))
    sp_ms = sorted(sp_times)[5]
    del flush
    # k_spmv_stage_fx: the 27-point box sum in fixed point from lines staged in
    # shared memory; no FP64 instruction without the p.Ap partials
    spmv = {"kernel": "k_spmv_stage_fx<6,0>", "ms": sp_ms, "fp64_instr_per_row": 0, "timing": "L2 flushed before each launch, median of 10",
            "g_fp64_instr_s": n * 1 / (sp_ms * 1e-3) / 1e9,
            "hbm_gbs_algorithmic": 16 * n / (sp_ms * 1e-3) / 1e9,
            "hbm_frac_of_measured": 16 * n / (sp_ms * 1e-3) / 1e9 / measured_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS)}
    del xs_, ys_

    # --- mixed vs FP64 time to 1e-9 (b = A x_true, x_true ~ U[-1,1], seed 1)
    xt = torch.as_tensor(mixed_precision_xtrue(n, seed=1), device=dev)
    bt = prob.spmv(xt)
    res = {}
    for prec in ["fp64", "mixed"]:
        p = prob if prec == "fp64" else HpcgProblem(NX, NY, NZ, levels=LEVELS, precision="mixed", device=dev)
        xs, st = p.pcg_solve(bt, max_iters=200, tol=1e-9)  # warm-up and graph capture
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        xs, st = p.pcg_solve(bt, max_iters=200, tol=1e-9)
        t1.record(stream)
        torch.cuda.synchronize()
        true_rel = float(torch.linalg.norm(bt - prob.spmv(xs)) / torch.linalg.norm(bt))
        res[prec] = {"ms": t0.elapsed_time(t1), "iters": st.iters, "restarts": st.restarts, "rel_res": st.rel_res,
                     "true_rel_res": true_rel, "err_vs_xtrue": float((xs - xt).abs().max() / xt.abs().max()),
                     "x": xs}
    # the same FP64 solve in other configurations of the library
    variants = {}
    for name, kw in [("fp64_storage_in_vcycle", {"block_fp": False}), ("persistent_coarse_kernel", {"persistent": True}),
                     ("plain_fp64_sums", {"fixed_point": False}), ("no_programmatic_dependent_launch", {"pdl": False})]:
        p_v = HpcgProblem(NX, NY, NZ, levels=LEVELS, device=dev, **kw)
        xv = torch.zeros(n, dtype=torch.float64, device=dev)
        p_v.pcg_solve(b, max_iters=ITERS, tol=0.0, out=xv)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        xv.zero_()
        p_v.pcg_solve(b, max_iters=ITERS, tol=0.0, out=xv)
        t1.record(stream)
        torch.cuda.synchronize()
        variants[name] = {"ms_per_step": t0.elapsed_time(t1), "max_abs_diff_x_vs_default": float((xv - x).abs().max())}
        if name == "persistent_coarse_kernel":
            variants[name]["first_level"] = persistent_first(p_v)
        del p_v, xv
    mixed_vs = {k: {kk: vv for kk, vv in v.items() if kk != "x"} for k, v in res.items()}
    mixed_vs["speedup"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    mixed_vs["mixed_vs_fp64_x"] = float((res["mixed"]["x"] - res["fp64"]["x"]).abs().max() / res["fp64"]["x"].abs().max())
    del res

    breakdown = {"fp64": time_breakdown(prob, b), "mixed": time_breakdown(
        HpcgProblem(NX, NY, NZ, levels=LEVELS, precision="mixed", device=dev), b)}
    forms = {} if args.skip_forms else other_forms(dev, stream)
    checks = {} if args.skip_forms else hpcg_checks(prob, dev, stream)
    # --- every form against the HBM roofline: the dominant kernel where one
    # kernel dominates (single-grid forms), and the whole solve against the
    # per-row byte model of algorithmic_bytes_per_iter
    mixed_l0_ms = breakdown["mixed"]["smoother_ms"][0]
    mixed_l0_bytes = 53.5 * n  # the method's 107 n with FP32 vectors (the kernels' own model: 74.5 n)
    # the binding roofline of one FP64 iteration, both terms: bytes over the
    # copy bandwidth, and the FP64-pipe warp instructions one iteration executes
    # (ncu count per finest-level row) over the FP64 issue rate measured live
    # by the library's probe
    fp64_rate = fp64_probe(dev)
    bytes_us = algorithmic_bytes_per_iter(NX, NY, NZ, LEVELS) / (hbm_peak * 1e9) * 1e6
    fp64_us = (FP64_WARP_INSTR_PER_ROW_ITER * n / fp64_rate["warp_instr_per_s"] * 1e6
               if FP64_WARP_INSTR_PER_ROW_ITER is not None else 0.0)
    by_form = {
        "fp64_192^3_50_iters": {
            "dominant_kernel": roofline["kernel"], "dominant_kernel_frac": roofline["frac"],
            "whole_solve_roofline": whole_solve_roofline(algorithmic_bytes_per_iter(NX, NY, NZ, LEVELS) * ITERS, ms, hbm_peak),
            "binding_roofline_per_iter": {"bytes_term_us": bytes_us, "fp64_term_us": fp64_us,
                                          "fp64_warp_instr_per_row": FP64_WARP_INSTR_PER_ROW_ITER,
                                          "fp64_rate": fp64_rate,
                                          "bound": "hbm" if bytes_us >= fp64_us else "fp64",
                                          "measured_us": ms * 1e3 / ITERS,
                                          "frac": max(bytes_us, fp64_us) / (ms * 1e3 / ITERS)}},
        "mixed_192^3_to_1e-9": {
            "dominant_kernel": "k_gs_lines<float,3,PAIR> (finest level, FP32 colour-pair runs)",
            "dominant_kernel_bytes_per_vcycle": mixed_l0_bytes, "dominant_kernel_ms_per_vcycle": mixed_l0_ms,
            "dominant_kernel_frac": mixed_l0_bytes / (mixed_l0_ms * 1e-3) / 1e9 / hbm_peak,
            "whole_solve_roofline": whole_solve_roofline(
                algorithmic_bytes_per_iter(NX, NY, NZ, LEVELS, "mixed") * mixed_vs["mixed"]["iters"], mixed_vs["mixed"]["ms"],
                hbm_peak)},
    }
    for k, v in forms.items():
        if "whole_solve_roofline" in v:
            by_form[k] = {"whole_solve_roofline": v["whole_solve_roofline"]}
    by_form["byte_model"] = ("whole solve: per CG iteration, finest SpMV 16 B/row (+8 kappa) + CG passes 88 (84 mixed); per "
                             "non-coarsest level 2 x 48 (symmetric smoother) + 9 (residual, restriction) + 2 (refinement), "
                             "coarsest 48; FP32 preconditioner halves its terms; = 226 B/row at 192^3 FP64")
    ell = {} if args.skip_forms else ell_study(b, x, dev, stream)

    # --- end to end through the public API with host buffers
    b_h = b.cpu().pin_memory()
    x_h = torch.zeros(n, dtype=torch.float64).pin_memory()
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()
    bd = torch.empty_like(b)
    xd = torch.empty_like(b)

    def e2e_step():
        bd.copy_(b_h, non_blocking=True)
        xd.copy_(x_h, non_blocking=True)
        prob.pcg_solve(bd, max_iters=ITERS, tol=0.0, out=xd)
        out_h.copy_(xd, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    e_steps = max(2, min(args.steps, 5))
    q0.record(stream)
    for _ in range(e_steps):
        e2e_step()
    q1.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks([q0.elapsed_time(q1) / e_steps], world, dev)[0]
    e2e = {"value": whole_job_gflops(world, flops_iter * ITERS, e_ms), "unit": "GFLOP/s", "h2d_bytes_per_step": 2 * n * 8,
           "d2h_bytes_per_step": n * 8, "ms_per_step": e_ms}

    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return 0
    cpu = cpu1 = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(parallel=True)
        cpu1 = cpu_baseline(parallel=False)
    fp64_rate = by_form["fp64_192^3_50_iters"]["binding_roofline_per_iter"]["fp64_rate"]
    if clocks.get("sm_mhz"):
        fp64_rate["lane_fma_per_sm_clock"] = fp64_rate["lane_fma_per_s"] / fp64_rate["sms"] / (clocks["sm_mhz"] * 1e6)
    detail = {
        "roofline": roofline, "mixed_vs_fp64_to_1e-9": mixed_vs, "roofline_by_form": by_form, "spmv": spmv,
        "iteration_breakdown": breakdown, "fp64_solve_variants": variants, "forms": forms, "hpcg_checks": checks,
        "materialised_ell": ell, "cpu_baseline_1thread": cpu1, "ms_per_step_spread": [min(step_ms), max(step_ms)],
    }
    detail_path = args.detail
    if detail_path:
        with open(detail_path, "w") as f:
            json.dump(detail, f, indent=1, default=float)

    def r3(v):
        return None if v is None else float("%.4g" % v)

    bw = by_form["fp64_192^3_50_iters"]
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (HPCG generates its own operator; b = A*ones)",
        "config": bench_config(world),
        "gpu_launches": launches,
        "roofline": {k: (r3(v) if isinstance(v, float) else v) for k, v in roofline.items()
                     if k not in ("launch_shapes_per_level", "timing", "peak_basis", "fp64_storage_kernel")},
        "hbm_gbs_whole_solve": r3(bw["whole_solve_roofline"]["gbs"]),
        "mixed_vs_fp64_to_1e-9": {"fp64_ms": r3(mixed_vs["fp64"]["ms"]), "fp64_iters": mixed_vs["fp64"]["iters"],
                                  "mixed_ms": r3(mixed_vs["mixed"]["ms"]), "mixed_iters": mixed_vs["mixed"]["iters"],
                                  "mixed_restarts": mixed_vs["mixed"]["restarts"], "speedup": r3(mixed_vs["speedup"]),
                                  "mixed_true_rel_res": r3(mixed_vs["mixed"]["true_rel_res"]),
                                  "mixed_vs_fp64_x": r3(mixed_vs["mixed_vs_fp64_x"])},
        "roofline_by_form": {k: {"kernel_frac": r3(v.get("dominant_kernel_frac")),
                                 "whole_solve_frac": r3(v["whole_solve_roofline"]["frac"])}
                             for k, v in by_form.items() if isinstance(v, dict) and "whole_solve_roofline" in v},
        "binding_roofline_per_iter_us": {"bytes": r3(bw["binding_roofline_per_iter"]["bytes_term_us"]),
                                         "fp64": r3(bw["binding_roofline_per_iter"]["fp64_term_us"]),
                                         "measured": r3(bw["binding_roofline_per_iter"]["measured_us"]),
                                         "fp64_tflops_probe": r3(fp64_rate["tflops"])},
        "spmv_hbm_frac": r3(spmv["hbm_frac_of_measured"]),
        "smoother_ms_per_level": [r3(v) for v in breakdown["fp64"]["smoother_ms"]],
        "iter_ms": r3(breakdown["fp64"]["total_ms"]),
        "max_abs_err_vs_ones": r3(err_ones),
        "e2e": {k: (r3(v) if isinstance(v, float) else v) for k, v in e2e.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "cpu_baseline_1thread_gflops": r3(cpu1["value"]) if cpu1 else None,
        "detail": detail_path,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=192, help="cubic grid edge (profiling runs; default 192)")
    ap.add_argument("--dims", default=None, help="nx,ny,nz of a non-cubic grid (profiling runs; overrides --grid)")
    ap.add_argument("--skip-forms", action="store_true", help="skip the batched and differentiable form timings")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="preconditioner precision of the timed solve (profiling runs; the bench line is FP64)")
    ap.add_argument("--shapes", default=None,
                    help="JSON list of per-level launch shapes [[row lines, row planes, line lines, line planes], ...] "
                         "to use instead of autotuning (repeatable profiling runs)")
    ap.add_argument("--ell-only", action="store_true",
                    help="run only the materialised-operator study (sliced-ELL, colour-sorted and natural order, two "
                         "sub-domains) at the grid size and print its JSON (profiling runs)")
    ap.add_argument("--detail", default=None,
                    help="file for the full measurement record (forms, variants, breakdowns); none by default")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="after the timed steps, one solve of this many CG iterations between cudaProfilerStart and "
                         "cudaProfilerStop (for ncu --profile-from-start off)")
    ap.add_argument("--vcycles", type=int, default=0,
                    help="time this many V-cycles alone and print per-level times (profiling runs of the preconditioner)")
    ap.add_argument("--cluster-tail", action="store_true", help="with --vcycles: hpcg_options.cluster_tail")
    ap.add_argument("--persistent", action="store_true", help="with --vcycles: hpcg_options.persistent")
    ap.add_argument("--size-sweep", default=None,
                    help="semicolon-separated nx,ny,nz grids: time the 50-iteration FP64 solve on each and print one "
                         "JSON line (how the rates change with problem size; the paper solves the largest that fits)")
    ap.add_argument("--quick", action="store_true",
                    help="time the FP64 solve only (no kernel roofline, mixed comparison, e2e or CPU baseline)")
    args = ap.parse_args()
    global NX, NY, NZ
    NX = NY = NZ = args.grid
    if args.dims:
        NX, NY, NZ = (int(v) for v in args.dims.split(","))
    if args.impl == "reference":
        return run_reference(args)
    if args.ell_only:
        return run_ell_only()
    if args.vcycles > 0:
        return run_vcycles(args)
    if args.size_sweep:
        return run_size_sweep(args)
    return run_gpu(args)


def run_size_sweep(args):
    """The FP64 MG-PCG solve (50 iterations, 4 levels, b = A ones) on each grid
    of --size-sweep: CUDA-event time of --steps solves after --warmup, the
    HPCG-rule rate, the whole solve against the per-row byte model, and the
    finest level's colour-pair runs against the method's 107 n bytes per
    V-cycle; with the colour-pair runs of one plane parity grouped into one
    launch as the autotuner chooses (auto), never (per_run) and always
    (grouped)."""
    import torch
    from paper_2304_08232_gb300 import HpcgProblem
    dev = torch.device("cuda", 0)
    peak = measured_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS)
    out = []
    for spec in args.size_sweep.split(";"):
        nx, ny, nz = (int(v) for v in spec.split(","))
        n = nx * ny * nz
        entry = {"grid": [nx, ny, nz], "rows": n}
        for name, fuse in (("auto", 0), ("per_run", -1), ("grouped", 1)):
            prob = HpcgProblem(nx, ny, nz, levels=LEVELS, fuse_planes=fuse, device=dev)
            b = prob.get_rhs()
            x = torch.zeros_like(b)
            for _ in range(max(args.warmup, 1)):
                prob.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                prob.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            prof = prob.profile_iteration(b)
            fine_ms = prof["smoother_ms"][0]
            entry[name] = {"ms_per_solve": round(ms, 3),
                           "gflops": round(hpcg_flops_per_iter(nx, ny, nz, LEVELS) * ITERS / (ms * 1e-3) / 1e9, 1),
                           "whole_solve_frac": round(whole_solve_roofline(algorithmic_bytes_per_iter(nx, ny, nz, LEVELS) * ITERS, ms,
                                                                          peak)["frac"], 4),
                           "finest_smoother_frac": round(107 * n / (fine_ms * 1e-3) / 1e9 / peak, 4),
                           "iteration_ms": round(prof["total_ms"], 4),
                           "smoother_ms_per_level": [round(v, 4) for v in prof["smoother_ms"]],
                           "max_abs_err_vs_ones": float((x - 1.0).abs().max())}
            del prob, b, x
            torch.cuda.empty_cache()
        out.append(entry)
        print(json.dumps(entry), file=sys.stderr, flush=True)
    print(json.dumps({"size_sweep": out, "levels": LEVELS, "cg_iters": ITERS, "hbm_peak_gbs": peak}), flush=True)
    return 0


def run_ell_only():
    import torch
    from paper_2304_08232_gb300 import HpcgProblem
    dev = torch.device("cuda", 0)
    prob = HpcgProblem(NX, NY, NZ, levels=LEVELS, device=dev)
    b = prob.get_rhs()
    x = torch.zeros_like(b)
    prob.pcg_solve(b, max_iters=ITERS, tol=0.0, out=x)
    torch.cuda.synchronize()
    print(json.dumps({"grid": [NX, NY, NZ], "materialised_ell": ell_study(b, x, dev, torch.cuda.current_stream())}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
