#!/usr/bin/env python
"""Jacobian-apply throughput of matrix-free Neo-Hookean hyperelasticity on B300.

One step = one Jacobian action y = J du (gather, sum-factorised collocated
gradient, pointwise linearised stress from stored quadrature data, transposed
contractions, atomic scatter, Dirichlet rows) through the C ABI call
nh_jacobian_apply.  Default workload: Q3 (q = 4 Gauss points) on 48^3
hexahedra of the unit cube, 9,145,875 DoF, FP64, 17 stored scalars per point.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nh|reference]

Prints ONE JSON line (rank 0).  N > 1 (torchrun) runs independent replicas,
one per GPU: the operator has no exchange step on a single-GPU mesh, so the
job value is the sum of all ranks' DoF over the slowest rank's time.
The reference arm (--impl reference) times the plain FP64 CPU oracle on a
bounded window of the same workload.  Besides the headline, the line carries the
roofline of the timed kernel, the end-to-end rate through the host-buffer entry
point, a sweep over Q2-Q4 and the three arithmetic paths, the unstructured-mesh
and quadrature-layout variants, and the solve comparison (plain FP64 p-MG
against the chosen solver), the multiscale solve and the atomics-vs-colouring
scatter timings.  Further modes print their own line instead: --multiscale (the
multiscale solve alone), --hex-solve (the solve workload through the
unstructured-mesh path) and --learned (the learned-coarse-space study on the
inclusion configuration).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobian apply GDoF/s Q2–Q4; solve time to rel. residual 1e-8, plain vs chosen"
NU = 0.3
PERTURB = 0.1
AMP = 0.05
SEED = 42
# Unit-count ALU peaks (148 SMs x DFMA or FFMA per clock x 2 flop x 2.032 GHz), used
# only when the measured ones (nh_fma_peak, measured at the start of every run) are missing
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# float-float: one FP64-accurate multiply-add (2 flops) costs 15 FP32 operations
# (FMA TwoProduct with the cross terms, TwoSum, Fast2Sum), and the FP32 pipe issues
# an add, a multiply or an FMA per lane per clock, so its ceiling in FP64 flops is
# the FP32 FMA rate (2 flops per instruction) / 15
FF_OPS_PER_FMA = 15
DEFAULT_N = {2: 74, 3: 48, 4: 37}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def n_dof_of(p, n):
    return 3 * (p * n + 1) ** 3


# dram__bytes_read.sum + dram__bytes_write.sum per apply launch from the ncu
# capture summarised in profiles/ (small case, scaled to the full launch by
# elements); reset to None whenever the kernel changes.
NCU_TRAFFIC = {("f64", 2, 74): 1.770e9, ("f64", 3, 48): 1.203e9, ("f64", 4, 37): 1.115e9,
               ("f32", 2, 74): 9.00e8, ("f32", 3, 48): 6.06e8, ("f32", 4, 37): 5.66e8,
               ("f64x", 2, 74): 1.795e9, ("f64x", 3, 48): 1.212e9, ("f64x", 4, 37): 1.179e9}


def apply_bytes(p, n, wbytes, S=17, bc_byte=True):
    """Algorithmic bytes of one apply: stored quadrature data, du read, y written,
    int32 element map, and (FP64 kernels) one Dirichlet-bit byte per node; the
    FP32 kernel reads the Dirichlet bits packed into its element map."""
    P, Q = p + 1, p + 1
    ne = n ** 3
    nn = (p * n + 1) ** 3
    return ne * Q ** 3 * S * wbytes + 2 * 3 * nn * wbytes + ne * P ** 3 * 4 + (nn if bc_byte else 0)


def apply_flops(p, n):
    """Algorithmic flops of one apply with sum factorisation and the collocated
    gradient: interpolation and its transpose 3 (P^3 Q + P^2 Q^2 + P Q^3) FMA each,
    gradient and its transpose 9 Q^4 FMA each, 168 flops pointwise per point."""
    P, Q = p + 1, p + 1
    fma = 6 * (P ** 3 * Q + P ** 2 * Q ** 2 + P * Q ** 3) + 18 * Q ** 4
    return n ** 3 * (2 * fma + 168 * Q ** 3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200", "-i", str(gpu_index)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the library arm
# ---------------------------------------------------------------------------
class Case:
    def __init__(self, nh, torch, ctx, p, n, layout=0):
        self.nh, self.ctx, self.p, self.n = nh, ctx, p, n
        from paper_2204_01722_b300 import inputs
        V = inputs.box_vertices(n, n, n, perturb=PERTURB, seed=SEED)
        self.space, self.nn, self.nd = nh.nh_space_box(ctx, n, n, n, V, p, p + 1)
        N = p * n + 1
        nh.nh_space_set_dirichlet(ctx, self.space, inputs.uniaxial_mask((N, N, N)))
        self.op = nh.nh_op_create(ctx, self.space, NU, None, 1.0, layout)
        X = nh.nh_space_coords(ctx, self.space, self.nn)
        u = inputs.smooth_field(X, AMP, seed=SEED + 1).ravel()
        self.minJ = nh.nh_qdata_setup(ctx, self.op, torch.from_numpy(u).cuda())
        self.du64 = torch.from_numpy(inputs.normal_vector(self.nd, seed=SEED + 2)).cuda()
        self.du32 = self.du64.float()
        self.y64 = torch.empty_like(self.du64)
        self.y32 = torch.empty_like(self.du32)

    def vecs(self, prec):
        return (self.du32, self.y32) if prec == "f32" else (self.du64, self.y64)

    def close(self):
        self.nh.nh_op_destroy(self.op)
        self.nh.nh_space_destroy(self.space)


class HexCase(Case):
    """The same workload on the unstructured-mesh path (`nh_space_hex`): every
    element's local frame a random cube rotation; ``shuffled`` also permutes the
    vertex ids and the element order (no locality left in the element map)."""

    def __init__(self, nh, torch, ctx, p, n, shuffled, morton=False):
        self.nh, self.ctx, self.p, self.n = nh, ctx, p, n
        from paper_2204_01722_b300 import inputs
        V = inputs.box_vertices(n, n, n, perturb=PERTURB, seed=SEED)
        Vh, H = inputs.hex_mesh_from_box(n, n, n, V, seed=SEED, permute=shuffled)
        if morton:  # elements reordered along the Z-order curve before numbering
            H = H[nh.nh_hex_morton_order(Vh, H)]
        self.space, self.nn, self.nd = nh.nh_space_hex(ctx, Vh, H, p, p + 1)
        X = nh.nh_space_coords(ctx, self.space, self.nn)
        m = np.zeros((self.nn, 3), dtype=bool)
        m[X[:, 0] < 1e-12, :] = True
        m[X[:, 0] > 1.0 - 1e-12, 0] = True
        nh.nh_space_set_dirichlet(ctx, self.space, m.ravel())
        self.op = nh.nh_op_create(ctx, self.space, NU, None, 1.0, 0)
        u = inputs.smooth_field(X, AMP, seed=SEED + 1).ravel()
        self.minJ = nh.nh_qdata_setup(ctx, self.op, torch.from_numpy(u).cuda())
        self.du64 = torch.from_numpy(inputs.normal_vector(self.nd, seed=SEED + 2)).cuda()
        self.du32 = self.du64.float()
        self.y64 = torch.empty_like(self.du64)
        self.y32 = torch.empty_like(self.du32)


def time_applies(nh, torch, ctx, stream, case, prec, steps, warmup, barrier):
    du, y = case.vecs(prec)
    for _ in range(warmup):
        nh.nh_jacobian_apply(ctx, case.op, du, y, prec=PREC[prec])
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = nh.nh_launch_count(ctx)
    e0.record(stream)
    for _ in range(steps):
        nh.nh_jacobian_apply(ctx, case.op, du, y, prec=PREC[prec])
    e1.record(stream)
    e1.synchronize()
    launches = nh.nh_launch_count(ctx) - l0
    barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), launches


PREC = {"f64": 0, "f32": 1, "f64x": 2}


def kernel_ms(nh, ctx, case, prec, steps):
    du, y = case.vecs(prec)
    nh.nh_profile_read(ctx)
    nh.nh_profile_enable(ctx, True)
    for _ in range(steps):
        nh.nh_jacobian_apply(ctx, case.op, du, y, prec=PREC[prec])
    tot, k = nh.nh_profile_read(ctx)
    nh.nh_profile_enable(ctx, False)
    return tot / max(k, 1)


def replica_max(dist, value, device):
    """Max over the ranks of a per-rank time: the slowest replica times the job."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, repeats, seconds):
    """Units per second over all replicas, in billions (GDoF/s for DoF)."""
    return world * units_per_rank * repeats / seconds / 1e9


def measure_alu_peaks(nh, ctx, gpu_index):
    """FP64 and FP32 FMA throughput measured on this GPU (nh_fma_peak: FMA chains
    on every SM, CUDA events), with the SM clock sampled meanwhile."""
    clocks = ClockSampler(gpu_index)
    f64, ms64 = nh.nh_fma_peak(ctx, 0, 16384)
    f32, ms32 = nh.nh_fma_peak(ctx, 1, 1 << 20)
    clk = clocks.stop()
    return {"fp64_tflops": round(f64, 4), "fp32_tflops": round(f32, 3),
            "float_float_tflops": round(f32 / FF_OPS_PER_FMA, 4), "fp64_ms": round(ms64, 2),
            "fp32_ms": round(ms32, 2), "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
            "how": "nh_fma_peak: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, one timed "
                   "launch after a warm-up; float-float = FP32 / %d FP32 operations per FP64-accurate FMA"
                   % FF_OPS_PER_FMA}


def run_nh(args):
    import torch
    from paper_2204_01722_b300 import nh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.Stream()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gpu_index = vis.split(",")[local] if vis and vis.split(",")[local].strip().isdigit() else str(local)
    out = {}
    with torch.cuda.stream(stream):
        ctx = nh.nh_create(local, stream.cuda_stream)
        p, n = args.p, args.n
        alu = measure_alu_peaks(nh, ctx, gpu_index)
        pk = {"f64": alu["fp64_tflops"], "f64x": alu["float_float_tflops"], "f32": alu["fp32_tflops"]}
        case = Case(nh, torch, ctx, p, n)
        clocks = ClockSampler(gpu_index)
        ms, launches = time_applies(nh, torch, ctx, stream, case, args.prec, args.steps, args.warmup, barrier)
        clk = clocks.stop()
        ms_max = replica_max(dist, ms, "cuda")
        value = whole_job_rate(world, case.nd, args.steps, ms_max * 1e-3)
        # roofline of the apply kernel alone (CUDA events around each launch)
        kms = kernel_ms(nh, ctx, case, args.prec, args.steps)
        hbm, hbm_src = peaks()
        wb = 4 if args.prec == "f32" else 8
        S, _ = nh.nh_op_info(ctx, case.op)
        if args.prec in ("f64", "f64x"):
            ach = apply_flops(p, n) / (kms * 1e-3) / 1e12
            src = ("measured FP64 DFMA throughput on this GPU (nh_fma_peak)" if args.prec == "f64" else
                   "measured FP32 FFMA throughput on this GPU / %d (float-float FMA cost)" % FF_OPS_PER_FMA)
            roof = {"bound": "alu", "achieved": round(ach, 4), "peak": pk[args.prec],
                    "unit": "TFLOP/s", "frac": round(ach / pk[args.prec], 4), "traffic": args.traffic,
                    "peak_source": src, "peak_unit_count": round(FP64_PEAK_TFLOPS, 4),
                    "kernel_ms": round(kms, 4), "hbm_frac": round(apply_bytes(p, n, wb, S) / (kms * 1e-3) / 1e9 / hbm, 4)}
        else:
            ach = apply_bytes(p, n, wb, S, bc_byte=False) / (kms * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "traffic": args.traffic, "peak_source": hbm_src + " (copy)",
                    "kernel_ms": round(kms, 4)}
        # end to end through the host-buffer entry point
        dt = np.float32 if args.prec == "f32" else np.float64
        hin = torch.from_numpy(np.ascontiguousarray(case.vecs(args.prec)[0].cpu().numpy())).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for _ in range(2):
            nh.nh_jacobian_apply_host(ctx, case.op, hin, hout, prec=PREC[args.prec])
        ek = max(3, args.steps // 10)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ek):
            nh.nh_jacobian_apply_host(ctx, case.op, hin, hout, prec=PREC[args.prec])
        te = time.perf_counter() - t0
        e2e = {"value": round(whole_job_rate(world, case.nd, ek, replica_max(dist, te, "cuda")), 4), "unit": "GDoF/s",
               "h2d_bytes_per_step": int(case.nd * np.dtype(dt).itemsize),
               "d2h_bytes_per_step": int(case.nd * np.dtype(dt).itemsize),
               "entry_point": "nh_jacobian_apply_host (pinned host du, y)"}
        minJ = case.minJ
        nd = case.nd
        case.close()
        sweep, hexes, layouts = [], [], []
        if args.sweep and rank == 0:
            for sp_ in (2, 3, 4):
                c = Case(nh, torch, ctx, sp_, DEFAULT_N[sp_])
                Sx, _ = nh.nh_op_info(ctx, c.op)
                for pr in ("f64", "f64x", "f32"):
                    k = kernel_ms(nh, ctx, c, pr, 5)  # warm (FP32 copy of the qdata on first use)
                    k = kernel_ms(nh, ctx, c, pr, 20)
                    w_ = 4 if pr == "f32" else 8
                    gbs = apply_bytes(sp_, c.n, w_, Sx, bc_byte=pr != "f32") / (k * 1e-3) / 1e9
                    tfl = apply_flops(sp_, c.n) / (k * 1e-3) / 1e12
                    sweep.append({"p": sp_, "n": c.n, "n_dof": c.nd, "prec": pr,
                                  "gdofs_kernel": round(c.nd / (k * 1e-3) / 1e9, 3), "kernel_ms": round(k, 4),
                                  "algorithmic_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                                  "tflops": round(tfl, 3), "alu_frac": round(tfl / pk[pr], 4),
                                  "traffic": NCU_TRAFFIC.get((pr, sp_, c.n))})
                c.close()
            for lay, lname in ((1, "initial tuned (27 scalars)"), (2, "AD-style tape (32 scalars)")):
                c = Case(nh, torch, ctx, 3, DEFAULT_N[3], layout=lay)
                for pr in ("f64", "f32"):
                    kernel_ms(nh, ctx, c, pr, 5)
                    k = kernel_ms(nh, ctx, c, pr, 20)
                    layouts.append({"layout": lname, "p": 3, "n": c.n, "n_dof": c.nd, "prec": pr,
                                    "gdofs_kernel": round(c.nd / (k * 1e-3) / 1e9, 3), "kernel_ms": round(k, 4)})
                c.close()
            for shuffled, morton in ((False, False), (True, False), (True, True)):
                c = HexCase(nh, torch, ctx, 3, DEFAULT_N[3], shuffled, morton)
                for pr in ("f64", "f32"):
                    kernel_ms(nh, ctx, c, pr, 5)
                    k = kernel_ms(nh, ctx, c, pr, 20)
                    # end to end through the host-buffer entry point (pinned du, y)
                    hin = c.vecs(pr)[0].cpu().pin_memory()
                    hout = torch.empty_like(hin).pin_memory()
                    nh.nh_jacobian_apply_host(ctx, c.op, hin, hout, prec=PREC[pr])
                    t0 = time.perf_counter()
                    for _ in range(5):
                        nh.nh_jacobian_apply_host(ctx, c.op, hin, hout, prec=PREC[pr])
                    te = (time.perf_counter() - t0) / 5
                    hexes.append({"mesh": "unstructured path, rotated element frames" +
                                          (", shuffled ids and elements" if shuffled else ", box element order") +
                                          (", then Z-order element order" if morton else ""),
                                  "p": 3, "n": c.n, "n_dof": c.nd, "prec": pr,
                                  "gdofs_kernel": round(c.nd / (k * 1e-3) / 1e9, 3), "kernel_ms": round(k, 4),
                                  "gdofs_e2e": round(c.nd / te / 1e9, 3)})
                c.close()
        sizes = []
        if args.sweep and rank == 0:
            # the ~1 M and ~50 M DoF rows of the Q2-Q4 sweep (the ~10 M rows are `sweep`)
            for sp_, n_ in ((2, 34), (2, 128), (3, 23), (3, 85), (4, 17), (4, 64)):
                c = Case(nh, torch, ctx, sp_, n_)
                Sx, _ = nh.nh_op_info(ctx, c.op)
                for pr in ("f64", "f64x", "f32"):
                    kernel_ms(nh, ctx, c, pr, 3)
                    k = kernel_ms(nh, ctx, c, pr, 10)
                    w_ = 4 if pr == "f32" else 8
                    gbs = apply_bytes(sp_, n_, w_, Sx, bc_byte=pr != "f32") / (k * 1e-3) / 1e9
                    tfl = apply_flops(sp_, n_) / (k * 1e-3) / 1e12
                    sizes.append({"p": sp_, "n": n_, "n_dof": c.nd, "prec": pr,
                                  "gdofs_kernel": round(c.nd / (k * 1e-3) / 1e9, 3), "kernel_ms": round(k, 4),
                                  "hbm_frac": round(gbs / hbm, 4), "alu_frac": round(tfl / pk[pr], 4)})
                c.close()
        scatter = []
        if args.sweep and rank == 0:
            # atomics against the eight-colour scatter (no atomics, eight launches), at
            # sizes whose x-element count is a multiple of the FP32 kernel's elements per block
            for sp_, n_ in ((2, 70), (3, 48), (4, 35)):
                c = Case(nh, torch, ctx, sp_, n_)
                for pr in ("f64", "f32"):
                    row = {"p": sp_, "n": n_, "n_dof": c.nd, "prec": pr}
                    for mode, key in ((0, "atomic"), (1, "colour8")):
                        nh.nh_op_set_scatter(ctx, c.op, mode)
                        kernel_ms(nh, ctx, c, pr, 5)
                        k = kernel_ms(nh, ctx, c, pr, 20)
                        row[key + "_ms"] = round(k, 4)
                        row[key + "_gdofs"] = round(c.nd / (k * 1e-3) / 1e9, 3)
                    nh.nh_op_set_scatter(ctx, c.op, 0)
                    scatter.append(row)
                c.close()
        solve = run_solves(nh, torch, ctx, stream, repeats=args.solve_repeats) if (args.solve and rank == 0) else None
        multi = multiscale_block(nh, torch, ctx, stream) if (args.multiscale_block and rank == 0) else None
        nh.nh_destroy(ctx)
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 4), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
               "config": {"workload": f"Jacobian apply, Q{p} (q={p + 1}) on {n}^3 hexahedra of the unit cube, "
                                      f"{nd} DoF, vertices perturbed 10% h, smooth displacement amplitude 0.05, "
                                      f"du ~ N(0,1), x=0 clamped + x=1 normal component fixed",
                          "p": p, "q": p + 1, "elements": n ** 3, "n_dof": nd, "layout": "current (17 scalars/point)",
                          "min_det_F": minJ, "l2": "inputs larger than L2 (quadrature data %.2f GB)"
                                                   % (n ** 3 * (p + 1) ** 3 * S * wb / 1e9),
                          "parallelism": f"replicas x{world}"},
               "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "alu_peaks": alu}
        if args.cpu_baseline:
            out["cpu_baseline"] = oracle_baseline_all_cores(p, n, args.cpu_seconds)
            out["cpu_baseline_1core"] = oracle_baseline(p, n, args.cpu_seconds)
        if sweep:
            out["sweep"] = sweep
        if hexes:
            out["hex"] = hexes
        if layouts:
            out["layouts"] = layouts
        if scatter:
            out["scatter"] = scatter
        if sizes:
            out["sweep_sizes"] = sizes
        if solve:
            out["solve"] = solve
        if multi:
            out["multiscale"] = multi
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# solve time to relative residual 1e-8, plain FP64 p-MG vs the chosen solver
# ---------------------------------------------------------------------------
SOLVE_ARMS = (  # name, mixed, fp64_kind, coarse_rediscretize, nonlinear, coarse_solver, coarse_fixed
    ("plain_fp64", 0, 0, 0, 0, 0, 0),
    ("lbfgs_fp64", 0, 0, 0, 1, 0, 0),
    ("newton_mixed_ff_rediscretized", 1, 1, 1, 0, 0, 0),
    ("chosen_lbfgs_mixed_ff_rediscretized_hmg", 1, 1, 1, 1, 1, 0),
    ("lbfgs_mixed_ff_rediscretized_hmg_fixed8", 1, 1, 1, 1, 1, 8),
)


def _report(rep):
    return {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.as_dict().items()}


def run_solves(nh, torch, ctx, stream, p=4, n=32, delta=0.10, steps=5, repeats=3):
    """Load-stepped p-MG solves of uniaxial compression, per solver arm: plain
    FP64 Newton-Krylov p-MG (the reference solver), FP64 L-BFGS with the V-cycle
    as initial inverse Hessian, Newton-Krylov with the faster V-cycle (FP32 on
    the p > 1 levels, FP64-accurate applies in float-float, rediscretised coarse
    levels), the chosen solver (L-BFGS with that V-cycle and the geometric
    multigrid coarse solve), and the same with the fixed coarse solve (8
    Chebyshev steps preconditioned by the geometric V-cycle).  Each arm: one
    discarded warm-up solve, then `repeats` timed solves, the arms' order rotated
    from one repeat to the next; reported: the median run's report, its time, and
    the spread of times and counts."""
    from paper_2204_01722_b300 import inputs
    V = inputs.box_vertices(n, n, n)
    sp, nn, nd = nh.nh_space_box(ctx, n, n, n, V, p, p + 1)
    N = p * n + 1
    nh.nh_space_set_dirichlet(ctx, sp, inputs.uniaxial_mask((N, N, N)))
    op = nh.nh_op_create(ctx, sp, NU, None, 1.0)
    g = torch.from_numpy(inputs.uniaxial_bc((N, N, N), delta)).cuda()
    mgs = {}
    for name, mixed, kind, redisc, nl, cs, fixed in SOLVE_ARMS:
        o = nh.nh_mg_default_opts(ctx, op, mixed=mixed, load_steps=steps, fp64_kind=kind,
                                  coarse_rediscretize=redisc, nonlinear=nl, coarse_solver=cs, coarse_fixed=fixed)
        mgs[name] = nh.nh_mg_create(ctx, op, o)
    runs = {name: [] for name in mgs}

    def solve(name):
        u = torch.zeros(nd, dtype=torch.float64, device="cuda")
        rep = nh.nh_solve(ctx, mgs[name], g, u, check=False)
        stream.synchronize()
        return rep

    for name in mgs:
        solve(name)                                   # warm-up, discarded
    names = list(mgs)
    for r in range(repeats):
        for name in names[r % len(names):] + names[:r % len(names)]:
            runs[name].append(solve(name))
    out = {}
    for name, reps in runs.items():
        secs = [x.seconds for x in reps]
        med = sorted(range(len(reps)), key=lambda i: secs[i])[len(reps) // 2]
        out[name] = _report(reps[med])
        out[name].update(seconds_all=[round(x, 3) for x in secs],
                         krylov_its_all=[x.krylov_its for x in reps], newton_its_all=[x.newton_its for x in reps])
        nh.nh_mg_destroy(mgs[name])
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(sp)
    out["workload"] = (f"Q{p} on {n}^3 ({nd} DoF), {int(delta * 100)}% uniaxial compression in {steps} load "
                       f"steps, p-MG {p}->2->1, Chebyshev(3)-Jacobi, Q1 coarse Jacobi-PCG 1e-3 (plain), "
                       f"FCG 1e-3, Newton to 1e-8")
    out["protocol"] = (f"per arm one discarded warm-up solve, then the median of {repeats} solves; "
                       f"arm order rotated between repeats")
    out["speedup"] = round(out["plain_fp64"]["seconds"] /
                           max(out["chosen_lbfgs_mixed_ff_rediscretized_hmg"]["seconds"], 1e-9), 3)
    return out


def run_hex_solves(args):
    """The solve workload (Q4 on 32^3, 10% compression in 5 load steps) passed
    through the unstructured-mesh path (`nh_space_hex`, every element's local
    frame a random cube rotation): the Q1 level is then the COO-assembled
    block-row matrix.  Prints one JSON line with plain FP64 Newton-Krylov p-MG
    and the chosen solver without the geometric coarse multigrid (box only)."""
    import torch
    from paper_2204_01722_b300 import inputs, nh
    p, n = 4, 32
    stream = torch.cuda.Stream()
    ctx = nh.nh_create(0, stream.cuda_stream)
    out = {"workload": f"Q{p} on {n}^3 through nh_space_hex (rotated element frames), 10% uniaxial compression "
                       f"in 5 load steps, relative residual 1e-8, Q1 level COO-assembled"}
    with torch.cuda.stream(stream):
        Vh, H = inputs.hex_mesh_from_box(n, n, n, inputs.box_vertices(n, n, n), seed=SEED, permute=False)
        sp, nn, nd = nh.nh_space_hex(ctx, Vh, H, p, p + 1)
        X = nh.nh_space_coords(ctx, sp, nn)
        m = np.zeros((nn, 3), dtype=bool)
        m[X[:, 0] < 1e-12, :] = True
        m[X[:, 0] > 1.0 - 1e-12, 0] = True
        nh.nh_space_set_dirichlet(ctx, sp, m.ravel())
        g = np.zeros((nn, 3))
        g[X[:, 0] > 1.0 - 1e-12, 0] = -0.10
        g = torch.from_numpy(g.ravel()).cuda()
        op = nh.nh_op_create(ctx, sp, NU, None, 1.0)
        for name, mixed, kind, redisc, nl in (("plain_fp64", 0, 0, 0, 0),
                                              ("lbfgs_mixed_ff_rediscretized", 1, 1, 1, 1)):
            o = nh.nh_mg_default_opts(ctx, op, mixed=mixed, load_steps=5, fp64_kind=kind,
                                      coarse_rediscretize=redisc, nonlinear=nl, coarse_solver=0)
            mg = nh.nh_mg_create(ctx, op, o)
            u = torch.zeros(nd, dtype=torch.float64, device="cuda")
            rep = nh.nh_solve(ctx, mg, g, u, check=False)
            stream.synchronize()
            out[name] = {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.as_dict().items()}
            nh.nh_mg_destroy(mg)
        nh.nh_op_destroy(op)
        nh.nh_space_destroy(sp)
    nh.nh_destroy(ctx)
    print(json.dumps({"hex_solve": out}), flush=True)


def multiscale_block(nh, torch, ctx, stream, p=3, n=64):
    """Mixed precision on the multiscale structure: Q3 on 64^3 elements (21.6 M DoF),
    per-element modulus from disjoint seeded spheres (volume fraction 0.3, radius
    2-6 elements, at least 2 elements between surfaces, contrast 1e3), 5% uniaxial
    compression in 5 load steps.  The chosen solver (L-BFGS, V-cycle with FP32
    applies/smoothers/transfers on p > 1 levels, float-float FP64-accurate fine
    residual path, rediscretised levels, geometric coarse multigrid) against the
    same solver with FP64 levels.  Each arm is warmed up by one load step of 0.5%
    on the same operator, then timed once; returns both reports, the relative
    difference of the two displacement solutions and min det F."""
    from paper_2204_01722_b300 import inputs
    out = {"workload": f"Q{p} on {n}^3, disjoint inclusions (vf 0.3, r 2-6 elements, gap >= 2 elements, "
                       f"E 1e3/1), 5% uniaxial compression in 5 load steps, relative residual 1e-8",
           "protocol": "per arm one warm-up solve (one load step of 0.5%), then one timed solve"}
    V = inputs.box_vertices(n, n, n)
    sp, nn, nd = nh.nh_space_box(ctx, n, n, n, V, p, p + 1)
    N = p * n + 1
    nh.nh_space_set_dirichlet(ctx, sp, inputs.uniaxial_mask((N, N, N)))
    E = inputs.inclusion_modulus(n, n, n, seed=SEED, gap=2.0)
    out["inclusion_fraction"] = round(float((E > 1.0).mean()), 4)
    op = nh.nh_op_create(ctx, sp, NU, E, 1.0)
    g = torch.from_numpy(inputs.uniaxial_bc((N, N, N), 0.05)).cuda()
    sols = {}
    for name, mixed, kind, redisc in (("chosen_mixed", 1, 1, 1), ("same_solver_fp64", 0, 0, 0)):
        o = nh.nh_mg_default_opts(ctx, op, mixed=mixed, load_steps=1, fp64_kind=kind,
                                  coarse_rediscretize=redisc, nonlinear=1, coarse_solver=1)
        mg = nh.nh_mg_create(ctx, op, o)
        u = torch.zeros(nd, dtype=torch.float64, device="cuda")
        nh.nh_solve(ctx, mg, g * 0.1, u, check=False)
        nh.nh_mg_destroy(mg)
        o.load_steps = 5
        mg = nh.nh_mg_create(ctx, op, o)
        u = torch.zeros(nd, dtype=torch.float64, device="cuda")
        rep = nh.nh_solve(ctx, mg, g, u, check=False)
        stream.synchronize()
        out[name] = _report(rep)
        out[name]["min_det_F"] = float("%.4g" % nh.nh_qdata_setup(ctx, op, u))
        sols[name] = u
        nh.nh_mg_destroy(mg)
    a, b = sols["chosen_mixed"], sols["same_solver_fp64"]
    out["rel_diff_mixed_vs_fp64"] = float("%.4g" % (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item())
    out["speedup"] = round(out["same_solver_fp64"]["seconds"] / max(out["chosen_mixed"]["seconds"], 1e-9), 3)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(sp)
    return out


def run_multiscale(args):
    """The multiscale block alone, as its own JSON line."""
    import torch
    from paper_2204_01722_b300 import nh
    stream = torch.cuda.Stream()
    ctx = nh.nh_create(0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        out = multiscale_block(nh, torch, ctx, stream, args.p, args.n)
    nh.nh_destroy(ctx)
    print(json.dumps({"multiscale": out}), flush=True)


def net_flops(N, channels):
    """Multiply-adds x 2 of one forward pass of the coarse-correction U-Net on an
    N^3 vertex grid (3x3x3 convolutions; stride-2 ones counted at their output)."""
    L = len(channels)
    Ng = [N]
    for _ in range(1, L):
        Ng.append((Ng[-1] - 1) // 2 + 1)
    conv = lambda ci, co, l: 2 * 27 * ci * co * Ng[l] ** 3
    f = conv(4, channels[0], 0) + conv(channels[0], channels[0], 0)
    for l in range(1, L):
        f += conv(channels[l - 1], channels[l], l) + conv(channels[l], channels[l], l)
    for l in range(L - 2, -1, -1):
        f += conv(channels[l + 1], channels[l], l) + conv(channels[l], channels[l], l)
    f += conv(channels[0], 3, 0)
    return f, f - conv(4, channels[0], 0)  # forward; input gradients (none for the network input)


def run_net(args):
    """Forward and Adam step of the coarse-correction network (BF16, 4 levels,
    16/32/48/64 channels) on the (n+1)^3 vertex grid, tensor cores against CUDA
    cores, CUDA events on the launching stream."""
    import torch
    from paper_2204_01722_b300 import nh
    N, ch, B = args.n + 1, (16, 32, 48, 64), 4
    stream = torch.cuda.Stream()
    ctx = nh.nh_create(0, stream.cuda_stream)
    out = {"workload": f"coarse-correction U-Net, {N}^3 vertex grid, channels 16/32/48/64, BF16", "steps": args.steps}
    with torch.cuda.stream(stream):
        net = nh.nh_net_create(ctx, N, len(ch), ch, bf16=True, seed=1)
        g = torch.Generator(device="cuda").manual_seed(1)
        x = torch.randn((B, 4, N, N, N), device="cuda", generator=g)
        t = torch.randn((B, 3, N, N, N), device="cuda", generator=g)
        y = torch.empty((3, N, N, N), device="cuda")

        def timed(fn, k):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / k

        for tc in (True, False):
            nh.nh_net_set_tensor_cores(ctx, net, tc)
            fwd = timed(lambda: nh.nh_net_forward(ctx, net, x[0], y), args.steps)
            step = timed(lambda: nh.nh_net_train_step(ctx, net, B, x, t, 1e-5), max(1, args.steps // 4))
            out["tensor_cores" if tc else "cuda_cores"] = {"forward_ms": round(fwd, 4),
                                                           "train_step_ms": round(step, 3)}
        nh.nh_net_destroy(net)
    nh.nh_destroy(ctx)
    ff, fdx = net_flops(N, ch)
    out["forward_gflop"] = round(ff / 1e9, 3)
    out["train_step_gflop"] = round(B * (2 * ff + fdx) / 1e9, 3)
    for k in ("tensor_cores", "cuda_cores"):
        out[k]["forward_tflops"] = round(ff / out[k]["forward_ms"] / 1e9, 2)
        out[k]["train_step_tflops"] = round(B * (2 * ff + fdx) / out[k]["train_step_ms"] / 1e9, 2)
    out["train_batch"] = B
    print(json.dumps({"net": out}), flush=True)


# ---------------------------------------------------------------------------
# oracle arm (CPU baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleWindow:
    """The plain FP64 oracle's Jacobian apply on a w^3-element window of the same
    workload (same p, q, material, perturbed mesh, displacement recipe), set up
    once; `time(seconds)` runs applies for at least that long (at least one)."""

    def __init__(self, p, n, w=8, index=0):
        from oracle import fem
        from paper_2204_01722_b300 import inputs
        self.fem, self.p, self.n, self.w = fem, p, n, w
        V = inputs.box_vertices(n, n, n, perturb=PERTURB, seed=SEED).reshape(n + 1, n + 1, n + 1, 3)
        x0 = (n - w) // 2
        z0 = (x0 + index * w) % (n - w + 1)   # window `index`: shifted along z
        sub = V[z0:z0 + w + 1, x0:x0 + w + 1, x0:x0 + w + 1].reshape(-1, 3)
        self.sp = fem.Space(w, w, w, sub, p, p + 1)
        mat = fem.Material(1.0, NU, self.sp.ne)
        u = inputs.smooth_field(self.sp.node_coords(), AMP, seed=SEED + 1).ravel()
        self.st = fem.qp_state(self.sp, mat, u)
        self.du = inputs.normal_vector(self.sp.n_dof, seed=SEED + 2)
        self.mask = np.zeros(self.sp.n_dof, dtype=bool)
        self.fem.jacobian_apply(self.sp, self.st, self.du, self.mask)

    def time(self, seconds):
        reps, t0 = 0, time.perf_counter()
        while True:
            self.fem.jacobian_apply(self.sp, self.st, self.du, self.mask)
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        return {"value": round(self.sp.n_dof * reps / el / 1e9, 6), "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                "sample": f"{reps} FP64 oracle applies on a {self.w}^3-element window (Q{self.p}, {self.sp.n_dof} "
                          f"DoF) of the {self.n}^3 workload, {el:.2f} s, single-threaded numpy"}


def oracle_baseline(p, n, seconds, w=8):
    """Time the plain FP64 oracle's Jacobian apply on a w^3-element window of the
    same workload for about `seconds`."""
    return OracleWindow(p, n, w).time(seconds)


def _oracle_worker(p, n, w, seconds, index, barrier, queue):
    """One host core: its own window, applies for `seconds` once every core is ready."""
    win = OracleWindow(p, n, w, index)
    try:
        barrier.wait(timeout=300)
    except Exception:
        queue.put((index, 0, 1.0, win.sp.n_dof))
        return
    reps, t0 = 0, time.perf_counter()
    while True:
        win.fem.jacobian_apply(win.sp, win.st, win.du, win.mask)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    queue.put((index, reps, el, win.sp.n_dof))


def oracle_baseline_all_cores(p, n, seconds, w=8):
    """The oracle on every host core at once: one process per core (spawned, one
    BLAS/OpenMP thread each), each applying the oracle on its own w^3-element
    window of the workload for about `seconds`; the rate is all windows' DoF
    over the slowest process's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    mpc = mp.get_context("spawn")
    barrier, queue = mpc.Barrier(cores), mpc.Queue()
    procs = [mpc.Process(target=_oracle_worker, args=(p, n, w, seconds, i, barrier, queue)) for i in range(cores)]
    for pr in procs:
        pr.start()
    res = [queue.get(timeout=600) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    el = max(r[2] for r in res)
    dofs = sum(r[1] * r[3] for r in res)
    return {"value": round(dofs / el / 1e9, 6), "unit": "GDoF/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, one per host core, each running FP64 oracle applies on its own "
                      f"{w}^3-element window (Q{p}) of the {n}^3 workload for {seconds:.0f} s; "
                      f"{sum(r[1] for r in res)} applies in {el:.2f} s"}


def run_reference(args):
    """The oracle as the reference arm: one step is one FP64 oracle apply on an
    8^3-element window of the workload (~0.06 s at Q3), set up once; W untimed
    steps, then K timed ones; the value is the window's DoF over the median step
    and ms_per_step that median, so steps x ms_per_step is the time spent."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    win = OracleWindow(args.p, args.n)
    for _ in range(args.warmup):
        win.fem.jacobian_apply(win.sp, win.st, win.du, win.mask)
    times, t0 = [], time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        win.fem.jacobian_apply(win.sp, win.st, win.du, win.mask)
        times.append(time.perf_counter() - t1)
    total = time.perf_counter() - t0
    step = statistics.median(times)
    v = round(win.sp.n_dof / step / 1e9, 6)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(step * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"Jacobian apply, Q{args.p} (q={args.p + 1}) on a {win.w}^3-element window "
                                  f"({win.sp.n_dof} DoF) of the {args.n}^3 hexahedra workload, plain FP64 CPU oracle",
                      "p": args.p, "window_elements": win.w ** 3, "window_n_dof": win.sp.n_dof,
                      "workload_n_dof": n_dof_of(args.p, args.n)},
           "cpu_baseline": {"value": v, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} single applies on the {win.w}^3-element window, median step "
                                      f"{step * 1e3:.1f} ms, {total:.1f} s in all, single-threaded numpy"},
           "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nh", choices=["nh", "reference"])
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "f64x"])
    ap.add_argument("--no-sweep", dest="sweep", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--solve-repeats", type=int, default=3)
    ap.add_argument("--no-multiscale", dest="multiscale_block", action="store_false",
                    help="skip the multiscale block of the default line")
    ap.add_argument("--hex-solve", action="store_true",
                    help="run the solve workload through the unstructured-mesh path instead of the bench")
    ap.add_argument("--multiscale", action="store_true",
                    help="run the mixed-precision multiscale solve (Q3 on 64^3 by default) instead of the bench")
    ap.add_argument("--learned", action="store_true",
                    help="run the learned-coarse-space study (training on 20 inclusion layouts of Q3 on 64^3, "
                         "5 held-out layouts; about 35 minutes) instead of the bench; prints its JSON line")
    ap.add_argument("--net", action="store_true",
                    help="time the coarse-correction network (forward and Adam step on the (n+1)^3 vertex grid, "
                         "tensor cores against CUDA cores) instead of the bench; prints its JSON line")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per apply from an ncu capture of this kernel (reported as is)")
    args = ap.parse_args()
    if args.hex_solve:
        run_hex_solves(args)
        return
    if args.learned:
        from paper_2204_01722_b300 import learned
        learned.main(["--n", str(args.n or 64), "--p", str(args.p), "--train", "20", "--test", "5", "--rhs", "1",
                      "--pairs", "16", "--epochs", "10", "--coarse-fixed", "30", "--vectors", "32,128"])
        return
    if args.net:
        args.n = args.n or 64
        run_net(args)
        return
    if args.multiscale:
        args.n = args.n or 64
        run_multiscale(args)
        return
    args.n = args.n or DEFAULT_N[args.p]
    if args.traffic is None:
        args.traffic = NCU_TRAFFIC.get((args.prec, args.p, args.n))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nh(args)


if __name__ == "__main__":
    main()
