"""Benchmark: operator matvecs per second of the grid-accelerated PMCHW operator
with surface-conductive absorbers, on the 12 um guide (19,420 triangles,
FFT grid 512 x 64 x 64, complex64), one GB300 per process.

A step is one full matvec y = A x (projection, FFT convolution with both
Green's functions, interpolation, near-field precorrection, testing of all
rows including the sigma-weighted absorber rows) on device-resident x.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

After the timed region the same line also carries (unless --no-extras):
the complex128 matvec rate, a 32-right-hand-side complex64 call, and the
time of one GMRES solve (complex64 operator, FP64 Arnoldi and refinement to
1e-8) with a Gaussian-beam excitation; a whole-matvec byte count beside the
dominant kernel's roofline.

N > 1 runs as N independent replicas (one per GPU, launched by
torch.distributed.run); the only collective is the max-over-ranks of the
timed region.  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

# the oracle baseline runs single-threaded; pin numpy's BLAS pools before import
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "operator matvecs/sec and GMRES solve time at N unknowns (%HBM roofline); FP32-batched vs FP64"
UNIT = "matvec/s"


def measured_traffic(stage, r_near_h=2.05):
    """DRAM bytes per launch of a stage's kernel from the committed ncu
    capture, or None when there is none, it was taken on another near radius,
    or the kernel source changed since."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "dram_traffic_guide_12um.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if abs(float(d.get("r_near_h", 2.05)) - r_near_h) > 1e-9:
        return None
    k = d.get("kernels", {}).get(stage)
    if not k:
        return None
    src = os.path.join(ROOT, k["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != k["source_sha256_16"]:
        return None
    return int(k["dram_read_bytes"] + k["dram_write_bytes"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_rate(case, seconds: float, max_tris: int | None = None):
    """Time the oracle's direct matvec (O1) on a bounded sample of edges (both
    triangles of each, so that their rows are complete) and extrapolate to a
    full matvec.  Returns (matvec/s, sample text, threads, seconds, rows) with
    rows = (x, row indices, O1 values at those rows) for the accuracy check."""
    from oracle import mesh, operator

    g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
    import cases

    sig = cases.sigma_points(case, g.qpts)
    med = operator.Media(*case.media)
    x = cases.synth.complex_normal(g.N, seed=1)
    rng = np.random.default_rng(0)
    order = rng.permutation(g.ne)
    row_of = mesh.row_index(g)
    done, ntri, t0 = 0, 0, time.perf_counter()
    threads = 1  # BLAS pools are pinned to one thread at start-up (see top of file)
    rows, vals = [], []
    while True:
        e = order[done]
        tris = g.edge_t[e]
        y = operator.matvec(g, med, x, sig, chunk=2, tris=tris)
        r = row_of[e][row_of[e] >= 0]
        rows.append(r)
        vals.append(y[r])
        done += 1
        ntri += len(tris)
        el = time.perf_counter() - t0
        if el >= seconds or done >= g.ne or (max_tris and ntri >= max_tris):
            break
    per_tri = el / ntri
    rate = 1.0 / (per_tri * g.nt)
    sample = (f"O1 direct matvec rows of {done} random edges ({ntri} target triangles of {g.nt}, {el:.1f} s), "
              "extrapolated")
    return rate, sample, threads, el, (x, np.concatenate(rows), np.concatenate(vals))


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------ byte models
def stage_bytes(info, ginfo, case, N, b):
    """Algorithmic HBM bytes per apply of each stage (one complex word = b
    bytes, one real word = b / 2).  Grid stages count only the covered grid
    points and active columns that the pruned transforms need."""
    n0, n1, n2 = case.grid.n
    P0 = 2 * n0
    nac, ngnz = ginfo["active_columns"], ginfo["covered_points"]
    oct_ = (P0 // 2 + 1) * (n1 + 1) * (n2 + 1)
    Q, q, p = info["qpoints"], case.q, case.grid.p
    nt = Q // q
    npairs = info["near_pairs"]
    r = b // 2
    return {
        # x in; summaries and point sources out; triangle and point geometry
        "summaries": b * (N + nt * 12 + Q * 12) + 4 * nt * 9 + 8 * (nt * 15 + Q * 4),
        # point sources in, the gather map (point, weight), 12 fields out
        "projection": b * (Q * 12 + 12 * ngnz) + Q * p**3 * (4 + r) + 8 * ngnz,
        "fft_axis0_fwd": b * 12 * nac * (n0 + P0),
        "fft_planes_green": b * (12 * P0 * nac + 16 * P0 * nac + 2 * oct_),
        "fft_axis0_inv": b * 16 * nac * (P0 + n0),
        # near records, the 16 potentials at covered points, summaries, tested
        # values out; per point: position, weight, stencil base and weights,
        # conductivity; per triangle: geometry
        "points": b * (npairs * q * 2 * 10 + 16 * ngnz + nt * 12 + nt * 12) + 4 * (nt + 1 + npairs)
        + Q * (24 + 8 + 12 + 2 * 3 * p * r + r) + nt * (16 + 3) * 8 + b * N + 4 * 12 * nt,
    }


def full_grid_model_bytes(info, case, N, b):
    """Whole-matvec bytes of the unpruned pFFT model: one round trip of each
    half-transformed field of the full transform grid (12 in, 16 out), both
    Green octants, the near records, the stencil data (read by projection and
    interpolation), per-point geometry, x in and y out."""
    n = 8 * case.grid.n[0] * case.grid.n[1] * case.grid.n[2]
    Q, p = info["qpoints"], case.grid.p
    nnz = info["near_pairs"] * case.q * 2 * 10
    return b * (2 * 28 * n // 2 + 2 * n // 8) + b * nnz + 2 * Q * (4 + 3 * p * (b // 2)) + Q * 48 + 2 * N * b


def run_gpu(args):
    ws, rank, local = dist_env()
    import cases

    case = cases.guide_full()
    case.r_near = args.near_radius_h * case.grid.h
    cpu = None
    o1_rows = None
    if rank == 0 and not args.no_cpu:
        rate, sample, threads, el, o1_rows = oracle_rate(case, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    import torch

    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_1004_5076_gb300 as sc
    from paper_1004_5076_gb300 import build

    build.build()
    m = case.mesh
    stream = torch.cuda.current_stream()
    t_setup = time.perf_counter()
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 1 if args.no_extras else 3, stream=stream)
    sc.scabem_set_sigma(op, segments=case.sigma_segments)
    t_setup = time.perf_counter() - t_setup
    info = sc.scabem_op_info(op)
    ginfo = sc.scabem_op_grid_info(op)
    N = sc.scabem_mesh_info(mh)[2]
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)

    def rand_x(shape, dtype):
        z = torch.complex(torch.randn(shape, device="cuda", generator=gen), torch.randn(shape, device="cuda",
                                                                                      generator=gen))
        return (z / math.sqrt(2)).to(dtype).contiguous()

    # the GPU operator against the oracle's dense operator (O1) on complete
    # sampled rows: the discretisation error of the grid method at (p, r_near)
    accuracy = None
    if o1_rows is not None:
        xo, ro, vo = o1_rows
        accuracy = {"rows": int(len(ro)), "reference": "oracle O1 (dense operator, direct matvec), same x",
                    "meaning": "grid-method (pFFT) discretisation error at this stencil order and near radius"}
        for name, prec, dt in (("c64", sc.SCABEM_C64, torch.complex64), ("c128", sc.SCABEM_C128, torch.complex128)):
            if name == "c128" and args.no_extras:
                continue
            xd = torch.as_tensor(xo).to(dt).cuda().contiguous()
            yd = torch.empty_like(xd)
            sc.scabem_apply(op, xd, yd, prec=prec, stream=stream)
            torch.cuda.synchronize()
            d = yd.cpu().numpy().astype(np.complex128)[ro] - vo
            accuracy["rel_l2_" + name] = float(np.linalg.norm(d) / np.linalg.norm(vo))
            accuracy["max_rel_" + name] = float(np.max(np.abs(d)) / np.max(np.abs(vo)))
    x = rand_x((N,), torch.complex64)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        sc.scabem_apply(op, x, y, prec=sc.SCABEM_C64, stream=stream)
    torch.cuda.synchronize()
    sc.scabem_profile(op, True, max(args.steps, 1))
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            sc.scabem_apply(op, x, y, prec=sc.SCABEM_C64, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    stages, napp = sc.scabem_profile_read(op)
    sc.scabem_profile(op, False)
    ms_max = max_over_ranks(ms, ws, device=torch.device("cuda", local))
    value = ws * args.steps / (ms_max / 1e3)

    # end to end through the C-ABI with pinned host buffers
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    sc.scabem_apply(op, xh, yh, prec=sc.SCABEM_C64, stream=stream)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sc.scabem_apply(op, xh, yh, prec=sc.SCABEM_C64, stream=stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, device=torch.device("cuda", local))
    barrier(ws)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    extras = None
    if not args.no_extras:
        # FP64 operator, single right-hand side
        x2 = x.to(torch.complex128)
        y2 = torch.empty_like(x2)
        ms128 = timed(lambda: sc.scabem_apply(op, x2, y2, prec=sc.SCABEM_C128, stream=stream), max(3, args.steps // 10))
        # complex64, 32 right-hand sides in one call (columns of a column-major N x 32 block)
        nb = 32
        X = rand_x((nb, N), torch.complex64)
        Y = torch.empty_like(X)
        msb = timed(lambda: sc.scabem_apply(op, X, Y, nrhs=nb, ld=N, prec=sc.SCABEM_C64, stream=stream), 3)
        # GMRES solve: Gaussian beam launched inside the core, complex64 operator with FP64
        # Arnoldi and FP64 iterative refinement to 1e-8
        src = [sc.make_source("beam", side="i", pos=(6.0, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.15)]
        bvec = torch.empty(N, dtype=torch.complex128, device="cuda")
        sc.scabem_rhs(op, src, bvec, prec=sc.SCABEM_C128, stream=stream)
        xs = torch.zeros_like(bvec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sinfo = sc.scabem_solve(op, bvec, xs, tol=1e-4, restart=100, maxit=20000, refine_tol=1e-8, max_refine=10,
                                prec=sc.SCABEM_C64, stream=stream)[0]
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        # transposed operator, adjoint solve and a conductivity gradient (16 B-spline coefficients)
        msa = timed(lambda: sc.scabem_apply_adjoint(op, x, y, prec=sc.SCABEM_C64, stream=stream),
                    max(3, args.steps // 10))
        g_rhs = torch.as_tensor(xs.cpu().numpy().conj()).cuda().contiguous()
        lam = torch.zeros_like(g_rhs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ainfo = sc.scabem_solve(op, g_rhs, lam, tol=1e-4, restart=100, maxit=20000, refine_tol=1e-8, max_refine=10,
                                prec=sc.SCABEM_C64, stream=stream, transpose=True)[0]
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        t0 = time.perf_counter()
        sc.scabem_sigma_gradient(op, xs, lam, src, bspline=(0.0, 12.0, 0, 16), stream=stream)
        t_grad = time.perf_counter() - t0
        # reflection of the solved field (the reflection configuration 2 asks for): E_y on the axis
        # between the beam source (x = 6 um) and the right absorber (x in [8, 12] um), two-wave fit
        refl = None
        try:
            t0 = time.perf_counter()
            rr = sc.scabem_reflection(op, xs, 0, 1, (0.0, 0.01, -0.005), 6.3, 7.7, 48, 8.0, 13.0, 1001, inc=src[0],
                                      stream=stream)[0]
            refl = {"abs_r": math.hypot(rr[0], rr[1]), "r": [rr[0], rr[1]], "beta_rad_per_um": rr[2],
                    "fit_residual": rr[3], "swr": rr[4], "r_from_swr": rr[5], "seconds": time.perf_counter() - t0,
                    "probe": "E_y at 48 axis points, x in [6.3, 7.7] um, beta scanned over [8, 13] rad/um",
                    "meaning": "reflection of the right-hand absorber seen by the beam launched at x = 6 um"}
        except sc.ScabemError as e:
            refl = {"error": str(e)}
        extras = {
            "reflection": refl,
            "c128": {"value": 1e3 / ms128, "unit": UNIT, "ms_per_step": ms128, "dtype": "c128"},
            "batched_c64": {"value": nb * 1e3 / msb, "unit": UNIT, "nrhs": nb, "ms_per_call": msb},
            "solve": {"seconds": t_solve, "iterations": sinfo["iters"], "refinements": sinfo["refinements"],
                      "relres": sinfo["relres"], "status": sinfo["status"],
                      "rhs": "Gaussian beam (waist 0.15 um) in the core at x = 6 um, y-polarised",
                      "mode": "GMRES(100) on the complex64 operator to 1e-4 with FP64 Arnoldi (classical Gram-Schmidt, repeated when the DGKS test asks), FP64 refinement to 1e-8"},
            "adjoint": {"matvec_per_s_c64": 1e3 / msa, "ms_per_step": msa,
                        "solve_seconds": t_adj, "solve_iterations": ainfo["iters"], "solve_relres": ainfo["relres"],
                        "sigma_gradient_seconds": t_grad,
                        "gradient": "d(lam^T (A x - b))/d coef for a 16-coefficient cubic B-spline over the guide"},
        }

    # roofline of the dominant kernel, and of the whole matvec
    hbm, src_peak = peaks()
    per = {k: v / max(napp, 1) for k, v in stages.items()}
    bmodel = stage_bytes(info, ginfo, case, N, 8)
    dom = max(per, key=per.get)
    roof = None
    if dom in bmodel:
        ach = bmodel[dom] / (per[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": measured_traffic(dom, args.near_radius_h), "peak_source": src_peak,
                "algorithmic_bytes": bmodel[dom]}
    t_mv = ms_max / args.steps / 1e3
    b_pruned = sum(bmodel.values())
    b_full = full_grid_model_bytes(info, case, N, 8)
    mv_roof = {
        "pruned_bytes": b_pruned, "pruned_frac": b_pruned / t_mv / 1e9 / hbm,
        "full_grid_model_bytes": b_full, "full_grid_model_frac": b_full / t_mv / 1e9 / hbm,
        "peak": hbm, "unit": "GB/s",
    }
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "guide_12um: 0.5x0.22 um eps 12.1 core in eps 2.1, 12 um, 4 um sigma0 (x/L)^3 "
                                   "absorbers at both ends, lambda 1.55 um",
                       "triangles": int(m.nt), "unknowns": int(N), "fft_grid": "512x64x64", "stencil_p": case.grid.p,
                       "q": case.q, "r_near_um": case.r_near, "r_near_h": args.near_radius_h,
                       "near_pairs": info["near_pairs"],
                       "covered_grid_points": ginfo["covered_points"], "active_columns": ginfo["active_columns"],
                       "l2": "working set per step > L2 (near data %.0f MB)" % (info["near_bytes_c64"] / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single GPU", "setup_s": t_setup},
            "e2e": {"value": ws * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(N * 8),
                    "d2h_bytes_per_step": int(N * 8)},
            "gpu_launches": 6 * args.steps,
            "stages_ms_per_step": per,
            "roofline": roof,
            "matvec_roofline": mv_roof,
            "cpu_baseline": cpu,
            "accuracy_vs_dense": accuracy,
            "clocks": clocks,
        }
        if extras:
            line.update(extras)
        print(json.dumps(line), flush=True)
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import cases

    case = cases.guide_full()
    case.r_near = args.near_radius_h * case.grid.h
    per_step = []
    sample = None
    threads = 1
    for i in range(args.warmup + args.steps):
        rate, sample, threads, el, _ = oracle_rate(case, args.ref_seconds)
        if i >= args.warmup:
            per_step.append(rate)
    value = float(np.mean(per_step))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "guide_12um (same as the GPU arm)", "triangles": int(case.mesh.nt)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--near-radius-h", type=float, default=2.05,
                    help="near-field radius in grid steps (2.05: the headline configuration)")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the c128, batched and solve measurements")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
