"""Benchmark: operator matvecs per second of the grid-accelerated PMCHW operator
with surface-conductive absorbers, on the 12 um guide (19,420 triangles,
FFT grid 512 x 64 x 64, complex64), one GB300 per process.

A step is one full matvec y = A x (projection, FFT convolution with both
Green's functions, interpolation, near-field precorrection, testing of all
rows including the sigma-weighted absorber rows) on device-resident x.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

After the timed region the same line also carries (unless --no-extras):
the complex128 matvec rate against the measured FP64 FMA peak, batched
complex64 calls of 8 and 32 right-hand sides, GMRES solves (complex64
operator, 48-bit Arnoldi and FP64 refinement to 1e-8) of one and of eight
excitations on the more accurate operator (near radius 3.05 grid steps) with
the reflection fitted from the solved field, the transposed operator and a
conductivity gradient, cuFFT on the full transform grid as a comparison, and
a whole-matvec byte count beside the dominant kernel's roofline.

N > 1 runs as N independent replicas (one per GPU, launched by
torch.distributed.run); the only collective is the max-over-ranks of the
timed region.  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import json
import math
import os
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
_O1 = {}


def _o1_init(case_name, r_near):
    """Worker set-up (spawned processes): the oracle's geometry of the workload."""
    import cases
    from oracle import mesh, operator

    case = cases.guide_full()
    case.r_near = r_near
    g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
    _O1.update(g=g, med=operator.Media(*case.media), sig=cases.sigma_points(case, g.qpts),
               x=cases.synth.complex_normal(g.N, seed=1), rows=mesh.row_index(g))


def _o1_edge(e):
    """O1 direct-matvec rows of edge e (both of its triangles as targets)."""
    from oracle import operator

    g = _O1["g"]
    tris = g.edge_t[e]
    y = operator.matvec(g, _O1["med"], _O1["x"], _O1["sig"], chunk=2, tris=tris)
    r = _O1["rows"][e][_O1["rows"][e] >= 0]
    return e, len(tris), r, y[r]


def oracle_rate_allcores(case, seconds: float):
    """The oracle's direct matvec (O1) on every host core: a pool of spawned
    processes evaluates the complete rows of random edges (both triangles of
    each) for `seconds` of wall time; the rate is extrapolated to a full
    matvec.  Returns (matvec/s, sample text, processes, seconds, rows) with
    rows = (x, row indices, O1 values) for the accuracy check."""
    import multiprocessing as mp

    from oracle import mesh

    g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
    import cases

    x = cases.synth.complex_normal(g.N, seed=1)
    order = np.random.default_rng(0).permutation(g.ne)
    nproc = os.cpu_count() or 1
    rows, vals, ntri, done = [], [], 0, 0
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(nproc, initializer=_o1_init, initargs=(case.name, case.r_near))
    try:
        list(pool.imap_unordered(_o1_edge, order[:nproc]))  # warm: every worker holds its geometry
        t0 = time.perf_counter()
        for e, nt_e, r, v in pool.imap_unordered(_o1_edge, order[nproc:], chunksize=1):
            rows.append(r)
            vals.append(v)
            ntri += nt_e
            done += 1
            if time.perf_counter() - t0 >= seconds:
                break
        el = time.perf_counter() - t0
    finally:
        pool.terminate()
        pool.join()
    rate = ntri / el / g.nt
    sample = (f"O1 direct matvec: complete rows of {done} random edges ({ntri} target triangles of {g.nt}) in "
              f"{el:.1f} s on {nproc} spawned processes, extrapolated to all {g.nt} triangles")
    return rate, sample, nproc, el, (x, np.concatenate(rows), np.concatenate(vals))


def o2_rate(case, targets: int = 24):
    """The oracle's grid operator (O2, the plain definition of the product the
    GPU computes) on one host core, with its near corrections precomputed as
    the GPU's set-up does: the grid part (projection, FFT convolution,
    interpolation) timed in full, the near-field application and testing
    timed on `targets` triangles and extrapolated.  Returns a dict."""
    import cases
    from oracle import mesh, operator, pfft
    from oracle.operator import current_sets, local_current, medium_fields, sigma_normalised, test_rows

    g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
    sig = cases.sigma_points(case, g.qpts)
    med = operator.Media(*case.media)
    x = cases.synth.complex_normal(g.N, seed=1)
    op = pfft.PFFT(g, med, case.grid, case.r_near)
    sets = current_sets(g, x[:, None])
    t0 = time.perf_counter()
    gf = op.grid_fields(sets, None)
    t_grid = time.perf_counter() - t0
    tg = np.arange(targets)
    pt, ps = pfft.near_pairs(g, op.r_near, tg)
    t0 = time.perf_counter()
    corr = pfft.near_corrections(op.grid, g, med, op.Gpad, pt, ps)
    t_corr = time.perf_counter() - t0
    t0 = time.perf_counter()
    (ke, ki), (ze, zi) = med.k, med.z
    q = g.q
    meds = []
    for m_, (k, z) in enumerate(((ke, ze), (ki, zi))):
        Js = sets[0] if m_ == 0 else sets[1]
        Ms = sets[2] if m_ == 0 else (-sets[2][0], -sets[2][1])
        Jn = pfft._near_fields(g, corr[m_], pt, ps, Js, tg)
        Mn = pfft._near_fields(g, corr[m_], pt, ps, Ms, tg)
        Jg, Mg = gf[m_]
        sel = (tg[:, None] * q + np.arange(q)[None, :]).reshape(-1)
        Jt = [Jg[i][sel].reshape((len(tg), q) + Jg[i].shape[1:]) + Jn[i] for i in range(4)]
        Mt = [Mg[i][sel].reshape((len(tg), q) + Mg[i].shape[1:]) + Mn[i] for i in range(4)]
        meds.append(medium_fields(Jt, Mt, k, z))
    Jsum = local_current(g, tg, sets[0]) + local_current(g, tg, sets[1])
    test_rows(g, tg, meds[0], meds[1], Jsum, local_current(g, tg, sets[2]), sigma_normalised(sig)[tg])
    t_near = time.perf_counter() - t0
    per_apply = t_grid + t_near * g.nt / targets
    return {"value": 1.0 / per_apply, "unit": UNIT, "cores": 1, "kind": "oracle O2 (grid operator definition)",
            "sample": (f"grid part timed in full ({t_grid:.1f} s); near-field application and testing of {targets} "
                       f"target triangles ({len(pt)} near pairs, {t_near:.2f} s) extrapolated to {g.nt}"),
            "setup_near_corrections_s_extrapolated": t_corr * g.nt / targets}


# ------------------------------------------------------------------ clocks
class Clocks:
    """SM clock and clock-event reasons sampled every 2 ms by a thread through
    NVML (read-only queries of libnvidia-ml), from entry to exit.  The GPU is
    matched to the CUDA device by UUID."""

    # clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.rows = []
        self.err = None
        self.max_mhz = None

    def _open(self):
        import ctypes as C

        nv = C.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        n = C.c_uint()
        nv.nvmlDeviceGetCount_v2(C.byref(n))
        want = None
        try:
            import torch

            want = str(torch.cuda.get_device_properties(self.cuda_index).uuid).lower().replace("gpu-", "")
        except Exception:
            pass
        dev = None
        for i in range(n.value):
            h = C.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(i, C.byref(h)) != 0:
                continue
            buf = C.create_string_buffer(96)
            nv.nvmlDeviceGetUUID(h, buf, 96)
            u = buf.value.decode().lower().replace("gpu-", "")
            if want is None or u == want or (n.value == 1):
                dev = h
                if want is None or u == want:
                    break
        if dev is None and self.cuda_index < n.value:
            h = C.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, C.byref(h)) == 0:
                dev = h
        if dev is None:
            raise RuntimeError("no NVML device matches the CUDA device")
        self.nv, self.dev = nv, dev
        mx = C.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(dev, 1, C.byref(mx)) == 0:  # NVML_CLOCK_SM = 1
            self.max_mhz = float(mx.value)
        self.get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons

    def _loop(self):
        import ctypes as C

        clk, rs = C.c_uint(), C.c_ulonglong()
        while not self.stop:
            if self.nv.nvmlDeviceGetClockInfo(self.dev, 1, C.byref(clk)) == 0 and \
                    self.get_reasons(self.dev, C.byref(rs)) == 0:
                self.rows.append((float(clk.value), int(rs.value)))
            time.sleep(0.002)

    def __enter__(self):
        import threading

        self.stop = False
        self.thread = None
        try:
            self._open()
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
        except Exception as e:  # no NVML on this host
            self.err = str(e)
        return self

    def __exit__(self, *a):
        self.stop = True
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, window):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"],
                    "error": self.err, "window": window}
        sm = [r[0] for r in self.rows]
        reasons = sorted({name for _, bits in self.rows for b, name in self.REASONS.items() if bits & b})
        return {"sm_mhz": float(np.median(sm)), "sm_min_mhz": float(min(sm)), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.rows), "source": "NVML, every 2 ms", "window": window}


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
def stage_bytes(info, ginfo, case, N, b, k=1):
    """Algorithmic HBM bytes per apply of each stage (one complex word = b
    bytes, one real word = b / 2) for a call of k right-hand sides: the near
    records, the tables and the geometry are read once per call, everything
    per right-hand side k times.  Grid stages count only the covered grid
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
        "summaries": k * b * (N + nt * 12 + Q * 12) + 4 * nt * 9 + 8 * (nt * 15 + Q * 4),
        # point sources in, the gather map (point, weight), 12 fields out
        "projection": k * b * (Q * 12 + 12 * ngnz) + Q * p**3 * (4 + r) + 8 * ngnz,
        "fft_axis0_fwd": k * b * 12 * nac * (n0 + P0),
        "fft_planes_green": k * b * (12 * P0 * nac + 16 * P0 * nac) + b * 2 * oct_,
        "fft_axis0_inv": k * b * 16 * nac * (P0 + n0),
        # near records, the 16 potentials at covered points, summaries, tested
        # values out; per point: position, weight, stencil base and weights,
        # conductivity; per triangle: geometry
        "points": b * npairs * q * 2 * 10 + k * b * (16 * ngnz + nt * 12 + nt * 12 + N) + 4 * (nt + 1 + npairs)
        + Q * (24 + 8 + 12 + 2 * 3 * p * r + r) + nt * (16 + 3) * 8 + 4 * 12 * nt,
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


def points_flops(info, case):
    """Floating-point operations of one apply's point stage (interpolation of
    the 16 potentials with value and gradient stencils, near-field
    corrections, testing), counted as the kernel performs them: each real
    stencil weight times a complex value is 2 FMAs, each complex multiply-add
    of the near records 4 FMAs; an FMA is 2 flops."""
    Q, p, q = info["qpoints"], case.grid.p, case.q
    interp = Q * 4 * p**3 * 4 * 4 * 2 * 2  # (medium, group) x stencil x 4 values x (v, gx, gy, gz) x 2 FMA x 2
    near = info["near_pairs"] * q * 4 * 19 * 4 * 2  # (pair, point, medium, group) x 19 complex MACs
    testing = Q * 3 * 4 * 60  # per (point, edge, row type): about 60 flops
    return interp + near + testing


def run_gpu(args):
    ws, rank, local = dist_env()
    import cases

    case = cases.guide_full()
    case.r_near = args.near_radius_h * case.grid.h
    cpu = None
    o1_rows = None
    o2 = None
    if rank == 0 and not args.no_cpu:
        # all host cores, in spawned processes, before this process touches the GPU
        rate, sample, nproc, el, o1_rows = oracle_rate_allcores(case, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample,
               "host": platform_info()}
        if not args.no_extras:
            o2 = o2_rate(case)
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

    def make_op(r_near, mask):
        t0 = time.perf_counter()
        o = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                                r_near, mask, stream=stream)
        sc.scabem_set_sigma(o, segments=case.sigma_segments)
        torch.cuda.synchronize()
        return o, time.perf_counter() - t0

    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op, t_setup = make_op(case.r_near, 1 if args.no_extras else 3)
    info = sc.scabem_op_info(op)
    ginfo = sc.scabem_op_grid_info(op)
    N = sc.scabem_mesh_info(mh)[2]
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)

    def rand_x(shape, dtype):
        z = torch.complex(torch.randn(shape, device="cuda", generator=gen), torch.randn(shape, device="cuda",
                                                                                      generator=gen))
        return (z / math.sqrt(2)).to(dtype).contiguous()

    def accuracy_of(o, precs):
        """The GPU operator against the oracle's dense operator (O1) on complete
        sampled rows: the discretisation error of the grid method."""
        if o1_rows is None:
            return None
        xo, ro, vo = o1_rows
        acc = {"rows": int(len(ro)), "reference": "oracle O1 (dense operator, direct matvec), same x",
               "meaning": "grid-method (pFFT) discretisation error at this stencil order and near radius"}
        for name, prec, dt in precs:
            xd = torch.as_tensor(xo).to(dt).cuda().contiguous()
            yd = torch.empty_like(xd)
            sc.scabem_apply(o, xd, yd, prec=prec, stream=stream)
            torch.cuda.synchronize()
            d = yd.cpu().numpy().astype(np.complex128)[ro] - vo
            acc["rel_l2_" + name] = float(np.linalg.norm(d) / np.linalg.norm(vo))
            acc["max_rel_" + name] = float(np.max(np.abs(d)) / np.max(np.abs(vo)))
        return acc

    precs = [("c64", sc.SCABEM_C64, torch.complex64)]
    if not args.no_extras:
        precs.append(("c128", sc.SCABEM_C128, torch.complex128))
    accuracy = accuracy_of(op, precs)
    x = rand_x((N,), torch.complex64)
    y = torch.empty_like(x)
    kb = max(1, args.batch)
    Xb = rand_x((kb, N), torch.complex64) if kb > 1 else x
    Yb = torch.empty_like(Xb)

    def step():
        sc.scabem_apply(op, Xb, Yb, nrhs=kb, ld=N, prec=sc.SCABEM_C64, stream=stream)

    ms = 0.0
    with Clocks(local) as clk:
        # keep the GPU loaded for about half a second before the timed region,
        # so that the clock samples describe the clocks under this load
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < args.load_seconds:
            for _ in range(50):
                step()
            torch.cuda.synchronize()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        sc.scabem_profile(op, True, max(args.steps, 1))
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    clocks = clk.summary("load, warm-up and timed applies (the timed region alone is too short for samples)")
    barrier(ws)
    stages, napp = sc.scabem_profile_read(op)
    sc.scabem_profile(op, False)
    ms_max = max_over_ranks(ms, ws, device=torch.device("cuda", local))
    value = ws * kb * args.steps / (ms_max / 1e3)

    # end to end through the C-ABI with pinned host buffers
    xh = Xb.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    sc.scabem_apply(op, xh, yh, nrhs=kb, ld=N, prec=sc.SCABEM_C64, stream=stream)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sc.scabem_apply(op, xh, yh, nrhs=kb, ld=N, prec=sc.SCABEM_C64, stream=stream)
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
    hbm, _ = peaks()
    if not args.no_extras:
        fp64_peak = sc.scabem_peak_fma(sc.SCABEM_C128, stream=stream)
        fp32x2_peak = sc.scabem_peak_fma(sc.SCABEM_C64, stream=stream)
        # FP64 operator, single right-hand side, with its stage times
        x2 = x.to(torch.complex128)
        y2 = torch.empty_like(x2)
        reps128 = max(3, args.steps // 20)
        sc.scabem_apply(op, x2, y2, prec=sc.SCABEM_C128, stream=stream)
        torch.cuda.synchronize()
        sc.scabem_profile(op, True, reps128)
        ms128 = timed(lambda: sc.scabem_apply(op, x2, y2, prec=sc.SCABEM_C128, stream=stream), reps128)
        st128, n128 = sc.scabem_profile_read(op)
        sc.scabem_profile(op, False)
        pts128_ms = st128["points"] / max(n128, 1)
        fl = points_flops(info, case)
        c128 = {"value": 1e3 / ms128, "unit": UNIT, "ms_per_step": ms128, "dtype": "c128",
                "stages_ms_per_step": {k: v / max(n128, 1) for k, v in st128.items()},
                "roofline": {"bound": "fp64_fma", "kernel": "points", "achieved": fl / (pts128_ms * 1e-3) / 1e12,
                             "peak": fp64_peak, "unit": "TFLOP/s", "frac": fl / (pts128_ms * 1e-3) / 1e12 / fp64_peak,
                             "flops_per_apply": fl, "peak_source": "measured (scabem_peak_fma: FP64 FMA chains)"}}
        # complex64, 8 and 32 right-hand sides in one call (column-major N x nrhs blocks)
        batched = {}
        for nb in (8, 32):
            X = rand_x((nb, N), torch.complex64)
            Y = torch.empty_like(X)
            sc.scabem_apply(op, X, Y, nrhs=nb, ld=N, prec=sc.SCABEM_C64, stream=stream)
            torch.cuda.synchronize()
            sc.scabem_profile(op, True, 5 * (nb // 8))
            msb = timed(lambda: sc.scabem_apply(op, X, Y, nrhs=nb, ld=N, prec=sc.SCABEM_C64, stream=stream), 5)
            stb, nbat = sc.scabem_profile_read(op)
            sc.scabem_profile(op, False)
            batched[f"nrhs{nb}"] = {"value": nb * 1e3 / msb, "unit": UNIT, "ms_per_call": msb,
                                    "vs_single_rhs": nb * 1e3 / msb / value,
                                    "stages_ms_per_8_columns": {k: v / max(nbat, 1) for k, v in stb.items()}}
            del X, Y
        # cuFFT on the full transform grid: the 12 forward and 16 inverse 3-D
        # transforms of an unpruned FFT convolution, as a comparison with the
        # pruned hand-written stages (axis-0 forward, (y, z) convolution, axis-0 inverse)
        Pd = tuple(2 * v for v in case.grid.n)
        F12 = rand_x((12,) + Pd, torch.complex64)
        F16 = rand_x((16,) + Pd, torch.complex64)
        ms_fft = timed(lambda: (torch.fft.fftn(F12, dim=(1, 2, 3)), torch.fft.ifftn(F16, dim=(1, 2, 3))), 5)
        del F12, F16
        own_fft = sum(stages[k] for k in ("fft_axis0_fwd", "fft_planes_green", "fft_axis0_inv")) / max(napp, 1)
        cufft = {"cufft_full_grid_ms": ms_fft, "hand_written_pruned_ms": own_fft,
                 "what": "torch.fft (cuFFT) fftn of 12 and ifftn of 16 fields of the 512x64x64 transform grid, "
                         "complex64; the hand-written stages transform only the covered columns and convolve in (y, z) "
                         "directly"}
        # the more accurate operator (near radius 3.05 grid steps) for solves and the reflection
        op2, t_setup2 = make_op(3.05 * case.grid.h, 3)
        acc2 = accuracy_of(op2, [("c64", sc.SCABEM_C64, torch.complex64)])
        xa = rand_x((N,), torch.complex64)
        ms_acc = timed(lambda: sc.scabem_apply(op2, xa, y, prec=sc.SCABEM_C64, stream=stream), max(3, args.steps // 10))
        # GMRES solve of one beam excitation: launched at x = 4.3 um (0.3 um past the left absorber)
        # along +x; the reflection of the right absorber (x > 8 um) is fitted from E_y on the axis over
        # x in [6.0, 7.8] um, 1.7 um or more from the source
        beam = dict(kind="beam", side="i", pos=(4.3, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.15)
        src = [sc.make_source(**beam)]
        bvec = torch.empty(N, dtype=torch.complex128, device="cuda")
        sc.scabem_rhs(op2, src, bvec, prec=sc.SCABEM_C128, stream=stream)
        xs = torch.zeros_like(bvec)
        sopt = dict(tol=1e-4, restart=200, maxit=20000, refine_tol=1e-8, max_refine=10, prec=sc.SCABEM_C64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sinfo = sc.scabem_solve(op2, bvec, xs, stream=stream, **sopt)[0]
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        refl = None
        try:
            rr = sc.scabem_reflection(op2, xs, 0, 1, (0.0, 0.01, -0.005), 6.0, 7.8, 64, 8.0, 13.0, 1001, inc=src[0],
                                      stream=stream)[0]
            ar = math.hypot(rr[0], rr[1])
            refl = {"abs_r": ar, "r": [rr[0], rr[1]], "beta_rad_per_um": rr[2], "fit_residual": rr[3], "swr": rr[4],
                    "r_from_swr": rr[5], "resolved": bool(rr[3] < 0.1 * ar),
                    "probe": "E_y at 64 axis points, x in [6.0, 7.8] um, beta scanned over [8, 13] rad/um",
                    "operator": "near radius 3.05 grid steps (accuracy_vs_dense below)",
                    "meaning": ("reflection of the right-hand absorber seen by a beam launched at x = 4.3 um; "
                                "resolved when the two-wave fit's residual is below a tenth of |r|")}
        except sc.ScabemError as e:
            refl = {"error": str(e)}
        # the same solve with the circulant preconditioners of Appendix B (Strang's and T. Chan's) on
        # the plain section's 100 regular slices (x in [4, 8] um: slices 100 .. 199 of 0.04 um),
        # each bounded to 6,000 iterations
        circ = {}
        for kind in ("strang", "chan"):
            try:
                t0 = time.perf_counter()
                sc.scabem_set_precond_circulant(op2, mh, axis=0, x0=0.0, dx=12.0 / 300, first=100, count=100,
                                                kind=kind, stream=stream)
                torch.cuda.synchronize()
                t_circ = time.perf_counter() - t0
                xc_ = torch.zeros_like(bvec)
                t0 = time.perf_counter()
                try:
                    cinfo = sc.scabem_solve(op2, bvec, xc_, stream=stream, **dict(sopt, maxit=6000))[0]
                    res = {"iterations": cinfo["iters"], "relres": cinfo["relres"], "status": cinfo["status"],
                           "solution_vs_block_diagonal": float((xc_ - xs).abs().norm() / xs.abs().norm())}
                except sc.ScabemError as e:
                    res = {"error": str(e), "maxit": 6000}
                finally:
                    sc.scabem_set_precond_circulant(op2, mh, count=0, stream=stream)
                torch.cuda.synchronize()
                circ[kind] = dict(res, setup_s=t_circ, seconds=time.perf_counter() - t0)
            except sc.ScabemError as e:
                circ[kind] = {"error": str(e)}
        circ["what"] = ("block circulant of the plain-surface block over slices 100-199 (192 unknowns each), "
                        "inverted by DFT over the slices; block-diagonal elsewhere; the same beam solve as 'solve'")
        # eight excitations in one call (2 polarisations x 4 launch points), batched GMRES in lockstep
        srcs8 = [sc.make_source("beam", "i", pos=(4.3 + 0.2 * k, 0.0, 0.0), dir=(1, 0, 0), pol=pol, b=0.15)
                 for pol in ((0, 1, 0), (0, 0, 1)) for k in range(4)]
        B8 = torch.empty((8, N), dtype=torch.complex128, device="cuda")
        sc.scabem_rhs(op2, srcs8, B8, ld=N, prec=sc.SCABEM_C128, stream=stream)
        X8 = torch.zeros_like(B8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info8 = sc.scabem_solve(op2, B8, X8, nrhs=8, ld=N, stream=stream, **sopt)
        torch.cuda.synchronize()
        t_solve8 = time.perf_counter() - t0
        solve = {"seconds": t_solve, "iterations": sinfo["iters"], "refinements": sinfo["refinements"],
                 "relres": sinfo["relres"], "status": sinfo["status"],
                 "rhs": "Gaussian beam (waist parameter 0.15 um) in the core at x = 4.3 um, y-polarised",
                 "operator": "near radius 3.05 grid steps", "matvec_per_s_c64": 1e3 / ms_acc,
                 "ms_per_iteration": t_solve * 1e3 / max(sinfo["iters"], 1),
                 "mode": ("GMRES(200) on the complex64 operator to 1e-4 with 48-bit Arnoldi (classical Gram-Schmidt "
                          "on FP32 (hi, lo) pairs, second pass by the DGKS test, Givens updates on the device), "
                          "FP64 refinement to 1e-8"),
                 "circulant_preconditioner": circ,
                 "nrhs8": {"seconds": t_solve8, "seconds_per_rhs": t_solve8 / 8,
                           "iterations": [i["iters"] for i in info8], "relres_max": max(i["relres"] for i in info8),
                           "status": [i["status"] for i in info8],
                           "rhs": "2 polarisations (y, z) x 4 launch points x = 4.3 .. 4.9 um",
                           "mode": "eight GMRES in lockstep sharing one batched operator apply per step"}}
        # transposed operator, adjoint solve and a conductivity gradient (16 B-spline coefficients)
        msa = timed(lambda: sc.scabem_apply_adjoint(op, x, y, prec=sc.SCABEM_C64, stream=stream),
                    max(3, args.steps // 10))
        g_rhs = torch.as_tensor(xs.cpu().numpy().conj()).cuda().contiguous()
        lam = torch.zeros_like(g_rhs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ainfo = sc.scabem_solve(op2, g_rhs, lam, stream=stream, transpose=True, **sopt)[0]
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        t0 = time.perf_counter()
        sc.scabem_sigma_gradient(op2, xs, lam, src, bspline=(0.0, 12.0, 0, 16), stream=stream)
        t_grad = time.perf_counter() - t0
        sc.scabem_op_destroy(op2)
        coupler = None if args.no_coupler else run_coupler(sc, torch, stream, timed, rand_x, hbm)
        extras = {
            "reflection": refl,
            "c128": c128,
            "batched_c64": batched,
            "fft_comparison": cufft,
            "peaks_measured": {"fp64_fma_tflops": fp64_peak, "fp32x2_fma_tflops": fp32x2_peak},
            "accurate_operator": {"r_near_h": 3.05, "setup_s": t_setup2, "matvec_per_s_c64": 1e3 / ms_acc,
                                  "accuracy_vs_dense": acc2},
            "solve": solve,
            "adjoint": {"matvec_per_s_c64": 1e3 / msa, "ms_per_step": msa,
                        "solve_seconds": t_adj, "solve_iterations": ainfo["iters"], "solve_relres": ainfo["relres"],
                        "sigma_gradient_seconds": t_grad,
                        "gradient": "d(lam^T (A x - b))/d coef for a 16-coefficient cubic B-spline over the guide"},
            "cpu_o2": o2,
            "coupler": coupler,
        }

    # roofline of the dominant kernel, and of the whole matvec
    _, src_peak = peaks()
    per = {k: v / max(napp, 1) for k, v in stages.items()}
    bmodel = stage_bytes(info, ginfo, case, N, 8, kb)
    dom = max(per, key=per.get)
    roof = None
    if dom in bmodel:
        ach = bmodel[dom] / (per[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": measured_traffic(dom, args.near_radius_h), "peak_source": src_peak,
                "algorithmic_bytes": bmodel[dom]}
    t_mv = ms_max / args.steps / 1e3 / kb  # per right-hand side
    b_pruned = sum(bmodel.values()) / kb
    b_full = full_grid_model_bytes(info, case, N, 8)
    mv_roof = {
        "pruned_bytes": b_pruned, "pruned_frac": b_pruned / t_mv / 1e9 / hbm,
        "full_grid_model_bytes": b_full, "full_grid_model_frac": b_full / t_mv / 1e9 / hbm,
        "peak": hbm, "unit": "GB/s",
    }
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
                       "parallelism": "replicas" if ws > 1 else "single GPU", "setup_s": t_setup,
                       "rhs_per_step": kb},
            "e2e": {"value": ws * kb * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(kb * N * 8),
                    "d2h_bytes_per_step": int(kb * N * 8)},
            "gpu_launches": 6 * ((kb + 7) // 8) * args.steps,
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


def run_coupler(sc, torch, stream, timed, rand_x, hbm):
    """Configuration 5: the two-guide directional coupler (128,440 triangles) on the 1024 x 256 x 256
    transform grid: set-up, complex64 matvec rates for one and eight right-hand sides, the point
    stage's roofline, and eight excitations (one beam per port pair and polarisation) solved in
    lockstep with a bounded iteration count."""
    import cases

    case = cases.coupler_full()
    m = case.mesh
    t0 = time.perf_counter()
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3, stream=stream)
    sc.scabem_set_sigma(op, segments=case.sigma_segments)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    info = sc.scabem_op_info(op)
    ginfo = sc.scabem_op_grid_info(op)
    N = sc.scabem_mesh_info(mh)[2]
    x = rand_x((N,), torch.complex64)
    y = torch.empty_like(x)
    sc.scabem_profile(op, True, 10)
    ms1 = timed(lambda: sc.scabem_apply(op, x, y, prec=sc.SCABEM_C64, stream=stream), 10)
    st, napp = sc.scabem_profile_read(op)
    sc.scabem_profile(op, False)
    pts_ms = st["points"] / max(napp, 1)
    bmodel = stage_bytes(info, ginfo, case, N, 8)
    X = rand_x((8, N), torch.complex64)
    Y = torch.empty_like(X)
    ms8 = timed(lambda: sc.scabem_apply(op, X, Y, nrhs=8, ld=N, prec=sc.SCABEM_C64, stream=stream), 3)
    del X, Y
    # eight excitations: beams launched inside either guide (y = -0.35 or 0.35 um) just past the left
    # absorber, y- or z-polarised, two waists
    srcs = [sc.make_source("beam", "i", pos=(4.3, yc, 0.0), dir=(1, 0, 0), pol=pol, b=bw)
            for yc in (-0.35, 0.35) for pol in ((0, 1, 0), (0, 0, 1)) for bw in (0.12, 0.15)]
    B = torch.empty((8, N), dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, srcs, B, ld=N, prec=sc.SCABEM_C128, stream=stream)
    Xs = torch.zeros_like(B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        sinfo = sc.scabem_solve(op, B, Xs, nrhs=8, ld=N, tol=1e-4, restart=100, maxit=1500, refine_tol=1e-8,
                                max_refine=3, prec=sc.SCABEM_C64, stream=stream)
        status = "converged"
    except sc.ScabemError as e:
        sinfo = None
        status = str(e)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    out = {"workload": "directional coupler: two 40 um guides, 0.2 um gap, 4 um absorbers at four ports",
           "triangles": int(m.nt), "unknowns": int(N), "fft_grid": "1024x256x256", "near_pairs": info["near_pairs"],
           "near_bytes_c64": info["near_bytes_c64"], "active_columns": ginfo["active_columns"],
           "transverse_direct": ginfo["transverse_direct"], "setup_s": t_setup,
           "matvec_per_s_c64": 1e3 / ms1, "ms_per_matvec_c64": ms1,
           "batched8": {"value": 8e3 / ms8, "unit": UNIT, "ms_per_call": ms8, "vs_single_rhs": ms1 * 8 / ms8},
           "points_roofline": {"bound": "hbm", "achieved": bmodel["points"] / (pts_ms * 1e-3) / 1e9, "peak": hbm,
                               "unit": "GB/s", "frac": bmodel["points"] / (pts_ms * 1e-3) / 1e9 / hbm,
                               "algorithmic_bytes": bmodel["points"], "stage_ms": pts_ms},
           "stages_ms_per_matvec": {k: v / max(napp, 1) for k, v in st.items()},
           "solve8": {"seconds": t_solve, "status": status, "maxit": 1500,
                      "iterations": [i["iters"] for i in sinfo] if sinfo else None,
                      "relres": [i["relres"] for i in sinfo] if sinfo else None,
                      "mode": "8 beams in lockstep, GMRES(100) on the complex64 operator with FP64 refinement, "
                              "bounded to 1,500 iterations"}}
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)
    torch.cuda.empty_cache()
    return out


def platform_info():
    import platform

    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"machine": platform.machine(), "cpu": model or platform.processor(), "nproc": os.cpu_count()}


def run_solve(args):
    """--mode solve: the GMRES iteration time on the 12 um guide.  The beam
    right-hand side is solved with the complex64 operator inside GMRES(100)
    (tol 1e-14, so that no column converges) for --solve-its and for three
    times as many iterations; the difference over 2 --solve-its iterations
    is the cost of one iteration without set-up.  The apply alone is timed
    beside it (200 back-to-back calls); their difference is the GMRES work.
    Rank 0 only (one GPU)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import cases
    import torch

    import paper_1004_5076_gb300 as sc
    from paper_1004_5076_gb300 import build

    build.build()
    case = cases.guide_full()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    r_near = args.near_radius_h * case.grid.h
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q, r_near, 3)
    sc.scabem_set_sigma(op, segments=case.sigma_segments)
    N = sc.scabem_mesh_info(mh)[2]
    src = [sc.make_source("beam", "i", pos=(4.3, 0, 0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.15)]
    b = torch.empty(N, dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, src, b, prec=sc.SCABEM_C128)
    x = torch.randn(N, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        sc.scabem_apply(op, x, y, prec=sc.SCABEM_C64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(200):
        sc.scabem_apply(op, x, y, prec=sc.SCABEM_C64)
    torch.cuda.synchronize()
    t_apply = (time.perf_counter() - t0) / 200

    def solve(its):
        xs = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.perf_counter()
        try:
            sc.scabem_solve(op, b, xs, tol=1e-14, restart=100, maxit=its, refine_tol=1e-14, max_refine=0,
                            prec=sc.SCABEM_C64)
        except sc.ScabemError:
            pass  # SCABEM_E_NOCONV: the iteration bound was the point
        torch.cuda.synchronize()
        return time.perf_counter() - t

    k = args.solve_its
    t1, t3 = solve(k), solve(3 * k)
    per_it = (t3 - t1) / (2 * k)
    line = {"metric": "GMRES iteration time (complex64 operator inside GMRES(100), beam right-hand side)",
            "value": per_it * 1e3, "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "c64",
            "data": "synthetic", "apply_ms": t_apply * 1e3, "gmres_work_ms": (per_it - t_apply) * 1e3,
            "iterations": [k, 3 * k], "seconds": [t1, t3],
            "config": {"workload": "guide_12um (as the matvec line)", "unknowns": int(N),
                       "r_near_h": args.near_radius_h, "restart": 100,
                       "basis_vectors": "0 .. 99 (mean about 50 over a cycle)"}}
    print(json.dumps(line), flush=True)
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import cases

    case = cases.guide_full()
    case.r_near = args.near_radius_h * case.grid.h
    per_step, samples = [], []
    nproc = 1
    for i in range(args.warmup + args.steps):
        rate, sample, nproc, el, _ = oracle_rate_allcores(case, args.ref_seconds)
        if i >= args.warmup:
            per_step.append(rate)
            samples.append(sample)
    value = float(np.mean(per_step))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "guide_12um (same as the GPU arm)", "triangles": int(case.mesh.nt)},
        "extrapolated": True,
        "step": (f"one bounded sample of about {args.ref_seconds:.0f} s of the oracle's direct matvec on "
                 f"{nproc} processes, extrapolated to a full matvec; value = mean rate over the {args.steps} samples"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": samples[-1],
                         "host": platform_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--mode", default="matvec", choices=["matvec", "solve"],
                    help="matvec: the benchmark line; solve: the GMRES iteration time on the same guide")
    ap.add_argument("--solve-its", type=int, default=200, help="--mode solve: iterations of the shorter solve")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--near-radius-h", type=float, default=2.05,
                    help="near-field radius in grid steps (2.05: the headline configuration)")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the c128, batched and solve measurements")
    ap.add_argument("--no-coupler", action="store_true", help="skip the directional-coupler measurements")
    ap.add_argument("--batch", type=int, default=1,
                    help="right-hand sides per timed step (one scabem_apply call of that many columns)")
    ap.add_argument("--load-seconds", type=float, default=0.5,
                    help="seconds of untimed applies before the warm-up (clock samples under load)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "solve":
        run_solve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
