"""Saliency throughput benchmark (voxels/s) of the GB300 CUDA path, with the FP64 CPU
oracle as the reference arm.

Default workload: the plain FP32 method on an F3-shaped synthetic volume
462 x 951 x 651 (time x crossline x inline, 286,024,662 voxels, 1.14 GB float32), local
cube L = 7, 26-neighbourhood, REFLECT boundary.  One step = one pass of the whole hot
path over the volume: spectral energies (fused local 3D DFT + projections + mean),
directional centre-surround, FP64 statistics and the normalised combination.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank processes its own copy of the workload (independent
volumes, no data-path collective; weak scaling); rank 0 prints one JSON line.
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

WORKLOADS = {
    # name: (shape, kind, seed)
    "f3": ((462, 951, 651), "f3", 1),
    "cube64": ((64, 64, 64), "basic", 0),
    "cube256": ((256, 256, 256), "basic", 2),
    "slab": ((462, 951, 160), "f3", 1),     # a profiling case: the F3 shape cut to 160 inlines
    "batch64": (None, "basic", 0),           # 64 volumes, every axis U[32, 192], seeds 0..63
}
STENCIL_NAMES = {"26": "26-neighbourhood", "line": "d x 1 lines along each axis (Sec. 2)",
                 "diag_tx": "d x 1 line along the t-x diagonal (Fig. 3)"}
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 sub-partitions x 32)
MUFU_PER_SM_CLK = 16             # square roots per SM and clock on the XU (MUFU) pipe

# DRAM bytes (read + write) of one spectral-energy launch, from one ncu capture of the same
# kernel build (dram__bytes_read.sum + dram__bytes_write.sum on the 462 x 951 x 160 slab,
# scaled to the full volume by the voxel count), keyed by (workload, L, precision).  Only
# the default tile shape; any other configuration reports null.
ENERGY_TRAFFIC = {
    ("f3", 7, "fp32"): (4.371e9, "profiles/traffic_slab_462x951x160_L7.md: "
                                 "(282.6 MB + 791.8 MB) on the slab x 4.0687"),
}


def algorithmic_flops_per_voxel(L: int, R: int = 4, BX: int = 8) -> float:
    """FP32 flops per voxel of the fused energy stage as the kernel's algorithm defines it (FMA = 2).

    Stage t on the real cube columns, once per voxel column (no halo recomputation).  Stage
    x on the mu >= 0 half over runs of BX outputs along x: output 0 by the +-k folded direct
    DFT, BX - 1 sliding updates (started in the phase of the direct output, so without a
    rotation).  Stage y per line over strips of R windows the same way, plus |F| = mul + add
    (or fma) + sqrt; 3 FMAs per (mu, |nu|, |omega|) weight group; final scale.
    """
    H = (L - 1) // 2
    real_pass = 5 * H + 4 * H * H                  # t stage, and the direct x output of mu = 0
    cplx_pass = 10 * H + 8 * H * H + 4 * H         # the direct x output of one mu > 0
    x_real = (real_pass + (BX - 1) * (2 + 4 * H)) / BX
    x_cplx = (cplx_pass + (BX - 1) * (5 + 16 * H)) / BX
    cline = 10 * H + 4 + H * (8 * H + 9) + (R - 1) * (9 + 25 * H)
    rline = 4 * H + H * (4 * H + 4) + (R - 1) * (2 + 12 * H)
    n_cl = H + H * (2 * H + 1)
    groups = H + H * (H + 1) + H * (H + 1) ** 2
    pair_adds = H * H * (H + 1)
    y = (n_cl * cline + rline) / R + 6 * groups + pair_adds
    return real_pass + (x_real + H * x_cplx) + y + 3


def lattice_size(n: int, s: int) -> int:
    return 1 if n <= 1 else (n - 2) // s + 2


def lattice_kernel_work(shape, L: int, s: int):
    """(FP32 flops on the FMA pipe, square roots) of one lattice-energy launch, counted from
    the kernel's own loops: per CTA of nj x nk lattice points and its RX x RY region, stage t
    once for every mu (real input, folded: L + 3h + 4h^2 per column); then for each
    mu = 0..h stage x at the lattice x (folded complex DFT of every nu: 8h^2 + 10h per column)
    and the folded stage y per (point, nu) line with |F|, the weights and the accumulation."""
    H = (L - 1) // 2
    BJ, BK = 8, 8
    while True:                                         # the launcher's block choice
        RXM, RYM = (BJ - 1) * s + L, (BK - 1) * s + L
        g1 = 2 * (H + 1) * RXM * RYM
        reg = (max(L * RXM * RYM, 2 * L * BJ * RYM) + 3) // 4 * 4
        need = 4 * (g1 + reg + 3 * BJ * BK * L)
        if (need <= 110 * 1024 and BJ * BK * L <= 1024 and BJ * RYM <= 512) or (BJ == 1 and BK == 1):
            break
        if BK >= BJ and BK > 1:
            BK //= 2
        else:
            BJ //= 2

    def blocks(n, B):
        nc = lattice_size(n, s)
        coord = lambda i: min(i * s, n - 1)
        sizes, regions = [], []
        for b0 in range(0, nc, B):
            nb = min(B, nc - b0)
            sizes.append(nb)
            regions.append(coord(b0 + nb - 1) - coord(b0) + 2 * H + 1)
        return np.array(sizes), np.array(regions)

    nj, RX = blocks(shape[1], BJ)
    nk, RY = blocks(shape[2], BK)
    if (L, s) in ((5, 2), (7, 2), (7, 3), (9, 2), (9, 3), (9, 4)):
        # compile-time geometry: every CTA works on its full block and region
        nj, RX = np.full(nj.size, BJ), np.full(nj.size, RXM)
        nk, RY = np.full(nk.size, BK), np.full(nk.size, RYM)
    Tc = lattice_size(shape[0], s)
    per_item = 8 * H * H + 23 * H + 15
    t_stage = (L + 3 * H + 4 * H * H) * RX.sum() * RY.sum()
    per_mu = (8 * H * H + 10 * H) * nj.sum() * RY.sum() + nj.sum() * nk.sum() * L * per_item
    flops = Tc * (t_stage + (H + 1) * per_mu + nj.sum() * nk.sum() * 3 * (L + 1))
    sqrts = Tc * (H + 1) * nj.sum() * nk.sum() * L * (1 + 2 * H)
    return float(flops - sqrts), float(sqrts)


def mufu_per_voxel(L: int) -> int:
    """Square roots (MUFU sqrt.approx) per voxel of the energy kernel: one per |F| of the half
    spectrum it forms, (L^3 - 1) / 2 (algorithmic_flops_per_voxel counts each as one flop)."""
    return (L ** 3 - 1) // 2


def measure_fma_rate(dev, stream, seconds: float = 1.0) -> dict:
    """Measured FP32 FMA rate of this GPU: the library's FMA-chain probe (scalar FFMA and
    packed f32x2 forms), 2048 threads per SM, timed with CUDA events on `stream` over about
    `seconds` with the SM clock sampled meanwhile.  TFLOP/s, FMA = 2 flops."""
    import torch

    from paper_1901_11095_gb300 import api

    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.empty(nsm * 2048, device=dev, dtype=torch.float32)
    iters = 1 << 15
    res = {"sms": nsm, "threads": out.numel(), "iters": iters}
    for packed in (False, True):
        api.sal_probe_fma_rate(out, iters, packed, stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = api.sal_probe_fma_rate(out, iters, packed, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        reps = max(1, int(seconds / 2 / max(e0.elapsed_time(e1) / 1e3, 1e-6)))
        with ClockSampler(dev.index) as clk:
            e0.record(stream)
            for _ in range(reps):
                api.sal_probe_fma_rate(out, iters, packed, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        res["packed" if packed else "scalar"] = {"tflops": flops / (ms / 1e3) / 1e12, "ms": ms, "reps": reps,
                                                 "clocks": clk.summary()}
    res["tflops"] = max(res["scalar"]["tflops"], res["packed"]["tflops"])
    return res


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx = [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, dist_mod, device) -> float:
    """The slowest rank's time: the job's step ends when its last rank ends (an all-reduce MAX
    of one FP64 value; `device` is the backend's device, a GPU for NCCL, the CPU for gloo)."""
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed (each rank its own, weak scaling)
    per second of the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(V: np.ndarray, L: int, target_s: float = 15.0):
    """Time the CPU oracle on a crop of the workload volume sized for about target_s seconds."""
    import oracle
    oracle.build()
    T, X, Y = V.shape
    cores = cpu_cores()
    probe = np.ascontiguousarray(V[:min(T, 32), :min(X, 16), :min(Y, 64)])
    t0 = time.perf_counter()
    oracle.saliency(probe, L=L, threads=cores)
    rate = probe.size / max(time.perf_counter() - t0, 1e-3)
    want = max(int(rate * target_s), 4096)
    ny = min(Y, 128)
    nx = max(1, min(X, want // (T * ny)))
    crop = np.ascontiguousarray(V[:, :nx, :ny])
    t0 = time.perf_counter()
    oracle.saliency(crop, L=L, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": crop.size / dt, "unit": "voxels/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, whole method on a {T}x{nx}x{ny} crop ({crop.size} voxels) of the "
                      f"workload volume, {dt:.1f} s, OpenMP over t"}, crop.shape, dt


def run_reference(args, rank: int, world: int) -> None:
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_1901_11095_gb300 import synth
    import oracle
    oracle.build()
    shape, kind, seed = WORKLOADS[args.workload]
    V = synth.make_volume(shape, seed=seed, kind=kind)
    cores = cpu_cores()
    T, X, Y = V.shape
    crop = np.ascontiguousarray(V[:, :min(X, 8), :min(Y, 64)])
    for _ in range(args.warmup):
        oracle.saliency(crop[:, :1, :], L=args.L, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.saliency(crop, L=args.L, threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = crop.size / (ms / 1e3)
    out = {"impl": "reference", "metric": "saliency voxels/s", "value": value, "unit": "voxels/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args),
           "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step: FP64 oracle on a {crop.shape[0]}x{crop.shape[1]}x{crop.shape[2]} "
                                      f"crop ({crop.size} voxels) of the workload volume"},
           "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_config(args) -> dict:
    if args.workload == "batch64":
        from paper_1901_11095_gb300 import synth
        shapes = synth.batch_shapes()
        nv = sum(a * b * c for a, b, c in shapes)
        return {"workload": f"plain method {args.precision.upper()}, 64 uneven synthetic volumes (axes U[32,192], "
                            f"seeds 0..63, {nv} voxels), local cube {args.L}, one persistent launch per stage in a "
                            f"library-captured CUDA graph, autotuned tile shape",
                "volumes": 64, "voxels": nv, "L": args.L, "precision": args.precision, "boundary": "reflect",
                "stencil": "26", "l2": "flush buffer (512 MB) written between steps"}
    shape = WORKLOADS[args.workload][0]
    stride = f", cubes at stride {args.stride} (E interpolated back)" if getattr(args, "stride", 1) > 1 else ""
    return {"workload": f"plain method {args.precision.upper()}, {'F3-shaped' if args.workload == 'f3' else 'synthetic'}"
                        f" volume {shape[0]}x{shape[1]}x{shape[2]}, local cube {args.L}, {STENCIL_NAMES[args.stencil]}{stride}",
            "stride": getattr(args, "stride", 1),
            "volume": list(shape), "L": args.L, "precision": args.precision, "boundary": "reflect",
            "stencil": args.stencil, "l2": "inputs larger than L2 (V 1.14 GB, E and S_m 3.4 GB each); no flush needed"
            if args.workload == "f3" else "flush buffer written between steps"}


def run_batch(args, rank: int, world: int) -> None:
    """64 uneven volumes as one graph replay per step (each stage one persistent launch)."""
    import torch
    import torch.distributed as dist

    from paper_1901_11095_gb300 import api, synth

    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    shapes = synth.batch_shapes()
    vols = [synth.make_volume(s, seed=i + 64 * rank) for i, s in enumerate(shapes)]
    Vs = [torch.from_numpy(v).to(dev) for v in vols]
    nvox = sum(v.size for v in vols)
    p = api.params(L=args.L, precision=args.precision)
    stream = torch.cuda.current_stream(dev)
    api.sal_autotune_clear()
    stats = torch.empty((len(Vs), 9), device=dev, dtype=torch.float64)
    g = api.SalGraph(Vs, p, stats=stats, stream=stream)
    choice = api.sal_autotune_query(args.L, p.precision, max(v.size for v in vols))
    flush = torch.empty(512 << 20, device=dev, dtype=torch.uint8)
    for _ in range(args.warmup):
        flush.zero_()
        g.launch(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            g.launch(stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)
    # end to end: host volumes in, host saliency maps out, through the public batched call
    Vh = [torch.from_numpy(v).pin_memory() for v in vols]
    Sh = [torch.empty(v.shape, dtype=torch.float32).pin_memory() for v in vols]
    ws = torch.empty(api.sal_batch_workspace_size([v.shape for v in vols], p), device=dev, dtype=torch.uint8)
    Ss = [torch.empty_like(V) for V in Vs]

    def e2e():
        for a, b in zip(Vs, Vh):
            a.copy_(b, non_blocking=True)
        api.sal_saliency_batched(Vs, p, Ss=Ss, stats=stats, ws=ws, stream=stream)
        for a, b in zip(Sh, Ss):
            a.copy_(b, non_blocking=True)

    e2e()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = max(1, min(args.steps, 5))
    e0.record(stream)
    for _ in range(n_e2e):
        e2e()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    g.close()
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    if rank != 0:
        return
    out = {"metric": "saliency voxels/s", "value": job_rate(world, nvox, ms), "unit": "voxels/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision], "data": "synthetic",
           "config": workload_config(args), "autotune_choice": choice,
           "e2e": {"value": job_rate(world, nvox, e2e_ms), "unit": "voxels/s", "h2d_bytes_per_step": 4 * nvox,
                   "d2h_bytes_per_step": 4 * nvox, "ms_per_step": e2e_ms},
           "gpu_launches": 4 * args.steps, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_sweep(args) -> None:
    """Precision sweep on a 256^3 volume: every precision at L = 5, 7, 9, 11, each a JSON line
    with its speed and its error against the whole-volume FP64 oracle, per component map
    (E_m and S_m, normwise) and for the final saliency map (normwise and relative L2)."""
    import torch

    import oracle
    from paper_1901_11095_gb300 import api, synth

    dev = torch.device("cuda:0")
    shape = (256, 256, 256)
    V_np = synth.make_volume(shape, seed=2)
    V = torch.from_numpy(V_np).to(dev)
    N = V_np.size
    stream = torch.cuda.current_stream(dev)
    cores = cpu_cores()

    def nerr(got, ref):
        return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))

    for L in (5, 7, 9, 11):
        t0 = time.perf_counter()
        S_ref, E_ref, Sm_ref, _ = oracle.saliency(V_np, L=L, threads=cores, full=True)
        oracle_s = time.perf_counter() - t0
        for prec in ("fp32", "tf32", "bf16"):
            p = api.params(L=L, precision=prec)
            E = torch.empty((3,) + shape, device=dev)
            ws = torch.empty(api.sal_workspace_size(api.dims_of(V), p), device=dev, dtype=torch.uint8)
            S = torch.empty_like(V)
            Sm, st = api.sal_directional_compare(api.sal_spectral_energy(V, p, E=E), p)
            for _ in range(2):
                api.sal_saliency(V, p, S=S, ws=ws)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            for _ in range(args.steps):
                api.sal_spectral_energy(V, p, E=E)
            e1.record(stream)
            for _ in range(args.steps):
                api.sal_saliency(V, p, S=S, ws=ws)
            e2.record(stream)
            torch.cuda.synchronize()
            api.sal_device_status()
            k1_ms = e0.elapsed_time(e1) / args.steps
            path_ms = e1.elapsed_time(e2) / args.steps
            err = {}
            Eh, Smh, Sh = E.double().cpu().numpy(), Sm.double().cpu().numpy(), S.double().cpu().numpy()
            for m, name in enumerate("txy"):
                err[f"E_{name}"] = nerr(Eh[m], E_ref[m])
                err[f"S_{name}"] = nerr(Smh[m], Sm_ref[m])
            err["S"] = nerr(Sh, S_ref)
            err["S_relL2"] = float(np.linalg.norm(Sh - S_ref) / np.linalg.norm(S_ref))
            print(json.dumps({"sweep": "precision", "volume": list(shape), "L": L, "precision": prec,
                              "voxels_per_s": N / (path_ms / 1e3), "ms_per_step": path_ms,
                              "spectral_energy_ms": k1_ms, "errors_vs_oracle": err,
                              "oracle": {"whole volume": True, "seconds": oracle_s, "cores": cores}}), flush=True)
            del E, Sm, S, ws


def run_surrogate(args) -> None:
    """The learned surrogate: trained on seeded 128^3 volumes labelled by the plain method,
    then inference on the F3-shaped volume with the per-block fallback (threshold 2e-2).
    Prints one JSON line: speed of the surrogate path and of the plain path, errors of the
    surrogate against the plain GPU method, fraction of blocks recomputed."""
    import torch

    from paper_1901_11095_gb300 import api, surrogate, synth

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    p = api.params(L=args.L)
    t0 = time.perf_counter()
    vols, labels = [], []
    for i in range(args.train_volumes):
        V = torch.from_numpy(synth.make_volume((128, 128, 128), seed=100 + i, kind="f3")).to(dev)
        vols.append(V)
        labels.append(api.sal_spectral_energy(V, p))
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    model = surrogate.Surrogate(dev, seed=0)
    t0 = time.perf_counter()
    hist = surrogate.train(model, vols, labels, steps=args.train_steps, crop=48, lr=args.train_lr,
                           lr_final=args.train_lr_final, seed=1,
                           log_every=max(1, args.train_steps // 20))
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0

    # held-out accuracy (volumes not trained on) against the plain method, next to the error on
    # training volumes and the untrained network's (the gain of training), and the fraction of
    # check blocks kept per threshold
    def rel_errs(m_, V_, E_):
        P = m_.forward(V_, training=True)
        return [float(torch.linalg.vector_norm((P[c] - E_[c]).double()) / torch.linalg.vector_norm(E_[c].double()))
                for c in range(3)]

    untrained = surrogate.Surrogate(dev, seed=0)
    held = [torch.from_numpy(synth.make_volume((128, 128, 128), seed=900 + i, kind="f3")).to(dev) for i in range(4)]
    held_E = [api.sal_spectral_energy(V, p) for V in held]
    accuracy = {"held_out_rel_l2": np.mean([rel_errs(model, V, E) for V, E in zip(held, held_E)], axis=0).tolist(),
                "train_rel_l2": np.mean([rel_errs(model, V, E) for V, E in zip(vols[:4], labels[:4])], axis=0).tolist(),
                "untrained_held_out_rel_l2": np.mean([rel_errs(untrained, V, E) for V, E in zip(held, held_E)],
                                                     axis=0).tolist()}
    kept = {}
    for thr in (2e-2, 5e-2, 1e-1, 2e-1, 5e-1):
        c_tr = model.infer(held[0], threshold=thr)[1].cpu().numpy()
        c_un = untrained.infer(held[0], threshold=thr)[1].cpu().numpy()
        kept[f"{thr:g}"] = {"trained": 1.0 - c_tr[0] / c_tr[1], "untrained": 1.0 - c_un[0] / c_un[1]}
    accuracy["blocks_kept_held_out"] = kept
    del vols, labels, held, held_E

    shape, kind, seed = WORKLOADS["f3"]
    V = torch.from_numpy(synth.make_volume(shape, seed=seed, kind=kind)).to(dev)
    N = V.numel()
    E_plain = api.sal_spectral_energy(V, p)
    Sm, st = api.sal_directional_compare(E_plain, p)
    S_plain = api.sal_combine(Sm, st, p)
    E = torch.empty_like(E_plain)
    S = torch.empty_like(V)
    dcs_ws = torch.empty(api.sal_dcs_workspace_size(api.dims_of(V), p), device=dev, dtype=torch.uint8)

    p_tc = api.params(L=args.L, precision="bf16")    # hidden layers on the tensor cores

    def surr_path(thr, pp=p):
        _, counts = model.infer(V, pp, threshold=thr, E=E)
        api.sal_directional_compare(E, p, Sm=Sm, stats=st, ws=dcs_ws)
        api.sal_combine(Sm, st, p, S=S)
        return counts

    def plain_path():
        api.sal_spectral_energy(V, p, E=E)
        api.sal_directional_compare(E, p, Sm=Sm, stats=st, ws=dcs_ws)
        api.sal_combine(Sm, st, p, S=S)

    out = {"impl": "surrogate", "metric": "saliency voxels/s", "unit": "voxels/s", "data": "synthetic",
           "config": {"workload": f"learned surrogate (5 x 3x3x3 conv, 24 channels, GELU, BF16 weights) trained on "
                                  f"{args.train_volumes} seeded 128^3 F3-kind volumes (3 faults, dome) labelled by "
                                  f"the plain FP32 method, "
                                  f"inference on the F3-shaped {shape[0]}x{shape[1]}x{shape[2]} volume, L={args.L}"},
           "training": {"volumes": args.train_volumes, "steps": args.train_steps, "crop": 48,
                        "seconds": t_train, "label_seconds": t_data, "loss_first": hist[0][1],
                        "loss_last": hist[-1][1], "lr": [args.train_lr, args.train_lr_final]},
           "accuracy": accuracy}
    for name, thr, pp in (("fallback_2e-2", 2e-2, p), ("surrogate_only", 1e30, p),
                          ("fallback_2e-2_tensor_cores", 2e-2, p_tc), ("surrogate_only_tensor_cores", 1e30, p_tc)):
        counts = surr_path(thr, pp)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            counts = surr_path(thr, pp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        errE = [float((E[m] - E_plain[m]).abs().max() / E_plain[m].abs().max()) for m in range(3)]
        errL2 = [float(torch.linalg.vector_norm((E[m] - E_plain[m]).double()) /
                       torch.linalg.vector_norm(E_plain[m].double())) for m in range(3)]
        errS = float(torch.linalg.vector_norm((S - S_plain).double()) / torch.linalg.vector_norm(S_plain.double()))
        out[name] = {"voxels_per_s": N / (ms / 1e3), "ms_per_step": ms, "E_err_vs_plain_normwise": errE,
                     "E_rel_l2_vs_plain": errL2,
                     "S_rel_l2_vs_plain": errS, "blocks_recomputed": int(counts[0]), "blocks": int(counts[1])}
    plain_path()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plain_path()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    out["plain_fp32"] = {"voxels_per_s": N / (ms / 1e3), "ms_per_step": ms}
    # the network alone (5 convolution layers, no check, no compare / combine)
    for name, pp in (("forward_cuda_cores", p), ("forward_tensor_cores", p_tc)):
        model.forward(V, E=E, p=pp)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            model.forward(V, E=E, p=pp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        macs = 27 * (1 * 24 + 3 * 24 * 24 + 24 * 3)
        out[name] = {"ms": ms, "voxels_per_s": N / (ms / 1e3), "macs_per_voxel": macs,
                     "tflops": 2 * macs * N / (ms / 1e3) / 1e12}
    api.sal_device_status()
    out["value"] = out["fallback_2e-2"]["voxels_per_s"]
    out["speedup_vs_plain"] = out["value"] / out["plain_fp32"]["voxels_per_s"]
    print(json.dumps(out), flush=True)


def run_surrogate_forward(args) -> None:
    """The surrogate network alone (seeded initial weights, no training) on an F3-kind volume of
    --surrogate-shape (default 128 x 128 x 256, a small, quick case for profiling the
    convolution kernels): milliseconds per forward on the CUDA cores and with layers 2..5 on
    the tensor cores."""
    import torch

    from paper_1901_11095_gb300 import api, surrogate, synth

    dev = torch.device("cuda:0")
    shape = tuple(int(v) for v in args.surrogate_shape.lower().split("x"))
    V = torch.from_numpy(synth.make_volume(shape, seed=0, kind="f3")).to(dev)
    model = surrogate.Surrogate(dev, seed=0)
    E = torch.empty((3,) + tuple(V.shape), device=dev, dtype=torch.float32)
    out = {"mode": "surrogate forward", "volume": list(V.shape), "steps": args.steps, "warmup": args.warmup}
    for name, prec in (("cuda_cores", "fp32"), ("tensor_cores", "bf16")):
        p = api.params(precision=prec)
        for _ in range(args.warmup):
            model.forward(V, E=E, p=p)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            model.forward(V, E=E, p=p)
        e1.record()
        torch.cuda.synchronize(dev)
        api.sal_device_status()
        out[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    print(json.dumps(out), flush=True)


def run_ours(args, rank: int, world: int) -> None:
    import torch
    import torch.distributed as dist

    from paper_1901_11095_gb300 import api, synth

    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    shape, kind, seed = WORKLOADS[args.workload]
    V_np = synth.make_volume(shape, seed=seed + rank, kind=kind)
    N = V_np.size
    p = api.params(L=args.L, precision=args.precision, stride=args.stride, stencil=args.stencil)
    V = torch.from_numpy(V_np).to(dev)
    E = torch.empty((3,) + shape, device=dev, dtype=torch.float32)
    lat = api.sal_lattice_dims(api.dims_of(V), p)
    Ec = torch.empty((3, lat.T, lat.X, lat.Y), device=dev, dtype=torch.float32) if args.stride > 1 else None
    Sm = torch.empty_like(E)
    S = torch.empty(shape, device=dev, dtype=torch.float32)
    stats = torch.empty(9, device=dev, dtype=torch.float64)
    dims = api.dims_of(V)
    ws_dcs = torch.empty(api.sal_dcs_workspace_size(dims, p), device=dev, dtype=torch.uint8)
    ws_all = torch.empty(api.sal_workspace_size(dims, p), device=dev, dtype=torch.uint8)
    stream = torch.cuda.current_stream(dev)
    flush = None if N * 4 > 256 << 20 else torch.empty(512 << 20, device=dev, dtype=torch.uint8)

    def step(ev=None):
        if flush is not None:
            flush.zero_()
        if ev is not None:
            ev[0].record(stream)
        if Ec is not None:          # coarse stride: lattice energies, then interpolation to every voxel
            api.sal_lattice_energy(V, p, Ec=Ec, stream=stream)
            api.sal_interpolate_lattice(Ec, shape, p, E=E, stream=stream)
        else:
            api.sal_spectral_energy(V, p, E=E, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        api.sal_directional_compare(E, p, Sm=Sm, stats=stats, ws=ws_dcs, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        api.sal_combine(Sm, stats, p, S=S, stream=stream)
        if ev is not None:
            ev[3].record(stream)

    # the measured FP32 FMA rate (denominator beside the derived peak), before the timed region
    fma_probe = measure_fma_rate(dev, stream) if args.precision == "fp32" and not args.no_fma_probe else None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        for i in range(args.steps):
            step(evs[i])
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    k1 = [e[0].elapsed_time(e[1]) for e in evs]
    k2 = [e[1].elapsed_time(e[2]) for e in evs]
    k4 = [e[2].elapsed_time(e[3]) for e in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][3])
    ms = total_ms / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)
    value = job_rate(world, N, ms)

    # end to end through the public C-ABI call on HOST buffers: sal_saliency_host copies the
    # pinned V in, runs the path and copies S back into pinned host memory; successive calls
    # overlap their copies with each other's kernels (double buffers in the workspace)
    Vh = torch.from_numpy(V_np).pin_memory()
    Shs = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    del ws_all                                # the host path keeps its own buffers in ws_host
    ws_host = torch.empty(api.sal_host_workspace_size(dims, p), device=dev, dtype=torch.uint8)
    e2e_calls = [0]

    def e2e_step():
        ev = torch.cuda.Event()
        api.sal_saliency_host(Vh, p, S_host=Shs[e2e_calls[0] % 2], stats=stats, ws=ws_host, stream=stream,
                              done_event=ev)
        e2e_calls[0] += 1
        return ev

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_e2e = max(1, args.steps)
    last = None
    for _ in range(n_e2e):
        last = e2e_step()
    stream.wait_event(last)                   # the timed region ends after the last copy of S
    e1.record(stream)
    torch.cuda.synchronize(dev)
    api.sal_host_release(ws_host)
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)

    # the other forms of the method on the same volume (BF16 and TF32 tensor-core y stage, cubes
    # at stride 3), each timed like the main step and compared with the FP32 path's E and S
    forms = {}
    if args.stride == 1 and args.precision == "fp32" and args.workload == "f3" and args.stencil == "26" and \
            not args.no_forms:
        E32 = E.clone()
        S32 = S.clone()
        lat3 = api.sal_lattice_dims(dims, api.params(L=args.L, stride=3))
        Ec3 = torch.empty((3, lat3.T, lat3.X, lat3.Y), device=dev, dtype=torch.float32)
        for name, pf in (("bf16", api.params(L=args.L, precision="bf16")),
                         ("tf32", api.params(L=args.L, precision="tf32")),
                         ("fp32_stride3", api.params(L=args.L, stride=3))):
            def fstep():
                if pf.stride > 1:
                    api.sal_lattice_energy(V, pf, Ec=Ec3, stream=stream)
                    api.sal_interpolate_lattice(Ec3, shape, pf, E=E, stream=stream)
                else:
                    api.sal_spectral_energy(V, pf, E=E, stream=stream)
                api.sal_directional_compare(E, pf, Sm=Sm, stats=stats, ws=ws_dcs, stream=stream)
                api.sal_combine(Sm, stats, pf, S=S, stream=stream)
            for _ in range(2):
                fstep()
            torch.cuda.synchronize(dev)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nf = max(3, min(args.steps, 10))
            f0.record(stream)
            for _ in range(nf):
                fstep()
            f1.record(stream)
            torch.cuda.synchronize(dev)
            api.sal_device_status()
            fms = f0.elapsed_time(f1) / nf
            e_err = [float((E[m] - E32[m]).abs().max() / E32[m].abs().max()) for m in range(3)]
            s_rel = float(torch.linalg.vector_norm((S - S32).double()) / torch.linalg.vector_norm(S32.double()))
            forms[name] = {"value": N / (fms / 1e3), "unit": "voxels/s", "ms_per_step": fms, "steps": nf,
                           "speedup_vs_fp32": ms / fms, "E_err_vs_fp32_normwise": e_err, "S_rel_l2_vs_fp32": s_rel}
        del E32, S32, Ec3

    if rank != 0:
        return
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 flops
    k1_ms = statistics.mean(k1)
    tile = api.sal_autotune_query(args.L, p.precision, N)     # the tile shape the launches used
    fpv = algorithmic_flops_per_voxel(args.L, BX=int(tile["bx"]))
    n_sqrt = mufu_per_voxel(args.L)
    fma_fpv = fpv - n_sqrt                                    # flops on the FMA pipe (sqrt excluded)
    n_mu = (args.L + 1) // 2
    direct_fpv = 2 * (args.L ** 2 + 4 * n_mu * args.L ** 2 * (1 + args.L) + 5 * n_mu * args.L ** 2)
    achieved = fma_fpv * N / (k1_ms / 1e3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    k2_gbs = 24 * N / (statistics.mean(k2) / 1e3) / 1e9
    k4_gbs = 16 * N / (statistics.mean(k4) / 1e3) / 1e9
    traffic = ENERGY_TRAFFIC.get((args.workload, args.L, args.precision))
    if args.stride > 1:
        lflops, lsqrt = lattice_kernel_work(shape, args.L, args.stride)
        mhz = clk.summary()["sm_mhz"] or sm_max
        roofline = {"bound": "alu", "kernel": f"lattice energies (cubes at stride {args.stride}) + trilinear "
                                              "interpolation back to every voxel",
                    "achieved": lflops / (k1_ms / 1e3) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": lflops / (k1_ms / 1e3) / 1e12 / alu_peak, "traffic": None, "traffic_source": None,
                    "peak_source": f"derived: {nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop/FMA x {sm_max:.0f} MHz",
                    "flops_per_launch": lflops, "lattice_points": int(lat.T * lat.X * lat.Y),
                    "xu": {"sqrt_per_launch": lsqrt, "frac": lsqrt / (k1_ms / 1e3) / (nsm * MUFU_PER_SM_CLK * mhz * 1e6)},
                    "note": "time of both launches (lattice energies and interpolation) against the lattice kernel's "
                            "own flops; the interpolation writes 12 B per voxel"}
    elif args.precision == "fp32":
        clk_sum = clk.summary()
        mhz = clk_sum["sm_mhz"] or sm_max
        xu_peak = nsm * MUFU_PER_SM_CLK * mhz * 1e6                  # square roots per second
        roofline = {"bound": "alu", "kernel": "spectral energy (fused local DFT, projections, mean)",
                    "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                    "traffic": traffic[0] if traffic else None,
                    "traffic_source": traffic[1] if traffic else None,
                    "peak_source": f"derived: {nsm} SMs (device properties) x {FP32_LANES_PER_SM} FP32 lanes x "
                                   f"2 flop/FMA x {sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json)",
                    "flops_per_voxel": fma_fpv,
                    "flops_note": "FP32 flops of the kernel's own algorithm on the FMA pipe (FMA = 2); the "
                                  f"{n_sqrt} square roots per voxel run on the XU pipe and are counted apart",
                    "tile": [tile["bt"], tile["bx"], tile["by"], tile["mode"]],
                    "xu": {"sqrt_per_voxel": n_sqrt, "achieved_per_s": n_sqrt * N / (k1_ms / 1e3),
                           "peak_per_s": xu_peak, "frac": n_sqrt * N / (k1_ms / 1e3) / xu_peak,
                           "peak_source": f"{nsm} SMs x {MUFU_PER_SM_CLK} per clock x {mhz:.0f} MHz "
                                          "(median SM clock sampled in the timed region)"},
                    # the same time against the operation count of the unfolded separable DFT
                    # (L^2 + 4 n_mu L^2 (1 + L) + 5 n_mu L^2 MACs per voxel): above 1, because the
                    # folding and the sliding recurrences do that method's work with fewer flops
                    "direct_method_flops_per_voxel": direct_fpv,
                    "direct_method_equivalent_tflops": direct_fpv * N / (k1_ms / 1e3) / 1e12,
                    "frac_direct_count": direct_fpv * N / (k1_ms / 1e3) / 1e12 / alu_peak}
        if fma_probe is not None:
            roofline["measured_fma_peak"] = fma_probe["tflops"]
            roofline["frac_of_measured_fma_peak"] = achieved / fma_probe["tflops"]
            roofline["measured_fma_probe"] = {
                "scalar_tflops": fma_probe["scalar"]["tflops"], "packed_tflops": fma_probe["packed"]["tflops"],
                "sm_mhz": fma_probe["packed"]["clocks"]["sm_mhz"],
                "how": f"sal_probe_fma_rate: {fma_probe['threads']} threads x {8} independent FMA chains x "
                       f"{fma_probe['iters']} steps, CUDA events, about 0.5 s per form"}
    else:
        # stage y as tensor-core products: the contraction it stands for is the length-L DFT of
        # every window of the n_mu L lines (4 n_mu L^3 real MACs per voxel), against the dense
        # peak of the operand type (BF16 measured; TF32 = BF16 x the nominal 1.1 / 2.25)
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        tc_peak = bf16 if args.precision == "bf16" else bf16 * 1.1 / 2.25
        tc_fpv = 2 * 4 * n_mu * args.L ** 3
        tc_achieved = tc_fpv * N / (k1_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "kernel": "spectral energy with stage y on tcgen05 "
                                                  f"({args.precision.upper()} operands, FP32 accumulation)",
                    "achieved": tc_achieved, "peak": tc_peak, "unit": "TFLOP/s", "frac": tc_achieved / tc_peak,
                    "traffic": None, "traffic_source": None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" +
                                   ("" if args.precision == "bf16" else " x 1.1 / 2.25 (nominal TF32 / BF16)"),
                    "flops_per_voxel": tc_fpv,
                    "note": "the CUDA-core part (stages t and x, |F| of every frequency, the weights) "
                            "bounds this kernel, not the products",
                    "fp32_algorithm_tflops": achieved}
    out = {
        "metric": "saliency voxels/s", "value": value, "unit": "voxels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision], "data": "synthetic",
        "config": workload_config(args),
        "roofline": roofline,
        "kernels_ms": {"spectral_energy": k1_ms, "directional_compare_and_stats": statistics.mean(k2),
                       "combine": statistics.mean(k4)},
        "hbm_stages": {"directional_compare_GBs": k2_gbs, "combine_GBs": k4_gbs, "peak_GBs": hbm,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)",
                       "bytes_per_voxel": {"directional_compare": 24, "combine": 16}},
        "e2e": {"value": job_rate(world, N, e2e_ms), "unit": "voxels/s", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * N, "ms_per_step": e2e_ms},
        "gpu_launches": (6 if args.stride > 1 else 5) * args.steps,
        "clocks": clk.summary(),
    }
    if forms:
        out["forms"] = forms
        out["forms_note"] = ("the same step with the y-stage DFT on the tensor cores (BF16, TF32 operands, FP32 "
                             "accumulation) and with cubes at stride 3 (E interpolated back); errors against this line's "
                             "FP32 E and S (the FP32 path is within 1e-4 of the FP64 oracle by the parity tests)")
    if not args.no_cpu_baseline:
        cb, _, _ = oracle_sample(V_np, args.L, target_s=args.cpu_seconds)
        out["cpu_baseline"] = cb
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="f3")
    ap.add_argument("--L", type=int, default=7)
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16"], default="fp32")
    ap.add_argument("--stride", type=int, default=1, help="cube stride (coarse-stride cubes, E interpolated back)")
    ap.add_argument("--stencil", choices=["26", "line", "diag_tx"], default="26", help="neighbourhood of Eq. 5")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fma-probe", action="store_true", help="skip the FP32 FMA-rate probe")
    ap.add_argument("--no-forms", action="store_true", help="skip the BF16 / TF32 / stride-3 forms")
    ap.add_argument("--fma-probe", action="store_true", help="only run the FP32 FMA-rate probe (one JSON line)")
    ap.add_argument("--sweep", action="store_true", help="precision sweep on 256^3 (several JSON lines)")
    ap.add_argument("--surrogate", action="store_true", help="train the learned surrogate and time its inference")
    ap.add_argument("--surrogate-forward", action="store_true",
                    help="time the surrogate network alone (seeded weights) on --surrogate-shape")
    ap.add_argument("--surrogate-shape", default="128x128x256", help="T x X x Y of --surrogate-forward")
    ap.add_argument("--train-volumes", type=int, default=200)
    ap.add_argument("--train-steps", type=int, default=60000)
    ap.add_argument("--train-lr", type=float, default=2e-3)
    ap.add_argument("--train-lr-final", type=float, default=2e-5)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    if args.fma_probe:
        import torch
        dev = torch.device("cuda:0")
        print(json.dumps({"mode": "fp32 fma rate", **measure_fma_rate(dev, torch.cuda.current_stream(dev), 2.0)}),
              flush=True)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.surrogate:
        run_surrogate(args)
        return
    if args.surrogate_forward:
        run_surrogate_forward(args)
        return
    (run_batch if args.workload == "batch64" else run_ours)(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
