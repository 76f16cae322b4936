"""Throughput of the PIE MLFMA matrix-vector product on one GB300 (or N replicas).

Workload: PEC sphere R = 1 m, icosahedral mesh subdivided 7 times
(327,680 triangles, 491,520 RWG functions, N = 819,200 unknowns -- the
"1M unknowns" point), kR = 1e-3, 7-level MLFMA (leaf box 1/32 m),
tau = 7, kappa a = 0.08, N_theta = 8 (P = 128).  One step = one product
y = Z x (all stages: coefficients, near part, aggregation, interpolation,
translations at levels 3..7, anterpolation, disaggregation, assembly) on a
complex-normal x (seed 1234) resident in HBM.  The headline `value` is the
MIXED form (near part complex float, far part complex double); the plain
FP64 form is reported beside it.  GMRES time to 1e-6 is reported for the
plain FP64 and MIXED solvers and for the nested solve (flexible GMRES on the
MIXED operator, inner GMRES cycles on the complex-float PIE_FP32H operator at
tau = 3, kappa a = 0.15, N_theta = 4).

cpu_baseline times the CPU FP64 oracle MLFMA on the host cores (products on
the 1280-triangle sphere, scaled to this workload by N x active levels);
--impl reference times the CPU FP64 oracle (the dense Galerkin product,
computed row by row) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="pec_sphere_icosphere7_1M", mesh="icosphere n=7, R=1 m", triangles=327680,
                rwg=491520, N=819200, kR=1e-3, levels=7, leaf_m=1.0 / 32, tau=7, kappa_a=0.08, ntheta=8, P=128,
                nrhs=1)
METRIC = "PIE MLFMA matvecs/s (1M unk)"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (vector and tensor), nominal; used only if the probe fails
FALLBACK_HBM_GBS = 6800.0
# DRAM read + write bytes per algorithmic flop of a stage's kernels, from one
# ncu capture (profiles/); valid while those kernels are unchanged.
# translation: k_trans<double>, one product at icosphere n=6 (levels 3..6),
# 74.84 MB for 1.3376e9 flop
NCU_BYTES_PER_FLOP = {"translation": 74.844416e6 / 1.33758976e9}
# inner operator of the nested solve and its settings
INNER = dict(tau=3, kappa_a=0.15, ntheta=4)
# (inner cycles of 20 steps to 0.05: shorter cycles were faster on some
# plane waves but took 5x more outer products on others, the count turning
# on the rounding of the far parts near the 1e-6 floor; the large sphere is
# allowed more outer products)
NESTED = dict(inner_restart=20, inner_tol=0.05, outer_restart=80, max_outer=1000, maxit=20000)
NESTED_LARGE = dict(inner_restart=20, inner_tol=0.05, outer_restart=80, max_outer=1500, maxit=30000)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=4, help="rows of the dense oracle product for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gmres", action="store_true", help="skip the GMRES time-to-tolerance measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 8-right-hand-side batched measurement")
    ap.add_argument("--no-multimesh", action="store_true",
                    help="skip the four-mesh, 64-right-hand-side group launch measurement")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch settings")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the nested solve on the 3,276,800-unknown sphere (icosphere n = 8, kR = 1e-4)")
    ap.add_argument("--gmres-tol", type=float, default=1e-6)
    ap.add_argument("--mesh-level", type=int, default=7,
                    help="icosphere subdivision n (L = n levels); 7 is the timed workload, smaller for profiling")
    ap.add_argument("--workload", default="1M", choices=["1M", "large", "inner", "cpu-oracle"],
                    help="large: the 3,276,800-unknown sphere (n = 8, kR = 1e-4), GMRES time to 1e-6 "
                         "in MIXED and FP64 and 8-right-hand-side product throughput; inner: products of the "
                         "nested solve's complex-float PIE_FP32H operator alone on the icosphere of --mesh-level "
                         "(for profiling); cpu-oracle: the CPU oracle alone on all host cores (no GPU): "
                         "GMRES time to 1e-6 on the 1280-triangle sphere at kR = 0.01 and products on the "
                         "1280- and 81,920-triangle spheres (several minutes)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region: the sampler is started and its first sample awaited before the
    region opens, and only samples taken between start() and stop() count."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.time(), line))

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return self
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        t = time.time()
        while not self.lines and time.time() - t < 5.0:
            time.sleep(0.02)
        return self

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.th.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = self.t0 if self.t0 is not None else -1e300
        t1 = self.t1 if self.t1 is not None else 1e300
        for ts, line in self.lines:
            if ts < t0 or ts > t1 + 0.1:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic(pr, stage, mixed):
    """(bound, amount, unit) of one launch group of a stage for one product."""
    P = pr.P
    L = pr.L
    T = pr.T
    c_far = 16  # far part is complex double in both forms
    if stage == "near":
        if mixed:
            # FP32 moments read once (8 complex64 per pair) + source coefficients + potentials
            return "hbm", pr.near_pairs * 64 + T * 6 * 16 * 2, "bytes"
        return "alu", pr.near_pairs * 12 * 8, "flops"
    if stage == "translation":
        nl = sum(len(pr.level(l)[2]) for l in range(3, L + 1))
        return "alu", nl * 5 * P * 8, "flops"
    if stage in ("interpolation", "anterpolation"):
        nc = sum(pr.boxes[l] for l in range(4, L + 1))
        return "alu", nc * 5 * P * P * 4, "flops"
    if stage in ("aggregation", "disaggregation"):
        return "alu", T * P * 8 * 8, "flops"
    return "hbm", pr.N * c_far * 2, "bytes"


def replica_max(v, world, device):
    """Largest value of v over the replicas (one process per GPU, each
    applying the whole operator to its own copy: no data exchange).  The
    timed region of a replica run is its slowest rank."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, ms_max):
    """Whole-job throughput: the units all replicas processed over the
    slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        return replica_max(v, world, "cuda")

    nlev = args.mesh_level
    xyz, tri = pi.icosphere(nlev)
    mesh = pg.Mesh(xyz, tri)
    k0 = 1e-3
    stream = torch.cuda.current_stream()
    try:  # FMA throughput of this GPU for the ALU-bound roofline
        probe = pg.measure_peaks()
    except pg.PieError:
        probe = None
    x_host = pi.complex_normal(mesh.nt + mesh.ne, 1234)
    results = {}
    for mode, prec in (("mixed", pg.PIE_MIXED), ("fp64", pg.PIE_FP64)):
        t0 = time.time()
        pr = pg.Problem(mesh, k0, nlev, root_side=2.0, precision=prec)
        setup_s = time.time() - t0
        tuning, tune_ms = (pr.tuning, None) if args.no_autotune else pr.autotune(nrhs=1, reps=5)
        x = torch.from_numpy(x_host).to(pr.torch_dtype).cuda()
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            pr.apply(x, y)
        torch.cuda.synchronize()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            clk.start()
            ev0.record(stream)
            for _ in range(args.steps):
                pr.apply(x, y)
            ev1.record(stream)
            torch.cuda.synchronize()
            clk.stop()
        barrier()
        ms = ev0.elapsed_time(ev1)
        ms_max = max_over_ranks(ms)
        # per-stage CUDA events (stages in order, near part not overlapped)
        pr.profile_begin(args.steps)
        for _ in range(args.steps):
            pr.apply(x, y)
        stage_ms, napplies = pr.profile_end()
        # end to end through the public API with host buffers
        xh = torch.from_numpy(x_host).to(pr.torch_dtype).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        xd = torch.empty_like(x)
        yd = torch.empty_like(x)
        for _ in range(2):
            xd.copy_(xh, non_blocking=True)
            pr.apply(xd, yd)
            yh.copy_(yd, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            xd.copy_(xh, non_blocking=True)
            pr.apply(xd, yd)
            yh.copy_(yd, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1))
        gm = nested = inner = None
        if not args.no_gmres:
            gm = gmres_run(pr, args.gmres_tol, k0, barrier, max_over_ranks)
            if mode == "mixed":
                nested, inner = nested_run(pg, mesh, nlev, pr, x_host, args.gmres_tol, k0, barrier,
                                           max_over_ranks, args.no_autotune)
        # coef, near, aggregation, interpolation (L-3), translation (L-2), anterpolation (L-3),
        # sum/difference patterns, disaggregation, assembly
        launches_per = 1 + 1 + 1 + (pr.L - 3) + (pr.L - 2) + (pr.L - 3) + 1 + 1 + 1
        results[mode] = dict(pr=pr, ms=ms_max, stage_ms=stage_ms, napplies=napplies, clocks=clk.summary(),
                             tuning=tuning,
                             e2e_ms=e2e_ms, setup_s=setup_s, launches=launches_per * args.steps,
                             bytes_io=x.numel() * x.element_size(), device_bytes=pr.device_bytes,
                             near_pairs=pr.near_pairs, gmres=gm, nested=nested, inner=inner)
        del x, y, xd, yd
    # batched right-hand sides: 8 columns per pass (MIXED)
    if not args.no_batched:
        nb = 8
        prb = pg.Problem(mesh, k0, nlev, root_side=2.0, precision=pg.PIE_MIXED, max_nrhs=nb)
        if not args.no_autotune:
            prb.autotune(nrhs=nb, reps=3)
        X = torch.from_numpy(np.stack([pi.complex_normal(mesh.nt + mesh.ne, 1234 + j) for j in range(nb)])).cuda()
        Y = torch.empty_like(X)
        for _ in range(args.warmup):
            prb.apply(X, Y)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            prb.apply(X, Y)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        results["batched"] = dict(nrhs=nb, ms=max_over_ranks(e0.elapsed_time(e1)), tuning=prb.tuning)
        del prb, X, Y
    if not args.no_multimesh:
        results["multimesh"] = multimesh_run(args, stream, barrier, max_over_ranks)
    if not args.no_large and not args.no_gmres and nlev == 7:
        results["large"] = large_nested_run(args, barrier, max_over_ranks)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    K = args.steps
    hbm, hbm_src = peaks()
    main = results["mixed"]
    pr = main["pr"]
    dom = max(main["stage_ms"], key=main["stage_ms"].get)
    bound, amount, unit = algorithmic(pr, dom, True)
    per_launch_ms = main["stage_ms"][dom] / max(1, main["napplies"])
    if bound == "hbm":
        achieved = amount / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": hbm_src, "algorithmic_bytes": amount, "traffic": None}
    else:
        achieved = amount / (per_launch_ms * 1e-3) / 1e12
        traffic = NCU_BYTES_PER_FLOP[dom] * amount if dom in NCU_BYTES_PER_FLOP else None
        # the probe's FP64 rate per SM clock, at the SM clock the timed step ran at
        sm_mhz = main["clocks"].get("sm_mhz") or 2070.0
        if probe and probe["fp64_mhz"] > 0:
            peak64 = probe["fp64_tflops"] * sm_mhz / probe["fp64_mhz"]
            src = (f"measured: FP64 FMA probe on this GPU (pie_measure_peaks), {probe['fp64_tflops']:.3f} TFLOP/s at "
                   f"{probe['fp64_mhz']:.0f} MHz, scaled to the {sm_mhz:.0f} MHz of the timed step")
        else:
            peak64, src = FP64_NOMINAL_TFLOPS, "nominal FP64"
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": achieved / peak64, "peak_source": src,
                "algorithmic_flops": amount, "traffic": traffic,
                "traffic_source": "ncu dram bytes per flop, scaled by flops (profiles/)" if traffic else None}
    stage_share = {k: round(v / sum(main["stage_ms"].values()), 4) for k, v in main["stage_ms"].items()}
    fp = results["fp64"]
    line = {
        "metric": METRIC,
        "value": replica_value(world, K, main["ms"]),
        "unit": "matvecs/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": main["ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 near + c128 far (mixed)",
        "data": "synthetic (icosphere mesh, seeded complex-normal x)",
        "config": dict(WORKLOAD if nlev == 7 else dict(workload=f"pec_sphere_icosphere{nlev}", N=pr.N, levels=pr.L),
                       precision="mixed", parallelism=f"replicas{world}",
                       l2="working set > L2 (near moments %.1f GB), no flush" % (main["near_pairs"] * 64 / 1e9)),
        "e2e": {"value": world * K / (main["e2e_ms"] * 1e-3), "unit": "matvecs/s",
                "h2d_bytes_per_step": main["bytes_io"], "d2h_bytes_per_step": main["bytes_io"]},
        "gpu_launches": main["launches"],
        "roofline": roof,
        "clocks": main["clocks"],
        "tuning": main["tuning"],
        "stage_ms_per_step": {k: round(v / K, 4) for k, v in main["stage_ms"].items()},
        "stage_share": stage_share,
        "setup_s": main["setup_s"],
        "device_bytes": main["device_bytes"],
        "multimesh": results.get("multimesh"),
        "batched8": ({"value": world * K * results["batched"]["nrhs"] / (results["batched"]["ms"] * 1e-3),
                      "unit": "matvecs/s", "nrhs": results["batched"]["nrhs"], "precision": "mixed",
                      "ms_per_batch": results["batched"]["ms"] / K, "tuning": results["batched"]["tuning"]}
                     if "batched" in results else None),
    }
    if not args.no_cpu_baseline and nlev == 7:
        line["cpu_baseline"] = cpu_baseline(args.cpu_rows)
    # the summaries the comparison rests on come last (the tail of the line)
    line["inner_fp32h"] = main["inner"]
    line["fp64"] = {"value": world * K / (fp["ms"] * 1e-3), "ms_per_step": fp["ms"] / K,
                    "e2e_value": world * K / (fp["e2e_ms"] * 1e-3),
                    "stage_ms_per_step": {k: round(v / K, 4) for k, v in fp["stage_ms"].items()}}
    line["peak_probe"] = probe
    line["gmres_fp64"] = fp["gmres"]
    line["gmres"] = main["gmres"]
    line["gmres_nested"] = main["nested"]
    line["large_nested"] = results.get("large")
    # one short record of the headline figures, last, so that it survives
    # wherever the line is cut
    def pick(d, *keys):
        for k in keys:
            d = d.get(k) if isinstance(d, dict) else None
        return d
    line["summary"] = {
        "matvecs_per_s_mixed": line["value"], "matvecs_per_s_mixed_e2e": line["e2e"]["value"],
        "matvecs_per_s_fp64": line["fp64"]["value"], "matvecs_per_s_fp64_e2e": line["fp64"]["e2e_value"],
        "matvecs_per_s_mixed_batched8": pick(line, "batched8", "value"),
        "matvecs_per_s_inner_fp32h": pick(line, "inner_fp32h", "matvecs_per_s"),
        "roofline_frac": roof["frac"], "roofline_kernel": roof["kernel"],
        "gmres_1e6_s_nested": pick(line, "gmres_nested", "seconds"),
        "gmres_1e6_s_nested_mean_4_waves": pick(line, "gmres_nested", "seconds_mean_4_waves"),
        "gmres_1e6_s_mixed": pick(line, "gmres", "seconds"), "gmres_1e6_s_fp64": pick(line, "gmres_fp64", "seconds"),
        "gmres_1e6_s_nested_3M": pick(line, "large_nested", "seconds"),
        "cpu_oracle_matvecs_per_s": pick(line, "cpu_baseline", "value")}
    print(json.dumps(line))


MULTIMESH = [  # name, mesh generator, root side (0 = bounding box), level range searched
    ("sphere", lambda pi: pi.icosphere(5), 2.0, (3, 6)),
    ("cube", lambda pi: pi.cube(32), 1.0, (3, 6)),
    ("ellipsoid_2_1_1", lambda pi: pi.octasphere(6, (1.0, 0.5, 0.5)), 0.0, (3, 7)),
    ("cylinder_capped", lambda pi: pi.cylinder(), 0.0, (3, 7)),
]


def multimesh_run(args, stream, barrier, max_over_ranks):
    """Four meshes of uneven size (20,480 to 40,960 triangles), kR = 1e-2,
    64 plane-wave right-hand sides each (32 directions on a uniform
    (theta, phi) grid x 2 polarisations), MIXED, in one group launch (one
    CUDA graph holding every member's product).  Level count and launch
    settings per mesh are chosen by the autotuner (set-up, untimed).  One
    step = one group launch = 4 x 64 products."""
    import numpy as np
    import torch

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi
    k0, nrhs = 1e-2, 64
    steps = min(args.steps, 20)  # one launch is 4 x 64 products (~0.15 s)
    waves = pi.planewave_set()
    members, info = [], []
    t0 = time.time()
    for name, gen, side, (lmin, lmax) in MULTIMESH:
        xyz, tri = gen(pi)
        mesh = pg.Mesh(xyz, tri)
        if args.no_autotune:
            L, lms = lmin + 1, {}
        else:
            # level search on 8-column products (per-column cost, smaller set-up)
            L, lms = pg.tune_levels(mesh, k0, lmin, lmax, nrhs=8, root_side=side, precision=pg.PIE_MIXED,
                                    max_nrhs=8)
        pr = pg.Problem(mesh, k0, L, root_side=side, precision=pg.PIE_MIXED, max_nrhs=nrhs)
        tuning = pr.tuning if args.no_autotune else pr.autotune(nrhs=nrhs, reps=3)[0]
        members.append(pr)
        info.append(dict(name=name, triangles=pr.T, N=pr.N, levels=L, ms_per_rhs_by_levels=lms, tuning=tuning))
    setup_s = time.time() - t0
    xs = [torch.stack([pr.rhs_planewave(kh, pol) for kh, pol in waves]) for pr in members]
    ys = [torch.empty_like(x) for x in xs]
    grp = pg.Group(members)
    for _ in range(args.warmup):
        grp.apply(xs, ys)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        grp.apply(xs, ys)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1)) / steps
    # the same products issued member after member on one stream, for contrast
    for pr, x, y in zip(members, xs, ys):
        pr.apply(x, y)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for pr, x, y in zip(members, xs, ys):
            pr.apply(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / steps
    g = grp.info()
    out = {"value": len(members) * nrhs / (ms * 1e-3), "unit": "matvecs/s (one mesh, one right-hand side each)",
           "unknown_matvecs_per_s": sum(m.N for m in members) * nrhs / (ms * 1e-3),
           "ms_per_launch": ms, "ms_member_by_member": seq_ms, "nrhs": nrhs, "kR": k0, "precision": "mixed",
           "graphs_captured": g["graphs"], "group_launches": g["launches"], "setup_and_tuning_s": setup_s,
           "meshes": info}
    del grp, xs, ys, members
    torch.cuda.empty_cache()
    return out


def large_nested_run(args, barrier, max_over_ranks):
    """The large sphere (icosphere n = 8: 1,310,720 triangles, N = 3,276,800,
    kR = 1e-4, 8 levels): nested solve to 1e-6 (MIXED outer operator,
    PIE_FP32H inner operator at INNER, settings NESTED_LARGE) for the x-polarised
    plane wave along -z, and the E-plane RCS of the solution against the
    Rayleigh limit.  Set-up untimed and reported; plain GMRES on this sphere
    runs under --workload large."""
    import torch

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi
    k0, n, L = 1e-4, 8, 8
    mesh = pg.Mesh(*pi.icosphere(n))
    t0 = time.time()
    po = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_MIXED)
    pin = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    setup_s = time.time() - t0
    if not args.no_autotune:
        po.autotune(nrhs=1, reps=3)
        pin.autotune(nrhs=1, reps=3)
    b = po.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    torch.cuda.synchronize()
    barrier()
    x, st = po.solve_nested(b, pin, tol=args.gmres_tol, **NESTED_LARGE)
    barrier()
    out = {"workload": "pec_sphere_icosphere8_3M", "N": po.N, "kR": k0, "levels": L, "tol": args.gmres_tol,
           "seconds": max_over_ranks(st["seconds"]), "converged": st["converged"], "rel_residual": st["rel_residual"],
           "inner_iterations": st["inner_iterations"], "outer_products": st["outer_products"],
           "inner_product_seconds": st["inner_product_seconds"], "outer_product_seconds": st["outer_product_seconds"],
           "rcs_max_db_err_vs_rayleigh": rcs_err_db(po, x, k0), "setup_s_both": setup_s,
           "device_bytes": po.device_bytes + pin.device_bytes, "settings": dict(NESTED_LARGE)}
    del po, pin, x, b
    torch.cuda.empty_cache()
    return out


def run_large(args):
    """Icosphere n = 8 (1,310,720 triangles, 1,966,080 RWG, N = 3,276,800),
    kR = 1e-4; level count by the autotuner among 8 and 9.  Per precision
    (MIXED, FP64): set-up time, product time (1 and 8 right-hand sides),
    GMRES(300) time to 1e-6 on the x-polarised plane wave along -z, and the
    E-plane RCS of the solution against the Rayleigh limit (exact to
    (kR)^2 = 1e-8)."""
    import numpy as np
    import torch

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    k0, n = 1e-4, 8
    steps = min(args.steps, 10)
    xyz, tri = pi.icosphere(n)
    mesh = pg.Mesh(xyz, tri)
    t0 = time.time()
    L, lms = pg.tune_levels(mesh, k0, 8, 9, nrhs=1, root_side=2.0, precision=pg.PIE_MIXED)
    tune_s = time.time() - t0
    out = {"metric": "PIE GMRES time to 1e-6 (3.3M unk)", "workload": "pec_sphere_icosphere8_3M", "N": mesh.nt + mesh.ne,
           "triangles": mesh.nt, "kR": k0, "levels": L, "ms_per_product_by_levels": lms, "level_search_s": tune_s}
    noop = lambda: None
    for mode, prec in (("mixed", pg.PIE_MIXED), ("fp64", pg.PIE_FP64)):
        nb = 8 if mode == "mixed" else 1
        t0 = time.time()
        pr = pg.Problem(mesh, k0, L, root_side=2.0, precision=prec, max_nrhs=nb)
        setup_s = time.time() - t0
        tuning, _ = pr.autotune(nrhs=nb, reps=3)
        X = torch.from_numpy(np.stack([pi.complex_normal(pr.N, 1234 + j) for j in range(nb)])).cuda()
        Y = torch.empty_like(X)
        res = {"setup_s": setup_s, "device_bytes": pr.device_bytes, "tuning": tuning}
        for cols in sorted({1, nb}):
            for _ in range(args.warmup):
                pr.apply(X[:cols], Y[:cols])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                pr.apply(X[:cols], Y[:cols])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            res[f"nrhs{cols}"] = {"ms_per_pass": ms, "matvecs_per_s": cols / (ms * 1e-3)}
        del X, Y
        res["gmres"] = gmres_run(pr, args.gmres_tol, k0, noop, lambda v: v)
        if mode == "mixed":
            pin = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
            pin.autotune(nrhs=1, reps=3)
            b = pr.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
            xs, st = pr.solve_nested(b, pin, tol=args.gmres_tol, **NESTED_LARGE)
            res["gmres_nested"] = {"seconds": st["seconds"], "converged": st["converged"],
                                   "inner_iterations": st["inner_iterations"],
                                   "outer_products": st["outer_products"],
                                   "rcs_max_db_err_vs_rayleigh": rcs_err_db(pr, xs, k0)}
            del pin
        out[mode] = res
        del pr
        torch.cuda.empty_cache()
    print(json.dumps(out))


def rayleigh_eplane(k0, R, cosg):
    """Bistatic E-plane RCS of a small PEC sphere (Rayleigh limit, relative
    error O((kR)^2)): 4 pi R^2 (kR)^4 (cos g - 1/2)^2."""
    return 4 * 3.141592653589793 * R * R * (k0 * R) ** 4 * (cosg - 0.5) ** 2


def gmres_run(pr, tol, k0, barrier, max_over_ranks):
    """GMRES(300) time to ||b - Z x|| <= tol ||b|| for the plane wave along -z,
    x-polarised, and the E-plane RCS of the solution against the Rayleigh
    limit (exact to ~(kR)^2 = 1e-6 at kR = 1e-3)."""
    import numpy as np
    import torch

    import pie_inputs as pi
    b = pr.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    torch.cuda.synchronize()
    barrier()
    x, st = pr.solve(b, tol=tol, maxit=3000, restart=300)
    barrier()
    rh = pi.bistatic_directions(181)
    E = pr.farfield(x, rh).cpu().numpy()
    s = 4 * np.pi * np.sum(np.abs(E) ** 2, axis=1)
    sm = rayleigh_eplane(k0, 1.0, -rh[:, 2])
    mask = sm > 1e-2 * sm.max()
    return {"tol": tol, "iterations": st["iterations"], "seconds": max_over_ranks(st["seconds"]),
            "product_seconds": st["product_seconds"], "reorthogonalizations": st["reorthogonalizations"],
            "rel_residual": st["rel_residual"], "converged": st["converged"], "restart": 300,
            "rcs_max_db_err_vs_rayleigh": float(np.max(np.abs(10 * np.log10(s[mask] / sm[mask]))))}


def rcs_err_db(pr, x, k0):
    """Largest |RCS - Rayleigh| in dB over the E-plane directions within 20 dB
    of the Rayleigh maximum (the null near 60 degrees is left out)."""
    import numpy as np

    import pie_inputs as pi
    rh = pi.bistatic_directions(181)
    E = pr.farfield(x, rh).cpu().numpy()
    s = 4 * np.pi * np.sum(np.abs(E) ** 2, axis=1)
    sm = rayleigh_eplane(k0, 1.0, -rh[:, 2])
    mask = sm > 1e-2 * sm.max()
    return float(np.max(np.abs(10 * np.log10(s[mask] / sm[mask]))))


def nested_run(pg, mesh, nlev, po, x_host, tol, k0, barrier, max_over_ranks, no_autotune):
    """Nested solve to ||b - Z x|| <= tol ||b|| (Z: the MIXED operator po) for
    the plane wave along -z, x-polarised: flexible GMRES on po, each outer
    step preconditioned by one GMRES cycle on the complex-float PIE_FP32H
    operator at INNER (set-up and autotuning untimed).  Also the inner
    operator's product time (1 and 8 right-hand sides per pass) and the HBM
    roofline of its near kernel."""
    import numpy as np
    import torch

    import pie_inputs as pi
    stream = torch.cuda.current_stream()
    pin = pg.Problem(mesh, k0, nlev, root_side=2.0, precision=pg.PIE_FP32H, max_nrhs=8, **INNER)
    if not no_autotune:
        pin.autotune(nrhs=1, reps=5)
    x = torch.from_numpy(x_host).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        pin.apply(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        pin.apply(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    pin.profile_begin(reps)
    for _ in range(reps):
        pin.apply(x, y)
    stage_ms, na = pin.profile_end()
    near_ms = stage_ms["near"] / max(1, na)
    # 8 right-hand sides per pass (launch settings tuned for 8 columns, then
    # restored): each pair's half moments are read once for several columns
    single = pin.tuning
    if not no_autotune:
        pin.autotune(nrhs=8, reps=5)
    else:
        pin.tuning = dict(single, rhs_chunk=8)
    batched_tuning = pin.tuning
    x8 = torch.from_numpy(np.stack([pi.complex_normal(pin.N, 77 + j) for j in range(8)])).to(torch.complex64).cuda()
    y8 = torch.empty_like(x8)
    for _ in range(3):
        pin.apply(x8, y8)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        pin.apply(x8, y8)
    e1.record(stream)
    torch.cuda.synchronize()
    ms8 = e0.elapsed_time(e1) / reps
    del x8, y8
    pin.tuning = single
    near_bytes = pin.near_pairs * 32 + pin.T * 6 * 8 * 2   # half moments once, float coefficients in, potentials out
    hbm, hbm_src = peaks()
    inner = {"point": dict(INNER), "precision": "fp32h", "ms_per_product": ms, "matvecs_per_s": 1e3 / ms,
             "stage_ms": {k: round(v / max(1, na), 4) for k, v in stage_ms.items()},
             "batched8": {"value": 8e3 / ms8, "unit": "matvecs/s", "ms_per_batch": ms8, "nrhs": 8,
                          "tuning": batched_tuning},
             "near_roofline": {"bound": "hbm", "achieved": near_bytes / (near_ms * 1e-3) / 1e9, "peak": hbm,
                               "unit": "GB/s", "frac": near_bytes / (near_ms * 1e-3) / 1e9 / hbm,
                               "peak_source": hbm_src, "algorithmic_bytes": near_bytes},
             "device_bytes": pin.device_bytes}
    b = po.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    torch.cuda.synchronize()
    barrier()
    xs, st = po.solve_nested(b, pin, tol=tol, **NESTED)
    barrier()
    # three more plane waves of the 64-wave set: near 1e-6 the iteration count
    # of this problem depends on the rounding of the far part, so a spread
    others = []
    waves = pi.planewave_set()
    for i in (5, 22, 41):
        _, so = po.solve_nested(po.rhs_planewave(*waves[i]), pin, tol=tol, **NESTED)
        others.append({"seconds": so["seconds"], "inner_iterations": so["inner_iterations"],
                       "outer_products": so["outer_products"], "converged": so["converged"]})
    nested = {"tol": tol, "seconds": max_over_ranks(st["seconds"]), "converged": st["converged"],
              "rel_residual": st["rel_residual"], "inner_iterations": st["inner_iterations"],
              "outer_iterations": st["outer_iterations"], "outer_products": st["outer_products"],
              "inner_product_seconds": st["inner_product_seconds"],
              "outer_product_seconds": st["outer_product_seconds"], "settings": dict(NESTED),
              "rcs_max_db_err_vs_rayleigh": rcs_err_db(po, xs, k0),
              "other_waves": others,
              "seconds_mean_4_waves": (st["seconds"] + sum(o["seconds"] for o in others)) / 4}
    del pin, x, y
    torch.cuda.empty_cache()
    return nested, inner


CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, ROOTDIR)
import numpy as np
import pie_inputs as pi
from oracle.dense import rows
from oracle.mesh import build_topology
from oracle.mlfma import MLFMA
out = {}
# oracle MLFMA on the 1280-triangle sphere (N = 3200), 3 levels
xyz, tri = pi.icosphere(3)
t0 = time.time()
M = MLFMA(xyz, tri, 1e-3, 3, side=2.0)
out["mlfma_setup_s"] = time.time() - t0
x = pi.complex_normal(M.top.N, 1234)
M.apply(x)
ts = []
c0, w0 = time.process_time(), time.time()
for _ in range(3):
    t0 = time.time()
    M.apply(x)
    ts.append(time.time() - t0)
# threads the products kept busy on average: process CPU time over wall time
out["mlfma_threads"] = (time.process_time() - c0) / max(time.time() - w0, 1e-9)
out["mlfma_mvm_s"] = float(np.median(ts))
out["mlfma_N"] = int(M.top.N)
# dense Galerkin rows of the 819,200-unknown sphere itself
xyz, tri = pi.icosphere(7)
top = build_topology(xyz, tri)
x = pi.complex_normal(top.N, 1234)
which = [0, top.E // 2, top.E + 5, top.N - 1][:NROWS]
rows(top, 1e-3, which[:1], x)          # warm-up (caches, page-in)
t0 = time.time()
rows(top, 1e-3, which, x)
out["rows"] = len(which)
out["rows_s"] = time.time() - t0
out["N"] = int(top.N)
print(json.dumps(out))
"""


CPU_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, ROOTDIR)
import numpy as np
import pie_inputs as pi
from oracle.dense import assemble
from oracle.excitation import rhs_planewave
from oracle.gmres import gmres
from oracle.mlfma import MLFMA
out = {}
# 1280-triangle sphere, kR = 0.01, L = 3: products and GMRES to 1e-6
xyz, tri = pi.icosphere(3)
t0 = time.time()
M = MLFMA(xyz, tri, 0.01, 3, side=2.0)
out["setup_s_1280"] = time.time() - t0
top = M.top
x = pi.complex_normal(top.N, 1234)
M.apply(x)
ts = []
c0, w0 = time.process_time(), time.time()
for _ in range(3):
    t0 = time.time()
    M.apply(x)
    ts.append(time.time() - t0)
out["mvm_threads_1280"] = (time.process_time() - c0) / max(time.time() - w0, 1e-9)
out["mvm_s_1280"] = float(np.median(ts))
# |Z_ii|^(-1/2) from the pairs of equal or edge-adjacent triangles, the
# scaling the GPU solver applies
t0 = time.time()
adj = [set([t]) for t in range(top.T)]
for n in range(top.E):
    a, b = int(top.edge_tri[n, 0]), int(top.edge_tri[n, 1])
    adj[a].add(b)
    adj[b].add(a)
Zp = assemble(top, 0.01, pair_mask=lambda t, s: np.array([int(q) in adj[int(p)] for p, q in zip(t, s)], bool))
D = 1.0 / np.sqrt(np.abs(np.diag(Zp)))
out["diag_s_1280"] = time.time() - t0
b = rhs_planewave(top, 0.01, np.array([0.0, 0.0, -1.0]), np.array([1.0, 0.0, 0.0]))
nprod = [0]
def op(v):
    nprod[0] += 1
    return D * M.apply(D * v)
t0, c0 = time.time(), time.process_time()
y, its, hist = gmres(op, D * b, tol=1e-6, restart=100, maxit=1500)
out["gmres_s_1280"] = time.time() - t0
out["gmres_threads_1280"] = (time.process_time() - c0) / max(out["gmres_s_1280"], 1e-9)
out["gmres_iterations_1280"] = int(its)
out["gmres_products_1280"] = nprod[0]
xs = D * y
out["gmres_true_rel_1280"] = float(np.linalg.norm(b - M.apply(xs)) / np.linalg.norm(b))
out["gmres_scaled_rel_1280"] = float(hist[-1])
out["N_1280"] = int(top.N)
if BIG:
    # 81,920-triangle sphere, kR = 1e-3, L = 6: set-up and one product
    xyz, tri = pi.icosphere(6)
    t0 = time.time()
    M = MLFMA(xyz, tri, 1e-3, 6, side=2.0)
    out["setup_s_81920"] = time.time() - t0
    x = pi.complex_normal(M.top.N, 1234)
    t0, c0 = time.time(), time.process_time()
    M.apply(x)
    out["mvm_s_81920"] = time.time() - t0
    out["mvm_threads_81920"] = (time.process_time() - c0) / max(out["mvm_s_81920"], 1e-9)
    out["N_81920"] = int(M.top.N)
print(json.dumps(out))
"""


def run_cpu_oracle(args):
    """The CPU FP64 oracle alone on all host cores (numpy with its BLAS on
    every core), for the small configurations the paper's method is first
    checked on: the 1280-triangle sphere at kR = 0.01 (3 levels; products,
    and GMRES(100) to 1e-6 on the system scaled by |Z_ii|^(-1/2), the GPU
    solver's scaling) and the 81,920-triangle sphere at kR = 1e-3 (6 levels;
    set-up and one product; left out with --mesh-level below 6).  One JSON
    line; no GPU work."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    ncpu = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(ncpu), OPENBLAS_NUM_THREADS=str(ncpu), MKL_NUM_THREADS=str(ncpu))
    code = CPU_ORACLE_SNIPPET.replace("ROOTDIR", repr(ROOT)).replace("BIG", str(args.mesh_level >= 6))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=5400)
    if out.returncode != 0:
        print(json.dumps({"workload": "cpu_oracle", "error": (out.stderr.strip().splitlines() or ["failed"])[-1]}))
        return
    d = json.loads(out.stdout.strip().splitlines()[-1])
    print(json.dumps({"workload": "cpu_oracle", "kind": "oracle MLFMA (numpy FP64)", "cores_available": ncpu,
                      "cpu_model": cpu_model(), **d}))


# One oracle process of the all-cores CPU leg: set up the 1280-triangle
# MLFMA, signal readiness, wait (bounded) until every process is ready, then
# time REPS products.  Single-threaded numpy per process.
CPU_WORKER = r"""
import json, os, sys, time
sys.path.insert(0, ROOTDIR)
import pie_inputs as pi
from oracle.mlfma import MLFMA
rank, n, d = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3]
xyz, tri = pi.icosphere(3)
M = MLFMA(xyz, tri, 1e-3, 3, side=2.0)
x = pi.complex_normal(M.top.N, 1234 + rank)
M.apply(x)
open(os.path.join(d, "ready%d" % rank), "w").close()
t_end = time.time() + 600
while sum(f.startswith("ready") for f in os.listdir(d)) < n and time.time() < t_end:
    time.sleep(0.01)
t0 = time.time()
for _ in range(REPS):
    M.apply(x)
print(json.dumps({"rank": rank, "seconds": time.time() - t0, "products": REPS}))
"""


def cpu_all_cores(ncpu, reps=10):
    """Oracle MLFMA products on every host core at once: ncpu independent
    single-threaded processes, each timing `reps` products of the
    1280-triangle sphere after all have set up.  Products per second of the
    whole host (total products over the slowest process's time), or None."""
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = CPU_WORKER.replace("ROOTDIR", repr(ROOT)).replace("REPS", str(int(reps)))
    with tempfile.TemporaryDirectory() as d:
        procs = [subprocess.Popen([sys.executable, "-c", code, str(r), str(ncpu), d], env=env,
                                  stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True) for r in range(ncpu)]
        res = []
        for p in procs:
            try:
                out, _ = p.communicate(timeout=900)
                res.append(json.loads(out.strip().splitlines()[-1]))
            except (subprocess.TimeoutExpired, ValueError, IndexError):
                p.kill()
                return None
    return sum(r["products"] for r in res) / max(r["seconds"] for r in res)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform_processor()


def platform_processor():
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(nrows):
    """The CPU FP64 oracle on all host cores: MLFMA products on the
    1280-triangle sphere (N = 3200, one translation level) in one
    single-threaded process per core at once (the numpy oracle keeps one
    thread busy), scaled to the 819,200-unknown, 5-translation-level
    workload by N x active levels (the O(N L) cost of the method, Section 4);
    beside it, one process alone and exact dense Galerkin rows of the
    workload itself."""
    ncpu = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(ncpu), OPENBLAS_NUM_THREADS=str(ncpu), MKL_NUM_THREADS=str(ncpu))
    code = CPU_SNIPPET.replace("ROOTDIR", repr(ROOT)).replace("NROWS", str(int(nrows)))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        return {"error": out.stderr.strip().splitlines()[-1] if out.stderr else "failed"}
    d = json.loads(out.stdout.strip().splitlines()[-1])
    scale = (WORKLOAD["N"] * (WORKLOAD["levels"] - 2)) / (d["mlfma_N"] * 1)
    one = 1.0 / (d["mlfma_mvm_s"] * scale)
    host = cpu_all_cores(ncpu)
    value, cores = (host / scale, ncpu) if host else (one, max(1, round(d["mlfma_threads"])))
    return {"value": value, "unit": "matvecs/s", "cores": cores, "cores_available": ncpu,
            "cpu_model": cpu_model(), "kind": "oracle MLFMA",
            "sample": (f"oracle MLFMA (numpy FP64) products on the 1280-triangle sphere (N = {d['mlfma_N']}, L = 3, "
                       f"one translation level), one single-threaded process per host core ({ncpu}), 10 products "
                       f"each after a common start: {host or 0:.1f} products/s for the host ({1 / d['mlfma_mvm_s']:.1f} "
                       f"for one process alone, {d['mlfma_setup_s']:.1f} s set-up); matvecs/s at N = 819,200, 5 "
                       f"translation levels = products/s / {scale:.0f}, the N x active-levels ratio"),
            "one_process": {"value": one, "threads_busy_avg": d["mlfma_threads"]},
            "mlfma_mvm_s_1280": d["mlfma_mvm_s"], "mlfma_setup_s_1280": d["mlfma_setup_s"],
            "dense_rows": {"value": d["rows"] / d["rows_s"] / d["N"], "unit": "matvecs/s",
                           "sample": f"{d['rows']} rows of the dense FP64 Galerkin product of this workload, "
                                     f"{d['rows_s']:.1f} s; matvecs/s = rows/s / N"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import pie_inputs as pi
    from oracle.dense import rows
    from oracle.mesh import build_topology
    xyz, tri = pi.icosphere(7)
    top = build_topology(xyz, tri)
    x = pi.complex_normal(top.N, 1234)
    rng = np.random.default_rng(0)
    # one step: an eighth of one row (the row's sum over a slice of the
    # source triangles), so that K steps stay within minutes
    parts = np.array_split(np.arange(top.T), 8)

    def step(i):
        rows(top, 1e-3, [int(rng.integers(top.N))], x, sources=parts[i % 8])

    for i in range(args.warmup):
        step(i)
    t0 = time.time()
    for i in range(args.steps):
        step(i)
    dt = time.time() - t0
    value = args.steps / 8 / dt / top.N
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic (icosphere mesh, seeded complex-normal x)", "config": dict(WORKLOAD, precision="fp64"),
        "cpu_baseline": {"value": value, "unit": "matvecs/s", "cores": 1, "kind": "oracle",
                         "sample": "one eighth of a row of the dense FP64 Galerkin product per step (the sum "
                                   "over a slice of the source triangles) on the same sphere; "
                                   "matvecs/s = rows/s / N"},
        "e2e": {"value": value, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_inner(args):
    """Products of the inner operator of the nested solve (PIE_FP32H at INNER,
    kR = 1e-3, L = n) on the icosphere of --mesh-level n: --warmup untimed,
    then --steps timed with CUDA events; one JSON line."""
    import torch

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.mesh_level
    mesh = pg.Mesh(*pi.icosphere(n))
    pin = pg.Problem(mesh, 1e-3, n, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    x = torch.from_numpy(pi.complex_normal(pin.N, 1234)).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        pin.apply(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pin.apply(x, y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"workload": f"inner_fp32h_icosphere{n}", "N": pin.N, "near_pairs": pin.near_pairs,
                      "ms_per_product": ms, "matvecs_per_s": 1e3 / ms, "point": INNER}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "large":
        run_large(a)
    elif a.workload == "inner":
        run_inner(a)
    elif a.workload == "cpu-oracle":
        run_cpu_oracle(a)
    else:
        run_ours(a)
