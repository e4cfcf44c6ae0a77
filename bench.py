"""Benchmark: MG-GCR solves per second to a true FP64 relative residual of 1e-10.

One step = the whole job for one gauge field: the adaptive setup at the
lightest mass (relaxation, group refinement, block orthonormalisation, Galerkin
coarse operator) followed by one MG-GCR solve at each mass of the sweep, the
setup being reused across masses.  Inputs (links, random starts, sources) are
resident on the device before the timed region; the `e2e` figure repeats the
step through the host-buffer C-ABI calls (links, starts and sources copied in,
solutions copied out, inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--prec fp32|fp64]

N > 1 (torchrun): every rank solves the same workload on its own GPU
(replicas: the method has no exchange step on one field); `value` = all
ranks' solves / max-over-ranks time.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1005_3043_gb300.workloads import WORKLOADS  # noqa: E402

DEFAULT_WORKLOAD = "wilson_16x16x16x32_nv20_beta6_5mass"
METRIC = "MG-GCR solves/sec to 1e-10 true residual"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="fp16", choices=["fp32", "fp16", "fp64"],
                    help="inner precision: fp16 = FP32 arithmetic with the coarse operator stored in FP16")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--quick", action="store_true", help="skip the other precision modes and the batch")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                f = [x.strip() for x in out.stdout.strip().split(",")]
                if len(f) >= 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_inputs(w):
    import synth
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed)
    plaq = synth.plaquette(U, w.dims)
    if np.isfinite(w.plaquette) and abs(plaq - w.plaquette) > 1e-10:
        raise RuntimeError(f"gauge field differs from the recorded one: plaquette {plaq!r} vs {w.plaquette!r}")
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    masses = w.masses()
    srcs = np.stack([synth.gaussian_spinor(w.dims, w.source_seed, stream=i) for i in range(len(masses))])
    return U, V0, srcs, masses, plaq


def batch_sources(w, n_gauss=4):
    """12 spin-colour point sources at the origin + n_gauss Gaussian sources."""
    import synth
    pts = [synth.point_source(w.dims, 0, s, c) for s in range(4) for c in range(3)]
    gs = [synth.gaussian_spinor(w.dims, w.source_seed, stream=100 + i) for i in range(n_gauss)]
    return np.stack(pts + gs)


def mg_params(w, prec):
    import paper_1005_3043_gb300 as wmg
    p = wmg.mg_default_params()
    for i in range(4):
        p.block[i] = w.block[i]
    p.nvec = w.nvec
    p.setup_group = 4          # Sec. IV: 10 relaxations, then groups of 4 prototypes,
    p.setup_iters = w.extra.get("setup_iters", 5)   # each refined by 5 truncated-MG iterations
    p.setup_init_relax = 10
    p.gcr_restart = 16
    p.tol = 1e-10
    p.max_outer = 4000
    p.smoother = w.extra.get("smoother", 0)                # 0: MR steps; 1: one GMRES(steps) application
    p.smoother_steps = w.extra.get("smoother_steps", 4)
    p.prec_inner = {"fp32": wmg.MG_FP32, "fp16": wmg.MG_FP16, "fp64": wmg.MG_FP64}[prec]
    p.delta = 0.0 if prec == "fp64" else 1e-4
    return p


def one_step_rate(wmg, torch, w, prec, U, dV0, dB, dX, masses, stream):
    """solves/s of one step (setup + one solve per mass) in another precision mode"""
    mg = wmg.WilsonMG(w.dims, mg_params(w, prec), stream=stream)
    mg.set_links(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mg.set_mass(w.setup_mass())
    mg.setup_device(dV0)
    iters = []
    for i, m in enumerate(masses):
        mg.set_mass(m)
        info = mg.solve_device(dB[i], dX[i])
        if info["status"] != 0:
            raise RuntimeError(f"{prec} solve failed at m={m}: {info}")
        iters.append(info["outer_iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    mg.close()
    ms = e0.elapsed_time(e1)
    return len(masses) / (ms / 1e3), ms, iters


def max_over_ranks(ms, device="cpu"):
    """The job's time is its slowest replica's: MAX of the per-rank times
    (identity when no process group is up)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: the units every rank processed / the max-over-ranks time."""
    return world * units_per_rank / (ms / 1e3)


def run_ours(args, w):
    import torch
    import paper_1005_3043_gb300 as wmg
    from paper_1005_3043_gb300 import build as wbuild

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wbuild.build()
    wmg.load()
    U, V0, srcs, masses, plaq = make_inputs(w)
    stream = torch.cuda.current_stream()
    mg = wmg.WilsonMG(w.dims, mg_params(w, args.prec), stream=stream)
    mg.set_links(U)
    dV0 = torch.from_numpy(V0.view(np.float64)).cuda()
    dB = torch.from_numpy(srcs.view(np.float64)).cuda()
    dX = torch.empty_like(dB)
    n_solve = len(masses)
    infos = []

    def step(record):
        mg.set_mass(w.setup_mass())
        mg.setup_device(dV0)
        for i, m in enumerate(masses):
            mg.set_mass(m)
            info = mg.solve_device(dB[i], dX[i])
            if record is not None:
                record.append(info)
            if info["status"] != 0:
                raise RuntimeError(f"solve failed at m={m}: {info}")

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(None)
    barrier()
    mg.profile_read()                       # reset the launch timer and the coarse counter
    mg.profile_enable(True)
    launches0 = wmg.mg_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(infos)
        ev1.record(stream)
        barrier()
    launches = wmg.mg_kernel_launches() - launches0
    prof, coarse_iters = mg.profile_read()
    mg.profile_enable(False)
    ms = max_over_ranks(ev0.elapsed_time(ev1), "cuda")
    ms_step = ms / args.steps
    value = job_rate(world, n_solve * args.steps, ms)

    # setup and solve phases of one more step, timed separately
    barrier()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    mg.set_mass(w.setup_mass())
    mg.setup_device(dV0)
    e1.record(stream)
    for i, m in enumerate(masses):
        mg.set_mass(m)
        mg.solve_device(dB[i], dX[i])
    e2.record(stream)
    torch.cuda.synchronize()
    setup_ms, solves_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)

    # end to end through the host-buffer C-ABI (copies inside the timed region)
    barrier()
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mg.set_links(U)
        mg.set_mass(w.setup_mass())
        mg.setup(V0)
        for i, m in enumerate(masses):
            mg.set_mass(m)
            x, info = mg.solve(srcs[i])
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = U.nbytes + V0.nbytes + srcs.nbytes
    d2h = srcs.nbytes

    # roofline of the kernel class with the most device time in the timed region
    real = 8 if args.prec == "fp64" else 4
    nc = 2 * w.nvec
    Vc = int(np.prod([d // b for d, b in zip(w.dims, w.block)]))
    V = int(np.prod(w.dims))
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    if dom == "coarse_solve":
        # per CG iteration: D_c read twice + 15 coarse-vector passes (minimum unique traffic)
        a_bytes = 2 * (2 if args.prec == "fp16" else real)   # one complex entry of D_c
        per_unit = 2 * 9 * nc * nc * Vc * a_bytes + 15 * Vc * nc * 2 * real
        total_bytes = coarse_iters * per_unit
        unit_desc = f"{coarse_iters:.0f} CG iterations x {per_unit} B"
    elif dom in ("dslash", "true_residual"):
        per_unit = V * (72 + 24 + 24) * (real if dom == "dslash" else 8)
        total_bytes = dom_n * per_unit
        unit_desc = f"{dom_n} launches x {per_unit} B"
    else:
        per_unit, total_bytes, unit_desc = None, None, "n/a"
    achieved = total_bytes / (dom_ms * 1e-3) / 1e9 if total_bytes else None
    # DRAM bytes per launch of the dominant kernel from one ncu capture of this
    # command (dram__bytes_read.sum + dram__bytes_write.sum); known only for the
    # kernel and workload that were captured
    traffic = {("wilson_16x16x16x32_nv20_beta6_5mass", "fp16", "coarse_solve"): 30.22e6 + 0.10e6}.get(
        (w.name, args.prec, dom))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    ds_prec = wmg.MG_FP64 if args.prec == "fp64" else wmg.MG_FP32
    ms_ds, bytes_ds = mg.time_dslash(ds_prec, 200)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    ms_dc, _ = mg.time_dslash_cold(flush.data_ptr(), flush.numel(), ds_prec, 50)
    del flush
    coarse_kernel = wmg.COARSE_KERNELS.get(mg.coarse_kernel(), "unknown")
    mg.close()

    # the other precision modes of the same step, and a batch of sources
    extra = {}
    if not args.quick:
        names = {"fp64": "plain_fp64", "fp32": "fp32_inner", "fp16": "fp16_storage"}
        for mode in ("fp64", "fp32", "fp16"):
            if mode == args.prec:
                continue
            r, msm, itm = one_step_rate(wmg, torch, w, mode, U, dV0, dB, dX, masses, stream)
            extra[names[mode]] = {"value": r, "ms_per_step": msm, "outer_iters": itm}
        if "plain_fp64" in extra:
            extra["vs_plain_fp64"] = value / world / extra["plain_fp64"]["value"]
        bsrc = batch_sources(w)
        mgb = wmg.WilsonMG(w.dims, mg_params(w, "fp32"), stream=stream)
        mgb.set_links(U)
        mgb.set_mass(w.setup_mass())
        mgb.setup_device(dV0)
        mgb.set_mass(masses[-1])
        dbb = torch.from_numpy(bsrc.view(np.float64)).cuda()
        dxb = torch.empty_like(dbb)
        mgb.solve_batched_device(dbb[:2], dxb[:2], 2)          # warm-up (graph capture, autotuner)
        eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eb0.record(stream)
        binfo = mgb.solve_batched_device(dbb, dxb, len(bsrc))
        eb1.record(stream)
        torch.cuda.synchronize()
        mgb.close()
        bms = eb0.elapsed_time(eb1)
        extra["batched"] = {"sources": len(bsrc), "mass": masses[-1], "solves_per_s": len(bsrc) / (bms / 1e3),
                            "ms": bms, "outer_iters": [b["outer_iters"] for b in binfo],
                            "max_true_rel_res": max(b["true_rel_res"] for b in binfo),
                            "status": sorted({b["status"] for b in binfo})}

    if rank == 0:
        iters = [i["outer_iters"] for i in infos[:n_solve]]
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32+f64", "fp16": "f16/f32+f64", "fp64": "f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": w.name, "lattice": "x".join(map(str, w.dims)), "nvec": w.nvec,
                       "block": "x".join(map(str, w.block)), "masses": masses, "solves_per_step": n_solve,
                       "step": "adaptive setup at the lightest mass + one MG-GCR solve per mass",
                       "l2": "working set > L2 (129 MB)", "parallelism": f"replicas{world}",
                       "plaquette": plaq, "prec_inner": args.prec},
            "outer_iters": iters, "true_rel_res": [i["true_rel_res"] for i in infos[:n_solve]],
            "setup_ms": setup_ms, "solves_ms": solves_ms, "solve_only_per_s": n_solve / (solves_ms / 1e3),
            "e2e": {"value": n_solve / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": {"coarse_solve": coarse_kernel, "dslash": "k_dslash",
                                    "true_residual": "k_dslash<double>"}.get(dom, dom),
                         "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1), "work": unit_desc,
                         "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()},
            "dslash_alone": {"ms": ms_dc, "GB/s": bytes_ds / (ms_dc * 1e-3) / 1e9,
                             "frac": bytes_ds / (ms_dc * 1e-3) / 1e9 / peak, "l2": "flushed before every launch",
                             "work": f"{V} sites x {(72 + 24 + 24) * (8 if args.prec == 'fp64' else 4)} B",
                             "back_to_back_ms": ms_ds},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        line.update(extra)
        if not args.no_baseline:
            line["cpu_baseline"] = cpu_baseline(w, U, srcs, masses, V0, oracle_iters(w, iters),
                                                mg_params(w, "fp64").setup_iters)
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def cpu_baseline(w, U, srcs, masses, V0, outer_iters, setup_iters, budget_s=25.0):
    """The FP64 CPU oracle on a bounded sample of the step, scaled to whole solves.

    Timed: one Wilson operator application, one block orthonormalisation and one
    Galerkin build from the random prototypes, and outer MG-GCR iterations at the
    heaviest mass until the budget is used.  Scaled: a solve costs its outer
    iteration count times the time of one outer iteration (the counts are the
    oracle's own, measured once per workload by tests/golden/make_oracle_iters.py;
    the GPU's counts where none are stored); the setup costs 10 MR relaxations of
    every prototype (two operator applications per step), Nv/4 groups x
    setup_iters x 4 truncated-cycle iterations (one outer iteration each) and
    1 + Nv/4 orthonormalisations and builds."""
    import oracle
    oracle.build()
    cores = os.cpu_count()
    t0 = time.perf_counter()
    oracle.dslash(U, srcs[0], masses[0], w.dims)
    t_d = time.perf_counter() - t0
    t0 = time.perf_counter()
    P, st = oracle.block_orthonormalize(V0, w.dims, w.block)
    t_ortho = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = oracle.coarse_build(U, P, masses[0], w.dims, w.block)
    t_build = time.perf_counter() - t0
    remaining = max(budget_s - t_ortho - t_build - t_d, 2.0)
    k = 1
    t_it = None
    while True:
        p = oracle.make_params(w.dims, w.block, nv=w.nvec, m=masses[0], tol=0.0, max_outer=k, gcr_restart=16,
                               smoother=w.extra.get("smoother", 0), mr_steps=w.extra.get("smoother_steps", 4))
        t1 = time.perf_counter()
        _, info = oracle.gcr_solve(p, U, P, A, srcs[0])
        dt = time.perf_counter() - t1
        t_it = dt / max(info["outer_iters"], 1)
        if dt * 2 > remaining or k >= 16:
            break
        k *= 2
    groups = w.nvec // 4
    n_builds = 1 + groups
    setup_s = 10 * w.nvec * 2 * t_d + groups * setup_iters * 4 * t_it + n_builds * (t_ortho + t_build)
    step_s = setup_s + t_it * sum(outer_iters)
    return {"value": len(masses) / step_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle (OpenMP, {cores} threads) timed on this workload: one operator application "
                       f"{t_d:.2f} s, block orthonormalisation {t_ortho:.2f} s, Galerkin build {t_build:.2f} s, "
                       f"{k} outer MG-GCR iterations ({t_it:.3f} s each); step = setup estimate {setup_s:.0f} s + "
                       f"{sum(outer_iters)} outer iterations ({list(outer_iters)} per mass)")}


def oracle_iters(w, fallback):
    """Outer iterations per mass of the oracle on this workload (stored), else the fallback."""
    it = w.extra.get("oracle_outer_iters")
    return list(it) if it else list(fallback)


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    U, V0, srcs, masses, plaq = make_inputs(w)
    iters = oracle_iters(w, [250] * len(masses))
    setup_iters = mg_params(w, "fp64").setup_iters
    t0 = time.perf_counter()
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(w, U, srcs, masses, V0, iters, setup_iters, budget_s=20.0)
    dt = time.perf_counter() - t0
    line = {"metric": METRIC, "value": cb["value"], "unit": "solves/s", "n_gpus": 0, "steps": args.steps,
            "warmup": 0, "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "lattice": "x".join(map(str, w.dims)), "nvec": w.nvec},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    if not np.isfinite(w.re_lambda_min_m0):
        raise SystemExit(f"workload {w.name} has no recorded mass yet")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
