"""Benchmark: MG-GCR solves per second to a true FP64 relative residual of 1e-10.

One step = the whole job for one gauge field: the adaptive setup at the
lightest mass (relaxation, group refinement, block orthonormalisation, Galerkin
coarse operator) followed by one MG-GCR solve at each mass of the sweep, the
setup being reused across masses.  Inputs (links, random starts, sources) are
resident on the device before the timed region; the `e2e` figure repeats the
step through the host-buffer C-ABI calls (links, starts and sources copied in
from pinned host memory, solutions copied out to it, inside the timed region).

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



def _load_workloads():
    """The workload table, loaded by file path: the reference arm must not
    import the CUDA package (nor map its library)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1005_3043_gb300", "workloads.py")
    spec = importlib.util.spec_from_file_location("_wmg_workloads", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["_wmg_workloads"] = mod
    spec.loader.exec_module(mod)
    return mod.WORKLOADS


WORKLOADS = _load_workloads()

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
    p.gcr_restart = w.extra.get("gcr_restart", 16)
    p.tol = 1e-10
    p.max_outer = 4000
    p.smoother = w.extra.get("smoother", 0)                # 0: MR steps; 1: one GMRES(steps) application
    p.smoother_steps = w.extra.get("smoother_steps", 4)
    p.prec_inner = {"fp32": wmg.MG_FP32, "fp16": wmg.MG_FP16, "fp64": wmg.MG_FP64}[prec]
    p.delta = 0.0 if prec == "fp64" else 1e-4
    return p


def one_step_rate(wmg, torch, w, prec, U, dV0, dB, dX, masses, stream):
    """solves/s of one step (setup + one solve per mass) in another precision
    mode, with the launch timer on the coarse solve only, as in the headline
    step; also the coarse CGNR's time per CG iteration in this mode"""
    mg = wmg.WilsonMG(w.dims, mg_params(w, prec), stream=stream)
    mg.set_links(U)
    mg.profile_read()
    mg.profile_classes(["coarse_solve"])
    mg.profile_enable(True)
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
    prof, coarse_iters = mg.profile_read()
    mg.profile_enable(False)
    kernel = wmg.COARSE_KERNELS.get(mg.coarse_kernel(), "unknown")
    mg.close()
    ms = e0.elapsed_time(e1)
    coarse = {"kernel": kernel, "cg_iterations": coarse_iters,
              "us_per_cg_iteration": 1e3 * prof["coarse_solve"][0] / coarse_iters if coarse_iters else None}
    return len(masses) / (ms / 1e3), ms, iters, coarse


def batched_leg(wmg, torch, stream, prec, name="wilson_24x24x24x64_nv24_beta6_76rhs", n_single=4):
    """Many right-hand sides on the 24^3 x 64 workload (Nv = 24, 48 coarse dof):
    12 spin-colour point sources at the origin + 64 Gaussian sources in one
    batched solve (lockstep flexible GCR(8), the coarse solve of all sources
    one CGLS on an RHS panel with the tensor-core stencil, its iterations
    replayed from a CUDA graph), against n_single of the same sources solved
    one at a time (the single-source path, on-chip or persistent coarse CG).
    Setup once at the workload's mass; both timed with CUDA events."""
    import synth
    w = WORKLOADS[name]
    U = synth.gauge_field(w.dims, beta=w.beta, sweeps=w.sweeps, n_or=w.n_or, seed=w.seed)
    plaq = synth.plaquette(U, w.dims)
    if abs(plaq - w.plaquette) > 1e-10:
        raise RuntimeError(f"{name}: plaquette {plaq!r} differs from the recorded {w.plaquette!r}")
    pts = [synth.point_source(w.dims, 0, sp, c) for sp in range(4) for c in range(3)]
    gs = [synth.gaussian_spinor(w.dims, w.source_seed, stream=200 + i) for i in range(w.extra["gaussian_sources"])]
    src = np.stack(pts + gs)
    del pts, gs
    V0 = synth.gaussian_vectors(w.dims, w.nvec, w.setup_seed)
    mg = wmg.WilsonMG(w.dims, mg_params(w, prec), stream=stream)
    mg.set_links(U)
    mg.set_mass(w.setup_mass())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mg.setup(V0)
    e1.record(stream)
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1)
    dB = torch.from_numpy(src.view(np.float64)).cuda()
    dX = torch.empty_like(dB)
    del src
    mg.solve_batched_device(dB[:2], dX[:2], 2)       # warm-up: workspace, graph capture, autotuner
    e0.record(stream)
    binfo = mg.solve_batched_device(dB, dX, dB.shape[0])
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1)
    # the tensor-core coarse stencil alone on a panel of this many columns
    tc_ms, tc_bytes, tc_flops = mg.time_coarse_batched(dB.shape[0], 20)
    pick = list(range(n_single // 2)) + list(range(12, 12 + n_single - n_single // 2))
    mg.solve_device(dB[0], dX[0])                   # warm-up of the single-source path
    e0.record(stream)
    sinfo = [mg.solve_device(dB[i], dX[i]) for i in pick]
    e1.record(stream)
    torch.cuda.synchronize()
    sms = e0.elapsed_time(e1)
    mg.close()
    del dB, dX
    n = len(binfo)
    out = {"workload": name, "lattice": "x".join(map(str, w.dims)), "nvec": w.nvec, "mass": w.setup_mass(),
           "plaquette": plaq, "sources": n, "gcr_restart": w.extra["gcr_restart"], "prec_inner": prec,
           "setup_ms": setup_ms, "batched_ms": bms, "batched_solves_per_s": n / (bms / 1e3),
           "batched_outer_iters": [b["outer_iters"] for b in binfo],
           "batched_max_true_rel_res": max(b["true_rel_res"] for b in binfo),
           "batched_status": sorted({b["status"] for b in binfo}),
           "single_sources": pick, "single_ms": sms, "single_solves_per_s": len(pick) / (sms / 1e3),
           "single_outer_iters": [i["outer_iters"] for i in sinfo],
           "single_max_true_rel_res": max(i["true_rel_res"] for i in sinfo)}
    out["batched_over_single"] = out["batched_solves_per_s"] / out["single_solves_per_s"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm, bf16 = peaks.get("hbm_gbs", 6800.0), peaks.get("bf16_tflops", 1900.0)
    out["tc_stencil"] = {"kernel": "k_coarse_apply_tc", "columns": n, "us": 1e3 * tc_ms,
                         "bytes": tc_bytes, "GB/s": tc_bytes / (tc_ms * 1e-3) / 1e9,
                         "hbm_frac": tc_bytes / (tc_ms * 1e-3) / 1e9 / hbm,
                         "useful_TFLOP/s": tc_flops / (tc_ms * 1e-3) / 1e12,
                         "tensor_frac": tc_flops / (tc_ms * 1e-3) / 1e12 / bf16,
                         "note": "bound by streaming the FP16 embedded operator (9 x (2Nv x 2)^2 halves per aggregate, "
                                 "larger than L2); useful flops exclude the padding of M to 128 and the hi/lo "
                                 "split; peaks of MEASURED_PEAKS.json (HBM copy, bf16 burst)"}
    return out


def coarse_tc_probe(nrhs=64, reps=20):
    """One small case of the tensor-core batched coarse stencil for a profiler:
    the 16^3 x 32 level after its setup, a panel of nrhs columns."""
    import torch
    import paper_1005_3043_gb300 as wmg
    wmg.load()
    w = WORKLOADS["wilson_16x16x16x32_nv20_beta6_5mass"]
    U, V0, srcs, masses, plaq = make_inputs(w)
    mg = wmg.WilsonMG(w.dims, mg_params(w, "fp16"), stream=torch.cuda.current_stream())
    mg.set_links(U)
    mg.set_mass(w.setup_mass())
    mg.setup(V0)
    ms, nb, fl = mg.time_coarse_batched(nrhs, reps)
    mg.close()
    print(json.dumps({"kernel": "k_coarse_apply_tc", "workload": w.name, "columns": nrhs, "us": 1e3 * ms,
                      "GB/s": nb / (ms * 1e-3) / 1e9, "useful_TFLOP/s": fl / (ms * 1e-3) / 1e12}), flush=True)


def three_level_leg(wmg, torch, w, U, dV0, dB, dX, masses, stream, prec, nv2=32, block2=(2, 2, 2, 2)):
    """The paper's favoured method (Sec. IV) on the same step: three levels (4^4
    then 2^4 aggregates, Nv2 = 32), the workload's GMRES post-smoother on the
    fine grid and GMRES(4) on level 1, two level-1 V-cycles per fine correction
    (the W-cycle), CG on the normal equations to 1e-3 on level 2; the step adds
    the level-2 setup (random level-1 starts, seeded) to the fine setup.  One
    warm-up step, one timed step (CUDA events)."""
    import synth
    p = mg_params(w, prec)
    p.levels, p.nvec2, p.smoother_steps1, p.cycles1 = 3, nv2, 4, 2
    for i in range(4):
        p.block2[i] = block2[i]
    Vc1 = int(np.prod([d // b for d, b in zip(w.dims, w.block)]))
    V2 = synth.gaussian(nv2 * Vc1 * 2 * w.nvec, w.setup_seed + 2, 0).reshape(nv2, Vc1, 2 * w.nvec)
    mg = wmg.WilsonMG(w.dims, p, stream=stream)
    mg.set_links(U)
    out = None
    for rep in range(2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        mg.set_mass(w.setup_mass())
        mg.setup_device(dV0)
        mg.setup_level2(V2)
        e1.record(stream)
        infos = []
        for i, m in enumerate(masses):
            mg.set_mass(m)
            info = mg.solve_device(dB[i], dX[i])
            if info["status"] != 0:
                raise RuntimeError(f"three-level solve failed at m={m}: {info}")
            infos.append(info)
        e2.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e2)
        out = {"levels": 3, "block2": "x".join(map(str, block2)), "nvec2": nv2, "smoother_steps1": 4, "cycles1": 2,
               "solves_per_s": len(masses) / (ms / 1e3), "ms_per_step": ms, "setup_ms": e0.elapsed_time(e1),
               "solves_ms": e1.elapsed_time(e2), "outer_iters": [i["outer_iters"] for i in infos],
               "level2_cg_iters": [i["coarse_iters"] for i in infos],
               "true_rel_res": [i["true_rel_res"] for i in infos]}
    mg.close()
    return out


def flops_mg(w, info):
    """Floating-point work of one MG-GCR solve, counted per fine site V and
    coarse site Vc: 1320 V per fine operator application, 144 nc^2 Vc per
    coarse CG iteration (D_c and D_c^dag, 9 complex nc x nc blocks each),
    96 Nv V per cycle for restriction and prolongation, and per cycle the
    Krylov vector work of the GMRES(k) smoother (k (k + 3) / 2 complex dots
    and updates over 12 V entries, 8 flops each) and of the flexible GCR
    (its average k / 2 + 2 dots and updates); reductions and scalars ignored."""
    V = int(np.prod(w.dims))
    nc = 2 * w.nvec
    Vc = V // int(np.prod(w.block))
    k = w.extra.get("smoother_steps", 4)
    cyc = info["outer_iters"]
    krylov = (k * (k + 3) / 2 + 16 / 2 + 2) * 2 * 8 * 12 * V
    return info["fine_matvecs"] * 1320.0 * V + info["coarse_iters"] * 144.0 * nc * nc * Vc + \
        cyc * (96.0 * w.nvec * V + krylov)


def learned_leg(wmg, torch, w, U, V0, src, stream, prec, members=(32, 33)):
    """The learned setup against the plain one on held-out fields of the
    network's ensemble (members 32 and 33 of the chain started from this
    workload's field; the network trained on members 0-31): per setup its
    device time, the outer iterations and time of one solve at the lightest
    mass, and the two-grid rate (MR(4) smoother, coarse solve to 1e-5).
    Variants: the plain Sec. IV schedule (10 relaxations, 5 refinement
    iterations), plain with 2 iterations, and the network's prototypes with 10
    relaxations + 2 iterations and with 2 iterations alone."""
    from paper_1005_3043_gb300 import learned_setup as ls
    if not os.path.exists(ls.WEIGHTS):
        return {"unavailable": "no trained weights"}
    base = mg_params(w, prec)
    mg = wmg.WilsonMG(w.dims, base, stream=stream)
    mg.nn_set_weights(wmg.nn_unflatten(np.load(ls.WEIGHTS)))
    eta = ls.starts(w, w.nvec, 9200)
    variants = (("plain", False, 10, 5), ("plain_r2", False, 10, 2), ("learned_relax_r2", True, 10, 2),
                ("learned_r2", True, 0, 2))
    out = {"fields": "held-out members %s of the training ensemble" % (list(members),), "mass": w.masses()[-1]}
    rows = {}
    for k, Uk in ls.ensemble(w, max(members) + 1):
        if k not in members:
            continue
        mg.set_links(Uk)
        for name, learned, relax, iters in variants:
            p = wmg.MgParams.from_buffer_copy(base)
            p.setup_init_relax, p.setup_iters = relax, iters
            mg.set_params(p)
            mg.set_mass(w.setup_mass())
            if learned:
                mg.setup_learned(eta, refine_iters=iters)
            else:
                mg.setup(V0)
            mg.set_mass(w.masses()[-1])
            x, info = mg.solve(src)
            rows.setdefault(name, []).append(
                {"member": k, "setup_ms": info["setup_ms"], "outer_iters": info["outer_iters"],
                 "solve_ms": info["solve_ms"], "true_rel_res": info["true_rel_res"],
                 "two_grid_rate": ls.two_grid_rate(wmg, mg, w)})
    mg.close()
    out.update(rows)
    return out


def eo_cg_leg(wmg, torch, w, U, dB, dX, masses, mg_infos, stream):
    """The comparison solver of Sec. IV (Fig. 1 and 2) on the same sources and
    masses: red-black preconditioned CG (FP32 iterations, FP64 reliable updates)
    to the same 1e-10, against the timed MG-GCR solves (FP16 mode, setup
    excluded as in the paper's Fig. 1).  Wilson products: every Dhat or
    Dhat^dag counts one (the fine work of Fig. 1); flops: 1320 V per product
    plus the CG's vector work (about 170 V per iteration) against flops_mg."""
    V = int(np.prod(w.dims))
    mg = wmg.WilsonMG(w.dims, mg_params(w, "fp32"), stream=stream)
    mg.set_links(U)
    out = {"solver": "red-black CG on the normal equations, FP32 iterations, FP64 reliable updates",
           "iters": [], "products": [], "ms": [], "true_rel_res": []}
    for i, m in enumerate(masses):
        mg.set_mass(m)
        info = mg.solve_eo_cg_device(dB[i], dX[i], tol=1e-10, maxit=500000, prec=wmg.MG_FP32)
        if info["status"] != 0:
            raise RuntimeError(f"red-black CG failed at m={m}: {info}")
        out["iters"].append(info["outer_iters"])
        out["products"].append(info["fine_matvecs"])
        out["ms"].append(info["solve_ms"])
        out["true_rel_res"].append(info["true_rel_res"])
    mg.close()
    out["mg_products"] = [i["fine_matvecs"] for i in mg_infos]
    out["mg_solve_ms"] = [i["solve_ms"] for i in mg_infos]
    out["matvec_ratio"] = [a / b for a, b in zip(out["products"], out["mg_products"])]
    out["time_ratio"] = [a / b for a, b in zip(out["ms"], out["mg_solve_ms"])]
    cg_fl = [p * 1320.0 * V + it * 170.0 * V for p, it in zip(out["products"], out["iters"])]
    out["flop_ratio"] = [a / flops_mg(w, i) for a, i in zip(cg_fl, mg_infos)]
    return out


def dslash_beyond_l2(wmg, torch, stream, peak):
    """The fine operator on a 24^3 x 64 lattice (hot-start links: the bandwidth
    does not depend on them): FP32 (480 B per site, 425 MB per application) and
    FP16 storage (264 B per site).  `frac` is timed back to back: the 425 MB
    working set is 3.3x the L2, so every launch reads it from HBM (inputs larger
    than L2); `flushed_*` with a 512 MB buffer written before every launch (that
    launch also pays the write-back of the flush's dirty lines)."""
    import synth
    L = (24, 24, 24, 64)
    U = synth.hot_gauge(L, 9)
    p = wmg.mg_default_params()
    p.nvec, p.setup_group = 2, 2
    mg = wmg.WilsonMG(L, p, stream=stream)
    mg.set_links(U)
    mg.set_mass(-0.5)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {"lattice": "24x24x24x64", "l2": "inputs larger than L2 (3.3x), back to back; flushed_*: a 512 MB "
                                             "buffer written before every launch", "peak_GBps": peak}
    for name, prec in (("fp32", wmg.MG_FP32), ("fp16", wmg.MG_FP16)):
        ms, nbytes = mg.time_dslash_cold(flush.data_ptr(), flush.numel(), prec, 50)
        ms2, _ = mg.time_dslash(prec, 200)
        gbs, gbs2 = nbytes / (ms * 1e-3) / 1e9, nbytes / (ms2 * 1e-3) / 1e9
        out[name] = {"us": 1e3 * ms2, "bytes": nbytes, "GB/s": gbs2, "frac": gbs2 / peak,
                     "flushed_us": 1e3 * ms, "flushed_GB/s": gbs, "flushed_frac": gbs / peak}
    del flush
    mg.close()
    return out


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
    # device time per kernel class from one profiled step outside the timed
    # region; the timed steps track only the class with the most device time
    # (its launch durations give the roofline), the others run without events
    mg.profile_read()                       # reset the launch timer and the coarse counter
    mg.profile_enable(True)
    step(None)
    barrier()
    prof_all, _ = mg.profile_read()
    dom = max(prof_all, key=lambda k: prof_all[k][0])
    mg.profile_classes([dom])
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
    mg.profile_classes(wmg.KERNEL_CLASSES)
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

    # end to end through the host-buffer C-ABI (copies inside the timed region),
    # the inputs and the solutions in pinned host memory
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
        t.numpy()[...] = a
        return t
    hU, hV0, hB = pinned(U), pinned(V0), pinned(srcs)
    hX = torch.empty(srcs.shape, dtype=torch.complex128, pin_memory=True)
    barrier()
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mg.set_links(hU.numpy())
        mg.set_mass(w.setup_mass())
        mg.setup(hV0.numpy())
        for i, m in enumerate(masses):
            mg.set_mass(m)
            x, info = mg.solve(hB.numpy()[i], out=hX.numpy()[i])
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = U.nbytes + V0.nbytes + srcs.nbytes
    d2h = srcs.nbytes

    # roofline of the kernel class with the most device time in the timed region
    real = 8 if args.prec == "fp64" else 4
    nc = 2 * w.nvec
    Vc = int(np.prod([d // b for d, b in zip(w.dims, w.block)]))
    V = int(np.prod(w.dims))
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
    traffic = {("wilson_16x16x16x32_nv20_beta6_5mass", "fp16", "coarse_solve"): 30.16e6 + 0.09e6}.get(
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
    latency = None
    if dom == "coarse_solve" and args.prec != "fp64" and coarse_iters > 0:
        # the on-chip coarse CG's floor: its two tagged stencils alone and its
        # exchange alone, on the same operator and launch shape
        try:
            us_st, us_x = mg.time_coarse_floor(500)
        except wmg.MGError as e:   # no on-chip shape for this operator: no floor to report
            us_st = us_x = None
            latency = {"unavailable": str(e)}
    if latency is None and dom == "coarse_solve" and args.prec != "fp64" and coarse_iters > 0:
        us_it = dom_ms * 1e3 / coarse_iters
        latency = {"us_per_cg_iteration": us_it, "us_two_stencils_only": us_st, "us_exchange_only": us_x,
                   "floor_frac": us_st / us_it,
                   "note": "operator resident on chip: the iteration is bound by the latency of its two "
                           "stencils (tagged neighbour staging, products, emission); the exchange overlaps "
                           "the second stencil; floor_frac = stencils-only time / time per CG iteration"}
    mg.close()

    # the other precision modes of the same step, and a batch of sources
    extra = {}
    if not args.quick:
        names = {"fp64": "plain_fp64", "fp32": "fp32_inner", "fp16": "fp16_storage"}
        for mode in ("fp64", "fp32", "fp16"):
            if mode == args.prec:
                continue
            r, msm, itm, cg = one_step_rate(wmg, torch, w, mode, U, dV0, dB, dX, masses, stream)
            extra[names[mode]] = {"value": r, "ms_per_step": msm, "outer_iters": itm, "coarse": cg}
        if "plain_fp64" in extra:
            extra["vs_plain_fp64"] = value / world / extra["plain_fp64"]["value"]
        bsrc = batch_sources(w)
        mgb = wmg.WilsonMG(w.dims, mg_params(w, args.prec), stream=stream)
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

    if not args.quick:
        extra["three_level"] = three_level_leg(wmg, torch, w, U, dV0, dB, dX, masses, stream, args.prec)
        extra["batched_24x24x24x64"] = batched_leg(wmg, torch, stream, args.prec)
        extra["eo_cg"] = eo_cg_leg(wmg, torch, w, U, dB, dX, masses, infos[:n_solve], stream)
        if w.name == "wilson_16x16x16x32_nv20_beta6_5mass":
            extra["learned_setup"] = learned_leg(wmg, torch, w, U, V0, srcs[-1], stream, args.prec)
        extra["dslash_24x24x24x64"] = dslash_beyond_l2(wmg, torch, stream, peak)

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
                         "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "latency_floor": latency},
            "kernel_ms": {k: round(v[0], 3) for k, v in prof_all.items()},
            "kernel_ms_note": "device time per kernel class of one step, profiled outside the timed region",
            "dslash_alone": {"ms": ms_dc, "GB/s": bytes_ds / (ms_dc * 1e-3) / 1e9,
                             "frac": bytes_ds / (ms_dc * 1e-3) / 1e9 / peak, "l2": "flushed before every launch",
                             "work": f"{V} sites x {(72 + 24 + 24) * (8 if args.prec == 'fp64' else 4)} B",
                             "back_to_back_ms": ms_ds},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        line.update(extra)
        if not args.no_baseline:
            cb = cpu_baseline(w, U, srcs, masses, V0)
            if cb is not None:
                line["cpu_baseline"] = {k: v for k, v in cb.items() if k not in ("step_s", "solve_s")}
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def oracle_counts(w):
    """The oracle's own work on this workload (setup at the setup mass, one solve
    per mass), recorded by tests/golden/make_oracle_iters.py: per solve outer
    iterations, coarse CG iterations and fine operator applications; for the
    setup its fine operator applications and coarse CG iterations."""
    path = os.path.join(ROOT, "tests", "golden", f"{w.name}_oracle_iters.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = [int(x) for x in v]
    return out


def cpu_baseline(w, U, srcs, masses, V0, budget_s=25.0):
    """The FP64 CPU oracle on this workload: its unit costs timed here, scaled by
    its own recorded work counts.

    Timed on this machine (oracle calls only, with the workload's field, random
    starts and sources): one fine operator application t_d; one block
    orthonormalisation and one Galerkin build; one coarse CG iteration t_cg
    (20 iterations of oracle.cgnr); and k outer MG-GCR iterations, whose time
    less their own fine applications and coarse iterations gives the rest of
    an outer iteration (GCR and smoother vector work, restriction,
    prolongation) t_rest.  Scaled by the counts the oracle itself produced on
    this workload: the step costs setup_fine_matvecs t_d + setup_coarse_iters
    t_cg + (1 + Nv/4) orthonormalisations and builds (the Nv/4 truncated
    levels scaled by (Nv-4)^2/Nv^2) + Nv/4 x setup_iters x 4 truncated cycles
    of t_rest, plus per mass fine_matvecs t_d + coarse_iters t_cg +
    outer_iters t_rest.  Without recorded counts it falls back to the GPU's
    outer iteration counts and says so."""
    import oracle
    oracle.build()
    cores = os.cpu_count()
    t_begin = time.perf_counter()
    t0 = time.perf_counter()
    for _ in range(3):
        oracle.dslash(U, srcs[0], masses[0], w.dims)
    t_d = (time.perf_counter() - t0) / 3
    t0 = time.perf_counter()
    P, st = oracle.block_orthonormalize(V0, w.dims, w.block)
    t_ortho = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = oracle.coarse_build(U, P, masses[-1], w.dims, w.block)
    t_build = time.perf_counter() - t0
    Lc = oracle.coarse_dims(w.dims, w.block)
    rc = oracle.restrict(P, srcs[0], w.dims, w.block)
    t0 = time.perf_counter()
    oracle.cgnr(A, rc, Lc, 0.0, 20)
    t_cg = (time.perf_counter() - t0) / 20
    sm, steps = w.extra.get("smoother", 0), w.extra.get("smoother_steps", 4)
    k = 1
    while True:
        p = oracle.make_params(w.dims, w.block, nv=w.nvec, m=masses[-1], tol=0.0, max_outer=k, gcr_restart=16,
                               smoother=sm, mr_steps=steps)
        t1 = time.perf_counter()
        _, info = oracle.gcr_solve(p, U, P, A, srcs[0])
        dt = time.perf_counter() - t1
        if dt * 2 > max(budget_s - (time.perf_counter() - t_begin), 2.0) or k >= 16:
            break
        k *= 2
    n_out = max(info["outer_iters"], 1)
    t_rest = max(dt - info["fine_matvecs"] * t_d - info["coarse_iters"] * t_cg, 0.0) / n_out
    try:
        c = oracle_counts(w)
        outer, coarse, mvs = c["outer_iters"], c["coarse_iters"], c["fine_matvecs"]
        s_mv, s_cg = c["setup_fine_matvecs"][0], c["setup_coarse_iters"][0]
        src = "the oracle's own recorded counts (tests/golden/make_oracle_iters.py)"
    except (OSError, KeyError):
        return None
    groups = w.nvec // 4
    setup_iters = w.extra.get("setup_iters", 5)
    trunc = ((w.nvec - 4) / w.nvec) ** 2
    setup_s = (s_mv * t_d + s_cg * t_cg + (t_ortho + t_build) * (1 + groups * trunc)
               + groups * setup_iters * 4 * t_rest)
    solve_s = [mvs[i] * t_d + coarse[i] * t_cg + outer[i] * t_rest for i in range(len(masses))]
    step_s = setup_s + sum(solve_s)
    return {"value": len(masses) / step_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "step_s": step_s, "setup_s": setup_s, "solve_s": solve_s,
            "sample": (f"oracle (OpenMP, {cores} threads) unit costs timed here on this workload: operator "
                       f"application {t_d:.3f} s, coarse CG iteration {t_cg * 1e3:.2f} ms, block "
                       f"orthonormalisation {t_ortho:.2f} s, Galerkin build {t_build:.2f} s, rest of an outer "
                       f"iteration {t_rest:.3f} s ({k} outer iterations timed); scaled by {src}: setup "
                       f"{s_mv} applications + {s_cg} coarse iterations, solves {outer} outer / {coarse} coarse "
                       f"iterations / {mvs} applications per mass")}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    U, V0, srcs, masses, plaq = make_inputs(w)
    cb = None
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(w, U, srcs, masses, V0, budget_s=20.0)
    sample_s = (time.perf_counter() - t0) / max(1, args.steps)
    if cb is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded oracle work counts for {w.name}"}))
        return
    line = {"metric": METRIC, "value": cb["value"], "unit": "solves/s", "n_gpus": 0, "steps": args.steps,
            "warmup": 0, "ms_per_step": 1e3 * cb["step_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "lattice": "x".join(map(str, w.dims)), "nvec": w.nvec},
            "cpu_baseline": {k: v for k, v in cb.items() if k not in ("step_s", "solve_s")},
            "sample_wall_s_per_step": sample_s,
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
