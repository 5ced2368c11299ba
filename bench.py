"""Benchmark: Fourier-order VRTE solves/s and full-BRDF seconds of the polarized
subsurface BRDF on one GB300 (and N independent replicas under torchrun).

A step is one full BRDF solve (every pipeline stage: tables, assembly, eigen,
boundary, particular, reconstruction, synthesis) of the N = 64, M = L = 128 Mie
layer with a 1024 x 1024 x 360 table. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

The headline is the mixed form (tensor-core contractions); the FP64 form is timed
beside it on the same layer ("fp64_plain", "speedup_vs_fp64_plain").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Fourier-order VRTE solves/s and full-BRDF seconds at N=64,M=128 vs FP64 plain"
UNIT = "order-solves/s"
WORKLOAD = 3


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def fp64_peak_tflops(sm_mhz):
    """FP64 CUDA-core peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 FLOP x SM clock."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def build_workload(grid=None):
    """The N=64, M=L=128 Mie layer; `grid` = (n_in, n_out, n_phi) replaces the 1024 x 1024
    x 360 table by a smaller one (profiling captures only; never a bench line)."""
    from vrte_inputs import angle_grids, make_config
    cfg = make_config(WORKLOAD)
    if grid:
        cfg["mu_in"], cfg["mu_out"], cfg["dphi"] = angle_grids(*grid)
        cfg["name"] = cfg["name"].rsplit("-", 2)[0] + "-%dx%dx%d-n1.5" % tuple(grid)
    ly = dict(cfg["layers"][0])
    ly["n_coef"] = ly["coef"].shape[0]
    return cfg, ly


def oracle_order(ly, m, mi, mo, dphi):
    """One Fourier order of the oracle on a sub-grid, with its share of the synthesis."""
    import oracle as O
    n_if = ly["n_interface"]
    nodes = O.gauss_legendre_01(ly["n_nodes"])
    R = O.fresnel_internal_reflection(nodes[0], n_if) if n_if > 1 else None
    sol = O.solve_order(m, ly["coef"], ly["omega"], ly["tau"], ly["n_nodes"], O.snell_mu(mi, n_if),
                        O.fresnel_beam_in(mi, n_if), R, nodes)
    Im = sol.reconstruct_top(O.snell_mu(mo, n_if))
    from oracle.brdf import synthesize
    return synthesize(Im[None], mi, mo, dphi, n_if)


def oracle_sample(ly, cfg, orders=(0, 64), grids=((2, 8), (8, 8), (2, 24), (8, 24))):
    """Time the oracle on sub-grids and extrapolate to the full grid per order.

    t(n_in, n_out) = a + b n_in + c n_out per order (least squares, non-negative) on
    four sub-grids (incident / outgoing cosines taken evenly from the workload's grids,
    all azimuths), averaged over the sampled orders. The oracle's cost is one eigen
    solve per order plus one dense 8N LU solve per incident cosine plus per-outgoing
    operator builds; its per-(incident, outgoing) work is small vectorised products.
    """
    mu_in_all, mu_out_all, dphi = cfg["mu_in"], cfg["mu_out"], cfg["dphi"]
    rows, times = [], []
    spent = 0.0
    for (ni, no) in grids:
        mi = mu_in_all[np.linspace(0, mu_in_all.size - 1, ni).astype(int)]
        mo = mu_out_all[np.linspace(0, mu_out_all.size - 1, no).astype(int)]
        t = 0.0
        for m in orders:
            t0 = time.perf_counter()
            oracle_order(ly, m, mi, mo, dphi)
            t += time.perf_counter() - t0
        spent += t
        rows.append([1.0, ni, no, ni * no])
        times.append(t / len(orders))
    A = np.array(rows)[:, :3]
    coef = np.linalg.lstsq(A, np.array(times), rcond=None)[0]
    coef = np.maximum(coef, 0.0)
    n_in, n_out = mu_in_all.size, mu_out_all.size
    t_order = float(coef @ np.array([1.0, n_in, n_out]))
    t_order = max(t_order, max(times))
    return t_order, spent, coef


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count()


def cpu_baseline(ly, cfg):
    t_order, spent, _ = oracle_sample(ly, cfg)
    return {
        "value": 1.0 / t_order,
        "unit": UNIT,
        "cores": blas_threads(),
        "cpu_model": cpu_model(),
        "nproc": os.cpu_count(),
        "kind": "oracle",
        "sample": ("FP64 numpy oracle (full 8N formulation) on orders m=0 and m=64 of the "
                   "N=64, L=128 layer for sub-grids (2,8), (8,8), (2,24), (8,24) incident x "
                   "outgoing cosines with all 360 azimuths; per-order time fitted as "
                   "a + b n_in + c n_out and evaluated at 1024 x 1024; "
                   f"{spent:.1f} s of CPU work"),
        "seconds_per_order_full_grid_est": t_order,
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, ly = build_workload()
    vals, t_all = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t_order, spent, _ = oracle_sample(ly, cfg)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(1.0 / t_order)
            t_all.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(t_all)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "mie-N64-M128-L128-1024x1024x360-n1.5", "N": 64, "M": 128, "L": 128,
                   "n_in": 1024, "n_out": 1024, "n_phi": 360,
                   "step": "bounded oracle sample (4 sub-grids x 2 orders), extrapolated"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(),
                         "cpu_model": cpu_model(), "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": "each step: oracle on orders 0 and 64, sub-grids (2,8),(8,8),"
                                   "(2,24),(8,24) x 360 azimuths, linear fit to 1024 x 1024"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_backward(vr, torch, dev, n_layers=16, steps=2, warmup=1):
    """The adjoint on the differentiation workload's shape (N = 48, M = L = 96 Mie layers with an
    interface, 64 x 64 x 90 FP32 tables): per step one vrte_solve_brdf and one
    vrte_brdf_backward of the loss 1/2 |F - F_target|^2 over `n_layers` of its 64 layers, on the
    plan's concurrent streams; F_target = the table of the layers with every parameter perturbed
    by a seeded 1-5 %."""
    from vrte_inputs import make_config
    cfg = make_config(5)
    layers = [dict(l, n_coef=l["coef"].shape[0]) for l in cfg["layers"][:n_layers]]
    rng = np.random.default_rng(5)
    pert = [dict(l, tau=l["tau"] * (1 + rng.uniform(0.01, 0.05)),
                 omega=min(0.999, l["omega"] * (1 + rng.uniform(0.01, 0.05))),
                 coef=l["coef"] * (1 + rng.uniform(-0.05, 0.05, l["coef"].shape))) for l in layers]
    Lmax = max(l["n_coef"] for l in layers)
    plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], 48, 96, Lmax, len(layers),
                   vr.VRTE_FP64, profile=True, adjoint=True)
    d_pert = torch.from_numpy(vr.pack_coefficients(pert, Lmax)).to(dev)
    plan.set_layers(pert, d_pert)
    target = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
    plan.solve(target)
    d_coef = torch.from_numpy(vr.pack_coefficients(layers, Lmax)).to(dev)
    plan.set_layers(layers, d_coef)
    F = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
    grad = torch.empty((len(layers), 3 + 6 * Lmax), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        plan.solve(F, stream)
        plan.backward(F - target, grad, stream)
    if plan.status() != 0:
        raise SystemExit("backward failed")
    if not bool(torch.isfinite(grad).all()):
        raise SystemExit("backward gradient not finite")
    plan.reset_stages()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        plan.solve(F, stream)
        G = F - target
        ev[i][1].record(stream)
        plan.backward(G, grad, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    bwd = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
    st = plan.status()
    stages = plan.stages()
    plan.close()
    orders = sum(min(l["n_orders"], l["n_coef"]) for l in layers)
    adj = next(x for x in stages if x["name"] == "adjoint")
    return {"workload": cfg["name"], "layers": len(layers), "order_solves": orders,
            "N": 48, "M": 96, "L": 96, "n_in": 64, "n_out": 64, "n_phi": 90,
            "forward_ms_per_step": fwd, "backward_ms_per_step": bwd,
            "backward_order_solves_per_s": orders / (bwd / 1000.0),
            "backward_over_forward": bwd / fwd, "status": int(st), "clocks": clk,
            "adjoint_stage_ms": round(adj["ms"] / steps, 2),
            "adjoint_stage_fp64_tflops": adj["flops"] / (adj["ms"] / 1000.0) / 1e12
            if adj["ms"] > 0 else None,
            "structure": "FP64 plan; backward recomputes each order batch in FP64 (eigen, "
                         "boundary, particular), then the adjoint kernels; gradient "
                         "[layers, 3 + 6 L] of omega, tau0, n, coefficients",
            "steps": steps, "warmup": warmup}


def time_slab(vr, torch, dev, n_sub=4, steps=2, warmup=1):
    """A multi-layer slab (vrte_solve_slab_brdf) of `n_sub` sub-layers of the differentiation
    workload's shape (N = 48, M = L = 96 Mie sub-layers, the first one's interface as the top,
    64 x 64 x 90 FP64 table), timed beside the same layers solved as independent layers
    (vrte_solve_brdf, FP64 plan): the slab's cost over the independent solves is its block
    elimination and the attenuated sum of the sub-layers' top radiances."""
    from vrte_inputs import make_config
    cfg = make_config(5)
    layers = [dict(l, n_coef=l["coef"].shape[0]) for l in cfg["layers"][:n_sub]]
    sub = [dict(l, n_interface=(l["n_interface"] if k == 0 else 1.0))
           for k, l in enumerate(layers)]
    Lmax = max(l["n_coef"] for l in layers)
    d_coef = torch.from_numpy(vr.pack_coefficients(sub, Lmax)).to(dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, slab in (("slab", True), ("independent", False)):
        plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], 48, 96, Lmax, n_sub,
                       vr.VRTE_FP64, profile=True, slab=slab)
        plan.set_layers(sub, d_coef)
        shape = plan.table_shape[1:] if slab else plan.table_shape
        out = torch.empty(shape, dtype=torch.float32, device=dev)
        run = plan.solve_slab if slab else plan.solve
        for _ in range(warmup):
            run(out, stream)
        torch.cuda.synchronize()
        plan.reset_stages()
        clocks = ClockSampler(torch.cuda.current_device())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            run(out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        st = plan.status()
        stages = {x["name"]: round(x["ms"] / steps, 2) for x in plan.stages() if x["ms"] > 0}
        plan.close()
        if st != 0:
            raise SystemExit(f"slab record: {name} solve failed ({st})")
        res[name] = {"ms_per_solve": e0.elapsed_time(e1) / steps, "stage_ms": stages,
                     "clocks": clk}
    orders = n_sub * 96
    return {"workload": f"slab of {n_sub} sub-layers of {cfg['name']}", "sub_layers": n_sub,
            "N": 48, "M": 96, "L": 96, "n_in": 64, "n_out": 64, "n_phi": 90,
            "ms_per_slab": res["slab"]["ms_per_solve"],
            "sub_layer_order_solves_per_s": orders / (res["slab"]["ms_per_solve"] / 1000.0),
            "independent_layers_ms": res["independent"]["ms_per_solve"],
            "slab_over_independent": res["slab"]["ms_per_solve"] /
            res["independent"]["ms_per_solve"],
            "slab_stage_ms": res["slab"]["stage_ms"],
            "independent_stage_ms": res["independent"]["stage_ms"],
            "clocks": res["slab"]["clocks"],
            "structure": "FP64 plans, FP32 tables; the slab runs its sub-layers in turn on one "
                         "stream, the independent solve on the plan's concurrent streams",
            "steps": steps, "warmup": warmup}


def _timed_solves(plan, out, stream, steps, warmup, torch):
    """Device time per vrte_solve_brdf call (CUDA events on `stream`, after `warmup` calls)."""
    for _ in range(warmup):
        plan.solve(out, stream)
    torch.cuda.synchronize()
    plan.reset_stages()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.solve(out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def time_batched(vr, torch, dev, subset_stride=16):
    """The batched workload (256 uneven layers, 64 x 64 x 90 FP32 tables) in one mixed-form
    call: one direct step after one warm-up, then the same call captured once into a CUDA graph
    and replayed as one graph launch per step. FP64-plain beside the mixed form on a stratified
    subset (every `subset_stride`-th layer), since 256 FP64 layers take minutes."""
    from vrte_inputs import make_config
    cfg = make_config(4)
    layers = [dict(l, n_coef=l["coef"].shape[0]) for l in cfg["layers"]]
    coef = vr.pack_coefficients(layers)
    d_coef = torch.from_numpy(coef).to(dev)
    stream = torch.cuda.Stream(dev)
    orders = lambda ls: sum(min(l["n_orders"], l["n_coef"]) for l in ls)
    rec = {"workload": cfg["name"], "layers": len(layers), "order_solves": orders(layers),
           "n_in": 64, "n_out": 64, "n_phi": 90, "out_dtype": "f32"}
    plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], max(l["n_nodes"] for l in layers),
                   max(l["n_orders"] for l in layers), coef.shape[1], len(layers), vr.VRTE_MIXED,
                   profile=False)
    plan.set_layers(layers, d_coef)
    out = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
    clocks = ClockSampler(torch.cuda.current_device())
    ms = _timed_solves(plan, out, stream, 1, 1, torch)
    launches = int(sum(st["launches"] for st in plan.stages()))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        plan.solve(out, stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        g.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    clk = clocks.stop()
    st = plan.status()
    del g
    plan.close()
    del out
    torch.cuda.empty_cache()
    if st != 0:
        raise SystemExit(f"batched record: solve failed ({st})")
    rec.update({"mixed_ms_per_step": ms, "order_solves_per_s": rec["order_solves"] / (ms / 1e3),
                "graph_ms_per_step": ms_graph,
                "graph_order_solves_per_s": rec["order_solves"] / (ms_graph / 1e3),
                "gpu_launches_per_step": launches, "host_launches_per_graph_step": 1,
                "clocks": clk})
    sub = layers[::subset_stride]
    scoef = vr.pack_coefficients(sub)
    d_scoef = torch.from_numpy(scoef).to(dev)
    sres = {}
    for name, prec in (("mixed", vr.VRTE_MIXED), ("fp64", vr.VRTE_FP64)):
        plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], max(l["n_nodes"] for l in sub),
                       max(l["n_orders"] for l in sub), scoef.shape[1], len(sub), prec)
        plan.set_layers(sub, d_scoef)
        out = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
        sres[name] = _timed_solves(plan, out, stream, 1, 1, torch)
        if plan.status() != 0:
            raise SystemExit(f"batched record: subset {name} solve failed")
        plan.close()
        del out
        torch.cuda.empty_cache()
    rec["subset"] = {"layers": len(sub), "every": subset_stride, "order_solves": orders(sub),
                     "mixed_ms": sres["mixed"], "fp64_plain_ms": sres["fp64"],
                     "mixed_over_fp64_speedup": sres["fp64"] / sres["mixed"]}
    rec["structure"] = ("one plan, one vrte_solve_brdf call per step; layers on up to 4 "
                        "concurrent streams (one workspace slot each), all orders of a layer "
                        "batched; graph: the same call captured once, one graph launch per step")
    rec["steps"], rec["warmup"] = 1, 1
    return rec


def max_over_ranks(x, dist, device):
    """Maximum of the float x over the ranks of the process group (x itself without one)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, seconds):
    """Units per second of the whole job: every rank processed units_per_rank per step, and the
    job took the slowest rank's time."""
    return world * units_per_rank * steps / seconds


def time_form(vr, torch, cfg, ly, precision, dev, steps, warmup, dist):
    """Warm up, then time `steps` full solves with CUDA events on the solve stream."""
    L = ly["n_coef"]
    plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], ly["n_nodes"], ly["n_orders"], L, 1,
                   precision, profile=True)
    coef = vr.pack_coefficients([ly])
    plan.set_layers([ly], torch.from_numpy(coef).to(dev))
    out = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        plan.solve(out, stream)
    st = plan.status()
    if st != 0:
        raise SystemExit(f"solve failed: {vr.STATUS_NAMES.get(st, st)}")
    plan.reset_stages()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)                       # evict L2 between timed steps
        ev[i][0].record(stream)
        plan.solve(out, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), dist, dev)
    st = plan.status()
    if st != 0:
        raise SystemExit(f"solve failed: {vr.STATUS_NAMES.get(st, st)}")
    stages = plan.stages()
    refined = plan.debug_buffer("refined")[0] if precision == vr.VRTE_MIXED else 0.0
    del out, flush
    return plan, coef, total_ms, clk, stages, refined


def run_batched(args):
    """Batched workload: 256 layers of uneven N, L, tau, omega and interface (8 materials x 32
    wavelengths) on a 64 x 64 x 90 table each, all in one plan and one solve call per
    step; the FP64 form is timed beside the mixed form. Prints its own JSON line."""
    import torch
    import paper_1707_05882_gb300 as vr
    from vrte_inputs import make_config
    cfg = make_config(4)
    layers = [dict(l, n_coef=l["coef"].shape[0]) for l in cfg["layers"]]
    coef = vr.pack_coefficients(layers)
    dev = torch.device("cuda", 0)
    d_coef = torch.from_numpy(coef).to(dev)
    M_total = sum(min(l["n_orders"], l["n_coef"]) for l in layers)
    res = {}
    for name, prec in (("mixed", vr.VRTE_MIXED), ("fp64", vr.VRTE_FP64)):
        if name == "fp64" and args.no_fp64_plain:
            continue
        plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"],
                       max(l["n_nodes"] for l in layers), max(l["n_orders"] for l in layers),
                       coef.shape[1], len(layers), prec, profile=True)
        plan.set_layers(layers, d_coef)
        out = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
        stream = torch.cuda.current_stream(dev)
        for _ in range(args.warmup):
            plan.solve(out, stream)
        if plan.status() != 0:
            raise SystemExit("batched solve failed")
        plan.reset_stages()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.solve(out, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        res[name] = {"ms_per_step": ms, "value": M_total / (ms / 1000.0), "clocks": clk,
                     "stages_ms": {st["name"]: round(st["ms"] / args.steps, 2)
                                   for st in plan.stages()},
                     "gpu_launches": int(sum(st["launches"] for st in plan.stages())) // args.steps}
        plan.close()
        del out
        torch.cuda.empty_cache()
    line = {"metric": "Fourier-order VRTE solves/s, batched uneven layers", "unit": UNIT,
            "value": res["mixed"]["value"], "ms_per_step": res["mixed"]["ms_per_step"],
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 via 7-slice (synthesis 5-slice) bf16 products on tcgen05 + f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "layers": len(layers), "order_solves": M_total,
                       "n_in": 64, "n_out": 64, "n_phi": 90, "out_dtype": "f32",
                       "structure": "one plan, one vrte_solve_brdf call per step; layers run "
                                    "on up to 4 concurrent streams (one workspace slot each), "
                                    "all orders of a layer batched",
                       "stages_ms": "summed over the concurrent streams, so above ms_per_step"},
            "mixed": res["mixed"], "fp64_plain": res.get("fp64"),
            "speedup_vs_fp64_plain": (res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
                                      if "fp64" in res else None)}
    print(json.dumps(line), flush=True)


# Committed ncu summaries that give the DRAM bytes per launch of a stage's dominant kernel
# (the stage's kernel, not the grid, decides them: k_eigen does not depend on the angular
# grid). A stage without a summary of its current kernel reports traffic null.
TRAFFIC_PROFILES = {"eigen": "profiles/eigen_mie-N64-M128.md",
                    "recon_part": "profiles/tc_gemm_part_mie-N64-M128-1024x1024x360.md"}


def profile_traffic(stage):
    """dram__bytes_read + dram__bytes_write (bytes per launch) from the stage's committed ncu
    summary table rows "| dram__bytes_read | X GB |", or None."""
    path = TRAFFIC_PROFILES.get(stage)
    if not path:
        return None
    try:
        total, seen = 0.0, set()
        for line in open(os.path.join(ROOT, path)):
            f = [x.strip() for x in line.strip().strip("|").split("|")]
            if len(f) >= 2 and f[0] in ("dram__bytes_read", "dram__bytes_write"):
                v, unit = f[1].split()[:2]
                total += float(v) * {"GB": 1e9, "MB": 1e6, "KB": 1e3, "B": 1.0}[unit]
                seen.add(f[0])
        return total if len(seen) == 2 else None
    except Exception:
        return None


def stage_roofline(st, pk, pk_src):
    """One stage against its bounding unit: tensor-core stages against the measured sustained
    BF16 peak (the slice products they issue), FP64 stages against the derived FP64 peak."""
    sec = st["ms"] / 1000.0 if st["ms"] > 0 else float("nan")
    if st.get("tc_flops", 0.0) > 0.0:
        # achieved: the stage's algorithmic (FP64-equivalent) FLOPs per second. Its ceiling is
        # the measured BF16 rate divided by the BF16 slice products the sliced scheme issues
        # per FP64 multiply-add (S(S+1)/2: 28 at 7 slices, 15 at 5), i.e. bf16 x flops/tc_flops.
        bf16 = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0)))
        ratio = st["flops"] / st["tc_flops"]
        achieved = st["flops"] / sec / 1e12
        peak = bf16 * ratio
        return {"stage": st["name"], "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "slice_products_tflops": st["tc_flops"] / sec / 1e12, "bf16_peak": bf16,
                "peak_source": f"bf16_tflops_sustained ({pk_src}) of measured x {ratio:.4f} "
                               "(algorithmic FP64 FLOPs per BF16 slice-product FLOP of the "
                               "stage's sliced contractions)"}
    peak = fp64_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    achieved = st["flops"] / sec / 1e12
    return {"stage": st["name"], "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "derived FP64: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x max SM clock"}


# Stages that run on a side stream beside the solve's own stream: their time is measured from
# their fork to their join and overlaps the eigen-decomposition, so they are never the
# headline's dominant stage.
CONCURRENT_STAGES = {"side_ops"}


def roofline(stages, clk, precision_name, grid=None):
    """Roofline of the dominant stage (the headline), with its DRAM traffic per launch from
    the committed ncu summary; `per_stage` holds every timed stage against its own unit."""
    pk, pk_src = peaks()
    timed = [s for s in stages if s["ms"] > 0 and s["flops"] > 0]
    dom = max((s for s in stages if s["name"] not in CONCURRENT_STAGES), key=lambda s: s["ms"])
    head = stage_roofline(dom, pk, pk_src)
    head["traffic"] = profile_traffic(dom["name"]) if WORKLOAD == 3 and not grid else None
    head["kernel_stage"] = head.pop("stage")
    head["launches"] = dom["launches"]
    per = []
    for s in timed:
        e = {k: (round(v, 4) if isinstance(v, float) else v)
             for k, v in stage_roofline(s, pk, pk_src).items() if k != "peak_source"}
        if s["name"] in CONCURRENT_STAGES:
            e["concurrent"] = "side stream, overlaps the eigen stage; ms from fork to join"
        per.append(e)
    head["per_stage"] = per
    return head


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true",
                    help="skip timing the FP64 form beside the mixed form")
    ap.add_argument("--grid", type=int, nargs=3, metavar=("N_IN", "N_OUT", "N_PHI"),
                    help="smaller table for profiling captures (not the benchmark workload)")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the adjoint record (vrte_brdf_backward on 16 layers of the "
                         "N=48, M=96 differentiation workload)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched record (256 uneven layers in one mixed-form call, "
                         "direct and graph-replayed; FP64-plain on a 16-layer subset)")
    ap.add_argument("--no-slab", action="store_true",
                    help="skip the multi-layer slab record (vrte_solve_slab_brdf on 4 sub-layers "
                         "of the N=48, M=96 workload)")
    ap.add_argument("--workload", default="brdf", choices=["brdf", "batched"],
                    help="brdf: the N=64, M=128 layer (the benchmark line); batched: 256 "
                         "uneven layers, its own JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)

    import torch
    import paper_1707_05882_gb300 as vr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    cfg, ly = build_workload(args.grid)
    L = ly["n_coef"]
    M_eff = min(ly["n_orders"], L)
    prec = vr.VRTE_FP64 if args.precision == "fp64" else vr.VRTE_MIXED

    fp64_plain = None
    if args.precision == "mixed" and not args.no_fp64_plain:
        plan64, _, ms64, clk64, stages64, _ = time_form(vr, torch, cfg, ly, vr.VRTE_FP64, dev,
                                                        args.steps, args.warmup, dist)
        plan64.close()
        torch.cuda.empty_cache()
        fp64_plain = {"ms_per_step": ms64 / args.steps,
                      "value": whole_job_rate(world, M_eff, args.steps, ms64 / 1000.0), "unit": UNIT,
                      "clocks": clk64,
                      "stages_ms": {s["name"]: round(s["ms"] / args.steps, 2) for s in stages64}}

    plan, coef, total_ms, clk, stages, refined = time_form(vr, torch, cfg, ly, prec, dev,
                                                           args.steps, args.warmup, dist)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, M_eff, args.steps, total_ms / 1000.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else
        "f64 via 7-slice (synthesis 5-slice) bf16 products on tcgen05 + f64",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "N": ly["n_nodes"], "M": ly["n_orders"], "L": L,
                   "n_in": int(cfg["mu_in"].size), "n_out": int(cfg["mu_out"].size),
                   "n_phi": int(cfg["dphi"].size), "n_interface": ly["n_interface"],
                   "tau": ly["tau"], "omega": ly["omega"], "precision": args.precision,
                   "out_dtype": "f32", "l2": "flushed by a 256 MiB device write before each step",
                   "parallelism": f"replicas x{world} (one independent layer solve per GPU)"},
        "full_brdf_seconds": ms_per_step / 1000.0,
        "clocks": clk,
        "gpu_launches": int(sum(s["launches"] for s in stages)),
        "roofline": roofline(stages, clk, args.precision, args.grid),
        "stages": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()}
                   for s in stages],
    }
    if args.precision == "mixed":
        line["refined_fp64_column_blocks_per_step"] = refined
    if fp64_plain:
        line["fp64_plain"] = fp64_plain
        line["speedup_vs_fp64_plain"] = fp64_plain["ms_per_step"] / ms_per_step

    if not args.no_e2e:
        stream = torch.cuda.current_stream(dev)
        h_coef = torch.from_numpy(coef).pin_memory()
        h_out = torch.empty(plan.table_shape, dtype=torch.float32, pin_memory=True)
        plan.solve_host(h_coef, h_out, stream)     # warm the staging buffers
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            plan.solve_host(h_coef, h_out, stream)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        # the device-to-host link alone: the same table copied from device to pinned host
        d_tab = torch.empty(plan.table_shape, dtype=torch.float32, device=dev)
        h_out.copy_(d_tab)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_out.copy_(d_tab)
        torch.cuda.synchronize()
        link_s = time.perf_counter() - t0
        d2h = int(h_out.numel() * 4)
        line["e2e"] = {"value": whole_job_rate(world, M_eff, args.steps, e2e_s), "unit": UNIT,
                       "h2d_bytes_per_step": int(h_coef.numel() * 8),
                       "d2h_bytes_per_step": d2h,
                       "seconds_per_step": e2e_s / args.steps,
                       "d2h_gbs_in_step": d2h / (e2e_s / args.steps) / 1e9,
                       "d2h_link_gbs_alone": d2h / link_s / 1e9,
                       "api": "vrte_solve_brdf_host (pinned host buffers; the layer is "
                              "reconstructed and synthesized in blocks of 64 incident cosines, "
                              "each block's copy overlapping the next block's work)"}
        del h_out, d_tab
    plan.close()
    torch.cuda.empty_cache()

    if not args.no_backward and not args.grid:
        line["backward"] = time_backward(vr, torch, dev)
    if not args.no_slab and not args.grid:
        line["slab"] = time_slab(vr, torch, dev)
    if not args.no_batched and not args.grid:
        line["batched"] = time_batched(vr, torch, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ly, cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
