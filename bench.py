"""Benchmark of the Pfaffian-sign hot path on one GB300 (or N replicas).

Workload: the synthetic 16^3 x 32 QCD+QED configuration (C* in x, y, z, periodic t,
SU(3) links exp(i 0.2 H), U(1) angles N(0, 0.3^2), c_sw = 1.9 / 1.0), doubled to
N_s = 262144 sites, target mass at kappa = 0.135.

One step = one full sign computation W_sgn(m0) with qs_pfaffian_sign (step A /
step B mass flow, low modes at every mass by the FP32 Chebyshev filter + FP64
Rayleigh-Ritz + mixed-precision Q^-2 power steps), cold start each step.  Its
working set (blocks of 16 spinors, 6 FP64 + 5 FP32 of 50 / 25 MB each) is far
larger than the 129 MB L2.

value   = operator throughput over the whole step: algorithmic bytes of every
          operator application in the step (per doubled site and right-hand side
          48 spinor reals, plus per launch 36 link + 36 SW-term reals per site) / step
          time (GB/s).  ms_per_step is the Pf-sign time per configuration.
e2e     = the same metric through the C-ABI with HOST inputs: every step loads the
          gauge field from host arrays (qs_load_gauge: copy, doubling, SW build) and
          returns the sign to the host.
roofline: the dominant kernel (FP32 operator), achieved = its algorithmic bytes /
          its CUDA-event time inside the timed steps, against the measured HBM copy
          bandwidth.
--op-only runs the operator alone (the earlier benchmark, used for ncu captures).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "qcdqed_16x16x16x32"
METRIC = "Dslash GB/s (% HBM peak); Pf-sign time/config, mixed+batched vs plain FP64 GPU"
KAPPA = 0.135


def reals_per_site(nrhs):
    return 48 * nrhs + 72


def kernel_source_hash():
    """sha256 of the sources the operator kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in ("dslash.cu", "dslash.cuh", "qs_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2108_11989_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(nrhs):
    """DRAM bytes per launch of the FP32 operator from the last ncu capture, if that
    capture was of the current kernel source and the same nrhs; else None."""
    p = os.path.join(ROOT, "profiles", "dslash_f32_tiled_16x16x16x32.traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != kernel_source_hash() or d.get("nrhs") != nrhs:
        return None
    return d["dram_bytes_per_launch"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = sorted(float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def max_over_ranks(x, ws):
    """Max of a per-rank scalar (the timed region is the slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(bytes_per_rank, ms_per_rank, ws):
    """Whole-job throughput: bytes of all ranks over the slowest rank's time (GB/s)."""
    ms = max_over_ranks(ms_per_rank, ws)
    return ws * bytes_per_rank / (ms * 1e-3) / 1e9, ms


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(cfg, m0, seconds=12.0):
    """The oracle's apply_Q (FP64, numpy) on sampled output sites of the same lattice."""
    import numpy as np
    from oracle.dirac import WilsonDirac
    from synth_inputs import random_spinor
    op = WilsonDirac(cfg, lazy=True)
    psi = random_spinor(1, cfg.T, cfg.L).reshape(-1)
    rng = np.random.default_rng(0)
    chunk = 2048
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        sites = rng.choice(cfg.n_sites, chunk, replace=False)
        op.apply_Q(psi, m0, sites)
        done += chunk
    dt = time.perf_counter() - t0
    gbs = done * reals_per_site(1) * 8 / dt / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} output sites of the {cfg.L}^3x{cfg.T} lattice in chunks of {chunk}, "
                      f"FP64 numpy, {dt:.1f} s; bytes counted with the same per-site model (nrhs=1, FP64)"}


def run_reference(args):
    ws, rank, _ = dist_init()
    if rank != 0:
        return
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config
    cfg = make_config(seed=0, **WORKLOADS[WORKLOAD])
    m0 = kappa_to_m0(KAPPA)
    vals = []
    per_step = max(0.3, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(cfg, m0, seconds=per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(cfg, m0, seconds=per_step))
    total = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    cb = dict(vals[-1])
    cb["value"] = v
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": WORKLOAD, "nrhs": 1, "prec": "f64",
                                 "l2": "oracle on host cores"},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_sign(args):
    import numpy as np
    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config

    cfg = make_config(seed=rank, **WORKLOADS[WORKLOAD])
    m0 = kappa_to_m0(KAPPA)
    stream = torch.cuda.current_stream()
    lat = qs.Lattice(cfg.L, cfg.T, device=local, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    opts = qs.sign_default_opts(eig={"k": args.k, "nwant": 2, "tol": args.tol, "cheb_degree": args.degree})
    opts.eig.warm_start = 0

    for _ in range(args.warmup):
        lat.pfaffian_sign(m0, opts)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    lat.set_profiling(True)
    l0 = qs.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = []
    for _ in range(args.steps):
        reps.append(lat.pfaffian_sign(m0, opts))
    e1.record(stream)
    torch.cuda.synchronize()
    launches = qs.kernel_launches() - l0
    barrier(ws)
    clk = clocks.stop()
    prof = lat.get_profile()
    lat.set_profiling(False)
    total_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    ms_step = total_ms / args.steps
    op_bytes = prof["f32"]["bytes"] + prof["f64"]["bytes"]
    value = ws * op_bytes / (total_ms * 1e-3) / 1e9 / 1.0
    f32 = prof["f32"]
    achieved = f32["bytes"] / (f32["ms"] * 1e-3) / 1e9 if f32["ms"] > 0 else 0.0
    peak, src = peaks()
    sign, rep = reps[-1]

    # end to end: host gauge arrays in, sign out, through the C-ABI
    e_steps = 1
    lat.set_profiling(True)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
        s_e, _ = lat.pfaffian_sign(m0, opts)
    torch.cuda.synchronize()
    e_s = max_over_ranks(time.perf_counter() - t0, ws)
    pe = lat.get_profile()
    lat.set_profiling(False)
    e2e = ws * (pe["f32"]["bytes"] + pe["f64"]["bytes"]) / e_s / 1e9
    h2d = cfg.su3.nbytes + (cfg.theta.nbytes if cfg.theta is not None else 0)

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={cfg.n_sites})",
                   "step": "qs_pfaffian_sign at kappa=0.135, cold start", "m0": m0,
                   "block_k": args.k, "cheb_degree": args.degree, "eig_tol": args.tol,
                   "precision": "FP32 filter + FP32 inner CG, FP64 Rayleigh-Ritz and defect correction",
                   "l2": "working set (>= 11 blocks of 16 spinors) far larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "pf_sign": {"s_per_config": ms_step / 1e3, "sign": sign, "masses": rep["n"],
                    "steps_a": rep["steps_a"], "steps_b": rep["steps_b"], "crossings": rep["crossings"],
                    "dslash_f32_per_config": rep["dslash_f32"], "dslash_f64_per_config": rep["dslash_f64"],
                    "cg_iterations": rep["cg_iterations"],
                    "f32_operator_share_of_step": f32["ms"] / total_ms if total_ms > 0 else None,
                    "f64_operator_ms_per_step": prof["f64"]["ms"] / args.steps},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(args.k),
                     "kernel": "dslash_kernel<float>",
                     "launches": f32["launches"], "avg_launch_us": 1e3 * f32["ms"] / max(1, f32["launches"]),
                     "peak_source": f"{src} hbm_gbs",
                     "bytes_model": "(48 nrhs + 72) reals/site x 4 B per launch"},
        "e2e": {"value": e2e, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                "s_per_config": e_s / e_steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_plain:
        # mixed (FP32 filter + mixed CG + FP64 Rayleigh-Ritz) vs plain FP64 form of the
        # eigensolver on the same GPU, one cold solve each at equal eigenvalue tolerance
        cmp = {}
        for name, prec in (("mixed", 1), ("plain_fp64", 0)):
            eo = qs.eig_default_opts(k=16, nwant=2, tol=1e-8, cheb_degree=args.degree, warm_start=0,
                                     max_iter=400, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, rs, st = lat.lowmodes_at_mass(m0, eo, allow_noconv=True)
            torch.cuda.synchronize()
            cmp[name] = {"s": time.perf_counter() - t0, "lambda_bar": abs(float(ev[0])),
                         "resid": float(rs[0]), "status": st["status"], "passes": st["iterations"],
                         "dslash_f32": st["dslash_f32"], "dslash_f64": st["dslash_f64"]}
        cmp["speedup_mixed_over_plain"] = cmp["plain_fp64"]["s"] / cmp["mixed"]["s"]
        cmp["lambda_bar_rel_diff"] = abs(cmp["mixed"]["lambda_bar"] - cmp["plain_fp64"]["lambda_bar"]) / \
            cmp["plain_fp64"]["lambda_bar"]
        out["eigensolve_mixed_vs_plain_fp64"] = cmp
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, m0)
    if rank == 0:
        print(json.dumps(out))
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--op-only", action="store_true", help="time the operator alone")
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--degree", type=int, default=48)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--tiled", action="store_true", help="--op-only with the solver's site-tiled layout")
    ap.add_argument("--workload", default=WORKLOAD, help="--op-only: synthetic workload name")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the mixed vs plain FP64 eigensolve")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if not args.op_only:
        return run_sign(args)

    import numpy as np
    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config, random_spinor

    cfg = make_config(seed=rank, **WORKLOADS[args.workload])
    m0 = kappa_to_m0(KAPPA)
    stream = torch.cuda.current_stream()
    lat = qs.Lattice(cfg.L, cfg.T, device=local, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    ns, R = cfg.n_sites, args.nrhs
    rdt = np.float32 if args.prec == "f32" else np.float64
    rsz = 4 if args.prec == "f32" else 8
    # rotate over 4 buffer sets unless one set alone is far larger than the L2
    nsets = 4 if ns * 24 * R * rsz < 1e9 else 1
    bufs = []
    for k in range(nsets):
        psi = random_spinor(100 + k, cfg.T, cfg.L, R)
        x = torch.from_numpy(psi.view(np.float64).astype(rdt)).cuda().reshape(-1)
        if args.tiled:
            x = qs.to_tiled(x, ns)
        bufs.append((x, torch.empty_like(x)))
    bytes_per_launch = ns * reals_per_site(R) * rsz
    launches_per_step = 1   # one operator launch covers all right-hand sides

    def step(k):
        x, y = bufs[k % nsets]
        lat.apply_Q(m0, x, y, tiled=args.tiled)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = time.perf_counter()
    for k in range(args.steps):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(ws)
    clk = clocks.stop()
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    total_ms = max_over_ranks(total_ms, ws)
    ms_step = total_ms / args.steps
    value = ws * bytes_per_launch * args.steps / (total_ms * 1e-3) / 1e9
    avg_step_s = sum(kern_ms) / len(kern_ms) * 1e-3
    achieved = bytes_per_launch / avg_step_s / 1e9
    peak, src = peaks()

    # end to end through the C-ABI with host buffers
    hx = torch.empty(bufs[0][0].numel(), dtype=bufs[0][0].dtype, pin_memory=True)
    hx.copy_(bufs[0][0].cpu())
    hy = torch.empty_like(hx, pin_memory=True)
    dx, dy = torch.empty_like(bufs[0][0]), torch.empty_like(bufs[0][0])
    e_steps = max(10, args.steps // 4)
    for _ in range(3):
        dx.copy_(hx, non_blocking=True); lat.apply_Q(m0, dx, dy); hy.copy_(dy, non_blocking=True)
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        dx.copy_(hx, non_blocking=True)
        lat.apply_Q(m0, dx, dy)
        hy.copy_(dy, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    e2e = ws * bytes_per_launch * e_steps / (e_ms * 1e-3) / 1e9

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={ns})",
                   "op": "Q = gamma5 D", "prec": args.prec, "nrhs": R, "m0": m0,
                   "layout": "site-tiled" if args.tiled else "canonical",
                   "l2": f"inputs larger than L2: {nsets} buffer set(s) of {ns * 24 * R * rsz / 1e6:.0f} MB",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{src} hbm_gbs", "bytes_model": f"{reals_per_site(R)} reals/site x {rsz} B"},
        "e2e": {"value": e2e, "unit": "GB/s", "h2d_bytes_per_step": hx.numel() * rsz,
                "d2h_bytes_per_step": hy.numel() * rsz},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if not args.no_plain:
        # mixed (FP32 filter + mixed CG + FP64 Rayleigh-Ritz) vs plain FP64 form of the
        # eigensolver on the same GPU, one cold solve each at equal eigenvalue tolerance
        cmp = {}
        for name, prec in (("mixed", 1), ("plain_fp64", 0)):
            eo = qs.eig_default_opts(k=16, nwant=2, tol=1e-8, cheb_degree=args.degree, warm_start=0,
                                     max_iter=400, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, rs, st = lat.lowmodes_at_mass(m0, eo, allow_noconv=True)
            torch.cuda.synchronize()
            cmp[name] = {"s": time.perf_counter() - t0, "lambda_bar": abs(float(ev[0])),
                         "resid": float(rs[0]), "status": st["status"], "passes": st["iterations"],
                         "dslash_f32": st["dslash_f32"], "dslash_f64": st["dslash_f64"]}
        cmp["speedup_mixed_over_plain"] = cmp["plain_fp64"]["s"] / cmp["mixed"]["s"]
        cmp["lambda_bar_rel_diff"] = abs(cmp["mixed"]["lambda_bar"] - cmp["plain_fp64"]["lambda_bar"]) / \
            cmp["plain_fp64"]["lambda_bar"]
        out["eigensolve_mixed_vs_plain_fp64"] = cmp
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, m0)
    if rank == 0:
        print(json.dumps(out))
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
