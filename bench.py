"""Benchmark of the Pfaffian-sign hot path on one GB300 (or N independent replicas).

Workload (the timed step): the synthetic 16^3 x 32 QCD+QED configuration (C* in x, y, z,
periodic t, SU(3) links exp(i 0.2 H), U(1) angles N(0, 0.3^2), c_sw = 1.9 / 1.0), doubled
to N_s = 262144 sites, target mass at kappa = 0.135.

One step = one full sign computation W_sgn(m0) with qs_pfaffian_sign (step A / step B
mass flow; low modes at every mass by the Chebyshev filter with 16-bit spinor storage
and FP32 arithmetic, FP64 Rayleigh-Ritz, mixed-precision Q^-2 power steps), cold start
every step.  Its working set (blocks of 32 spinors, 6 FP64 + 5 FP32 of 50 / 25 MB each
per vector) is far larger than the 129 MB L2.

value   = operator throughput over the whole step: algorithmic bytes of every operator
          launch in the step (per doubled site: each right-hand side's spinor in and out,
          two more spinors for the fused Chebyshev step, and once per launch 36 link + 36
          SW-term reals) / step time (GB/s).  ms_per_step is the Pf-sign time per
          configuration.
e2e     = the same metric through the C-ABI with HOST inputs: the step loads the gauge
          field from host arrays (qs_load_gauge: copy, doubling, SW build) and returns the
          sign to the host.
roofline: the dominant operator kernel in the step (by summed event time), achieved =
          its algorithmic bytes / its CUDA-event time inside the timed steps, against the
          measured HBM copy bandwidth.
extras (after the timed region, once): the same W_sgn with the FP32 filter and in the
          plain FP64 form (signs must agree; time per configuration each), and on the
          32^3 x 64 configuration the operator alone (FP32 and FP16 storage, 24 right-hand
          sides) and the low modes at the target mass with FP16 filter storage against an
          FP64 GPU Rayleigh-Ritz of the same block (per-eigenvalue error).
--op-only times the operator alone (the form used for ncu captures).
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
BIG = "qcdqed_32x32x32x64"
METRIC = "Dslash GB/s (% HBM peak); Pf-sign time/config, mixed+batched vs plain FP64 GPU"
KAPPA = 0.135
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}


def op_bytes_per_site(nrhs, prec, cheb=False):
    """Algorithmic bytes per doubled site of one operator launch (see module doc)."""
    spinor = {"f64": 192, "f32": 96, "f16": 52, "bf16": 52}[prec]
    links = 72 * (8 if prec == "f64" else 4)
    return spinor * (4 if cheb else 2) * nrhs + links


def kernel_source_hash():
    """sha256 of the sources the FP32-arithmetic operator kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in ("dslash32.cu", "dslash.cuh", "stencil.cuh", "qs_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2108_11989_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kind, algorithmic_bytes_per_launch):
    """DRAM bytes per launch of the operator, from the committed ncu summary of one launch
    of the current kernel source: the capture's ratio of DRAM bytes (read + write) to
    algorithmic bytes, applied to this launch's algorithmic bytes (traffic scales with the
    sites and right-hand sides a launch processes).  None if no capture of the current
    source and storage exists."""
    p = os.path.join(ROOT, "profiles", "dslash32_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kind)
    if not e or d.get("source_sha256") != kernel_source_hash():
        return None
    return algorithmic_bytes_per_launch * e["dram_bytes"] / e["algorithmic_bytes"]


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


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(cfg, m0, seconds=12.0):
    """The oracle's plain-loop C operator (FP64, OpenMP on all host cores) applying Q to
    the whole lattice, repeated for about `seconds`."""
    from oracle.dirac import WilsonDiracC
    from synth_inputs import random_spinor
    t_build = time.perf_counter()
    op = WilsonDiracC(cfg)
    t_build = time.perf_counter() - t_build
    psi = random_spinor(1, cfg.T, cfg.L).reshape(-1)
    op.apply_Q(psi, m0)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        op.apply_Q(psi, m0)
        done += 1
    dt = time.perf_counter() - t0
    gbs = done * cfg.n_sites * op_bytes_per_site(1, "f64") / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", cpu_cores()))
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{done} applications of Q to one vector on the whole {cfg.L}^3x{cfg.T} lattice "
                      f"(oracle/dirac_c.c, FP64, OpenMP, {dt:.1f} s; operator set-up {t_build:.0f} s not "
                      f"counted); bytes counted with the same per-site model (nrhs=1, FP64)"}


def run_reference(args):
    ws, rank, _ = dist_init()
    if rank != 0:
        return
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config
    cfg = make_config(seed=0, **WORKLOADS[args.workload])
    m0 = kappa_to_m0(KAPPA)
    vals = []
    per_step = max(0.5, min(8.0, 120.0 / max(1, args.steps + args.warmup)))
    from oracle.dirac import WilsonDiracC
    op = WilsonDiracC(cfg)
    from synth_inputs import random_spinor
    psi = random_spinor(1, cfg.T, cfg.L).reshape(-1)

    def sample(seconds):
        done, t0 = 0, time.perf_counter()
        while True:
            op.apply_Q(psi, m0)
            done += 1
            if time.perf_counter() - t0 >= seconds:
                break
        return done * cfg.n_sites * op_bytes_per_site(1, "f64") / (time.perf_counter() - t0) / 1e9, done

    for _ in range(args.warmup):
        sample(per_step)
    t0 = time.perf_counter()
    napp = 0
    for _ in range(args.steps):
        v, d = sample(per_step)
        vals.append(v)
        napp += d
    total = time.perf_counter() - t0
    v = sum(vals) / len(vals)
    cores = int(os.environ.get("OMP_NUM_THREADS", cpu_cores()))
    cb = {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
          "sample": f"{napp} applications of Q (FP64, oracle/dirac_c.c with OpenMP) to one vector on the "
                    f"whole {cfg.L}^3x{cfg.T} lattice, about {per_step:.1f} s per step"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": args.workload, "nrhs": 1, "prec": "f64",
                                 "l2": "oracle on host cores"},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def sign_opts(qs, args, precision):
    o = qs.sign_default_opts(eig={"k": args.k, "nwant": 2, "tol": args.tol, "cheb_degree": args.degree,
                                  "precision": precision, "max_iter": 400})
    o.eig.warm_start = 0
    return o


def dominant(prof):
    """(name, entry) of the operator precision with the largest summed event time."""
    name = max(prof, key=lambda n: prof[n]["ms"])
    return name, prof[name]


def device_spinors(qs, lat, ns, nrhs, prec, seed):
    """Seeded Gaussian spinors made on the device, in the tiled layout of `prec`."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x64 = torch.randn(nrhs * ns * 24, dtype=torch.float64, device="cuda", generator=g) / 2 ** 0.5
    if prec == "f64":
        return x64
    if prec == "f32":
        return x64.float()
    out = torch.empty(nrhs * ns * qs.Q16_BYTES_PER_SITE, dtype=torch.uint8, device="cuda")
    qs.convert_spinors(lat.h, x64, qs.QS_F64, out, PREC[prec], nrhs)
    return out


def time_operator(qs, lat, cfg, m0, prec, nrhs, steps, warmup, nsets=None):
    """CUDA-event time of `steps` operator launches in the tiled layout, inputs rotated
    over buffer sets that together exceed the L2; returns (us per launch, GB/s)."""
    import torch
    ns = cfg.n_sites
    vb = nrhs * ns * (qs.Q16_BYTES_PER_SITE if prec in ("f16", "bf16") else 24 * (8 if prec == "f64" else 4))
    if nsets is None:
        nsets = 1 if vb > 1e9 else 4
    bufs = []
    for k in range(nsets):
        x = device_spinors(qs, lat, ns, nrhs, prec, 100 + k)
        bufs.append((x, torch.empty_like(x)))
    p = PREC[prec]
    stream = torch.cuda.current_stream()
    for k in range(warmup):
        x, y = bufs[k % nsets]
        lat.apply_Q(m0, x, y, tiled=True, prec=p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        x, y = bufs[k % nsets]
        lat.apply_Q(m0, x, y, tiled=True, prec=p)
    e1.record(stream)
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / steps
    gbs = ns * op_bytes_per_site(nrhs, prec) / (us * 1e-6) / 1e9
    del bufs
    torch.cuda.empty_cache()
    return us, gbs


def big_extras(qs, args, peak):
    """32^3 x 64: operator alone (FP32, FP16) and the low modes at the target mass with
    FP16 filter storage against an FP64 Rayleigh-Ritz of the same block."""
    import numpy as np
    import torch
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config
    t0 = time.perf_counter()
    cfg = make_config(seed=0, **WORKLOADS[BIG])
    t_gen = time.perf_counter() - t0
    m0 = kappa_to_m0(KAPPA)
    stream = torch.cuda.current_stream()
    lat = qs.Lattice(cfg.L, cfg.T, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    del cfg.su3
    out = {"workload": BIG, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={cfg.n_sites})",
           "field_generation_s": t_gen}
    ops = {}
    for prec in ("f32", "f16"):
        us, gbs = time_operator(qs, lat, cfg, m0, prec, 24, 20, 3)
        ops[prec] = {"nrhs": 24, "us_per_launch": us, "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "bytes_model": f"{op_bytes_per_site(24, prec)} B/site"}
    out["operator"] = ops
    if not args.no_big_eig:
        k = 24
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        eo = qs.eig_default_opts(k=k, nwant=4, tol=1e-8, cheb_degree=args.degree, warm_start=0,
                                 max_iter=40, precision=2)
        ev, rs, st = lat.lowmodes_at_mass(m0, eo, allow_noconv=True)
        torch.cuda.synchronize()
        t_mixed = time.perf_counter() - t1
        # FP64 GPU reference: plain FP64 Rayleigh-Ritz passes from the block just found
        ep = qs.eig_default_opts(k=k, nwant=4, tol=1e-11, cheb_degree=8, warm_start=1, max_iter=2,
                                 precision=0)
        t1 = time.perf_counter()
        ev64, rs64, st64 = lat.lowmodes_at_mass(m0, ep, allow_noconv=True)
        torch.cuda.synchronize()
        t_ref = time.perf_counter() - t1
        nw = 4
        err = [abs(float(ev[i]) - float(ev64[i])) / abs(float(ev64[i])) for i in range(nw)]
        out["lowmodes_fp16_filter"] = {
            "k": k, "nwant": nw, "tol": 1e-8, "s": t_mixed, "status": st["status"],
            "passes": st["iterations"], "filter_passes": st["filter_passes"], "refine_passes": st["refine_passes"],
            "eigenvalues": [float(x) for x in ev[:nw]], "residuals": [float(x) for x in rs[:nw]],
            "fp64_reference_eigenvalues": [float(x) for x in ev64[:nw]],
            "fp64_reference_residuals": [float(x) for x in rs64[:nw]], "fp64_reference_s": t_ref,
            "rel_error_vs_fp64_per_eigenvalue": err, "max_rel_error": max(err)}
    lat.close()
    torch.cuda.empty_cache()
    return out


def run_sign(args):
    import numpy as np
    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config

    cfg = make_config(seed=rank, **WORKLOADS[WORKLOAD])
    m0 = kappa_to_m0(KAPPA)
    # a stream of its own: the library captures the filter loop as a CUDA graph on it
    stream = torch.cuda.Stream()
    lat = qs.Lattice(cfg.L, cfg.T, device=local, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    eprec = PREC[args.eig_prec]
    opts = sign_opts(qs, args, eprec)

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
    stream.synchronize()
    torch.cuda.synchronize()
    launches = qs.kernel_launches() - l0
    barrier(ws)
    clk = clocks.stop()
    prof = lat.get_profile()
    lat.set_profiling(False)
    total_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    ms_step = total_ms / args.steps
    op_bytes = sum(p["bytes"] for p in prof.values())
    value = ws * op_bytes / (total_ms * 1e-3) / 1e9
    dname, dom = dominant(prof)
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9 if dom["ms"] > 0 else 0.0
    peak, src = peaks()
    sign, rep = reps[-1]

    # end to end: host gauge arrays in, sign out, through the C-ABI
    lat.set_profiling(True)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    s_e, _ = lat.pfaffian_sign(m0, opts)
    torch.cuda.synchronize()
    e_s = max_over_ranks(time.perf_counter() - t0, ws)
    pe = lat.get_profile()
    lat.set_profiling(False)
    e2e = ws * sum(p["bytes"] for p in pe.values()) / e_s / 1e9
    h2d = cfg.su3.nbytes + (cfg.theta.nbytes if cfg.theta is not None else 0)

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{args.eig_prec}+f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={cfg.n_sites})",
                   "step": "qs_pfaffian_sign at kappa=0.135, cold start", "m0": m0,
                   "block_k": args.k, "cheb_degree": args.degree, "eig_tol": args.tol,
                   "precision": f"{args.eig_prec} filter storage with FP32 arithmetic, FP32 inner CG, "
                                "FP64 Rayleigh-Ritz and defect correction",
                   "l2": "working set (>= 11 blocks of 32 spinors) far larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "pf_sign": {"s_per_config": ms_step / 1e3, "sign": sign, "masses": rep["n"],
                    "steps_a": rep["steps_a"], "steps_b": rep["steps_b"], "crossings": rep["crossings"],
                    "dslash_f32_arith_per_config": rep["dslash_f32"], "dslash_f64_per_config": rep["dslash_f64"],
                    "cg_iterations": rep["cg_iterations"],
                    "operator_ms_share_of_step": {n: p["ms"] / total_ms for n, p in prof.items() if p["ms"] > 0}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic(dname, dom["bytes"] / max(1, dom["launches"])),
                     "kernel": f"dslash32_kernel ({dname} storage, FP32 arithmetic)" if dname != "f64"
                     else "dslash_kernel<double>",
                     "launches": dom["launches"], "avg_launch_us": 1e3 * dom["ms"] / max(1, dom["launches"]),
                     "peak_source": f"{src} hbm_gbs (of measured)",
                     "bytes_model": "per doubled site: spinor in + out per right-hand side (+ 2 spinors for the "
                                    "fused Chebyshev step) + 72 link/SW reals per launch"},
        "e2e": {"value": e2e, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                "s_per_config": e_s},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_extras:
        forms = {f"mixed_{args.eig_prec}_filter": {"s_per_config": ms_step / 1e3, "sign": sign, "masses": rep["n"]}}
        for name, prec in (("mixed_f32_filter", 1), ("plain_fp64", 0)):
            if name.startswith("plain") and not args.plain_sign:
                continue
            o = sign_opts(qs, args, prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                s, r = lat.pfaffian_sign(m0, o)
                forms[name] = {"s_per_config": time.perf_counter() - t0, "sign": s, "masses": r["n"],
                               "dslash_f64": r["dslash_f64"], "dslash_f32_arith": r["dslash_f32"]}
            except qs.QStarError as e:
                forms[name] = {"error": str(e)}
        # one cold low-mode solve at the target mass, mixed (16-bit filter) vs plain FP64,
        # at equal eigenvalue tolerance
        cmp = {}
        for name, prec in (("mixed_f16_filter", 2), ("plain_fp64", 0)):
            eo = qs.eig_default_opts(k=16, nwant=2, tol=1e-8, cheb_degree=args.degree, warm_start=0,
                                     max_iter=400, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, rs, st = lat.lowmodes_at_mass(m0, eo, allow_noconv=True)
            torch.cuda.synchronize()
            cmp[name] = {"s": time.perf_counter() - t0, "lambda_bar": abs(float(ev[0])), "resid": float(rs[0]),
                         "status": st["status"], "passes": st["iterations"], "dslash_f64": st["dslash_f64"],
                         "dslash_f32_arith": st["dslash_f32"]}
        cmp["speedup_mixed_over_plain"] = cmp["plain_fp64"]["s"] / cmp["mixed_f16_filter"]["s"]
        cmp["lambda_bar_rel_diff"] = abs(cmp["mixed_f16_filter"]["lambda_bar"] - cmp["plain_fp64"]["lambda_bar"]) / \
            cmp["plain_fp64"]["lambda_bar"]
        out["eigensolve_mixed_vs_plain_fp64"] = cmp
        base = forms.get("plain_fp64", {}).get("s_per_config")
        if base:
            for f in forms.values():
                if "s_per_config" in f:
                    f["speedup_over_plain_fp64"] = base / f["s_per_config"]
        forms["signs_identical"] = len({f["sign"] for f in forms.values() if isinstance(f, dict) and "sign" in f}) == 1
        out["pf_sign_forms"] = forms
    lat.close()
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_extras and not args.no_big:
        out["headline_32x32x32x64"] = big_extras(qs, args, peaks()[0])
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, m0)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_op_only(args):
    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config

    cfg = make_config(seed=rank, **WORKLOADS[args.workload])
    m0 = kappa_to_m0(KAPPA)
    stream = torch.cuda.current_stream()
    lat = qs.Lattice(cfg.L, cfg.T, device=local, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    ns, R, prec = cfg.n_sites, args.nrhs, args.prec
    clocks = Clocks(local)
    barrier(ws)
    us, gbs = time_operator(qs, lat, cfg, m0, prec, R, args.steps, args.warmup)
    barrier(ws)
    clk = clocks.stop()
    total_ms = max_over_ranks(us * args.steps * 1e-3, ws)
    bytes_per_launch = ns * op_bytes_per_site(R, prec)
    value = ws * bytes_per_launch * args.steps / (total_ms * 1e-3) / 1e9
    peak, src = peaks()

    # end to end through the C-ABI with host buffers (pinned host -> device, operator, back)
    x = device_spinors(qs, lat, ns, R, prec, 7)
    hx = torch.empty(x.numel(), dtype=x.dtype, pin_memory=True)
    hx.copy_(x.cpu())
    hy = torch.empty_like(hx, pin_memory=True)
    dx, dy = torch.empty_like(x), torch.empty_like(x)
    e_steps = max(5, args.steps // 4)
    for _ in range(2):
        dx.copy_(hx, non_blocking=True); lat.apply_Q(m0, dx, dy, tiled=True, prec=PREC[prec])
        hy.copy_(dy, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        dx.copy_(hx, non_blocking=True)
        lat.apply_Q(m0, dx, dy, tiled=True, prec=PREC[prec])
        hy.copy_(dy, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    e2e = ws * bytes_per_launch * e_steps / (e_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={ns})",
                   "op": "Q = gamma5 D", "prec": prec, "nrhs": R, "m0": m0, "layout": "site-tiled",
                   "l2": "inputs rotated over buffer sets larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "traffic": measured_traffic(prec, bytes_per_launch), "peak_source": f"{src} hbm_gbs (of measured)",
                     "bytes_model": f"{op_bytes_per_site(R, prec)} B/site"},
        "e2e": {"value": e2e, "unit": "GB/s", "h2d_bytes_per_step": hx.numel() * hx.element_size(),
                "d2h_bytes_per_step": hy.numel() * hy.element_size()},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out))
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_w_mass(args):
    """One stochastic estimate of W_mass (Sec. 4) on the synthetic field: n factors of the
    optimal rational approximation on [r_a, r_b] = [0.02, 8], nsrc sources, FP64 CG."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config, random_spinor

    cfg = make_config(seed=0, **WORKLOADS[args.workload])
    m = kappa_to_m0(KAPPA)
    mp = m + 0.002
    stream = torch.cuda.current_stream()
    lat = qs.Lattice(cfg.L, cfg.T, stream=stream)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    A, nu, mu, delta = qs.ratapprox(args.wm_n, 0.02, 8.0)
    eta = random_spinor(11, cfg.T, cfg.L, nrhs=args.wm_nsrc).reshape(args.wm_nsrc, -1)
    dev = torch.from_numpy(np.ascontiguousarray(np.stack([eta.real, eta.imag], -1))).cuda()
    clocks = Clocks(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q, lw, iters = lat.w_mass(m, mp, nu, mu, dev, tol=1e-10)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    ns = cfg.n_sites
    # full-lattice equivalents of the FP64 operator (per RHS): D_hat applies it to each parity
    # once, Q_hat^2 twice per CG iteration, four more D_hat per factor outside the CG
    n_dslash = (2 * iters + 4 * args.wm_n) * args.wm_nsrc
    gflops = n_dslash * ns * 2160 / secs / 1e9
    out = {
        "metric": "W_mass stochastic estimate (Sec. 4), time per estimate", "value": secs, "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={ns})", "m": m,
                   "m_prime": mp, "n": args.wm_n, "nsrc": args.wm_nsrc, "r_a": 0.02, "r_b": 8.0,
                   "ratapprox_delta": delta, "cg_tol": 1e-10},
        "result": {"log_w_mass": lw, "q": q.tolist(), "cg_iterations": iters},
        "roofline": {"bound": "alu", "achieved": gflops, "peak": 1250.0, "unit": "GFLOP/s (FP64)",
                     "frac": gflops / 1250.0, "traffic": None,
                     "peak_source": "nominal FP64 rate of GB300 (no measured FP64 peak)",
                     "flops_model": "2160 flop per site and RHS per full-lattice FP64 operator "
                                    "application; D_hat = one (half on each parity); Q_hat^2 per CG "
                                    "iteration = two; four D_hat per factor outside the CG; the odd-site "
                                    "block solves are not counted"},
        "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(out))
    lat.close()


def run_solve(args):
    """x = D^-1 b on the synthetic field: the even-odd preconditioned solve of Sec. 4 against
    CG on the full-lattice Q^2, FP64, one right-hand side, tol 1e-10."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS, kappa_to_m0, make_config, random_spinor

    cfg = make_config(seed=0, **WORKLOADS[args.workload])
    m0 = kappa_to_m0(KAPPA)
    lat = qs.Lattice(cfg.L, cfg.T, stream=torch.cuda.current_stream())
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    b = random_spinor(3, cfg.T, cfg.L, nrhs=1).reshape(1, -1)
    bd = torch.from_numpy(np.ascontiguousarray(np.stack([b.real, b.imag], -1))).cuda()
    ns = cfg.n_sites
    res = {}
    for eo in (True, False):
        lat.solve_D(m0, bd, torch.empty_like(bd), even_odd=eo, tol=1e-4)   # warm-up (autotuner, allocator)
        xd = torch.empty_like(bd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = lat.solve_D(m0, bd, xd, even_odd=eo, tol=1e-10)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        # full-lattice FP64 operator equivalents: Q^2 (2) or Q_hat^2 (2 halves twice) per iteration
        gfl = 2 * it * ns * 2160 / secs / 1e9
        res["even_odd" if eo else "full"] = {"s": secs, "cg_iterations": it, "operator_gflops": gfl}
        res["x_norm_" + ("even_odd" if eo else "full")] = float(torch.linalg.vector_norm(xd))
    out = {
        "metric": "D x = b, FP64, even-odd preconditioned vs full-lattice CG (Sec. 4)",
        "value": res["full"]["s"] / res["even_odd"]["s"], "unit": "speedup", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"{cfg.L}^3x{cfg.T} (doubled N_s={ns})", "m0": m0,
                   "nrhs": 1, "tol": 1e-10},
        "result": res,
    }
    print(json.dumps(out))
    lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--op-only", action="store_true", help="time the operator alone")
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--degree", type=int, default=48)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--eig-prec", default="f16", choices=["f32", "f16", "bf16"],
                    help="filter storage of the timed sign computation")
    ap.add_argument("--nrhs", type=int, default=24)
    ap.add_argument("--prec", default="f16", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--workload", default=None,
                    help="synthetic workload of --op-only (default 32^3x64) or of the reference arm "
                         "(default the timed step's 16^3x32)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other forms and the 32^3x64 lines")
    ap.add_argument("--plain-sign", action="store_true",
                    help="also time W_sgn in the plain FP64 form (several minutes on 16^3x32)")
    ap.add_argument("--no-big", action="store_true", help="skip the 32^3x64 lines")
    ap.add_argument("--no-big-eig", action="store_true", help="skip the 32^3x64 low-mode solve")
    ap.add_argument("--w-mass", action="store_true", help="time one W_mass estimate (Sec. 4) instead")
    ap.add_argument("--solve", action="store_true",
                    help="time D x = b, even-odd preconditioned against the full-lattice CG, instead")
    ap.add_argument("--wm-n", type=int, default=6, help="order of the rational approximation for --w-mass")
    ap.add_argument("--wm-nsrc", type=int, default=1, help="sources per factor for --w-mass")
    args = ap.parse_args()
    if args.w_mass:
        args.workload = args.workload or WORKLOAD
        return run_w_mass(args)
    if args.solve:
        args.workload = args.workload or WORKLOAD
        return run_solve(args)
    if args.impl == "reference":
        args.workload = args.workload or WORKLOAD
        return run_reference(args)
    if args.op_only:
        args.workload = args.workload or BIG
        return run_op_only(args)
    return run_sign(args)


if __name__ == "__main__":
    main()
