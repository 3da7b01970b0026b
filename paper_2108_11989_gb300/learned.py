"""Training data and training loop of the step-proposal network.

Samples come from the sign flows the library itself runs (report["windows"] with
trace=True): for every step-A move from mass m_i to m_{i+1} the features are the
windows of the step-A masses up to m_i (newest first, 8 of them, divided by
lambda_bar(m_i), zero where missing) -- the same features qs_pfaffian_sign builds
for its proposals -- and the targets are
  y0 = log(dm* / lambda_bar_i), dm* = 0.95 ((lb_i - r_i) + (lb_{i+1} - r_{i+1})),
the longest step the no-crossing certificate of the observed pair would have
accepted, and, for each of the 24 window slots j, whether the signed value in slot j
changed sign between the two masses.  So T has 1 + 24 = 25 columns, the output width
of the step network.
"""
import numpy as np

WINDOW = 24
HIST = 8
N_IN = HIST * WINDOW     # network inputs: 8 windows of 24 scaled eigenvalues
N_OUT = 1 + WINDOW       # network outputs: log step + one crossing logit per slot


def samples_from_flow(report):
    """(X [n][8*24], T [n][1 + 24]) float32 from one flow report with windows."""
    W = report["windows"]
    ph = report["phase"]
    m = np.asarray(report["mass"])
    lb = np.asarray(report["lambda_bar"])
    r = np.asarray(report["resid"])
    a_idx = [i for i in range(len(ph)) if ph[i] == "A"]
    X, T = [], []
    for q in range(len(a_idx) - 1):
        i, j = a_idx[q], a_idx[q + 1]
        if j != i + 1 or not m[j] > m[i]:
            continue
        hist = [W[a_idx[p]] for p in range(q, max(-1, q - HIST), -1)]
        x = np.zeros((HIST, WINDOW))
        for h, w in enumerate(hist):
            x[h] = w / lb[i]
        dm = 0.95 * ((lb[i] - r[i]) + (lb[j] - r[j]))
        if not dm > 0:
            continue
        t = np.zeros(N_OUT)
        t[0] = np.log(dm / lb[i])
        t[1:] = (np.sign(W[i][:WINDOW]) * np.sign(W[j][:WINDOW]) < 0).astype(float)
        X.append(x.ravel())
        T.append(t)
    if not X:
        return np.zeros((0, N_IN), np.float32), np.zeros((0, N_OUT), np.float32)
    return np.asarray(X, np.float32), np.asarray(T, np.float32)


def train(net, X, T, steps=400, lr=2e-3, batch=256, seed=0):
    """Adam on random mini-batches, every step through qs_mlp_train_step; returns losses."""
    import torch
    rng = np.random.default_rng(seed)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    losses = []
    for _ in range(steps):
        idx = torch.from_numpy(rng.integers(0, len(X), size=min(batch, len(X)))).cuda()
        losses.append(net.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), lr))
    return losses


def run_study(train_L=8, train_T=16, flows=200, eval_L=16, eval_T=32, eval_configs=4, steps=600, seed=0,
              kappas=(0.1345, 0.135, 0.1355), out=None, log=print):
    """Train the step network on flows the library computes and measure what it gains.

    Training flows: `flows` synthetic fields of train_L^3 x train_T with the link
    distribution of the 16^3 x 32 workload (SU(3) exp(i 0.2 H), U(1) N(0, 0.3^2), c_sw 1.9
    / 1.0), seeds 1000 + i, target masses cycling through `kappas`.  Evaluation:
    `eval_configs` held-out fields of eval_L^3 x eval_T (seeds 5000 + j) at kappa = 0.135,
    each flow run plainly and with the network; the signs must agree and the report gives
    masses visited and seconds per configuration for both.  Returns a dict."""
    import time

    import torch

    import paper_2108_11989_gb300 as qs
    from synth_inputs import kappa_to_m0, make_config, mlp_init

    field = dict(eps=0.2, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0)
    opts = qs.sign_default_opts(eig={"k": 32, "nwant": 2, "tol": 1e-5, "cheb_degree": 48, "precision": 2})
    stream = torch.cuda.Stream()
    Xs, Ts, t0 = [], [], time.perf_counter()
    for i in range(flows):
        cfg = make_config(T=train_T, L=train_L, seed=1000 + i, **field)
        lat = qs.Lattice(cfg.L, cfg.T, stream=stream)
        lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
        try:
            _, rep = lat.pfaffian_sign(kappa_to_m0(kappas[i % len(kappas)]), opts, trace=True)
            X, T = samples_from_flow(rep)
            Xs.append(X)
            Ts.append(T)
        except qs.QStarError as e:
            log(f"[learned] training flow {i}: {e} (fail_reason {getattr(e, 'report', {}).get('fail_reason')})")
        lat.close()
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    t_gen = time.perf_counter() - t0
    log(f"[learned] {len(X)} samples from {flows} flows in {t_gen:.1f} s")
    net = qs.MLP(N_IN, 128, N_OUT, max_batch=1024, stream=stream)
    net.set_params(mlp_init(seed, N_IN, 128, N_OUT))
    t0 = time.perf_counter()
    losses = train(net, X, T, steps=steps, lr=2e-3, batch=512, seed=seed)
    t_train = time.perf_counter() - t0
    log(f"[learned] loss {losses[0]:.3f} -> {losses[-1]:.3f} in {t_train:.1f} s")
    rows = []
    for j in range(eval_configs):
        cfg = make_config(T=eval_T, L=eval_L, seed=5000 + j, **field)
        lat = qs.Lattice(cfg.L, cfg.T, stream=stream)
        lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
        m = kappa_to_m0(0.135)
        res = {}
        for name, model in (("plain", None), ("learned", net)):
            stream.synchronize()
            t1 = time.perf_counter()
            try:
                s, rep = lat.pfaffian_sign(m, opts, step_model=model)
                res[name] = {"sign": s, "masses": rep["n"], "s": time.perf_counter() - t1,
                             "accepted": rep["learned_accepted"], "rejected": rep["learned_rejected"]}
            except qs.QStarError as e:
                rep = getattr(e, "report", {})
                res[name] = {"error": str(e), "fail_reason": rep.get("fail_reason"), "masses": rep.get("n"),
                             "s": time.perf_counter() - t1}
            stream.synchronize()
        rows.append(res)
        log(f"[learned] eval {j}: {res}")
        lat.close()
    ok = [r for r in rows if "sign" in r["plain"] and "sign" in r["learned"]]
    plain_n = sum(r["plain"]["masses"] for r in ok)
    learned_n = sum(r["learned"]["masses"] for r in ok)
    out_d = {"train": {"lattice": f"{train_L}^3x{train_T}", "flows": flows, "samples": int(len(X)),
                       "kappas": list(kappas), "s_flows": t_gen, "s_train": t_train,
                       "loss_first": float(losses[0]), "loss_last": float(losses[-1]), "adam_steps": steps},
             "eval": {"lattice": f"{eval_L}^3x{eval_T}", "configs": eval_configs, "rows": rows,
                      "completed_both": len(ok), "masses_plain": plain_n, "masses_learned": learned_n,
                      "s_plain": sum(r["plain"]["s"] for r in ok),
                      "s_learned": sum(r["learned"]["s"] for r in ok),
                      "signs_identical": all(r["plain"]["sign"] == r["learned"]["sign"] for r in ok)}}
    net.close()
    if out:
        import json
        with open(out, "w") as f:
            json.dump(out_d, f, indent=1)
    return out_d


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the step network on library flows and measure its gain")
    ap.add_argument("--flows", type=int, default=200)
    ap.add_argument("--train-lattice", default="8x16", help="L x T of the training fields")
    ap.add_argument("--eval-lattice", default="16x32", help="L x T of the held-out fields")
    ap.add_argument("--eval-configs", type=int, default=4)
    ap.add_argument("--steps", type=int, default=600, help="Adam steps")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    tl, tt = (int(v) for v in a.train_lattice.split("x"))
    el, et = (int(v) for v in a.eval_lattice.split("x"))
    r = run_study(tl, tt, a.flows, el, et, a.eval_configs, a.steps, out=a.out)
    print(json.dumps(r["eval"] | {"train": r["train"]}))
