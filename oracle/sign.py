"""Sign of the Pfaffian W_sgn (Sec. 3).

Three routes, all FP64 on the CPU:

1. ``sign_by_pfaffian``: the definition.  W_sgn(m0) = sign of pf[CTD(m0)] relative to
   pf[CTD(m_big)], with m_big = 3 (c_sw + c_sw,U(1)) + 1.  Reading: the paper fixes
   the overall sign by pf > 0 as m0 -> +inf (Sec. 3); D has no zero mode for
   m0 > 3 (c_sw + c_sw,U(1)) because the hopping part has norm <= 4 and the SW term
   norm <= 3 c_sw per group, so pf keeps its sign above that mass and the ratio to
   pf(m_big) is the basis-independent sign.  The ratio must be real (checked).
2. ``sign_by_eigencount``: pf[CTD] = prod_{n=1}^{12V} lambda_n (Sec. 3), one lambda per
   degenerate pair, so W_sgn = (-1)^(N_-/2) with N_- the number of negative
   eigenvalues of the dense Q counted with multiplicity.
3. ``pfaffian_sign_flow``: the mass-flow algorithm.  Step A as the enumerated
   algorithm of Sec. 3 (steps 1-5, c slightly below 2), each certification made with
   lower bounds lambda_bar - ||r||; a step that leaves the crossing-free interval
   (m - lambda_bar, m + lambda_bar) of eq. derivativebound uncovered is shortened to
   its edge (m + 0.95 (lambda_bar - r)) instead of being accepted.  Step B is not
   described in the paper (it cites other work); our reading: from the last
   certified mass, walk upward in steps dm chosen inside a spectral gap of the
   tracked window (gap between sorted |lambda|: s_i < a < s_{i+1},
   dm <= (s_{i+1} - s_i)/2 minus residual margins), and add the change of the number
   of eigenvalues in (-a, 0).  By |lambda'| <= 1 (eq. derivativebound) no eigenvalue
   outside (-a, a) can change sign in the step, and the eigenvalues inside stay
   inside, so the change of N_- is exact.  Return to step A as soon as lambda_bar
   grows again.  Step 4 also fires when m + (lambda_bar - r) > m0_max: the interval
   (m - lambda_bar, m + lambda_bar) of eq. derivativebound already covers m0_max.

Pinned by tests/test_oracle_sign.py: routes 1 and 2 agree (the theorem of
Sec. 3), sign +1 above m0_max, and the flow agrees with both on tiny lattices,
including configurations with negative signs.
"""
import numpy as np

from .pfaffian import pfaffian, pfaffian_c

UNDECIDED = 0


def m_big(cfg):
    return 3.0 * (cfg.csw_su3 + cfg.csw_u1) + 1.0


def m0_max_default(cfg):
    return 3.0 * (cfg.csw_su3 + cfg.csw_u1)


def sign_by_pfaffian(op, m0, use_c=None):
    n = op.n
    pf = pfaffian_c if (use_c or (use_c is None and n > 1000)) else pfaffian
    la, pa = pf(op.dense_CTD(m0))
    lb, pb = pf(op.dense_CTD(m_big(op.cfg)))
    r = pa / pb
    if abs(r.imag) > 1e-8:
        raise ArithmeticError(f"Pfaffian ratio is not real: {r}")
    if la == -np.inf:
        return UNDECIDED, r
    return (1 if r.real > 0 else -1), r


def negative_count(op, m0):
    return int(np.sum(np.linalg.eigvalsh(op.dense_Q(m0)) < 0))


def sign_by_eigencount(op, m0):
    nneg = negative_count(op, m0)
    assert nneg % 2 == 0
    return 1 if (nneg // 2) % 2 == 0 else -1


def _lambda_bar(modes):
    w, r = modes
    i = int(np.argmin(np.abs(w)))
    return abs(w[i]), r[i]


def pfaffian_sign_flow(modes_fn, m_target, m0_max, c=1.9, max_steps=200, min_step=1e-9):
    """W_sgn(m_target) by the mass flow.  modes_fn(m) -> (signed eigenvalues of Q(m)
    closest to zero sorted by |lambda|, their residual bounds); it must return the
    k lowest |lambda| with k >= 4.  Returns (sign, report)."""
    report = {"masses": [], "lambda_bar": [], "phase": [], "crossings": 0, "evals": 0}

    def modes(m):
        report["evals"] += 1
        w, r = modes_fn(m)
        report["masses"].append(m)
        report["lambda_bar"].append(float(np.min(np.abs(w))))
        return np.asarray(w), np.asarray(r)

    m = m_target
    cur = modes(m)
    lb, rb = _lambda_bar(cur)
    report["phase"].append("A")
    if lb - rb <= 0:
        return UNDECIDED, report
    flips = 0          # change of N_- / 2 accumulated by step B (mod 2 decides)
    steps = 0
    while steps < max_steps:
        # ---- step A (steps 1-5 of the enumerated algorithm) ----------------
        go_b = False
        while steps < max_steps:
            lb, rb = _lambda_bar(cur)
            if m > m0_max or m + (lb - rb) > m0_max:   # step 4 (or its interval covers m0_max)
                return (1 if flips % 2 == 0 else -1), report
            m_new = m + c * lb                           # step 5
            new = modes(m_new)
            report["phase"].append("A")
            steps += 1
            lb2, rb2 = _lambda_bar(new)
            covered = (lb - rb) + (lb2 - rb2) >= (m_new - m)
            if not covered:
                # the step went past the interval (m - lb, m + lb) of eq. derivativebound
                # that is free of crossings: retreat to its edge
                m_new = m + 0.95 * (lb - rb)
                new = modes(m_new)
                report["phase"].append("A")
                steps += 1
                lb2, rb2 = _lambda_bar(new)
            m, cur = m_new, new
            if lb2 < lb:                                 # step 3: lambda_bar decreases
                go_b = True
                break
        if not go_b:
            break
        # ---- step B (our reading, see module doc) --------------------------
        while steps < max_steps:
            w, r = cur
            s = np.abs(w)
            order = np.argsort(s, kind="stable")
            s, w, r = s[order], w[order], r[order]
            best_g, best_i = -1.0, -1
            for i in range(len(s) - 1):
                g = (s[i + 1] - r[i + 1]) - (s[i] + r[i])
                if g > best_g:
                    best_g, best_i = g, i
            dm = 0.5 * best_g * 0.95
            if dm < min_step:
                raise ArithmeticError("step B: no spectral gap in the tracked window")
            a = 0.5 * ((s[best_i] + r[best_i]) + (s[best_i + 1] - r[best_i + 1]))
            before = int(np.sum((w < 0) & (np.abs(w) < a)))
            lb_old = s[0]
            m = m + dm
            cur = modes(m)
            report["phase"].append("B")
            steps += 1
            w2, r2 = cur
            after = int(np.sum((w2 < 0) & (np.abs(w2) < a)))
            d = after - before
            if d % 2:
                raise ArithmeticError("step B: odd change of the negative count")
            flips += d // 2
            report["crossings"] += abs(d) // 2
            if np.min(np.abs(w2)) > lb_old:           # lambda_bar grows again: back to A
                break
    raise ArithmeticError("mass flow did not terminate")
