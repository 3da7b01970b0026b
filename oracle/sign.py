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
3. ``pfaffian_sign_flow``: the mass-flow algorithm.  Step A is the enumerated
   algorithm of Sec. 3 in its order: (1) m^(0) = m_target; (2) lambda_bar^(n); (3) if
   lambda_bar^(n) < lambda_bar^(n-1), go to step B; (4) if m^(n) > m0_max, W_sgn is the
   sign found so far; (5) m^(n+1) = m^(n) + c lambda_bar^(n), c slightly below 2.
   Finite accuracy: lambda_bar is the smallest |lambda| of the window and
   lo = min (|lambda_j| - r_j) its certified lower bound; the step m^(n) -> m^(n+1) is
   covered by the crossing-free intervals of eq. derivativebound iff
   lo^(n) + lo^(n+1) >= m^(n+1) - m^(n).  With exact eigenvalues that holds whenever
   lambda_bar does not decrease (c < 2); a step that is not covered is treated as step 3
   and step B starts from m^(n), the last mass the flow is certified up to; after a
   covered step where lambda_bar decreased, step B starts from m^(n+1).  Step 4 also
   fires when m + lo > m0_max (the interval around m already covers m0_max).
   ``retreat=True`` (an option, not the paper's algorithm): an uncovered step is first
   shortened to m^(n) + 0.95 lo^(n), the edge of the crossing-free interval around m^(n).
   Step B is not described in the paper (it cites other work); our reading: from the
   start mass, walk upward in steps dm chosen inside a spectral gap of the tracked
   window (gap between sorted |lambda|: s_i < a < s_{i+1}, dm <= (s_{i+1} - s_i)/2 minus
   residual margins), and add the change of the number of eigenvalues in (-a, 0).  By
   |lambda'| <= 1 (eq. derivativebound) no eigenvalue outside (-a, a) can change sign in
   the step, and the eigenvalues inside stay inside, so the change of N_- is exact.
   Return to step A as soon as lambda_bar grows again.

Pins (tests/test_oracle_sign.py): routes 1 and 2 agree with each other and with
the real eigenvalues of D(0) (det D(m0) = prod (mu + m0)) on a rough field with
negative signs (the theorem of Sec. 3); sign +1 above m0_max; the flow, with and
without the retreat option, reproduces the definition on that field, and its step-A
trace obeys the paper's rules (steps of exactly c lambda_bar while lambda_bar grows).
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
    """(lambda_bar, lo): the smallest |lambda| and min (|lambda_j| - r_j) of a window."""
    w, r = modes
    a = np.abs(np.asarray(w))
    return float(np.min(a)), float(np.min(a - np.asarray(r)))


def pfaffian_sign_flow(modes_fn, m_target, m0_max, c=1.9, max_steps=200, min_step=1e-9, retreat=False):
    """W_sgn(m_target) by the mass flow.  modes_fn(m) -> (signed eigenvalues of Q(m)
    closest to zero sorted by |lambda|, their residual bounds); it must return the
    k lowest |lambda| with k >= 4.  Returns (sign, report)."""
    report = {"masses": [], "lambda_bar": [], "phase": [], "crossings": 0, "evals": 0}

    def modes(m, phase):
        report["evals"] += 1
        w, r = modes_fn(m)
        report["masses"].append(m)
        report["lambda_bar"].append(float(np.min(np.abs(w))))
        report["phase"].append(phase)
        return np.asarray(w), np.asarray(r)

    m = m_target                                         # step 1
    cur = modes(m, "A")                                  # step 2
    lb, lo = _lambda_bar(cur)
    if lo <= 0:
        return UNDECIDED, report
    flips = 0          # change of N_- / 2 accumulated by step B (mod 2 decides)
    steps = 0
    while steps < max_steps:
        # ---- step A (steps 1-5 of the enumerated algorithm) ----------------
        go_b = False
        while steps < max_steps:
            lb, lo = _lambda_bar(cur)
            if m > m0_max or m + lo > m0_max:            # step 4 (or its interval covers m0_max)
                return (1 if flips % 2 == 0 else -1), report
            m_new = m + c * lb                           # step 5
            new = modes(m_new, "A")                      # step 2 at n + 1
            steps += 1
            lb2, lo2 = _lambda_bar(new)
            covered = lo + lo2 >= (m_new - m)
            if not covered:
                if not retreat:                          # step 3: B from the certified mass m
                    go_b = True
                    break
                m_new = m + 0.95 * lo                    # retreat option
                new = modes(m_new, "A")
                steps += 1
                lb2, lo2 = _lambda_bar(new)
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
            cur = modes(m, "B")
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
