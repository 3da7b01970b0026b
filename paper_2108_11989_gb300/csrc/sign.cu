// Sign of the Pfaffian by the mass flow (Sec. 3).  Host control flow only: every
// eigenvalue it uses comes from the GPU eigensolver with its residual bound r
// (some eigenvalue of Q lies within r of each Ritz value theta).
//
// Step A follows the enumerated algorithm of Sec. 3: m_{n+1} = m_n + c lambda_bar_n;
// stop for step B when lambda_bar decreases, stop with the sign once m > m0_max.
// The no-crossing certificate of eq. derivativebound (|lambda'| <= 1) is checked
// with lower bounds: (lb_n - r_n) + (lb_{n+1} - r_{n+1}) >= m_{n+1} - m_n.
//
// Step B (our reading; the paper defers to other work): at mass m with tracked
// window |theta_0| <= ... (all with residual bounds), pick the widest gap between
// consecutive |theta| bounds, put a in its middle and step by dm = 0.95 * gap / 2.
// No eigenvalue can cross |lambda| = a during the step, so eigenvalues outside
// (-a, a) keep their sign and the change of N_- equals the change of the number of
// tracked eigenvalues in (-a, 0).  Each change of N_- by 2 (a degenerate pair) flips
// the sign.  Back to step A as soon as lambda_bar grows again.
#include "blas.cuh"

#include <math.h>
#include <string.h>
#include <time.h>

#include <algorithm>


extern "C" void qs_sign_default_opts(qs_sign_opts *o)
{
    if (!o) return;
    o->c = 1.9;
    o->m0_max = 0.0;
    o->max_steps = 400;
    qs_eig_default_opts(&o->eig);
    // certificates carry the residual bound r, so any r < |theta| is rigorous; a
    // moderate relative accuracy keeps every mass point cheap
    o->eig.tol = 1e-5;
}

namespace {

struct Flow {
    qs_lattice *lat;
    qs_sign_opts o;
    qs_sign_report *rep;
    int steps;
    double t0;
};

double now_s()
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

int modes(Flow &f, double m, char phase, Ritz *rz)
{
    qs_eig_opts e = f.o.eig;
    e.warm_start = 1;
    // step B reads the whole window, but only through residual bounds: the gap it
    // steps in lies between bounds s_i + r_i and s_{i+1} - r_{i+1}, so Ritz values far
    // from convergence just make that gap narrower; only the leading ones must converge
    if (phase == 'B' && e.nwant < 4) e.nwant = 4 < e.k - 2 ? 4 : e.k - 2;
    int conv = 0;
    qs_eig_stats st;
    memset(&st, 0, sizeof(st));
    int s = qs_lowmodes_impl(f.lat, m, &e, rz, &conv, &st);
    if (s != QS_OK) return s;
    qs_sign_report *r = f.rep;
    r->dslash_f32 += st.dslash_f32;
    r->dslash_f64 += st.dslash_f64;
    r->cg_iterations += st.cg_iterations;
    if (r->n < QS_TRACE_MAX) {
        r->mass[r->n] = m;
        r->lambda_bar[r->n] = fabs(rz->theta[0]);
        r->resid[r->n] = rz->res[0];
        r->phase[r->n] = phase;
    }
    r->n++;
    if (phase == 'A') r->steps_a++; else r->steps_b++;
    return conv ? QS_OK : QS_ENOCONV;
}

}  // namespace

extern "C" int qs_pfaffian_sign(qs_lattice *lat, double m_target, const qs_sign_opts *opts, int *sign,
                                qs_sign_report *report)
{
    if (!lat || !sign) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    qs_sign_report local;
    qs_sign_report *rep = report ? report : &local;
    memset(rep, 0, sizeof(*rep));
    Flow f;
    f.lat = lat;
    if (opts) f.o = *opts; else qs_sign_default_opts(&f.o);
    if (!(f.o.c > 0 && f.o.c < 2) || f.o.eig.k < 4 || f.o.max_steps < 1) return QS_EINVAL;
    f.rep = rep;
    f.steps = 0;
    f.t0 = now_s();
    const double m0max = f.o.m0_max > 0 ? f.o.m0_max : 3.0 * (lat->csw_su3 + lat->csw_u1);
    const int kw = f.o.eig.k - 2;   // tracked window in step B
    int st;
    auto finish = [&](int status) {
        rep->seconds = now_s() - f.t0;
        return status;
    };

    double m = m_target;
    Ritz cur, prev_r;
    st = modes(f, m, 'A', &cur);
    if (st != QS_OK) return finish(st);
    if (fabs(cur.theta[0]) - cur.res[0] <= 0) return finish(QS_EUNDECIDED);
    long flips = 0;
    while (f.steps < f.o.max_steps) {
        // ---- step A -------------------------------------------------------------
        int n = 0;
        bool go_b = false;
        double pm = m, plb = 0, prb = 0;
        while (f.steps < f.o.max_steps) {
            double lb = fabs(cur.theta[0]), rb = cur.res[0];
            if (n >= 1) {
                bool covered = (plb - prb) + (lb - rb) >= (m - pm);
                if (lb < plb || !covered) {          // step 3, or the certificate fails
                    go_b = true;
                    if (!covered) { m = pm; cur = prev_r; }
                    break;
                }
            }
            // step 4; also stop once the no-crossing interval (m - lb, m + lb) of
            // eq. derivativebound already reaches past m0_max
            if (m > m0max || m + (lb - rb) > m0max) {
                *sign = (flips % 2 == 0) ? 1 : -1;
                return finish(QS_OK);
            }
            pm = m; prev_r = cur; plb = lb; prb = rb;
            m = m + f.o.c * lb;                      // step 5
            st = modes(f, m, 'A', &cur);
            if (st != QS_OK) return finish(st);
            ++n;
            ++f.steps;
        }
        if (!go_b) break;
        // ---- step B -------------------------------------------------------------
        while (f.steps < f.o.max_steps) {
            double s[64], r[64];
            for (int i = 0; i < kw; ++i) { s[i] = fabs(cur.theta[i]); r[i] = cur.res[i]; }
            double best = -1;
            int bi = -1;
            for (int i = 0; i + 1 < kw; ++i) {
                double g = (s[i + 1] - r[i + 1]) - (s[i] + r[i]);
                if (g > best) { best = g; bi = i; }
            }
            double dm = 0.5 * best * 0.95;
            if (bi < 0 || !(dm > 1e-13)) return finish(QS_ENOCONV);
            double a = 0.5 * ((s[bi] + r[bi]) + (s[bi + 1] - r[bi + 1]));
            int before = 0;
            for (int i = 0; i < kw; ++i) before += (cur.theta[i] < 0 && fabs(cur.theta[i]) < a);
            double lb_old = s[0];
            m += dm;
            st = modes(f, m, 'B', &cur);
            if (st != QS_OK) return finish(st);
            ++f.steps;
            int after = 0;
            for (int i = 0; i < kw; ++i) after += (cur.theta[i] < 0 && fabs(cur.theta[i]) < a);
            int d = after - before;
            if (d % 2) return finish(QS_ENUMERIC);   // the degenerate pairs must stay paired
            flips += d / 2;
            rep->crossings += abs(d) / 2;
            if (fabs(cur.theta[0]) > lb_old) break;  // lambda_bar grows again: step A
        }
    }
    return finish(QS_ENOCONV);
}
