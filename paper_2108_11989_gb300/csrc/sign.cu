// Sign of the Pfaffian by the mass flow (Sec. 3).  Host control flow only: every
// eigenvalue it uses comes from the GPU eigensolver with its residual bound r
// (some eigenvalue of Q lies within r of each Ritz value theta).
//
// lambda_bar at a mass is the smallest |theta| of the block and lo = min (|theta_j| - r_j)
// its certified lower bound, both over the values that carry information (the converged
// ones, and every other value with r_j <= |theta_j| / 2).
//
// Step A follows the enumerated algorithm of Sec. 3: m_{n+1} = m_n + c lambda_bar_n;
// step 3 (lambda_bar decreases) hands over to step B, step 4 (m > m0_max) ends with the
// sign found so far.  At finite accuracy the no-crossing certificate of eq.
// derivativebound (|lambda'| <= 1) is checked with lower bounds,
// lo_n + lo_{n+1} >= m_{n+1} - m_n; with exact eigenvalues and c < 2 it holds whenever
// lambda_bar does not decrease.  A step that fails it is treated as step 3: step B starts
// from m_n, the last mass up to which the flow is certified.  With the `retreat` option
// an uncertified step is instead shortened to m_n + 0.95 lo_n (the edge of the interval
// around m_n that is free of crossings), and step B starts there if lambda_bar decreased.
//
// Step B (our reading; the paper defers to other work): at mass m with tracked
// window |theta_0| <= ... (all with residual bounds), pick the widest gap between
// consecutive |theta| bounds, put a in its middle and step by dm = 0.95 * gap / 2.
// No eigenvalue can cross |lambda| = a during the step, so eigenvalues outside
// (-a, a) keep their sign and the change of N_- equals the change of the number of
// tracked eigenvalues in (-a, 0).  Each change of N_- by 2 (a degenerate pair) flips
// the sign.  Back to step A as soon as lambda_bar grows again.
#include "blas.cuh"

#include <nvtx3/nvToolsExt.h>

#include <math.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <thread>
#include <vector>


extern "C" void qs_sign_default_opts(qs_sign_opts *o)
{
    if (!o) return;
    o->c = 1.9;
    o->m0_max = 0.0;
    o->max_steps = 400;
    o->step_model = nullptr;
    o->window_trace = nullptr;
    o->retreat = 0;
    o->log_path = nullptr;
    o->checkpoint_path = nullptr;
    o->resume = 0;
    qs_eig_default_opts(&o->eig);
    // certificates carry the residual bound r, so any r < |theta| is rigorous; a
    // moderate relative accuracy keeps every mass point cheap
    o->eig.tol = 1e-5;
}

cudaStream_t qs_mlp_stream(const qs_mlp *n);

namespace {

struct Window {
    double v[QS_WINDOW];
};

struct Flow {
    int nb;            // step-B prefix size (values that must converge)
    std::vector<Window> hist;   // windows of the step-A masses, oldest first
    float *dX, *dY;    // device buffers of the step model (features, outputs)
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

// lambda_bar (smallest |theta|) and its certified lower bound min (|theta_j| - r_j) over
// the values of the block that carry information: the nwant converged ones and every
// other value with r_j <= |theta_j| / 2 (larger residuals belong to unconverged mixtures).
// The solver orders the block by theta^2 + r^2, so the smallest lower bound need not
// belong to theta[0].
void lambda_bar(const Ritz &rz, int k, int nwant, double *lb, double *lo)
{
    double b = 1e300, l = 1e300;
    for (int j = 0; j < k; ++j) {
        const double t = fabs(rz.theta[j]), r = rz.res[j];
        if (j < nwant || r <= 0.5 * t) {
            b = std::min(b, t);
            l = std::min(l, t - r);
        }
    }
    *lb = b;
    *lo = l;
}

int modes(Flow &f, double m, char phase, Ritz *rz)
{
    qs_eig_opts e = f.o.eig;
    // the first mass starts as the caller asks (cold or from the handle's last
    // subspace); every later mass starts from the previous one
    if (f.rep->n > 0) e.warm_start = 1;
    // step B converges a prefix of k/2 Ritz values; the rest of the block are guard
    // vectors whose Ritz values enter only through their residual bounds
    if (phase == 'B') {
        e.nwant = std::max(e.nwant, f.nb);
        // the counts only need bounds that separate at the gap
        e.tol = std::max(e.tol, 1e-4);
    }
    int conv = 0;
    qs_eig_stats st;
    memset(&st, 0, sizeof(st));
    char label[64];
    snprintf(label, sizeof(label), "modes %c m=%.6f", phase, m);
    nvtxRangePushA(label);
    int s = qs_lowmodes_impl(f.lat, m, &e, rz, &conv, &st);
    nvtxRangePop();
    if (s != QS_OK) { f.rep->fail_reason = 1; return s; }
    qs_sign_report *r = f.rep;
    r->dslash_f32 += st.dslash_f32;
    r->dslash_f64 += st.dslash_f64;
    r->cg_iterations += st.cg_iterations;
    double lb, lo;
    lambda_bar(*rz, e.k, e.nwant, &lb, &lo);
    if (r->n < QS_TRACE_MAX) {
        r->mass[r->n] = m;
        r->lambda_bar[r->n] = lb;
        r->resid[r->n] = lb - lo;
        r->phase[r->n] = phase;
    }
    if (f.o.log_path) {   // one JSON line per mass visited, appended
        FILE *fp = fopen(f.o.log_path, "a");
        if (fp) {
            fprintf(fp,
                    "{\"step\": %d, \"mass\": %.17g, \"phase\": \"%c\", \"lambda_bar\": %.17g, "
                    "\"lower_bound\": %.17g, \"converged\": %d, \"dslash_f32\": %lld, \"dslash_f64\": %lld, "
                    "\"cg_iterations\": %lld, \"seconds\": %.6f}\n",
                    r->n, m, phase, lb, lo, conv, (long long)st.dslash_f32, (long long)st.dslash_f64,
                    (long long)st.cg_iterations, now_s() - f.t0);
            fclose(fp);
        }
    }
    if (f.o.window_trace && r->n < f.o.max_steps)
        for (int i = 0; i < QS_WINDOW; ++i)
            f.o.window_trace[(size_t)r->n * QS_WINDOW + i] = i < e.k ? rz->theta[i] : 0.0;
    r->n++;
    if (phase == 'A') r->steps_a++; else r->steps_b++;
    if (!conv) r->fail_reason = 1;
    return conv ? QS_OK : QS_ENOCONV;
}

Window window_of(const Ritz &rz, int k)
{
    Window w;
    for (int i = 0; i < QS_WINDOW; ++i) w.v[i] = i < k ? rz.theta[i] : 0.0;
    return w;
}

// dm proposed by the step model from the last 8 step-A windows (newest first,
// divided by the newest lambda_bar), clamped to [c lb, 8 lb]: a proposal can only
// lengthen the plain step of Sec. 3, never shorten it
int propose(Flow &f, double lb, double *dm)
{
    float x[8 * QS_WINDOW];
    int nh = (int)f.hist.size();
    for (int j = 0; j < 8; ++j)
        for (int i = 0; i < QS_WINDOW; ++i)
            x[j * QS_WINDOW + i] = j < nh ? (float)(f.hist[nh - 1 - j].v[i] / lb) : 0.f;
    // the network may run on another stream than the lattice: order the copies by
    // synchronising each stream before the next one uses the data
    cudaStream_t st = f.lat->stream, ns = qs_mlp_stream(f.o.step_model);
    QS_CUDA(cudaMemcpyAsync(f.dX, x, sizeof(x), cudaMemcpyHostToDevice, st));
    QS_CUDA(cudaStreamSynchronize(st));
    QS_TRY(qs_mlp_forward(f.o.step_model, f.dX, 1, f.dY));
    QS_CUDA(cudaStreamSynchronize(ns));
    float y0 = 0.f;
    QS_CUDA(cudaMemcpy(&y0, f.dY, sizeof(float), cudaMemcpyDeviceToHost));
    double ly = std::min(std::max((double)y0, log(f.o.c)), log(8.0));
    *dm = lb * exp(ly);
    return QS_OK;
}

// ---- checkpoint of the flow at a certified mass -----------------------------------------
struct Checkpoint {
    double m_target, m, csw_su3, csw_u1;
    long flips;
    int crossings, steps, L, T, cstar_y, cstar_z, t_anti;
};

bool write_checkpoint(const char *path, const Checkpoint &c)
{
    char tmp[4096];
    if (snprintf(tmp, sizeof(tmp), "%s.tmp", path) >= (int)sizeof(tmp)) return false;
    FILE *fp = fopen(tmp, "w");
    if (!fp) return false;
    const int n = fprintf(fp,
                          "{\"qstar_sign_checkpoint\": 1, \"m_target\": %.17g, \"m\": %.17g, \"flips\": %ld, "
                          "\"crossings\": %d, \"steps\": %d, \"L\": %d, \"T\": %d, \"cstar_y\": %d, "
                          "\"cstar_z\": %d, \"t_anti\": %d, \"csw_su3\": %.17g, \"csw_u1\": %.17g}\n",
                          c.m_target, c.m, c.flips, c.crossings, c.steps, c.L, c.T, c.cstar_y, c.cstar_z, c.t_anti,
                          c.csw_su3, c.csw_u1);
    const bool ok = n > 0 && fflush(fp) == 0;
    if (fclose(fp) != 0 || !ok) { remove(tmp); return false; }
    return rename(tmp, path) == 0;
}

// the number after "key": in a one-object JSON text; false if the key is missing
bool json_number(const char *txt, const char *key, double *v)
{
    char pat[64];
    snprintf(pat, sizeof(pat), "\"%s\":", key);
    const char *p = strstr(txt, pat);
    if (!p) return false;
    char *end = nullptr;
    *v = strtod(p + strlen(pat), &end);
    return end != p + strlen(pat);
}

bool read_checkpoint(const char *path, Checkpoint *c)
{
    FILE *fp = fopen(path, "r");
    if (!fp) return false;
    char txt[2048];
    const size_t n = fread(txt, 1, sizeof(txt) - 1, fp);
    fclose(fp);
    txt[n] = 0;
    double v[13];
    const char *keys[13] = {"qstar_sign_checkpoint", "m_target", "m", "flips", "crossings", "steps", "L", "T",
                            "cstar_y", "cstar_z", "t_anti", "csw_su3", "csw_u1"};
    for (int i = 0; i < 13; ++i)
        if (!json_number(txt, keys[i], &v[i])) return false;
    if (v[0] != 1) return false;
    c->m_target = v[1];
    c->m = v[2];
    c->flips = (long)v[3];
    c->crossings = (int)v[4];
    c->steps = (int)v[5];
    c->L = (int)v[6];
    c->T = (int)v[7];
    c->cstar_y = (int)v[8];
    c->cstar_z = (int)v[9];
    c->t_anti = (int)v[10];
    c->csw_su3 = v[11];
    c->csw_u1 = v[12];
    return true;
}

Checkpoint state_of(const Flow &f, double m_target, double m, long flips)
{
    Checkpoint c;
    c.m_target = m_target;
    c.m = m;
    c.flips = flips;
    c.crossings = f.rep->crossings;
    c.steps = f.steps;
    c.L = f.lat->g.L;
    c.T = f.lat->g.T;
    c.cstar_y = f.lat->g.cstar_y;
    c.cstar_z = f.lat->g.cstar_z;
    c.t_anti = f.lat->g.t_anti;
    c.csw_su3 = f.lat->csw_su3;
    c.csw_u1 = f.lat->csw_u1;
    return c;
}

bool same_problem(const Checkpoint &a, const Checkpoint &b)
{
    return a.m_target == b.m_target && a.L == b.L && a.T == b.T && a.cstar_y == b.cstar_y &&
           a.cstar_z == b.cstar_z && a.t_anti == b.t_anti && a.csw_su3 == b.csw_su3 && a.csw_u1 == b.csw_u1;
}

}  // namespace

extern "C" int qs_block_bounds(const double *theta, const double *res, int k, int nwant, double *lb, double *lo)
{
    if (!theta || !res || !lb || !lo || k < 1 || k > 64) return QS_EINVAL;
    Ritz rz;
    for (int j = 0; j < k; ++j) { rz.theta[j] = theta[j]; rz.res[j] = res[j]; }
    lambda_bar(rz, k, nwant, lb, lo);
    return QS_OK;
}

extern "C" int qs_pfaffian_sign(qs_lattice *lat, double m_target, const qs_sign_opts *opts, int *sign,
                                qs_sign_report *report)
{
    if (!lat || !sign) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    qs_sign_report local;
    qs_sign_report *rep = report ? report : &local;
    memset(rep, 0, sizeof(*rep));
    Flow f;
    f.lat = lat;
    if (opts) f.o = *opts; else qs_sign_default_opts(&f.o);
    if (!(f.o.c > 0 && f.o.c < 2) || f.o.eig.k < 4 || f.o.max_steps < 1) return QS_EINVAL;
    f.rep = rep;
    f.steps = 0;
    f.nb = 2;
    f.dX = f.dY = nullptr;
    if (f.o.step_model) {
        if (cudaMalloc(&f.dX, 8 * QS_WINDOW * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&f.dY, 64 * sizeof(float)) != cudaSuccess) {
            cudaFree(f.dX);
            return QS_ENOMEM;
        }
    }
    f.t0 = now_s();
    nvtxRangePushA("qs_pfaffian_sign");
    const double m0max = f.o.m0_max > 0 ? f.o.m0_max : 3.0 * (lat->csw_su3 + lat->csw_u1);
    int st;
    auto finish = [&](int status) {
        nvtxRangePop();
        rep->seconds = now_s() - f.t0;
        cudaFree(f.dX);
        cudaFree(f.dY);
        return status;
    };

    double m = m_target;
    long flips = 0;
    rep->resumed_from = m_target;
    if (f.o.resume && f.o.checkpoint_path) {
        // continue from the certified mass of an earlier run on the same problem
        Checkpoint c;
        if (read_checkpoint(f.o.checkpoint_path, &c) && same_problem(c, state_of(f, m_target, m, 0))) {
            m = c.m;
            rep->resumed_from = m;
            flips = c.flips;
            rep->crossings = c.crossings;
            f.steps = c.steps;
        }
    }
    auto checkpoint = [&]() {
        if (f.o.checkpoint_path && !write_checkpoint(f.o.checkpoint_path, state_of(f, m_target, m, flips)))
            rep->checkpoint_errors++;
    };
    const int kk = f.o.eig.k, nw = f.o.eig.nwant;
    Ritz cur;
    st = modes(f, m, 'A', &cur);
    if (st != QS_OK) return finish(st);
    {
        double lb0, lo0;
        lambda_bar(cur, kk, nw, &lb0, &lo0);
        if (!(lo0 > 0)) { rep->fail_reason = 6; return finish(QS_EUNDECIDED); }
    }
    checkpoint();
    while (f.steps < f.o.max_steps) {
        // ---- step A -------------------------------------------------------------
        bool go_b = false;
        while (f.steps < f.o.max_steps) {
            double lb, lo;
            lambda_bar(cur, kk, nw, &lb, &lo);
            if (!(lo > 0)) { rep->fail_reason = 6; return finish(QS_EUNDECIDED); }
            // step 4; also stop once the no-crossing interval (m - lo, m + lo) of
            // eq. derivativebound already reaches past m0_max
            if (m > m0max || m + lo > m0max) {
                *sign = (flips % 2 == 0) ? 1 : -1;
                return finish(QS_OK);
            }
            f.hist.push_back(window_of(cur, kk));
            double mn = m + f.o.c * lb;              // step 5
            bool learned = false;
            if (f.o.step_model) {
                double dm = 0;
                st = propose(f, lb, &dm);
                if (st != QS_OK) return finish(st);
                mn = m + dm;
                learned = true;
            }
            Ritz nw_r;
            st = modes(f, mn, 'A', &nw_r);
            if (st != QS_OK) return finish(st);
            ++f.steps;
            double lb2, lo2;
            lambda_bar(nw_r, kk, nw, &lb2, &lo2);
            bool certified = lo + lo2 >= (mn - m);
            if (learned) { if (certified) rep->learned_accepted++; else rep->learned_rejected++; }
            if (learned && !certified) {
                // the plain rule is the fallback: take the step of Sec. 3 instead
                mn = m + f.o.c * lb;
                st = modes(f, mn, 'A', &nw_r);
                if (st != QS_OK) return finish(st);
                ++f.steps;
                lambda_bar(nw_r, kk, nw, &lb2, &lo2);
                certified = lo + lo2 >= (mn - m);
            }
            if (!certified) {
                // With exact eigenvalues and c < 2 this happens only when lambda_bar
                // decreased, i.e. at step 3.  The flow is certified up to m: step B
                // starts there (cur is still the window at m).
                if (!f.o.retreat) { go_b = true; break; }
                // retreat option: shorten the step to the edge of the crossing-free
                // interval around m instead
                mn = m + 0.95 * lo;
                st = modes(f, mn, 'A', &nw_r);
                if (st != QS_OK) return finish(st);
                ++f.steps;
                lambda_bar(nw_r, kk, nw, &lb2, &lo2);
            }
            m = mn;
            cur = nw_r;
            if (lo2 > 0) checkpoint();   // a certified mass from which step A can restart
            if (lb2 < lb) { go_b = true; break; }   // step 3: lambda_bar decreases
        }
        if (!go_b) break;
        // ---- step B -------------------------------------------------------------
        // The window is the whole block; every Ritz value t_i stands for an
        // eigenvalue in [t_i - r_i, t_i + r_i].  The step dm is taken inside a gap
        // (a - g, a + g) of the |lambda| bounds, g >= dm: either between two values of
        // the converged prefix (sorted by |theta|) or above the prefix, below the lower
        // bounds of all other Ritz values.  Then no eigenvalue crosses |lambda| = a in
        // the step (|lambda'| <= 1), and the change of N_- is the change of the number
        // of values certainly in (-a, 0).  A value whose bounds straddle a at the new
        // mass leaves the step uncertified (QS_ENOCONV).  Values are counted over the
        // converged prefix (ended at a gap of the window); for the gap above it the guard
        // values beyond it must lie certainly above a at both masses.
        // prefix size: end the prefix at the widest relative gap of the window, among
        // sizes 2 .. 3k/4, so it never cuts into a cluster
        auto pick_prefix = [&](const Ritz &rz) {
            // q_i = sqrt(theta_i^2 + r_i^2) = ||Q v_i||, the order the window is kept in:
            // close to |lambda| for converged values, large for unconverged ones
            int best_n = std::max(2, f.o.eig.nwant);
            double best_g = -1e300;
            for (int n = std::max(2, f.o.eig.nwant); n <= (3 * kk) / 4; n += 2) {
                double qa = hypot(rz.theta[n - 1], rz.res[n - 1]), qb = hypot(rz.theta[n], rz.res[n]);
                double g = (qb - qa) / (qb + 1e-300);
                if (g > best_g) { best_g = g; best_n = n; }
            }
            return best_n;
        };
        f.nb = pick_prefix(cur);
        int nb = f.nb;
        // the window at the start mass m was solved for step A (few values converged):
        // solve it again (warm) for the step-B prefix
        st = modes(f, m, 'B', &cur);
        if (st != QS_OK) return finish(st);
        while (f.steps < f.o.max_steps) {
            int idx[64];
            for (int i = 0; i < nb; ++i) idx[i] = i;
            std::sort(idx, idx + nb, [&](int x, int y) { return fabs(cur.theta[x]) < fabs(cur.theta[y]); });
            // lowest lower bound among the guard values (the block beyond the prefix);
            // guards with r > |theta| / 2 are unconverged mixtures that say nothing about
            // where the next eigenvalue lies and are skipped
            auto guard_low = [&](const Ritz &rz) {
                double lo = 1e300;
                int any = 0;
                for (int j = nb; j < kk; ++j)
                    if (rz.res[j] <= 0.5 * fabs(rz.theta[j])) { lo = std::min(lo, fabs(rz.theta[j]) - rz.res[j]); any = 1; }
                return any ? lo : -1e300;
            };
            double guard_lo = guard_low(cur);
            double best = -1, a = 0;
            int above_gap = 0;
            // inner gaps: a prefix value above a already bounds (block containing the
            // lowest eigenvalues) every eigenvalue outside the prefix from below
            for (int q = 0; q + 1 < nb; ++q) {
                int i = idx[q], j = idx[q + 1];
                double lo = fabs(cur.theta[i]) + cur.res[i], hi = fabs(cur.theta[j]) - cur.res[j];
                if (hi - lo > best) { best = hi - lo; a = 0.5 * (lo + hi); above_gap = 0; }
            }
            // the gap above the prefix needs the guard values' lower bounds
            {
                double lo = fabs(cur.theta[idx[nb - 1]]) + cur.res[idx[nb - 1]];
                if (guard_lo - lo > best) { best = guard_lo - lo; a = 0.5 * (lo + guard_lo); above_gap = 1; }
            }
            double dm = 0.5 * best * 0.95;
            if (!(dm > 1e-13)) { rep->fail_reason = 2; return finish(QS_ENOCONV); }
            // count over the converged prefix.  *ok: for an inner gap some prefix value
            // lies certainly above a; for the gap above the prefix every guard value does
            auto count_below = [&](const Ritz &rz, int *neg, int *straddle, int *ok) {
                *neg = 0; *straddle = 0;
                int pre_above = 0, guards_above = 1;
                for (int i = 0; i < nb; ++i) {
                    double t = fabs(rz.theta[i]), r = rz.res[i];
                    if (t + r < a) *neg += rz.theta[i] < 0;
                    else if (t - r <= a) ++*straddle;
                    else pre_above = 1;
                }
                if (!(guard_low(rz) > a)) guards_above = 0;
                *ok = above_gap ? guards_above : pre_above;
            };
            int before, sb, ab, after = 0, sa = 0, aa = 0;
            count_below(cur, &before, &sb, &ab);
            if (sb || !ab) { rep->fail_reason = 3; return finish(QS_ENOCONV); }
            double lb_old, lo_old;
            lambda_bar(cur, kk, nb, &lb_old, &lo_old);
            const double m_prev = m;
            for (int tries = 0;; ++tries) {
                m = m_prev + dm;
                st = modes(f, m, 'B', &cur);
                if (st != QS_OK) return finish(st);
                ++f.steps;
                count_below(cur, &after, &sa, &aa);
                if (!sa && aa) break;
                // the count at the new mass is not certified (a value's bounds straddle
                // a, or the window no longer bounds everything above a).  The gap at
                // m_prev rules out a crossing of a for every shorter step too: halve it
                if (tries == 3 || f.steps >= f.o.max_steps) { rep->fail_reason = 3; return finish(QS_ENOCONV); }
                dm *= 0.5;
            }
            int d = after - before;
            if (d % 2) { rep->fail_reason = 4; return finish(QS_ENUMERIC); }   // pairs must stay paired
            flips += d / 2;
            rep->crossings += abs(d) / 2;
            double lb_new, lo_new;
            lambda_bar(cur, kk, nb, &lb_new, &lo_new);
            if (lb_new > lb_old) break;  // lambda_bar grows again: step A
            f.nb = nb = pick_prefix(cur);
        }
    }
    rep->fail_reason = 5;
    return finish(QS_ENOCONV);
}

// The batched form: the flows of several configurations are independent (Sec. 3: the
// algorithm is run on each configuration), each with its own sequence of masses, so they
// run concurrently -- one host thread per configuration, each on its handle's stream --
// and the GPU executes their kernels side by side.
extern "C" int qs_pfaffian_sign_batch(qs_lattice *const *lats, int n, const double *m0_targets,
                                      const qs_sign_opts *opts, int *signs, int *status, qs_sign_report *reports)
{
    if (!lats || n < 1 || !m0_targets || !signs || !status) return QS_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!lats[i] || !lats[i]->gauge_loaded) return QS_EINVAL;
        for (int j = 0; j < i; ++j)
            if (lats[j] == lats[i]) return QS_EINVAL;   // a handle serves one flow at a time
    }
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i)
        th.emplace_back([=] {
            status[i] = qs_pfaffian_sign(lats[i], m0_targets[i], opts, &signs[i], reports ? &reports[i] : nullptr);
        });
    for (auto &t : th) t.join();
    for (int i = 0; i < n; ++i)
        if (status[i] != QS_OK) return status[i];
    return QS_OK;
}
