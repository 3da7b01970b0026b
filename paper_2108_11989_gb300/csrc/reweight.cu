// Mass reweighting and the even-odd preconditioned solve (Sec. 4).
//
// qs_ratapprox: the (n, n) rational function R(y) = A prod_i (y + nu_i^2) / (y + mu_i^2) of
// least uniform relative error |R(y) y^(1/4) - 1| on y in [r_a^2, r_b^2] (eq. ratapprox; R
// stands for (Q_hat^2)^(-1/4) in eq. detQ2).  Host code: a Remez exchange in which the
// 2n + 2 equioscillation equations at the reference points are solved by damped Newton in
// the logarithms of A, nu_i^2 and mu_i^2 (all positive), then the reference moves to the
// extrema of the error (located on a grid, refined by golden-section search).  The first
// guess is a staircase: n factors with equal log-steps spread over the interval and a margin
// on both sides, each lowering log R by 1/4 of its share of log y.
//
// qs_w_mass: the stochastic estimate of W_mass = det[R(Q_hat_m^2) R^-1(Q_hat_m'^2)]
// (eq. Wmass): for every j and source eta, q = (eta, R_j eta), R_j = X^+ + X + X^+ X,
// X = delta D S_j, delta D = D_hat(m') - D_hat(m), with
//   S_j = b^-1 i gamma_5 (mu_j - nu_j) a^-1,  a = D_hat(m) + i gamma_5 nu_j,
//                                              b = D_hat(m') + i gamma_5 mu_j,
// which is the printed three-term S_j after b^-1 (b - a - delta D) a^-1 is multiplied out.
// a^-1 v = (Q_hat_m - i nu)(Q_hat_m^2 + nu^2)^-1 gamma_5 v (gamma_5 a = Q_hat_m + i nu), the
// inverse by FP64 conjugate gradients on the positive operator Q_hat^2 + nu^2.  The estimate
// is prod_j (1/N) sum_l exp(-q_jl) (E[exp(-(eta, R_j eta))] = 1/det(1 + R_j) for sources of
// density ~ exp(-(eta, eta))).
//
// qs_solve_D: x = D^-1 b through the Schur complement on the even sites, with the same FP64
// CG (on Q_hat^2) and the odd-site inverses; or, for comparison, CG on the full-lattice Q^2.
#include "evenodd.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace {

// ---- rational approximation (host) -------------------------------------------------------

const double kP = 0.25;   // R approximates y^-p

inline double log_add_exp(double a, double b)
{
    const double mx = a > b ? a : b;
    return mx + log1p(exp(-fabs(a - b)));
}

// log(R(y) y^p) at S = log y; u = (log A, log nu_i^2 (n), log mu_i^2 (n))
double log_ratio(const double *u, int n, double S)
{
    double g = u[0] + kP * S;
    for (int i = 0; i < n; ++i) g += log_add_exp(S, u[1 + i]) - log_add_exp(S, u[1 + n + i]);
    return g;
}

inline double rel_err(const double *u, int n, double S) { return expm1(log_ratio(u, n, S)); }

// solve M x = b (m x m, row-major) by Gaussian elimination with partial pivoting; b <- x
bool dense_solve(std::vector<double> &M, std::vector<double> &b, int m)
{
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(M[r * m + c]) > fabs(M[piv * m + c])) piv = r;
        if (!(fabs(M[piv * m + c]) > 0)) return false;
        if (piv != c) {
            for (int j = 0; j < m; ++j) std::swap(M[c * m + j], M[piv * m + j]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < m; ++r) {
            const double f = M[r * m + c] / M[c * m + c];
            if (f == 0) continue;
            for (int j = c; j < m; ++j) M[r * m + j] -= f * M[c * m + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = m - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < m; ++j) s -= M[r * m + j] * b[j];
        b[r] = s / M[r * m + r];
    }
    return true;
}

// residuals of the levelled equations g(S_k) = log(1 + sg_k delta); u[2n+1] = delta
double level_residual(const std::vector<double> &u, int n, const std::vector<double> &S,
                      const std::vector<double> &sg, std::vector<double> *F)
{
    const int m = 2 * n + 2;
    const double d = u[2 * n + 1];
    double nrm = 0;
    for (int k = 0; k < m; ++k) {
        const double a = 1 + sg[k] * d;
        const double f = a > 0 ? log_ratio(u.data(), n, S[k]) - log(a) : INFINITY;
        if (F) (*F)[k] = f;
        nrm += f * f;
    }
    return sqrt(nrm);
}

// damped Newton on the levelled equations at a fixed reference
void newton_level(std::vector<double> &u, int n, const std::vector<double> &S, const std::vector<double> &sg)
{
    const int m = 2 * n + 2;
    std::vector<double> F(m), J(m * m), du(m), un(m);
    for (int it = 0; it < 60; ++it) {
        const double nF = level_residual(u, n, S, sg, &F);
        if (!(nF > 1e-15)) return;
        const double d = u[2 * n + 1];
        for (int k = 0; k < m; ++k) {
            double *row = &J[k * m];
            row[0] = 1;
            for (int i = 0; i < n; ++i) {
                row[1 + i] = exp(u[1 + i] - log_add_exp(S[k], u[1 + i]));
                row[1 + n + i] = -exp(u[1 + n + i] - log_add_exp(S[k], u[1 + n + i]));
            }
            row[2 * n + 1] = -sg[k] / (1 + sg[k] * d);
            du[k] = -F[k];
        }
        if (!dense_solve(J, du, m)) return;
        double lam = 1;
        bool ok = false;
        while (lam > 1e-6) {
            for (int k = 0; k < m; ++k) un[k] = u[k] + lam * du[k];
            if (fabs(un[2 * n + 1]) < 0.9) {
                const double nn = level_residual(un, n, S, sg, nullptr);
                if (std::isfinite(nn) && nn < (1 - 1e-4 * lam) * nF) { ok = true; break; }
            }
            lam *= 0.5;
        }
        if (!ok) return;
        u = un;
    }
}

// refine an extremum of |e| inside [a, b] by golden-section search
double refine_extremum(const std::vector<double> &u, int n, double a, double b)
{
    const double gr = 0.5 * (sqrt(5.0) - 1);
    double c = b - gr * (b - a), d = a + gr * (b - a);
    double fc = fabs(rel_err(u.data(), n, c)), fd = fabs(rel_err(u.data(), n, d));
    for (int it = 0; it < 60 && b - a > 1e-12 * (1 + fabs(a)); ++it) {
        if (fc > fd) { b = d; d = c; fd = fc; c = b - gr * (b - a); fc = fabs(rel_err(u.data(), n, c)); }
        else { a = c; c = d; fc = fd; d = a + gr * (b - a); fd = fabs(rel_err(u.data(), n, d)); }
    }
    return 0.5 * (a + b);
}

// the alternating extrema of the error on the grid (largest |e| of each run of one sign),
// trimmed to m by dropping the weaker end; refined off the grid.  Returns how many were found.
int find_extrema(const std::vector<double> &u, int n, const std::vector<double> &grid, int m,
                 std::vector<double> *S, std::vector<double> *sg, double *emax)
{
    const int ng = (int)grid.size();
    std::vector<double> e(ng);
    *emax = 0;
    for (int i = 0; i < ng; ++i) {
        e[i] = rel_err(u.data(), n, grid[i]);
        *emax = std::max(*emax, fabs(e[i]));
    }
    std::vector<int> ext;
    int start = 0;
    for (int i = 1; i <= ng; ++i)
        if (i == ng || (e[i] >= 0) != (e[start] >= 0)) {
            int best = start;
            for (int j = start; j < i; ++j)
                if (fabs(e[j]) > fabs(e[best])) best = j;
            ext.push_back(best);
            start = i;
        }
    while ((int)ext.size() > m) {
        if (fabs(e[ext.front()]) < fabs(e[ext.back()])) ext.erase(ext.begin());
        else ext.pop_back();
    }
    const int ne = (int)ext.size();
    if (ne < m) return ne;
    S->assign(m, 0);
    sg->assign(m, 0);
    for (int k = 0; k < m; ++k) {
        const int i = ext[k];
        double x = grid[i];
        if (i > 0 && i < ng - 1) x = refine_extremum(u, n, grid[i - 1], grid[i + 1]);
        const double ex = rel_err(u.data(), n, x);
        (*S)[k] = x;
        (*sg)[k] = ex >= 0 ? 1.0 : -1.0;
        *emax = std::max(*emax, fabs(ex));
    }
    return m;
}

}  // namespace

extern "C" int qs_ratapprox(int n, double ra, double rb, double *A, double *nu, double *mu, double *delta)
{
    if (n < 0 || n > 32 || !(ra > 0) || !(rb > ra) || !A || !delta || (n > 0 && (!nu || !mu)))
        return QS_EINVAL;
    const double la = 2 * log(ra), lb = 2 * log(rb), L = lb - la;
    if (n == 0) {   // best constant: A y^p - 1 = -delta at y_a, +delta at y_b
        const double a = exp(kP * la), b = exp(kP * lb);
        *A = 2 / (a + b);
        *delta = (b - a) / (b + a);
        return QS_OK;
    }
    const int m = 2 * n + 2;
    std::vector<double> u(m, 0.0);
    const double margin = 2.5;
    const double w = kP * (L + 2 * margin) / n;
    for (int i = 0; i < n; ++i) {
        const double c = la - margin + (L + 2 * margin) * (i + 0.5) / n;
        u[1 + i] = c + 0.5 * w;
        u[1 + n + i] = c - 0.5 * w;
    }
    const int ng = 4000 + 2000 * n;
    std::vector<double> grid(ng);
    for (int i = 0; i < ng; ++i) grid[i] = la + L * i / (ng - 1);
    {   // centre the error of the staircase
        double gmin = INFINITY, gmax = -INFINITY;
        for (int i = 0; i < ng; i += 7) {
            const double g = log_ratio(u.data(), n, grid[i]);
            gmin = std::min(gmin, g);
            gmax = std::max(gmax, g);
        }
        u[0] = -0.5 * (gmin + gmax);
    }
    std::vector<double> S, sg;
    double emax = 0;
    if (find_extrema(u, n, grid, m, &S, &sg, &emax) < m) {
        S.resize(m);
        sg.resize(m);
        for (int k = 0; k < m; ++k) {
            S[k] = 0.5 * (la + lb) - 0.5 * L * cos(M_PI * k / (m - 1));
            sg[k] = (k % 2) ? -1.0 : 1.0;
        }
    }
    bool done = false;
    for (int outer = 0; outer < 100 && !done; ++outer) {
        const std::vector<double> u0 = u;
        u[2 * n + 1] = 0;
        newton_level(u, n, S, sg);
        std::vector<double> S2, sg2;
        // a Newton solution that loses the alternation went too far: move only part of the way
        int found = find_extrema(u, n, grid, m, &S2, &sg2, &emax);
        const std::vector<double> u1 = u;
        for (int h = 1; h <= 12 && found < m; ++h) {
            const double f = ldexp(1.0, -h);
            for (int k = 0; k < m; ++k) u[k] = u0[k] + f * (u1[k] - u0[k]);
            found = find_extrema(u, n, grid, m, &S2, &sg2, &emax);
        }
        if (found < m) return QS_ENOCONV;
        double emin = INFINITY;
        for (int k = 0; k < m; ++k) emin = std::min(emin, fabs(rel_err(u.data(), n, S2[k])));
        S = S2;
        sg = sg2;
        done = emax - emin <= std::max(1e-9 * emax, 2e-13);   // the rounding floor of log_ratio
    }
    if (!done) return QS_ENOCONV;
    *A = exp(u[0]);
    std::vector<double> a(u.begin() + 1, u.begin() + 1 + n), b(u.begin() + 1 + n, u.begin() + 1 + 2 * n);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    for (int i = 0; i < n; ++i) {
        nu[i] = exp(0.5 * a[i]);
        mu[i] = exp(0.5 * b[i]);
    }
    *delta = emax;
    return QS_OK;
}

// ---- W_mass (GPU) -------------------------------------------------------------------------
namespace {

#define RW_PARTS 304   // blocks per right-hand side in the reductions (2 x 152 SMs)

struct Coef {
    double v[64];
};

// y_r += a_r x_r over vectors of len doubles each
__global__ void rw_axpy(double *__restrict__ y, const double *__restrict__ x, Coef a, int64_t len)
{
    const int r = blockIdx.y;
    const double c = a.v[r];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        y[r * len + i] += c * x[r * len + i];
}

// p_r = z_r + b_r p_r
__global__ void rw_xpby(double *__restrict__ p, const double *__restrict__ z, Coef b, int64_t len)
{
    const int r = blockIdx.y;
    const double c = b.v[r];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        p[r * len + i] = z[r * len + i] + c * p[r * len + i];
}

// out = in + c i x (complex, c real); in may equal out
__global__ void rw_add_ix(double2 *out, const double2 *in, const double2 *__restrict__ x, double c, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = in[i], b = x[i];
        out[i] = make_double2(a.x - c * b.y, a.y + c * b.x);
    }
}

// out = c i gamma_5 x (c real; chiral basis: spins 2, 3 negated); out may equal x
__global__ void rw_ig5(double2 *out, const double2 *x, double c, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = (i % 12) >= 6 ? -c : c;
        const double2 b = x[i];
        out[i] = make_double2(-s * b.y, s * b.x);
    }
}

// out = gamma_5 x; out may equal x
__global__ void rw_g5(double2 *out, const double2 *x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 b = x[i];
        out[i] = (i % 12) >= 6 ? make_double2(-b.x, -b.y) : b;
    }
}

// part[r][blk] = sum over the block's share of conj(x_r) y_r (complex), fixed order
__global__ void rw_dot_part(const double2 *__restrict__ x, const double2 *__restrict__ y, int64_t n,
                            double2 *__restrict__ part)
{
    __shared__ double2 sh[256];
    const int r = blockIdx.y;
    double re = 0, im = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = x[r * n + i], b = y[r * n + i];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    sh[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[threadIdx.x].x += sh[threadIdx.x + s].x;
            sh[threadIdx.x].y += sh[threadIdx.x + s].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[r * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void rw_dot_sum(const double2 *__restrict__ part, int nparts, double2 *__restrict__ out)
{
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    double re = 0, im = 0;
    for (int b = 0; b < nparts; ++b) {
        re += part[r * nparts + b].x;
        im += part[r * nparts + b].y;
    }
    out[r] = make_double2(re, im);
}

struct RwWork {
    qs_lattice *lat;
    int nrhs;
    int64_t len;          // doubles per vector
    double *eta, *t, *x, *r, *p, *ap, *tmp, *dwork;
    double2 *part, *dots;
    int full;             // 1: Q^2 of the full-lattice operator instead of Q_hat^2
    // odd-site block inverses at the two masses of the estimate
    double mass[2];
    const double2 *inv[2];
    const double2 *inv_for(double m) const { return m == mass[0] ? inv[0] : m == mass[1] ? inv[1] : nullptr; }
};

int rw_check(const char *where)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { qs_record_cuda_error(e, where); return QS_ECUDA; }
    return QS_OK;
}

// out[r] = (x_r, y_r) on the host
int rw_dot(RwWork &w, const double *x, const double *y, double2 *out)
{
    cudaStream_t st = w.lat->stream;
    rw_dot_part<<<dim3(RW_PARTS, w.nrhs), 256, 0, st>>>((const double2 *)x, (const double2 *)y, w.len / 2, w.part);
    rw_dot_sum<<<w.nrhs, 32, 0, st>>>(w.part, RW_PARTS, w.dots);
    qs_note_launches(2);
    QS_TRY(rw_check("rw_dot"));
    QS_CUDA(cudaMemcpyAsync(out, w.dots, w.nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaStreamSynchronize(st));
    return QS_OK;
}

unsigned rw_grid(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4 * 152); }

// out = Q_hat(m)^2 in + sigma in
int rw_q2(RwWork &w, double m, double sigma, const double *in, double *out)
{
    if (w.full) {
        double mm[64];
        for (int r = 0; r < w.nrhs; ++r) mm[r] = m;
        QS_TRY(qs_dslash_run(w.lat, QS_F64, mm, in, w.tmp, w.nrhs, 1, 0));
        QS_TRY(qs_dslash_run(w.lat, QS_F64, mm, w.tmp, out, w.nrhs, 1, 0));
    } else {
        QS_TRY(qs_dhat_run(w.lat, m, in, w.tmp, w.nrhs, 1, w.dwork, w.inv_for(m)));
        QS_TRY(qs_dhat_run(w.lat, m, w.tmp, out, w.nrhs, 1, w.dwork, w.inv_for(m)));
    }
    Coef c;
    for (int r = 0; r < w.nrhs; ++r) c.v[r] = sigma;
    rw_axpy<<<dim3(rw_grid(w.len), w.nrhs), 256, 0, w.lat->stream>>>(out, in, c, w.len);
    qs_note_launches(1);
    return rw_check("rw_q2");
}

// x = (Q_hat(m)^2 + sigma)^-1 b by conjugate gradients (x0 = 0), every right-hand side to
// ||r|| <= tol ||b||; *iters: iterations taken
int rw_cg(RwWork &w, double m, double sigma, const double *b, double *x, double tol, int max_iter, int *iters)
{
    cudaStream_t st = w.lat->stream;
    const size_t bytes = (size_t)w.nrhs * w.len * sizeof(double);
    QS_CUDA(cudaMemsetAsync(x, 0, bytes, st));
    QS_CUDA(cudaMemcpyAsync(w.r, b, bytes, cudaMemcpyDeviceToDevice, st));
    QS_CUDA(cudaMemcpyAsync(w.p, b, bytes, cudaMemcpyDeviceToDevice, st));
    double2 d[64];
    QS_TRY(rw_dot(w, w.r, w.r, d));
    double rr[64], stop[64];
    bool live[64];
    for (int r = 0; r < w.nrhs; ++r) {
        rr[r] = d[r].x;
        stop[r] = tol * tol * rr[r];
        live[r] = rr[r] > 0;
    }
    const unsigned gx = rw_grid(w.len);
    for (int it = 0; it < max_iter; ++it) {
        bool any = false;
        for (int r = 0; r < w.nrhs; ++r) any |= live[r];
        if (!any) { *iters = it; return QS_OK; }
        QS_TRY(rw_q2(w, m, sigma, w.p, w.ap));
        QS_TRY(rw_dot(w, w.p, w.ap, d));
        Coef a, na;
        for (int r = 0; r < w.nrhs; ++r) {
            a.v[r] = live[r] && d[r].x > 0 ? rr[r] / d[r].x : 0.0;
            na.v[r] = -a.v[r];
        }
        rw_axpy<<<dim3(gx, w.nrhs), 256, 0, st>>>(x, w.p, a, w.len);
        rw_axpy<<<dim3(gx, w.nrhs), 256, 0, st>>>(w.r, w.ap, na, w.len);
        qs_note_launches(2);
        QS_TRY(rw_dot(w, w.r, w.r, d));
        Coef beta;
        for (int r = 0; r < w.nrhs; ++r) {
            const double rn = d[r].x;
            beta.v[r] = live[r] && rr[r] > 0 ? rn / rr[r] : 0.0;
            if (live[r] && rn <= stop[r]) live[r] = false;
            rr[r] = rn;
        }
        rw_xpby<<<dim3(gx, w.nrhs), 256, 0, st>>>(w.p, w.r, beta, w.len);
        qs_note_launches(1);
        QS_TRY(rw_check("rw_cg"));
    }
    *iters = max_iter;
    for (int r = 0; r < w.nrhs; ++r)
        if (live[r]) return QS_ENOCONV;
    return QS_OK;
}

// out = a^-1 in with a = D_hat(m) + i gamma_5 shift: (Q_hat(m) - i shift)(Q_hat^2 + shift^2)^-1 gamma_5 in
int rw_shifted_inverse(RwWork &w, double m, double shift, const double *in, double *out, double tol, int max_iter,
                       int *iters)
{
    const int64_t nc = (int64_t)w.nrhs * w.len / 2;
    cudaStream_t st = w.lat->stream;
    rw_g5<<<rw_grid(nc), 256, 0, st>>>((double2 *)w.t, (const double2 *)in, nc);
    qs_note_launches(1);
    QS_TRY(rw_cg(w, m, shift * shift, w.t, w.x, tol, max_iter, iters));
    QS_TRY(qs_dhat_run(w.lat, m, w.x, out, w.nrhs, 1, w.dwork, w.inv_for(m)));
    rw_add_ix<<<rw_grid(nc), 256, 0, st>>>((double2 *)out, (const double2 *)out, (const double2 *)w.x, -shift, nc);
    qs_note_launches(1);
    return rw_check("rw_shifted_inverse");
}

}  // namespace

extern "C" int qs_w_mass(qs_lattice *lat, double m, double mp, int n, const double *nu, const double *mu,
                         const void *eta, int nsrc, double tol, int max_iter, double *q, double *log_w,
                         int *cg_iterations)
{
    if (!lat || !nu || !mu || !eta || !q || n < 1 || n > 32 || nsrc < 1 || nsrc > 64) return QS_EINVAL;
    if (!(tol > 0) || max_iter < 1 || ((uintptr_t)eta & 15)) return QS_EINVAL;
    for (int j = 0; j < n; ++j)
        if (!(nu[j] > 0) || !(mu[j] > 0)) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    const Geom &g = lat->g;
    if ((g.T | g.L) & 1) return QS_EINVAL;   // hopping must connect opposite parities only
    QS_CUDA(cudaSetDevice(lat->device));
    RwWork w;
    w.lat = lat;
    w.full = 0;
    w.nrhs = nsrc;
    w.len = g.Ns * 24;
    const int64_t vl = (int64_t)nsrc * w.len;   // doubles per block of nsrc vectors
    double *buf = nullptr;
    const size_t inv_len = (size_t)36 * g.Vphys;   // complex entries of the inverses at one mass
    QS_CUDA(cudaMalloc(&buf, 12 * vl * sizeof(double) + (size_t)nsrc * (RW_PARTS + 1) * sizeof(double2) +
                                 2 * inv_len * sizeof(double2)));
    w.eta = buf;
    w.t = buf + vl;
    w.x = buf + 2 * vl;
    w.r = buf + 3 * vl;
    w.p = buf + 4 * vl;
    w.ap = buf + 5 * vl;
    w.tmp = buf + 6 * vl;
    w.dwork = buf + 7 * vl;   // 3 blocks
    double *v1 = buf + 10 * vl, *v2 = buf + 11 * vl;
    w.part = (double2 *)(buf + 12 * vl);
    w.dots = w.part + (size_t)nsrc * RW_PARTS;
    double2 *inv = w.dots + nsrc;
    w.mass[0] = m;
    w.mass[1] = mp;
    w.inv[0] = inv;
    w.inv[1] = inv + inv_len;
    cudaStream_t st = lat->stream;
    const int64_t nc = vl / 2;
    int s = QS_OK, total_it = 0;
    double lw = 0;
    do {
        if ((s = qs_even_mask(lat, (const double *)eta, w.eta, nsrc)) != QS_OK) break;
        if ((s = qs_clover_inverse_odd(lat, m, (double2 *)w.inv[0])) != QS_OK) break;
        if ((s = qs_clover_inverse_odd(lat, mp, (double2 *)w.inv[1])) != QS_OK) break;
        for (int j = 0; j < n && s == QS_OK; ++j) {
            int it = 0;
            // v1 = i gamma_5 (mu - nu) a^-1 eta, v2 = b^-1 v1 = S_j eta
            if ((s = rw_shifted_inverse(w, m, nu[j], w.eta, v1, tol, max_iter, &it)) != QS_OK) break;
            total_it += it;
            rw_ig5<<<rw_grid(nc), 256, 0, st>>>((double2 *)v1, (const double2 *)v1, mu[j] - nu[j], nc);
            qs_note_launches(1);
            if ((s = rw_shifted_inverse(w, mp, mu[j], v1, v2, tol, max_iter, &it)) != QS_OK) break;
            total_it += it;
            // v1 = X eta = D_hat(m') S_j eta - D_hat(m) S_j eta
            if ((s = qs_dhat_run(lat, mp, v2, v1, nsrc, 0, w.dwork, w.inv_for(mp))) != QS_OK) break;
            if ((s = qs_dhat_run(lat, m, v2, w.tmp, nsrc, 0, w.dwork, w.inv_for(m))) != QS_OK) break;
            Coef c;
            for (int r = 0; r < nsrc; ++r) c.v[r] = -1.0;
            rw_axpy<<<dim3(rw_grid(w.len), nsrc), 256, 0, st>>>(v1, w.tmp, c, w.len);
            qs_note_launches(1);
            // q = (eta, R_j eta) = 2 Re (eta, X eta) + ||X eta||^2
            double2 ex[64], xx[64];
            if ((s = rw_dot(w, w.eta, v1, ex)) != QS_OK) break;
            if ((s = rw_dot(w, v1, v1, xx)) != QS_OK) break;
            double mx = -INFINITY;
            for (int l = 0; l < nsrc; ++l) {
                q[(size_t)j * nsrc + l] = 2 * ex[l].x + xx[l].x;
                mx = std::max(mx, -q[(size_t)j * nsrc + l]);
            }
            double sum = 0;   // log of the mean of exp(-q), shifted by the largest exponent
            for (int l = 0; l < nsrc; ++l) sum += exp(-q[(size_t)j * nsrc + l] - mx);
            lw += mx + log(sum / nsrc);
        }
    } while (0);
    cudaFree(buf);
    if (cg_iterations) *cg_iterations = total_it;
    if (s == QS_OK && log_w) *log_w = lw;
    return s;
}

// ---- the even-odd preconditioned solve of D x = b (Sec. 4) ---------------------------------
namespace {
int rw_copy(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_solve_D copy"); return QS_ECUDA; }
    return QS_OK;
}
}  // namespace

// even_odd = 1:  b'_e = b_e - D_eo (D_oo)^-1 b_o;  D_hat x_e = b'_e by CG on Q_hat^2
// (x_e = Q_hat (Q_hat^2)^-1 gamma_5 b'_e);  x_o = (D_oo)^-1 (b_o - D_oe x_e).
// even_odd = 0:  x = Q (Q^2)^-1 gamma_5 b by CG on the full-lattice Q^2 (the comparison).
extern "C" int qs_solve_D(qs_lattice *lat, double m0, const void *b, void *x, int nrhs, int even_odd, double tol,
                          int max_iter, int *iterations)
{
    if (!lat || !b || !x || nrhs < 1 || nrhs > 64 || !(tol > 0) || max_iter < 1) return QS_EINVAL;
    if (((uintptr_t)b | (uintptr_t)x) & 15) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    const Geom &g = lat->g;
    if (even_odd && ((g.T | g.L) & 1)) return QS_EINVAL;
    const size_t bytes = (size_t)nrhs * g.Ns * 24 * sizeof(double);
    const char *pa = (const char *)b, *pb = (const char *)x;
    if (pa < pb + bytes && pb < pa + bytes) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    RwWork w;
    w.lat = lat;
    w.full = even_odd ? 0 : 1;
    w.nrhs = nrhs;
    w.len = g.Ns * 24;
    const int64_t vl = (int64_t)nrhs * w.len;
    const size_t inv_len = even_odd ? (size_t)36 * g.Vphys : 0;
    double *buf = nullptr;
    QS_CUDA(cudaMalloc(&buf, 11 * vl * sizeof(double) + (size_t)nrhs * (RW_PARTS + 1) * sizeof(double2) +
                                 inv_len * sizeof(double2)));
    w.eta = nullptr;
    w.t = buf;
    w.x = buf + vl;
    w.r = buf + 2 * vl;
    w.p = buf + 3 * vl;
    w.ap = buf + 4 * vl;
    w.tmp = buf + 5 * vl;
    w.dwork = buf + 6 * vl;   // 3 blocks
    double *a1 = buf + 9 * vl, *a2 = buf + 10 * vl;
    w.part = (double2 *)(buf + 11 * vl);
    w.dots = w.part + (size_t)nrhs * RW_PARTS;
    double2 *inv = even_odd ? w.dots + nrhs : nullptr;
    w.mass[0] = w.mass[1] = m0;
    w.inv[0] = w.inv[1] = inv;
    cudaStream_t st = lat->stream;
    const int64_t nc = vl / 2;
    Coef minus, plus;
    for (int r = 0; r < nrhs; ++r) { minus.v[r] = -1.0; plus.v[r] = 1.0; }
    const dim3 ga(rw_grid(w.len), nrhs);
    int s = QS_OK, it = 0;
    do {
        if (even_odd) {
            if ((s = qs_clover_inverse_odd(lat, m0, inv)) != QS_OK) break;
            if ((s = qs_oo_inverse_apply(lat, inv, (const double *)b, a1, nrhs, 1.0)) != QS_OK) break;
            if ((s = qs_dslash64_parity(lat, m0, a1, a2, nrhs, 0)) != QS_OK) break;   // D_eo D_oo^-1 b_o
            if ((s = qs_even_mask(lat, (const double *)b, w.t, nrhs)) != QS_OK) break;
            rw_axpy<<<ga, 256, 0, st>>>(w.t, a2, minus, w.len);                          // b'_e
            rw_g5<<<rw_grid(nc), 256, 0, st>>>((double2 *)w.t, (const double2 *)w.t, nc);
            qs_note_launches(2);
            if ((s = rw_cg(w, m0, 0.0, w.t, w.x, tol, max_iter, &it)) != QS_OK) break;
            if ((s = qs_dhat_run(lat, m0, w.x, a1, nrhs, 1, w.dwork, inv)) != QS_OK) break;   // x_e
            if ((s = qs_dslash64_parity(lat, m0, a1, a2, nrhs, 1)) != QS_OK) break;            // D_oe x_e
            if ((s = rw_copy(w.t, b, bytes, st)) != QS_OK) break;
            rw_axpy<<<ga, 256, 0, st>>>(w.t, a2, minus, w.len);                          // b_o - D_oe x_e
            qs_note_launches(1);
            if ((s = qs_oo_inverse_apply(lat, inv, w.t, a2, nrhs, 1.0)) != QS_OK) break;     // x_o
            if ((s = rw_copy(x, a1, bytes, st)) != QS_OK) break;
            rw_axpy<<<ga, 256, 0, st>>>((double *)x, a2, plus, w.len);
            qs_note_launches(1);
        } else {
            rw_g5<<<rw_grid(nc), 256, 0, st>>>((double2 *)w.t, (const double2 *)b, nc);
            qs_note_launches(1);
            if ((s = rw_cg(w, m0, 0.0, w.t, w.x, tol, max_iter, &it)) != QS_OK) break;
            double mm[64];
            for (int r = 0; r < nrhs; ++r) mm[r] = m0;
            if ((s = qs_dslash_run(lat, QS_F64, mm, w.x, x, nrhs, 1, 0)) != QS_OK) break;    // x = Q y
        }
        if ((s = rw_check("qs_solve_D")) != QS_OK) break;
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_solve_D"); s = QS_ECUDA; }
    } while (0);
    cudaFree(buf);
    if (iterations) *iterations = it;
    return s;
}
