// Exact even-odd factor of the mass reweighting (Sec. 4):
//   W_eo(m -> m') = |det[D^oo_m' (D^oo_m)^-1]|^(1/2),
// D^oo = D restricted to the odd sites of the doubled lattice.  Hopping connects
// opposite parities only, so D^oo is site-diagonal: 4 + m0 + A(x), two 6 x 6 chiral
// blocks per site, and log|det D^oo| = sum over odd sites and blocks of log|det|.
// A physical site and its mirror have the same parity (L is even) and the mirror
// block S conj(A) S has the same (real) determinant, so the sum runs over odd physical
// sites and counts each twice.  One thread per physical site, a complex LU with
// partial pivoting per block in FP64, then a fixed-order two-stage sum.
#include "blas.cuh"
#include "evenodd.cuh"

#include <math.h>
#include <stdlib.h>

namespace {

#define EO_MAX_MASS 16
#define EO_BLOCKS 304

__device__ double block_logdet(const double *__restrict__ clov, int64_t V, int64_t p, int b, double dm)
{
    double re[6][6], im[6][6];
    const double *cb = clov + (int64_t)b * 36 * V + p;
    for (int i = 0; i < 6; ++i) {
        re[i][i] = dm + cb[(int64_t)i * V];
        im[i][i] = 0.0;
        for (int j = 0; j < i; ++j) {
            const int k = 6 + 2 * qs_tri(i, j);
            re[i][j] = cb[(int64_t)k * V];
            im[i][j] = cb[(int64_t)(k + 1) * V];
            re[j][i] = re[i][j];          // Hermitian: upper = conj(lower)
            im[j][i] = -im[i][j];
        }
    }
    double acc = 0.0;
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = re[c][c] * re[c][c] + im[c][c] * im[c][c];
        for (int r = c + 1; r < 6; ++r) {
            const double a = re[r][c] * re[r][c] + im[r][c] * im[r][c];
            if (a > best) { best = a; piv = r; }
        }
        if (piv != c)
            for (int j = 0; j < 6; ++j) {
                double t = re[c][j]; re[c][j] = re[piv][j]; re[piv][j] = t;
                t = im[c][j]; im[c][j] = im[piv][j]; im[piv][j] = t;
            }
        acc += 0.5 * log(best);           // log|u_cc|; a zero pivot gives -inf
        if (!(best > 0.0)) continue;
        const double ir = re[c][c] / best, ii = -im[c][c] / best;   // 1 / u_cc
        for (int r = c + 1; r < 6; ++r) {
            const double lr = re[r][c] * ir - im[r][c] * ii, li = re[r][c] * ii + im[r][c] * ir;
            for (int j = c + 1; j < 6; ++j) {
                re[r][j] -= lr * re[c][j] - li * im[c][j];
                im[r][j] -= lr * im[c][j] + li * re[c][j];
            }
        }
    }
    return acc;
}

__global__ void logdet_oo_kernel(Geom g, const double *__restrict__ clov, int nmass, const double *__restrict__ m0,
                                 double *part)
{
    __shared__ double sh[EO_MAX_MASS][8];
    double acc[EO_MAX_MASS];
    for (int q = 0; q < nmass; ++q) acc[q] = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.Vphys; p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % g.L);
        int64_t row = p / g.L;
        const int y = (int)(row % g.L);
        row /= g.L;
        const int z = (int)(row % g.L);
        const int t = (int)(row / g.L);
        if (((t + z + y + x) & 1) == 0) continue;
        for (int q = 0; q < nmass; ++q)
            for (int b = 0; b < 2; ++b) acc[q] += 2.0 * block_logdet(clov, g.Vphys, p, b, 4.0 + m0[q]);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int q = 0; q < nmass; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) sh[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < nmass) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[threadIdx.x][i];
        part[threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void sum_parts_kernel(const double *part, int nb, int nmass, double *out)
{
    const int q = threadIdx.x;
    if (q >= nmass) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[q * nb + i];
    out[q] = s;
}

}  // namespace

extern "C" int qs_log_det_oo(qs_lattice *lat, int nmass, const double *m0, double *logdet)
{
    if (!lat || !m0 || !logdet || nmass < 1 || nmass > EO_MAX_MASS) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    double *d = nullptr;
    const size_t n = (size_t)EO_MAX_MASS + (size_t)EO_MAX_MASS * EO_BLOCKS + EO_MAX_MASS;
    QS_CUDA(cudaMalloc(&d, n * sizeof(double)));
    double *dm = d, *part = d + EO_MAX_MASS, *out = part + (size_t)EO_MAX_MASS * EO_BLOCKS;
    cudaError_t e = cudaMemcpyAsync(dm, m0, nmass * sizeof(double), cudaMemcpyHostToDevice, lat->stream);
    if (e == cudaSuccess) {
        logdet_oo_kernel<<<EO_BLOCKS, 256, 0, lat->stream>>>(lat->g, lat->clov64, nmass, dm, part);
        sum_parts_kernel<<<1, 32, 0, lat->stream>>>(part, EO_BLOCKS, nmass, out);
        qs_note_launches(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(logdet, out, nmass * sizeof(double), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    cudaFree(d);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "qs_log_det_oo");
        return QS_ECUDA;
    }
    for (int q = 0; q < nmass; ++q)
        if (!isfinite(logdet[q])) return QS_ENUMERIC;
    return QS_OK;
}

extern "C" int qs_w_eo(qs_lattice *lat, double m, double mp, double *w_eo, double *log_w_eo)
{
    if (!w_eo && !log_w_eo) return QS_EINVAL;
    double ms[2] = {m, mp}, ld[2];
    QS_TRY(qs_log_det_oo(lat, 2, ms, ld));
    const double lw = 0.5 * (ld[1] - ld[0]);
    if (log_w_eo) *log_w_eo = lw;
    if (w_eo) *w_eo = exp(lw);
    return QS_OK;
}

// ---- the even-odd preconditioned operator (Sec. 4) --------------------------------
// D_hat = D_ee - D_eo (D_oo)^-1 D_oe on the even sites, Q_hat = gamma_5 D_hat.  With x the
// even part of the input (odd entries zero): (D x)_e = D_ee x_e and (D x)_o = D_oe x_e, so
//   D_hat x_e = (D x)_e - (D u)_e,  u = (D_oo)^-1 (D x)_o  (u zero on even sites),
// two applications of the full FP64 operator, a site-local solve and parity masks.
namespace {

__device__ __forceinline__ int site_parity(const Geom &g, int64_t s)
{
    const int x = (int)(s % g.L2);
    int64_t r = s / g.L2;
    const int y = (int)(r % g.L);
    r /= g.L;
    const int z = (int)(r % g.L);
    const int t = (int)(r / g.L);
    return (t + z + y + x) & 1;
}

// out = in on sites of parity `keep`, 0 elsewhere (canonical FP64 layout, k vectors)
__global__ void parity_mask_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, Geom g, int k,
                                   int keep)
{
    const int64_t n = g.Ns * 12 * k;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = (i / 12) % g.Ns;
    out[i] = site_parity(g, s) == keep ? in[i] : make_double2(0, 0);
}

// v = x on even sites and v = -(4 + m0 + A(x))^-1 t on odd sites (two 6 x 6 chiral blocks,
// complex Gaussian elimination with partial pivoting in FP64); one thread per (vector, site).
// The mirror site's block is S conj(A) S: entry (i, j) = sign * conj(A[i +- 3][j +- 3]),
// sign = -1 across the two spin halves.
__global__ void clover_solve_odd_kernel(const double *__restrict__ clov, const double2 *__restrict__ t,
                                        const double2 *__restrict__ xe, double2 *__restrict__ u, Geom g, int k,
                                        double dm)
{
    const int64_t n = g.Ns * k;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = i % g.Ns;
    const double2 *ti = t + i * 12;
    double2 *ui = u + i * 12;
    if (site_parity(g, s) == 0) {
        const double2 *xi = xe + i * 12;
        for (int c = 0; c < 12; ++c) ui[c] = xi[c];
        return;
    }
    const int x = (int)(s % g.L2);
    const bool mir = x >= g.L;
    const int64_t p = (s / g.L2) * g.L + (mir ? x - g.L : x);
    const int64_t V = g.Vphys;
    for (int b = 0; b < 2; ++b) {
        const double *cb = clov + (int64_t)b * 36 * V + p;
        double ar[6][6], ai[6][6], rr[6], ri[6];
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) {
                const int ii = mir ? (r + 3) % 6 : r, jj = mir ? (c + 3) % 6 : c;
                double er, ei;
                if (ii == jj) { er = cb[(int64_t)ii * V]; ei = 0; }
                else if (ii > jj) {
                    const int kk = 6 + 2 * qs_tri(ii, jj);
                    er = cb[(int64_t)kk * V]; ei = cb[(int64_t)(kk + 1) * V];
                } else {
                    const int kk = 6 + 2 * qs_tri(jj, ii);
                    er = cb[(int64_t)kk * V]; ei = -cb[(int64_t)(kk + 1) * V];
                }
                if (mir) {
                    ei = -ei;
                    if ((r < 3) != (c < 3)) { er = -er; ei = -ei; }
                }
                ar[r][c] = er + (r == c ? dm : 0.0);
                ai[r][c] = ei;
            }
        for (int r = 0; r < 6; ++r) { rr[r] = ti[6 * b + r].x; ri[r] = ti[6 * b + r].y; }
        for (int c = 0; c < 6; ++c) {
            int piv = c;
            double best = ar[c][c] * ar[c][c] + ai[c][c] * ai[c][c];
            for (int r = c + 1; r < 6; ++r) {
                const double a2 = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
                if (a2 > best) { best = a2; piv = r; }
            }
            if (piv != c) {
                for (int j = 0; j < 6; ++j) {
                    double tt = ar[c][j]; ar[c][j] = ar[piv][j]; ar[piv][j] = tt;
                    tt = ai[c][j]; ai[c][j] = ai[piv][j]; ai[piv][j] = tt;
                }
                double tt = rr[c]; rr[c] = rr[piv]; rr[piv] = tt;
                tt = ri[c]; ri[c] = ri[piv]; ri[piv] = tt;
            }
            const double ir = ar[c][c] / best, ii2 = -ai[c][c] / best;   // 1 / pivot
            for (int r = c + 1; r < 6; ++r) {
                const double lr = ar[r][c] * ir - ai[r][c] * ii2, li = ar[r][c] * ii2 + ai[r][c] * ir;
                for (int j = c; j < 6; ++j) {
                    ar[r][j] -= lr * ar[c][j] - li * ai[c][j];
                    ai[r][j] -= lr * ai[c][j] + li * ar[c][j];
                }
                rr[r] -= lr * rr[c] - li * ri[c];
                ri[r] -= lr * ri[c] + li * rr[c];
            }
        }
        for (int r = 5; r >= 0; --r) {   // back substitution
            double sr = rr[r], si = ri[r];
            for (int j = r + 1; j < 6; ++j) {
                sr -= ar[r][j] * rr[j] - ai[r][j] * ri[j];
                si -= ar[r][j] * ri[j] + ai[r][j] * rr[j];
            }
            const double d2 = ar[r][r] * ar[r][r] + ai[r][r] * ai[r][r];
            rr[r] = (sr * ar[r][r] + si * ai[r][r]) / d2;
            ri[r] = (si * ar[r][r] - sr * ai[r][r]) / d2;
        }
        for (int r = 0; r < 6; ++r) ui[6 * b + r] = make_double2(-rr[r], -ri[r]);
    }
}

// inv = (4 + m0 + A(x))^-1 for every odd physical site x, both chiral blocks, by Gauss-Jordan
// elimination with partial pivoting in FP64; layout [block][6][6][V_phys / 2] complex, the odd
// physical site p at index p / 2 (L is even, so the odd sites of a row of L alternate).  The mirror site's block S conj(M) S has the inverse
// S conj(M^-1) S, formed on the fly when it is applied.
__global__ void clover_inverse_kernel(const double *__restrict__ clov, Geom g, double dm, double2 *__restrict__ inv)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= g.Vphys) return;
    const int x = (int)(p % g.L);
    int64_t row = p / g.L;
    const int y = (int)(row % g.L);
    row /= g.L;
    const int z = (int)(row % g.L);
    const int t = (int)(row / g.L);
    if (((t + z + y + x) & 1) == 0) return;
    const int64_t V = g.Vphys;
    for (int b = 0; b < 2; ++b) {
        const double *cb = clov + (int64_t)b * 36 * V + p;
        double ar[6][6], ai[6][6], br[6][6], bi[6][6];
        for (int i = 0; i < 6; ++i) {
            ar[i][i] = dm + cb[(int64_t)i * V];
            ai[i][i] = 0.0;
            for (int j = 0; j < i; ++j) {
                const int k = 6 + 2 * qs_tri(i, j);
                ar[i][j] = cb[(int64_t)k * V];
                ai[i][j] = cb[(int64_t)(k + 1) * V];
                ar[j][i] = ar[i][j];      // Hermitian: upper = conj(lower)
                ai[j][i] = -ai[i][j];
            }
            for (int j = 0; j < 6; ++j) { br[i][j] = i == j ? 1.0 : 0.0; bi[i][j] = 0.0; }
        }
        for (int c = 0; c < 6; ++c) {
            int piv = c;
            double best = ar[c][c] * ar[c][c] + ai[c][c] * ai[c][c];
            for (int r = c + 1; r < 6; ++r) {
                const double a2 = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
                if (a2 > best) { best = a2; piv = r; }
            }
            if (piv != c)
                for (int j = 0; j < 6; ++j) {
                    double q = ar[c][j]; ar[c][j] = ar[piv][j]; ar[piv][j] = q;
                    q = ai[c][j]; ai[c][j] = ai[piv][j]; ai[piv][j] = q;
                    q = br[c][j]; br[c][j] = br[piv][j]; br[piv][j] = q;
                    q = bi[c][j]; bi[c][j] = bi[piv][j]; bi[piv][j] = q;
                }
            const double pr = ar[c][c] / best, pim = -ai[c][c] / best;   // 1 / pivot
            for (int j = 0; j < 6; ++j) {
                double q = ar[c][j] * pr - ai[c][j] * pim;
                ai[c][j] = ar[c][j] * pim + ai[c][j] * pr;
                ar[c][j] = q;
                q = br[c][j] * pr - bi[c][j] * pim;
                bi[c][j] = br[c][j] * pim + bi[c][j] * pr;
                br[c][j] = q;
            }
            for (int r = 0; r < 6; ++r) {
                if (r == c) continue;
                const double fr = ar[r][c], fi = ai[r][c];
                for (int j = 0; j < 6; ++j) {
                    ar[r][j] -= fr * ar[c][j] - fi * ai[c][j];
                    ai[r][j] -= fr * ai[c][j] + fi * ar[c][j];
                    br[r][j] -= fr * br[c][j] - fi * bi[c][j];
                    bi[r][j] -= fr * bi[c][j] + fi * br[c][j];
                }
            }
        }
        const int64_t V2 = V / 2, q = p >> 1;   // odd sites of a row of L have one index parity each
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) inv[((int64_t)b * 36 + i * 6 + j) * V2 + q] = make_double2(br[i][j], bi[i][j]);
    }
}

// v = x on even sites, v = -(4 + m0 + A(x))^-1 t on odd sites from the stored inverses.  Thread
// j takes the j-th odd site (x = 2 jx or 2 jx + 1 in its row) and copies its even x partner.
__global__ void clover_apply_inv_kernel(const double2 *__restrict__ inv, const double2 *__restrict__ t,
                                        const double2 *__restrict__ xe, double2 *__restrict__ v, Geom g, int k)
{
    const int64_t half = g.Ns / 2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= half * k) return;
    const int64_t r = i / half, j = i - r * half;
    const int64_t row = j / g.L;
    const int jx = (int)(j - row * g.L);
    const int y = (int)(row % g.L), z = (int)((row / g.L) % g.L), tt = (int)(row / ((int64_t)g.L * g.L));
    const int x = 2 * jx + ((1 + tt + z + y) & 1);
    const int64_t s = row * g.L2 + x;
    {
        const int64_t e = (r * g.Ns + (s ^ 1)) * 12;
        for (int c = 0; c < 12; ++c) v[e + c] = xe[e + c];
    }
    const double2 *ti = t + (r * g.Ns + s) * 12;
    double2 *vi = v + (r * g.Ns + s) * 12;
    const bool mir = x >= g.L;
    const int64_t p = row * g.L + (mir ? x - g.L : x);
    const int64_t V2 = g.Vphys / 2, q = p >> 1;
    for (int b = 0; b < 2; ++b)
        for (int rr = 0; rr < 6; ++rr) {
            double accr = 0, acci = 0;
            for (int c = 0; c < 6; ++c) {
                const int ii = mir ? (rr + 3) % 6 : rr, jj = mir ? (c + 3) % 6 : c;
                double2 e = inv[((int64_t)b * 36 + ii * 6 + jj) * V2 + q];
                if (mir) {
                    e.y = -e.y;
                    if ((rr < 3) != (c < 3)) { e.x = -e.x; e.y = -e.y; }
                }
                const double2 w = ti[6 * b + c];
                accr += e.x * w.x - e.y * w.y;
                acci += e.x * w.y + e.y * w.x;
            }
            vi[6 * b + rr] = make_double2(-accr, -acci);
        }
}

// out = scale (4 + m0 + A(x))^-1 t on odd sites (stored inverses), 0 on even sites; thread j
// takes the j-th odd site and zeroes its even x partner
__global__ void oo_inverse_kernel(const double2 *__restrict__ inv, const double2 *__restrict__ t,
                                  double2 *__restrict__ out, Geom g, int k, double scale)
{
    const int64_t half = g.Ns / 2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= half * k) return;
    const int64_t r = i / half, j = i - r * half;
    const int64_t row = j / g.L;
    const int jx = (int)(j - row * g.L);
    const int y = (int)(row % g.L), z = (int)((row / g.L) % g.L), tt = (int)(row / ((int64_t)g.L * g.L));
    const int x = 2 * jx + ((1 + tt + z + y) & 1);
    const int64_t s = row * g.L2 + x;
    {
        double2 *o = out + (r * g.Ns + (s ^ 1)) * 12;
        for (int c = 0; c < 12; ++c) o[c] = make_double2(0.0, 0.0);
    }
    const double2 *ti = t + (r * g.Ns + s) * 12;
    double2 *oi = out + (r * g.Ns + s) * 12;
    const bool mir = x >= g.L;
    const int64_t p = row * g.L + (mir ? x - g.L : x);
    const int64_t V2 = g.Vphys / 2, q = p >> 1;
    for (int b = 0; b < 2; ++b)
        for (int rr = 0; rr < 6; ++rr) {
            double accr = 0, acci = 0;
            for (int c = 0; c < 6; ++c) {
                const int ii = mir ? (rr + 3) % 6 : rr, jj = mir ? (c + 3) % 6 : c;
                double2 e = inv[((int64_t)b * 36 + ii * 6 + jj) * V2 + q];
                if (mir) {
                    e.y = -e.y;
                    if ((rr < 3) != (c < 3)) { e.x = -e.x; e.y = -e.y; }
                }
                const double2 w = ti[6 * b + c];
                accr += e.x * w.x - e.y * w.y;
                acci += e.x * w.y + e.y * w.x;
            }
            oi[6 * b + rr] = make_double2(scale * accr, scale * acci);
        }
}

}  // namespace

// D_hat (or Q_hat) of nrhs FP64 vectors, asynchronous on the lattice's stream; work holds
// 3 * nrhs * N_s * 24 doubles.  in and out must not overlap work; in may equal out.
// With x the even part of the input, u = (D_oo)^-1 (D x)_o and v = x - u (even part x,
// odd part -u):  D_hat x = (D x)_e - (D u)_e = (D v)_e, so the operator is applied twice,
// each time on the output sites of one parity only.
int qs_oo_inverse_apply(qs_lattice *lat, const double2 *inv, const double *in, double *out, int nrhs, double scale)
{
    const int64_t n = lat->g.Ns / 2 * nrhs;
    oo_inverse_kernel<<<(unsigned)((n + 127) / 128), 128, 0, lat->stream>>>(inv, (const double2 *)in, (double2 *)out,
                                                                          lat->g, nrhs, scale);
    qs_note_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_oo_inverse_apply"); return QS_ECUDA; }
    return QS_OK;
}

int qs_dslash64_parity(qs_lattice *lat, double m0, const double *in, double *out, int nrhs, int parity)
{
    DslashArgs<double> d;
    d.g = lat->g;
    d.links = lat->links64;
    d.clov = lat->clov64;
    d.nrhs = nrhs;
    for (int r = 0; r < nrhs; ++r) d.m0[r] = m0;
    d.in = in;
    d.out = out;
    d.gamma5 = 0;
    const cudaError_t e = qs_dslash64_parity_launch(d, parity, lat->stream);
    qs_note_launches(1);
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_dslash64_parity"); return QS_ECUDA; }
    return QS_OK;
}

int qs_clover_inverse_odd(qs_lattice *lat, double m0, double2 *inv)
{
    const int64_t V = lat->g.Vphys;
    clover_inverse_kernel<<<(unsigned)((V + 127) / 128), 128, 0, lat->stream>>>(lat->clov64, lat->g, 4.0 + m0, inv);
    qs_note_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_clover_inverse_odd"); return QS_ECUDA; }
    return QS_OK;
}

int qs_dhat_run(qs_lattice *lat, double m0, const double *in, double *out, int nrhs, int gamma5, double *work,
                const double2 *inv)
{
    const Geom &g = lat->g;
    cudaStream_t st = lat->stream;
    const int64_t vlen = (int64_t)nrhs * g.Ns * 24;
    double *x = work, *dx = work + vlen, *v = work + 2 * vlen;
    DslashArgs<double> d;
    d.g = g;
    d.links = lat->links64;
    d.clov = lat->clov64;
    d.nrhs = nrhs;
    for (int r = 0; r < nrhs; ++r) d.m0[r] = m0;
    const int64_t n = g.Ns * 12 * nrhs;
    const unsigned nb = (unsigned)((n + 255) / 256), nbs = (unsigned)((g.Ns * nrhs + 127) / 128);
    parity_mask_kernel<<<nb, 256, 0, st>>>((const double2 *)in, (double2 *)x, g, nrhs, 0);
    d.in = x;
    d.out = dx;
    d.gamma5 = 0;
    cudaError_t e = qs_dslash64_parity_launch(d, 1, st);                                     // (D x)_o
    if (e == cudaSuccess) {
        if (inv)
            clover_apply_inv_kernel<<<(unsigned)((g.Ns / 2 * nrhs + 127) / 128), 128, 0, st>>>(
                inv, (const double2 *)dx, (const double2 *)x, (double2 *)v, g, nrhs);          // v = x - u
        else
            clover_solve_odd_kernel<<<nbs, 128, 0, st>>>(lat->clov64, (const double2 *)dx, (const double2 *)x,
                                                         (double2 *)v, g, nrhs, 4.0 + m0);

        d.in = v;
        d.out = out;
        d.gamma5 = gamma5;
        e = qs_dslash64_parity_launch(d, 0, st);                                             // (D v)_e
    }
    qs_note_launches(4);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_dhat_run"); return QS_ECUDA; }
    return QS_OK;
}

int qs_even_mask(qs_lattice *lat, const double *in, double *out, int nrhs)
{
    const int64_t n = lat->g.Ns * 12 * nrhs;
    parity_mask_kernel<<<(unsigned)((n + 255) / 256), 256, 0, lat->stream>>>((const double2 *)in, (double2 *)out,
                                                                             lat->g, nrhs, 0);
    qs_note_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_even_mask"); return QS_ECUDA; }
    return QS_OK;
}

extern "C" int qs_apply_Dhat(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int gamma5)
{
    if (!lat || !in || !out || nrhs < 1 || nrhs > 64) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    const Geom &g = lat->g;
    if ((g.T | g.L) & 1) return QS_EINVAL;   // hopping must connect opposite parities only
    const size_t bytes = (size_t)nrhs * g.Ns * 24 * sizeof(double);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return QS_EINVAL;
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    double *buf = nullptr;
    QS_CUDA(cudaMalloc(&buf, 3 * bytes));
    int s = qs_dhat_run(lat, m0, (const double *)in, (double *)out, nrhs, gamma5, buf, nullptr);
    if (s == QS_OK) {
        const cudaError_t e = cudaStreamSynchronize(lat->stream);
        if (e != cudaSuccess) { qs_record_cuda_error(e, "qs_apply_Dhat"); s = QS_ECUDA; }
    }
    cudaFree(buf);
    return s;
}
