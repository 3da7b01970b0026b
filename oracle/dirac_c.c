/* Plain-loop FP64 restatement of the O(a)-improved Wilson-Dirac operator on the
 * C*-doubled lattice (test infrastructure only: the CPU oracle).
 *
 *   (D psi)(x) = (4 + m0) psi(x) + A(x) psi(x)
 *                - 1/2 sum_mu [ bf_mu(x) (1 - g_mu) V(x, mu) psi(x + mu)
 *                             + bb_mu(x) (1 + g_mu) V(x - mu, mu)^+ psi(x - mu) ]
 *
 * (Sec. 2 operator; Sec. 3 doublet on the doubled lattice.)  Every input is the
 * oracle's own Python construction: the doubled links V (U exp(i theta), mirror half
 * conjugated), the 12 x 12 SW blocks A(x), the neighbour tables with their fermion
 * boundary factors, and the four gamma matrices.  Index order of a spinor: site,
 * spin, colour.  One output site per loop iteration; OpenMP over sites.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>

typedef double complex cplx;

/* out = D(m0) in (gamma5 = 0) or Q(m0) in = gamma_5 D(m0) in (gamma5 = 1).
 * V[ns][4][3][3], A[ns][12][12], fw/bw[4][ns] neighbour sites, bcf/bcb[4][ns] factors,
 * gam[4][4][4]; in/out[ns][4][3]. */
void wd_apply(long ns, const cplx *V, const cplx *A, const long *fw, const long *bw, const double *bcf,
              const double *bcb, const cplx *gam, double m0, int gamma5, const cplx *in, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (long x = 0; x < ns; ++x) {
        cplx r[12];
        for (int k = 0; k < 12; ++k) {
            cplx s = (4.0 + m0) * in[x * 12 + k];
            for (int l = 0; l < 12; ++l) s += A[(x * 12 + k) * 12 + l] * in[x * 12 + l];
            r[k] = s;
        }
        for (int mu = 0; mu < 4; ++mu) {
            const long y = fw[mu * ns + x], z = bw[mu * ns + x];
            const cplx *Uf = V + (x * 4 + mu) * 9;     /* V(x, mu) */
            const cplx *Ub = V + (z * 4 + mu) * 9;     /* V(x - mu, mu) */
            const cplx *g = gam + mu * 16;
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                    cplx hf = 0, hb = 0;
                    for (int b = 0; b < 4; ++b) {
                        const cplx pm = (a == b ? 1.0 : 0.0) - g[a * 4 + b];   /* (1 - g_mu)_ab */
                        const cplx pp = (a == b ? 1.0 : 0.0) + g[a * 4 + b];   /* (1 + g_mu)_ab */
                        for (int j = 0; j < 3; ++j) {
                            hf += pm * Uf[i * 3 + j] * in[y * 12 + b * 3 + j];
                            hb += pp * conj(Ub[j * 3 + i]) * in[z * 12 + b * 3 + j];
                        }
                    }
                    r[a * 3 + i] -= 0.5 * (bcf[mu * ns + x] * hf + bcb[mu * ns + x] * hb);
                }
        }
        for (int k = 0; k < 12; ++k) out[x * 12 + k] = (gamma5 && k >= 6) ? -r[k] : r[k];
    }
}

/* ||Q(m0) v_i - theta_i v_i|| for k vectors v (each ns * 12 complex), Q as wd_apply */
void wd_residuals(long ns, const cplx *V, const cplx *A, const long *fw, const long *bw, const double *bcf,
                  const double *bcb, const cplx *gam, double m0, int k, const cplx *vecs, const double *theta,
                  cplx *work, double *res)
{
    for (int i = 0; i < k; ++i) {
        const cplx *v = vecs + (size_t)i * ns * 12;
        wd_apply(ns, V, A, fw, bw, bcf, bcb, gam, m0, 1, v, work);
        double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
        for (long q = 0; q < ns * 12; ++q) {
            cplx d = work[q] - theta[i] * v[q];
            s += creal(d) * creal(d) + cimag(d) * cimag(d);
        }
        res[i] = sqrt(s);
    }
}
