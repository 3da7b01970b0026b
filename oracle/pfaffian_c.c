/* Pfaffian of a complex antisymmetric matrix by Parlett-Reid elimination with
 * partial pivoting (Wimmer, ACM TOMS 38, 30 (2012)); plain C, test
 * infrastructure of the CPU oracle only.  Same steps as oracle/pfaffian.py:
 * for k = 0, 2, 4, ...: bring the largest |A[k][j]|, j > k, to column k+1
 * (a swap of index k+1 and p flips the sign), take a = A[k][k+1] into the
 * product, and replace the trailing block by A' + (c b^T - b c^T) / a with
 * b = A[k][k+2:], c = A[k+1][k+2:].  The result is (log|pf|, phase).
 * A (row-major, n x n) is overwritten.  Returns 0, or 1 if pf = 0. */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

int pf_parlett_reid(long n, double complex *A, double *logabs, double *ph_re, double *ph_im)
{
    double la = 0.0;
    double complex ph = 1.0;
    if (n % 2) { *logabs = -INFINITY; *ph_re = 0; *ph_im = 0; return 1; }
    double complex *b = malloc(sizeof(double complex) * n);
    double complex *c = malloc(sizeof(double complex) * n);
    for (long k = 0; k + 1 < n; k += 2) {
        long p = k + 1;
        double best = cabs(A[k * n + k + 1]);
        for (long j = k + 2; j < n; ++j) {
            double v = cabs(A[k * n + j]);
            if (v > best) { best = v; p = j; }
        }
        if (p != k + 1) {
            for (long j = 0; j < n; ++j) {           /* swap rows */
                double complex t = A[(k + 1) * n + j];
                A[(k + 1) * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
            for (long i = 0; i < n; ++i) {           /* swap columns */
                double complex t = A[i * n + k + 1];
                A[i * n + k + 1] = A[i * n + p];
                A[i * n + p] = t;
            }
            ph = -ph;
        }
        double complex a = A[k * n + k + 1];
        if (a == 0.0) { free(b); free(c); *logabs = -INFINITY; *ph_re = 0; *ph_im = 0; return 1; }
        la += log(cabs(a));
        ph *= a / cabs(a);
        long m = n - k - 2;
        if (m <= 0) break;
        for (long j = 0; j < m; ++j) {
            b[j] = A[k * n + k + 2 + j];
            c[j] = A[(k + 1) * n + k + 2 + j] / a;
        }
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < m; ++i) {
            double complex ci = c[i], bi = b[i];
            double complex *row = A + (k + 2 + i) * n + k + 2;
            for (long j = 0; j < m; ++j)
                row[j] += ci * b[j] - bi * c[j];
        }
    }
    free(b); free(c);
    *logabs = la; *ph_re = creal(ph); *ph_im = cimag(ph);
    return 0;
}
