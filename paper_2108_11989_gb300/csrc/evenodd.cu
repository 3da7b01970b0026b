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
