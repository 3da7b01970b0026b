// Vector, block and reduction kernels of the eigensolver and the CG.
// Reductions are two-stage with a fixed grid (QS_RED_BLOCKS partials per
// vector, then one fixed-order pass), so results are bit-reproducible.
#include "blas.cuh"

#include <type_traits>

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum (blockDim.x a multiple of 32, <= 1024); result valid in thread 0
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

template <typename R>
__global__ void norm2_part(const R *__restrict__ v, int64_t nr, double *part)
{
    const R *x = v + (int64_t)blockIdx.y * nr;
    R acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        R a = x[i];
        acc += a * a;
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// sum of nb partials per output (one block per output), fixed order
__global__ void finalize_sum(const double *part, int nb, int stride_out, double *out)
{
    const double *p = part + (int64_t)blockIdx.x * nb;
    double acc = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += p[i];
    double s = block_sum(acc);
    if (threadIdx.x == 0) out[(int64_t)blockIdx.x * stride_out] = s;
}

template <typename R>
__global__ void dot_part(const R *__restrict__ a, const R *__restrict__ b, int64_t nr, double *part)
{
    const R *x = a + (int64_t)blockIdx.y * nr;
    const R *y = b + (int64_t)blockIdx.y * nr;
    R re = 0, im = 0;
    int64_t nc = nr / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        R ar = x[2 * i], ai = x[2 * i + 1], br = y[2 * i], bi = y[2 * i + 1];
        re += ar * br + ai * bi;
        im += ar * bi - ai * br;
    }
    double sr = block_sum((double)re);
    double si = block_sum((double)im);
    if (threadIdx.x == 0) {
        part[(2 * blockIdx.y) * gridDim.x + blockIdx.x] = sr;
        part[(2 * blockIdx.y + 1) * gridDim.x + blockIdx.x] = si;
    }
}

__global__ void resid_part(const double *__restrict__ a, const double *__restrict__ b, const double *theta,
                           int64_t nr, double *part)
{
    const double *x = a + (int64_t)blockIdx.y * nr;
    const double *y = b + (int64_t)blockIdx.y * nr;
    double t = theta[blockIdx.y];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        double d = x[i] - t * y[i];
        acc += d * d;
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Gram partials: each block accumulates G[i][j] over chunks of GCH complex
// elements staged in shared memory; pair q = i * kb + j, thread owns q = tid + 256 m.
#define GCH 32
#define GMAXP 16
// LOWP: products and the sum over one chunk of GCH elements in FP32, chunk sums
// accumulated in FP64 (one FP64 add per chunk instead of four FMAs per element)
template <bool LOWP>
__global__ void __launch_bounds__(256) gram_part(const double *__restrict__ A, int ka,
                                                 const double *__restrict__ B, int kb, int64_t nc,
                                                 double *part)
{
    // FP64 staging: double2 [ka + kb][GCH]; FP32 staging (LOWP): float2, converted once
    // per element when loaded (FP64 -> FP32 conversions run on the FP64 pipe)
    extern __shared__ double2 gsh[];
    float2 *gsf = reinterpret_cast<float2 *>(gsh);
    const double2 *A2 = reinterpret_cast<const double2 *>(A);
    const double2 *B2 = reinterpret_cast<const double2 *>(B);
    const int P = ka * kb;
    double ar[GMAXP], ai[GMAXP];
#pragma unroll
    for (int m = 0; m < GMAXP; ++m) { ar[m] = 0; ai[m] = 0; }
    int64_t nchunks = (nc + GCH - 1) / GCH;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int64_t e0 = ch * GCH;
        __syncthreads();
        for (int t = threadIdx.x; t < (ka + kb) * GCH; t += blockDim.x) {
            int v = t / GCH, e = t % GCH;
            int64_t idx = e0 + e;
            double2 val = make_double2(0, 0);
            if (idx < nc) val = v < ka ? A2[(int64_t)v * nc + idx] : B2[(int64_t)(v - ka) * nc + idx];
            if (LOWP) gsf[t] = make_float2((float)val.x, (float)val.y);
            else gsh[t] = val;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < GMAXP; ++m) {
            int q = threadIdx.x + 256 * m;
            if (q < P) {
                int i = q / kb, j = q % kb;
                if (LOWP) {
                    const float2 *x = gsf + i * GCH, *y = gsf + (ka + j) * GCH;
                    float re = 0.f, im = 0.f;
#pragma unroll 8
                    for (int e = 0; e < GCH; ++e) {
                        float2 u = x[e], w = y[e];
                        re = fmaf(u.x, w.x, fmaf(u.y, w.y, re));
                        im = fmaf(u.x, w.y, fmaf(-u.y, w.x, im));
                    }
                    ar[m] += re; ai[m] += im;
                } else {
                    const double2 *x = gsh + i * GCH, *y = gsh + (ka + j) * GCH;
                    double re = ar[m], im = ai[m];
#pragma unroll 8
                    for (int e = 0; e < GCH; ++e) {
                        double2 u = x[e], w = y[e];
                        re = fma(u.x, w.x, fma(u.y, w.y, re));
                        im = fma(u.x, w.y, fma(-u.y, w.x, im));
                    }
                    ar[m] = re; ai[m] = im;
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < GMAXP; ++m) {
        int q = threadIdx.x + 256 * m;
        if (q < P) {
            part[((int64_t)2 * q) * gridDim.x + blockIdx.x] = ar[m];
            part[((int64_t)2 * q + 1) * gridDim.x + blockIdx.x] = ai[m];
        }
    }
}

// LOWP: the k-term sums in FP32 (inputs rounded to FP32), stored as FP64
template <bool LOWP>
__global__ void rotate_kernel(const double *__restrict__ W, int ka, const double2 *__restrict__ C, int kc,
                              int64_t nc, double *__restrict__ V)
{
    extern __shared__ double2 csh[];
    float2 *csf = reinterpret_cast<float2 *>(csh);
    for (int t = threadIdx.x; t < ka * kc; t += blockDim.x) {
        if (LOWP) csf[t] = make_float2((float)C[t].x, (float)C[t].y);
        else csh[t] = C[t];
    }
    __syncthreads();
    const double2 *W2 = reinterpret_cast<const double2 *>(W);
    double2 *V2 = reinterpret_cast<double2 *>(V);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
        for (int j0 = 0; j0 < kc; j0 += 8) {
            typedef typename std::conditional<LOWP, float, double>::type T;
            T re[8], im[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) { re[jj] = 0; im[jj] = 0; }
            for (int i = 0; i < ka; ++i) {
                double2 w = W2[(int64_t)i * nc + e];
                T wx = (T)w.x, wy = (T)w.y;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    if (j0 + jj < kc) {
                        T cx, cy;
                        if (LOWP) { float2 c = csf[i * kc + j0 + jj]; cx = c.x; cy = c.y; }
                        else { double2 c = csh[i * kc + j0 + jj]; cx = (T)c.x; cy = (T)c.y; }
                        re[jj] = wx * cx - wy * cy + re[jj];
                        im[jj] = wx * cy + wy * cx + im[jj];
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (j0 + jj < kc) V2[(int64_t)(j0 + jj) * nc + e] = make_double2((double)re[jj], (double)im[jj]);
        }
    }
}

__global__ void d2f_kernel(const double *__restrict__ x, float *__restrict__ y, const double *scale, int64_t nr)
{
    double s = scale ? scale[blockIdx.y] : 1.0;
    const double *a = x + (int64_t)blockIdx.y * nr;
    float *b = y + (int64_t)blockIdx.y * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)(a[i] * s);
}

__global__ void f2d_kernel(const float *__restrict__ x, double *__restrict__ y, int64_t nr)
{
    const float *a = x + (int64_t)blockIdx.y * nr;
    double *b = y + (int64_t)blockIdx.y * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

__global__ void axpy_f2d_kernel(double *__restrict__ x, const float *__restrict__ e, const double *coef, int64_t nr)
{
    double c = coef[blockIdx.y];
    double *a = x + (int64_t)blockIdx.y * nr;
    const float *b = e + (int64_t)blockIdx.y * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += c * (double)b[i];
}

__global__ void scale_cols_kernel(double *x, const double *scale, int64_t nr)
{
    double c = scale[blockIdx.y];
    double *a = x + (int64_t)blockIdx.y * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        a[i] *= c;
}

__global__ void scaled_copy_kernel(double *x, const double *b, const double *coef, int64_t nr)
{
    double c = coef[blockIdx.y];
    double *a = x + (int64_t)blockIdx.y * nr;
    const double *q = b + (int64_t)blockIdx.y * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = c * q[i];
}

template <typename R>
__global__ void cheb_kernel(R *__restrict__ ynew, const R *__restrict__ ay, const R *__restrict__ y,
                            const R *__restrict__ x, R c, R s1, R s2, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ynew[i] = s1 * (ay[i] - c * y[i]) - s2 * x[i];
}

template <typename R>
__global__ void axpby_kernel(R a, const R *__restrict__ x, R b, R *__restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void gauss_kernel(double *x, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t h1 = splitmix64(seed ^ splitmix64(2 * (uint64_t)i));
        uint64_t h2 = splitmix64(seed ^ splitmix64(2 * (uint64_t)i + 1));
        double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double u2 = ((h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

__global__ void map_scalars_kernel(const double *in, double *out, int k, int mode)
{
    int r = threadIdx.x;
    if (r >= k) return;
    double v = in[r];
    if (mode == 0) out[r] = v > 0 ? 1.0 / sqrt(v) : 0.0;      // 1/sqrt
    else if (mode == 1) out[r] = sqrt(v > 0 ? v : 0.0);        // sqrt
    else if (mode == 2) out[r] = v != 0 ? 1.0 / (v * v) : 0.0; // theta^-2
    else out[r] = v;
}

// ---- CG (FP32 vectors, FP64 scalars) ----------------------------------------
__global__ void cg_update_kernel(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
                                 const float *__restrict__ ap, CgScalars s, int64_t nr, double *part)
{
    int q = blockIdx.y;
    double al = (s.active[q] && s.pap[q] > 0) ? s.rr[q] / s.pap[q] : 0.0;
    float a = (float)al;
    float *xq = x + (int64_t)q * nr, *rq = r + (int64_t)q * nr;
    const float *pq = p + (int64_t)q * nr, *aq = ap + (int64_t)q * nr;
    float acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        xq[i] += a * pq[i];
        float rv = rq[i] - a * aq[i];
        rq[i] = rv;
        acc += rv * rv;
    }
    double sm = block_sum((double)acc);
    if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = sm;
}

__global__ void cg_finalize_kernel(CgScalars s, double tol2, int k, const double *part, int nb, int *nactive)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int q = 0; q < k; ++q) {
        double acc = 0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[q * nb + i];
        double rn = block_sum(acc);
        if (threadIdx.x == 0) {
            int act = s.active[q];
            s.beta[q] = (act && s.rr[q] > 0) ? rn / s.rr[q] : 0.0;
            if (act) s.rr[q] = rn;
            act = act && (rn > tol2 * s.rr0[q]) && isfinite(rn);
            s.active[q] = act;
            cnt += act;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *nactive = cnt;
}

__global__ void cg_p_kernel(float *__restrict__ p, const float *__restrict__ r, CgScalars s, int64_t nr)
{
    int q = blockIdx.y;
    if (!s.active[q]) return;
    float b = (float)s.beta[q];
    float *pq = p + (int64_t)q * nr;
    const float *rq = r + (int64_t)q * nr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
        pq[i] = rq[i] + b * pq[i];
}

__global__ void cg_init_kernel(CgScalars s, const double *rr, int k)
{
    int q = threadIdx.x;
    if (q >= k) return;
    s.rr[q] = rr[q];
    s.rr0[q] = rr[q];
    s.beta[q] = 0;
    s.active[q] = rr[q] > 0;
}

inline int grid_for(int64_t n, int per = 256)
{
    int64_t b = (n + per - 1) / per;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

}  // namespace

template <typename R>
cudaError_t qs_norm2(const R *v, int k, int64_t nr, double *part, double *out, cudaStream_t st)
{
    dim3 g(QS_RED_BLOCKS, k);
    norm2_part<R><<<g, QS_RED_THREADS, 0, st>>>(v, nr, part);
    finalize_sum<<<k, 256, 0, st>>>(part, QS_RED_BLOCKS, 1, out);
    qs_note_launches(2);
    return cudaGetLastError();
}
template cudaError_t qs_norm2<float>(const float *, int, int64_t, double *, double *, cudaStream_t);
template cudaError_t qs_norm2<double>(const double *, int, int64_t, double *, double *, cudaStream_t);

template <typename R>
cudaError_t qs_dot(const R *a, const R *b, int k, int64_t nr, double *part, double *out, cudaStream_t st)
{
    dim3 g(QS_RED_BLOCKS, k);
    dot_part<R><<<g, QS_RED_THREADS, 0, st>>>(a, b, nr, part);
    finalize_sum<<<2 * k, 256, 0, st>>>(part, QS_RED_BLOCKS, 1, out);
    qs_note_launches(2);
    return cudaGetLastError();
}
template cudaError_t qs_dot<float>(const float *, const float *, int, int64_t, double *, double *, cudaStream_t);
template cudaError_t qs_dot<double>(const double *, const double *, int, int64_t, double *, double *, cudaStream_t);

cudaError_t qs_resid2(const double *a, const double *b, const double *theta, int k, int64_t nr,
                      double *part, double *out, cudaStream_t st)
{
    dim3 g(QS_RED_BLOCKS, k);
    resid_part<<<g, QS_RED_THREADS, 0, st>>>(a, b, theta, nr, part);
    finalize_sum<<<k, 256, 0, st>>>(part, QS_RED_BLOCKS, 1, out);
    qs_note_launches(2);
    return cudaGetLastError();
}

cudaError_t qs_gram(const double *A, int ka, const double *B, int kb, int64_t nr, double *part,
                    double2 *G, cudaStream_t st, int lowp)
{
    if (ka * kb > 256 * GMAXP) return cudaErrorInvalidValue;
    int64_t nc = nr / 2;
    size_t sm = (size_t)(ka + kb) * GCH * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gram_part<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * GCH * 16);
        cudaFuncSetAttribute(gram_part<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * GCH * 16);
        attr = true;
    }
    int64_t nch = (nc + GCH - 1) / GCH;
    int nb = (int)(nch < QS_RED_BLOCKS ? nch : QS_RED_BLOCKS);
    if (lowp) gram_part<true><<<nb, 256, sm, st>>>(A, ka, B, kb, nc, part);
    else gram_part<false><<<nb, 256, sm, st>>>(A, ka, B, kb, nc, part);
    finalize_sum<<<2 * ka * kb, 256, 0, st>>>(part, nb, 1, reinterpret_cast<double *>(G));
    qs_note_launches(2);
    return cudaGetLastError();
}

cudaError_t qs_rotate(const double *W, int ka, const double2 *C, int kc, int64_t nr, double *V, cudaStream_t st,
                      int lowp)
{
    int64_t nc = nr / 2;
    size_t sm = (size_t)ka * kc * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rotate_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * 16);
        cudaFuncSetAttribute(rotate_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * 16);
        attr = true;
    }
    if (lowp) rotate_kernel<true><<<grid_for(nc, 256), 256, sm, st>>>(W, ka, C, kc, nc, V);
    else rotate_kernel<false><<<grid_for(nc, 256), 256, sm, st>>>(W, ka, C, kc, nc, V);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_d2f(const double *x, float *y, const double *scale, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    d2f_kernel<<<g, 256, 0, st>>>(x, y, scale, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_f2d(const float *x, double *y, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    f2d_kernel<<<g, 256, 0, st>>>(x, y, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_axpy_f2d(double *x, const float *e, const double *coef, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    axpy_f2d_kernel<<<g, 256, 0, st>>>(x, e, coef, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_scale_cols(double *x, const double *scale, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    scale_cols_kernel<<<g, 256, 0, st>>>(x, scale, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_scaled_copy(double *x, const double *b, const double *coef, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    scaled_copy_kernel<<<g, 256, 0, st>>>(x, b, coef, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

template <typename R>
cudaError_t qs_cheb_step(R *ynew, const R *ay, const R *y, const R *x, double c, double s1, double s2,
                         int64_t n, cudaStream_t st)
{
    cheb_kernel<R><<<grid_for(n), 256, 0, st>>>(ynew, ay, y, x, (R)c, (R)s1, (R)s2, n);
    qs_note_launches(1);
    return cudaGetLastError();
}
template cudaError_t qs_cheb_step<float>(float *, const float *, const float *, const float *, double, double, double, int64_t, cudaStream_t);
template cudaError_t qs_cheb_step<double>(double *, const double *, const double *, const double *, double, double, double, int64_t, cudaStream_t);

template <typename R>
cudaError_t qs_axpby(double a, const R *x, double b, R *y, int64_t n, cudaStream_t st)
{
    axpby_kernel<R><<<grid_for(n), 256, 0, st>>>((R)a, x, (R)b, y, n);
    qs_note_launches(1);
    return cudaGetLastError();
}
template cudaError_t qs_axpby<float>(double, const float *, double, float *, int64_t, cudaStream_t);
template cudaError_t qs_axpby<double>(double, const double *, double, double *, int64_t, cudaStream_t);

cudaError_t qs_fill_gauss(double *x, int64_t n, uint64_t seed, cudaStream_t st)
{
    gauss_kernel<<<grid_for(n), 256, 0, st>>>(x, n, seed);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_map_scalars(const double *in, double *out, int k, int mode, cudaStream_t st)
{
    map_scalars_kernel<<<1, 64, 0, st>>>(in, out, k, mode);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_cg_update(float *x, float *r, const float *p, const float *ap, CgScalars s, int k, int64_t nr,
                         double *part, cudaStream_t st)
{
    dim3 g(QS_RED_BLOCKS, k);
    cg_update_kernel<<<g, QS_RED_THREADS, 0, st>>>(x, r, p, ap, s, nr, part);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_cg_finalize(CgScalars s, double tol2, int k, double *part, int *nactive, cudaStream_t st)
{
    cg_finalize_kernel<<<1, 256, 0, st>>>(s, tol2, k, part, QS_RED_BLOCKS, nactive);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_cg_pupdate(float *p, const float *r, CgScalars s, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    cg_p_kernel<<<g, 256, 0, st>>>(p, r, s, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_cg_init(CgScalars s, const double *rr, int k, cudaStream_t st)
{
    cg_init_kernel<<<1, 64, 0, st>>>(s, rr, k);
    qs_note_launches(1);
    return cudaGetLastError();
}
