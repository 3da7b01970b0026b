// Vector, block and reduction kernels of the eigensolver and the CG.
// Reductions are two-stage with a fixed grid (QS_RED_BLOCKS partials per
// vector, then one fixed-order pass), so results are bit-reproducible.
#include "blas.cuh"

#include <mutex>
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

template <typename R>
__global__ void resid_part(const R *__restrict__ a, const R *__restrict__ b, const double *theta,
                           int64_t nr, double *part)
{
    const R *x = a + (int64_t)blockIdx.y * nr;
    const R *y = b + (int64_t)blockIdx.y * nr;
    const R t = (R)theta[blockIdx.y];
    R acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        R d = x[i] - t * y[i];
        acc += d * d;
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Gram partials G[i][j] = sum_e conj(A_i[e]) B_j[e] (i < ka, j < kb <= 64).  A block
// stages a chunk of GE elements of all ka + kb vectors in shared memory, element-major
// ([e][vector], row padded by one complex to spread the banks); each thread owns a 4 x 4
// tile of (i, j) and a residue class of the chunk's elements, so every staged value it
// reads feeds four complex multiply-adds.  The element classes of a tile are summed in
// shared memory at the end, in a fixed order.  LOWP: values rounded to FP32, products
// and the sum over one chunk in FP32, chunk sums added in FP64.
#define GE 64
// (hi, lo) += x, with hi + lo exact to the rounding of the final add (Knuth's two-sum)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}
__device__ __forceinline__ void two_sum_acc(double &hi, double &lo, double x) { hi += x; }

template <bool LOWP, typename TIn = double2>
__global__ void __launch_bounds__(256, LOWP ? 2 : 1) gram_tile_kernel(const TIn *__restrict__ A_, int ka,
                                                           const TIn *__restrict__ B_, int kb, int64_t nc,
                                                           double *part)
{
    typedef typename std::conditional<LOWP, float2, double2>::type V2;
    typedef typename std::conditional<LOWP, float, double>::type T;
    extern __shared__ __align__(16) unsigned char gsm_raw[];
    V2 *sv = reinterpret_cast<V2 *>(gsm_raw);
    const int kk = ka + kb, row = kk + 1;            // padded row of one element
    const int ti_n = (ka + 3) / 4, tj_n = (kb + 3) / 4, ntile = ti_n * tj_n;
    const int eg_n = 256 / ntile;                     // element classes (>= 1)
    const int t = threadIdx.x;
    const int tile = t % ntile, eg = t / ntile;
    const bool active = eg < eg_n;
    const int i0 = 4 * (tile / tj_n), j0 = 4 * (tile % tj_n);
    // running totals: FP64 (FP64 products), or an FP32 (hi, lo) pair per real sum kept
    // exact to ~2^-48 by Knuth's two-sum (FP32 products: GB300's FP64 pipe is too slow
    // for a per-chunk FP64 add)
    typedef typename std::conditional<LOWP, float, double>::type A;
    A acc[4][4][2], accl[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = accl[a][b][0] = accl[a][b][1] = (A)0;
    const int64_t nch = (nc + GE - 1) / GE;
    const int nq = kk * GE;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int64_t e0 = ch * GE;
        __syncthreads();
        // staging: SU independent loads in flight per thread before their stores
        constexpr int SU = LOWP ? 4 : 8;
        for (int q0 = t; q0 < nq; q0 += 256 * SU) {
            TIn val[SU];
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int q = q0 + 256 * u;
                val[u].x = 0;
                val[u].y = 0;
                if (q < nq) {
                    const int v = q / GE, e = q % GE;
                    const int64_t idx = e0 + e;
                    if (idx < nc) val[u] = v < ka ? __ldg(A_ + (int64_t)v * nc + idx) : __ldg(B_ + (int64_t)(v - ka) * nc + idx);
                }
            }
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int q = q0 + 256 * u;
                if (q < nq) {
                    V2 x;
                    x.x = (T)val[u].x;
                    x.y = (T)val[u].y;
                    sv[(q % GE) * row + q / GE] = x;
                }
            }
        }
        __syncthreads();
        if (!active) continue;
        if constexpr (LOWP) {
            // FP32 sums over the chunk, added to the (hi, lo) totals once per chunk
            float cr[4][4], ci[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cr[a][b] = ci[a][b] = 0.f;
            for (int e = eg; e < GE; e += eg_n) {
                const V2 *r = sv + e * row;
                V2 x[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a] = (i0 + a < ka) ? r[i0 + a] : V2{0.f, 0.f};
#pragma unroll
                for (int b = 0; b < 4; ++b) y[b] = (j0 + b < kb) ? r[ka + j0 + b] : V2{0.f, 0.f};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {   // conj(x) y
                        cr[a][b] = fmaf(x[a].x, y[b].x, fmaf(x[a].y, y[b].y, cr[a][b]));
                        ci[a][b] = fmaf(x[a].x, y[b].y, fmaf(-x[a].y, y[b].x, ci[a][b]));
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    two_sum_acc(acc[a][b][0], accl[a][b][0], cr[a][b]);
                    two_sum_acc(acc[a][b][1], accl[a][b][1], ci[a][b]);
                }
        } else {
            for (int e = eg; e < GE; e += eg_n) {
                const V2 *r = sv + e * row;
                V2 x[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a] = (i0 + a < ka) ? r[i0 + a] : V2{0.0, 0.0};
#pragma unroll
                for (int b = 0; b < 4; ++b) y[b] = (j0 + b < kb) ? r[ka + j0 + b] : V2{0.0, 0.0};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {   // conj(x) y
                        acc[a][b][0] = fma(x[a].x, y[b].x, fma(x[a].y, y[b].y, acc[a][b][0]));
                        acc[a][b][1] = fma(x[a].x, y[b].y, fma(-x[a].y, y[b].x, acc[a][b][1]));
                    }
            }
        }
    }
    // sum the element classes of each tile (fixed order), reusing the staging buffer
    __syncthreads();
    double *red = reinterpret_cast<double *>(gsm_raw);   // [ntile][32] partial of class 0 ...
    for (int c = 0; c < eg_n; ++c) {
        if (active && eg == c) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    double *d = red + tile * 32 + (a * 4 + b) * 2;
                    const double v0 = (double)acc[a][b][0] + (double)accl[a][b][0];
                    const double v1 = (double)acc[a][b][1] + (double)accl[a][b][1];
                    if (c == 0) { d[0] = v0; d[1] = v1; }
                    else { d[0] += v0; d[1] += v1; }
                }
        }
        __syncthreads();
    }
    for (int q = t; q < ntile * 16; q += 256) {
        const int tl = q / 16, ab = q % 16, a = ab / 4, b = ab % 4;
        const int i = 4 * (tl / tj_n) + a, j = 4 * (tl % tj_n) + b;
        if (i < ka && j < kb) {
            const int pq = i * kb + j;
            part[((int64_t)2 * pq) * gridDim.x + blockIdx.x] = red[tl * 32 + ab * 2];
            part[((int64_t)2 * pq + 1) * gridDim.x + blockIdx.x] = red[tl * 32 + ab * 2 + 1];
        }
    }
}

// V_j = sum_i W_i C[i][j] (j < kc): each thread computes RE elements for a block of
// up to RJ output vectors, the coefficients read from shared memory (the same word for
// all threads of a warp); each W value it loads feeds RJ multiply-adds.  LOWP: values and
// coefficients rounded to FP32, the sums in FP32.
#define RE 2
template <bool LOWP, typename TIn = double2, typename TOut = double2>
__global__ void __launch_bounds__(256, 2) rotate_tile_kernel(const TIn *__restrict__ W, int ka,
                                                             const double2 *__restrict__ C, int kc, int64_t nc,
                                                             TOut *__restrict__ V)
{
    typedef typename std::conditional<LOWP, float2, double2>::type V2;
    typedef typename std::conditional<LOWP, float, double>::type T;
    constexpr int RJ = LOWP ? 16 : 8;   // output columns per pass (register budget)
    extern __shared__ __align__(16) unsigned char rsm_raw[];
    V2 *cs = reinterpret_cast<V2 *>(rsm_raw);         // [ka][kc]
    for (int q = threadIdx.x; q < ka * kc; q += blockDim.x) {
        V2 x;
        x.x = (T)C[q].x;
        x.y = (T)C[q].y;
        cs[q] = x;
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * RE;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * RE + threadIdx.x; base < nc; base += stride) {
        for (int j0 = 0; j0 < kc; j0 += RJ) {
            T ar[RE][RJ], ai[RE][RJ];
#pragma unroll
            for (int u = 0; u < RE; ++u)
#pragma unroll
                for (int jj = 0; jj < RJ; ++jj) ar[u][jj] = ai[u][jj] = (T)0;
            for (int i0 = 0; i0 < ka; i0 += 4) {
                // four input vectors' values loaded together (independent loads in flight)
                T wr[4][RE], wi[4][RE];
#pragma unroll
                for (int di = 0; di < 4; ++di)
#pragma unroll
                    for (int u = 0; u < RE; ++u) {
                        const int64_t e = base + (int64_t)u * blockDim.x;
                        TIn w;
                        w.x = 0;
                        w.y = 0;
                        if (e < nc && i0 + di < ka) w = __ldg(W + (int64_t)(i0 + di) * nc + e);
                        wr[di][u] = (T)w.x;
                        wi[di][u] = (T)w.y;
                    }
#pragma unroll
                for (int di = 0; di < 4; ++di) {
                    if (i0 + di >= ka) break;
                    const V2 *crow = cs + (i0 + di) * kc + j0;
#pragma unroll
                    for (int jj = 0; jj < RJ; ++jj) {
                        if (j0 + jj < kc) {
                            const V2 c = crow[jj];
#pragma unroll
                            for (int u = 0; u < RE; ++u) {
                                ar[u][jj] = fma(wr[di][u], c.x, fma(-wi[di][u], c.y, ar[u][jj]));
                                ai[u][jj] = fma(wr[di][u], c.y, fma(wi[di][u], c.x, ai[u][jj]));
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < RJ; ++jj)
                if (j0 + jj < kc)
#pragma unroll
                    for (int u = 0; u < RE; ++u) {
                        const int64_t e = base + (int64_t)u * blockDim.x;
                        if (e < nc) {
                            TOut o;
                            o.x = ar[u][jj];
                            o.y = ai[u][jj];
                            V[(int64_t)(j0 + jj) * nc + e] = o;
                        }
                    }
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

template <typename R>
__global__ void scale_cols_kernel(R *x, const double *scale, int64_t nr)
{
    const R c = (R)scale[blockIdx.y];
    R *a = x + (int64_t)blockIdx.y * nr;
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

template <typename R>
cudaError_t qs_resid2(const R *a, const R *b, const double *theta, int k, int64_t nr,
                      double *part, double *out, cudaStream_t st)
{
    dim3 g(QS_RED_BLOCKS, k);
    resid_part<R><<<g, QS_RED_THREADS, 0, st>>>(a, b, theta, nr, part);
    finalize_sum<<<k, 256, 0, st>>>(part, QS_RED_BLOCKS, 1, out);
    qs_note_launches(2);
    return cudaGetLastError();
}
template cudaError_t qs_resid2<double>(const double *, const double *, const double *, int, int64_t, double *,
                                       double *, cudaStream_t);
template cudaError_t qs_resid2<float>(const float *, const float *, const double *, int, int64_t, double *, double *,
                                      cudaStream_t);

cudaError_t qs_gram(const double *A, int ka, const double *B, int kb, int64_t nr, double *part,
                    double2 *G, cudaStream_t st, int lowp)
{
    if (ka < 1 || kb < 1 || ka > 64 || kb > 64) return cudaErrorInvalidValue;
    int64_t nc = nr / 2;
    const int row = ka + kb + 1;
    const size_t stage = (size_t)GE * row * (lowp ? sizeof(float2) : sizeof(double2));
    const size_t red = (size_t)((ka + 3) / 4) * ((kb + 3) / 4) * 32 * sizeof(double);
    const size_t sm = stage > red ? stage : red;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(gram_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(gram_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    int64_t nch = (nc + GE - 1) / GE;
    int nb = (int)(nch < QS_RED_BLOCKS ? nch : QS_RED_BLOCKS);
    if (lowp) gram_tile_kernel<true><<<nb, 256, sm, st>>>((const double2 *)A, ka, (const double2 *)B, kb, nc, part);
    else gram_tile_kernel<false><<<nb, 256, sm, st>>>((const double2 *)A, ka, (const double2 *)B, kb, nc, part);
    finalize_sum<<<2 * ka * kb, 256, 0, st>>>(part, nb, 1, reinterpret_cast<double *>(G));
    qs_note_launches(2);
    return cudaGetLastError();
}

cudaError_t qs_rotate(const double *W, int ka, const double2 *C, int kc, int64_t nr, double *V, cudaStream_t st,
                      int lowp)
{
    if (ka < 1 || kc < 1 || ka > 64 || kc > 64) return cudaErrorInvalidValue;
    int64_t nc = nr / 2;
    size_t sm = (size_t)ka * kc * (lowp ? sizeof(float2) : sizeof(double2));
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(rotate_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * 16);
        cudaFuncSetAttribute(rotate_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * 16);
    });
    int64_t blocks = (nc + 256 * RE - 1) / (256 * RE);
    int nb = (int)(blocks < 4 * 152 ? blocks : 4 * 152);
    if (lowp) rotate_tile_kernel<true><<<nb, 256, sm, st>>>((const double2 *)W, ka, C, kc, nc, (double2 *)V);
    else rotate_tile_kernel<false><<<nb, 256, sm, st>>>((const double2 *)W, ka, C, kc, nc, (double2 *)V);
    qs_note_launches(1);
    return cudaGetLastError();
}

// the same contractions on FP32 blocks (products and per-chunk sums in FP32)
cudaError_t qs_gram32(const float *A, int ka, const float *B, int kb, int64_t nr, double *part, double2 *G,
                      cudaStream_t st)
{
    if (ka < 1 || kb < 1 || ka > 64 || kb > 64) return cudaErrorInvalidValue;
    int64_t nc = nr / 2;
    const int row = ka + kb + 1;
    const size_t stage = (size_t)GE * row * sizeof(float2);
    const size_t red = (size_t)((ka + 3) / 4) * ((kb + 3) / 4) * 32 * sizeof(double);
    const size_t sm = stage > red ? stage : red;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(gram_tile_kernel<true, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    int64_t nch = (nc + GE - 1) / GE;
    int nb = (int)(nch < QS_RED_BLOCKS ? nch : QS_RED_BLOCKS);
    gram_tile_kernel<true, float2><<<nb, 256, sm, st>>>((const float2 *)A, ka, (const float2 *)B, kb, nc, part);
    finalize_sum<<<2 * ka * kb, 256, 0, st>>>(part, nb, 1, reinterpret_cast<double *>(G));
    qs_note_launches(2);
    return cudaGetLastError();
}

cudaError_t qs_rotate32(const float *W, int ka, const double2 *C, int kc, int64_t nr, float *V, cudaStream_t st)
{
    if (ka < 1 || kc < 1 || ka > 64 || kc > 64) return cudaErrorInvalidValue;
    int64_t nc = nr / 2;
    size_t sm = (size_t)ka * kc * sizeof(float2);
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(rotate_tile_kernel<true, float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             64 * 64 * 8);
    });
    int64_t blocks = (nc + 256 * RE - 1) / (256 * RE);
    int nb = (int)(blocks < 4 * 152 ? blocks : 4 * 152);
    rotate_tile_kernel<true, float2, float2><<<nb, 256, sm, st>>>((const float2 *)W, ka, C, kc, nc, (float2 *)V);
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

template <typename R>
cudaError_t qs_scale_cols(R *x, const double *scale, int k, int64_t nr, cudaStream_t st)
{
    dim3 g(grid_for(nr) / k + 1, k);
    scale_cols_kernel<R><<<g, 256, 0, st>>>(x, scale, nr);
    qs_note_launches(1);
    return cudaGetLastError();
}
template cudaError_t qs_scale_cols<double>(double *, const double *, int, int64_t, cudaStream_t);
template cudaError_t qs_scale_cols<float>(float *, const double *, int, int64_t, cudaStream_t);

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
