// The operator D and Q = gamma_5 D with FP32 arithmetic (Sec. 2 operator on the
// C*-doubled lattice, Sec. 3 doublet and Q) for FP32 or 16-bit spinor storage.
//
//   out = (4 + m0) psi + A psi - 1/2 sum_mu [ V (1 - g_mu) psi(x+mu) + V^+ (1 + g_mu) psi(x-mu) ]
//
// Thread map.  A block has 128 threads.  Each warp covers 32 / RL consecutive sites
// and RL "RHS lanes"; a thread computes its site for G right-hand sides.  The RL
// lanes of one site load the same link and SW-term words in the same instruction, so
// a link or SW word leaves L1 once for RL * G right-hand sides, and a thread applies
// every link it loads to G right-hand sides.  Blocks run through all sites of one
// group of RL * G right-hand sides before the next group starts, so the spinor
// neighbours a block needs were read recently by its neighbouring blocks (the
// working set of one group, a few time slices of RL * G vectors, stays in L2).
//
// Storage.  FP32: the solver's site-tiled layout [site / 16][12][site % 16] float2 or
// the canonical [site][12] float2.  FP16 / BF16: tiles of 16 sites, 12 x 16 half2 (or
// bf162) components followed by 16 FP32 scales (832 B per tile); a site's 24 reals are
// stored divided by the largest of their magnitudes, which is its scale.  Arithmetic
// is FP32 throughout.
//
// Epilogue.  PLAIN: out = D in or Q in.  CHEB: one step of the scaled Chebyshev
// recurrence of the filter, out = s1 (Q in - c y) - s2 x, with y, x in the same
// storage (saves a separate pass over four vectors).
#include "qs_internal.cuh"
#include "dslash.cuh"
#include "stencil.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

namespace {

typedef float2 cf;

__device__ __forceinline__ cf cadd(cf a, cf b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cf csub(cf a, cf b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cf cneg(cf a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ cf cmi(cf a) { return make_float2(-a.y, a.x); }   // i a
// c + a b
__device__ __forceinline__ cf cfma(cf a, cf b, cf c)
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// ---- storage formats ------------------------------------------------------
struct StF32Tiled {
    static constexpr int64_t kBytesPerSite = 96;
    static constexpr bool kScaled = false;
    __device__ static void ld(const char *__restrict__ base, int s, cf v[12])
    {
        const cf *b = reinterpret_cast<const cf *>(base) + ((int64_t)(s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = __ldg(b + c * 16);
    }
    __device__ static void st(char *__restrict__ base, int s, const cf v[12])
    {
        cf *b = reinterpret_cast<cf *>(base) + ((int64_t)(s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) b[c * 16] = v[c];
    }
};

struct StF32Canon {
    static constexpr int64_t kBytesPerSite = 96;
    static constexpr bool kScaled = false;
    __device__ static void ld(const char *__restrict__ base, int s, cf v[12])
    {
        const float4 *q = reinterpret_cast<const float4 *>(base) + (int64_t)s * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float4 a = __ldg(q + i);
            v[2 * i] = make_float2(a.x, a.y);
            v[2 * i + 1] = make_float2(a.z, a.w);
        }
    }
    __device__ static void st(char *__restrict__ base, int s, const cf v[12])
    {
        float4 *q = reinterpret_cast<float4 *>(base) + (int64_t)s * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    }
};

// 16-bit storage with a per-site FP32 scale: tile = 12 x 16 words of two 16-bit
// reals, then 16 scales.
template <typename H2>
struct StScaled {
    static constexpr int64_t kBytesPerSite = 52;
    static constexpr bool kScaled = true;
    static constexpr int kTile = 832;
    __device__ static float2 cvt(H2 h);
    __device__ static H2 pack(float a, float b);
    // the stored (site-normalised) values and the site's scale
    __device__ static void ld_raw(const char *__restrict__ base, int s, cf v[12], float *scale)
    {
        const char *t = base + (int64_t)(s >> 4) * kTile;
        const unsigned *w = reinterpret_cast<const unsigned *>(t) + (s & 15);
        *scale = __ldg(reinterpret_cast<const float *>(t + 768) + (s & 15));
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            unsigned u = __ldg(w + c * 16);
            H2 h = *reinterpret_cast<H2 *>(&u);
            v[c] = cvt(h);
        }
    }
    __device__ static void ld(const char *__restrict__ base, int s, cf v[12])
    {
        const char *t = base + (int64_t)(s >> 4) * kTile;
        const unsigned *w = reinterpret_cast<const unsigned *>(t) + (s & 15);
        const float sc = __ldg(reinterpret_cast<const float *>(t + 768) + (s & 15));
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            unsigned u = __ldg(w + c * 16);
            H2 h = *reinterpret_cast<H2 *>(&u);
            float2 f = cvt(h);
            v[c] = make_float2(f.x * sc, f.y * sc);
        }
    }
    __device__ static void st(char *__restrict__ base, int s, const cf v[12])
    {
        char *t = base + (int64_t)(s >> 4) * kTile;
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].x), fabsf(v[c].y)));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        unsigned *w = reinterpret_cast<unsigned *>(t) + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            H2 h = pack(v[c].x * inv, v[c].y * inv);
            w[c * 16] = *reinterpret_cast<unsigned *>(&h);
        }
        reinterpret_cast<float *>(t + 768)[s & 15] = m;
    }
};
template <> __device__ float2 StScaled<__half2>::cvt(__half2 h) { return __half22float2(h); }
template <> __device__ __half2 StScaled<__half2>::pack(float a, float b) { return __floats2half2_rn(a, b); }
template <> __device__ float2 StScaled<__nv_bfloat162>::cvt(__nv_bfloat162 h) { return __bfloat1622float2(h); }
template <> __device__ __nv_bfloat162 StScaled<__nv_bfloat162>::pack(float a, float b) { return __floats2bfloat162_rn(a, b); }

typedef StScaled<__half2> StF16;
typedef StScaled<__nv_bfloat162> StBF16;

// ---- spin projection / reconstruction (chiral basis, see dslash.cu) ---------
// half spinor h for direction MU, forward (FW: 1 - g_mu) or backward (1 + g_mu)
template <int MU, bool FW>
__device__ __forceinline__ void project(const cf v[12], cf h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cf p0 = v[c], p1 = v[3 + c], p2 = v[6 + c], p3 = v[9 + c];
        if (MU == 0) {
            h[0][c] = FW ? cadd(p0, p2) : csub(p0, p2);
            h[1][c] = FW ? cadd(p1, p3) : csub(p1, p3);
        } else if (MU == 1) {
            h[0][c] = FW ? cadd(p0, cmi(p3)) : csub(p0, cmi(p3));
            h[1][c] = FW ? cadd(p1, cmi(p2)) : csub(p1, cmi(p2));
        } else if (MU == 2) {
            h[0][c] = FW ? cadd(p0, p3) : csub(p0, p3);
            h[1][c] = FW ? csub(p1, p2) : cadd(p1, p2);
        } else {
            h[0][c] = FW ? cadd(p0, cmi(p2)) : csub(p0, cmi(p2));
            h[1][c] = FW ? csub(p1, cmi(p3)) : cadd(p1, cmi(p3));
        }
    }
}

// acc += (x, lower(x)), lower = -+ e_mu^+ x
template <int MU, bool FW>
__device__ __forceinline__ void reconstruct(cf acc[12], const cf x[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cadd(acc[c], x[0][c]);
        acc[3 + c] = cadd(acc[3 + c], x[1][c]);
        if (MU == 0) {
            acc[6 + c] = FW ? cadd(acc[6 + c], x[0][c]) : csub(acc[6 + c], x[0][c]);
            acc[9 + c] = FW ? cadd(acc[9 + c], x[1][c]) : csub(acc[9 + c], x[1][c]);
        } else if (MU == 1) {
            acc[6 + c] = FW ? csub(acc[6 + c], cmi(x[1][c])) : cadd(acc[6 + c], cmi(x[1][c]));
            acc[9 + c] = FW ? csub(acc[9 + c], cmi(x[0][c])) : cadd(acc[9 + c], cmi(x[0][c]));
        } else if (MU == 2) {
            acc[6 + c] = FW ? csub(acc[6 + c], x[1][c]) : cadd(acc[6 + c], x[1][c]);
            acc[9 + c] = FW ? cadd(acc[9 + c], x[0][c]) : csub(acc[9 + c], x[0][c]);
        } else {
            acc[6 + c] = FW ? csub(acc[6 + c], cmi(x[0][c])) : cadd(acc[6 + c], cmi(x[0][c]));
            acc[9 + c] = FW ? cadd(acc[9 + c], cmi(x[1][c])) : csub(acc[9 + c], cmi(x[1][c]));
        }
    }
}

__host__ __device__ constexpr int tri(int i, int j) { return i * (i - 1) / 2 + j; }

// entry (i, j) of a packed SW block P (pairs: 3 of real diagonals, 15 of strict-lower
// complex entries), for a physical site
template <int I, int J>
__device__ __forceinline__ cf sw_entry(const cf P[18])
{
    if constexpr (I > J) {
        return P[3 + tri(I, J)];
    } else {
        cf e = P[3 + tri(J, I)];
        return make_float2(e.x, -e.y);
    }
}
// entry (i, j) of the mirror site's block S conj(A) S: sign (same spin half ? + : -)
// times conj(A[i +- 3][j +- 3])
template <int I, int J>
__device__ __forceinline__ cf sw_entry_mirror(const cf P[18])
{
    constexpr int II = (I + 3) % 6, JJ = (J + 3) % 6;
    cf e = sw_entry<II, JJ>(P);
    e.y = -e.y;
    if ((I < 3) != (J < 3)) e = cneg(e);
    return e;
}
template <int I>
__device__ __forceinline__ float sw_diag(const cf P[18], bool mir)
{
    constexpr int II = (I + 3) % 6;
    const float d0 = (I & 1) ? P[I / 2].y : P[I / 2].x;
    const float dm = (II & 1) ? P[II / 2].y : P[II / 2].x;
    return mir ? dm : d0;
}

template <int I, int J, int G>
__device__ __forceinline__ void sw_row_term(const cf P[18], bool mir, int b, const cf v[G][12], cf acc[G][12])
{
    if constexpr (I == J) {
        const float d = sw_diag<I>(P, mir);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            acc[g][6 * b + I].x = fmaf(d, v[g][6 * b + J].x, acc[g][6 * b + I].x);
            acc[g][6 * b + I].y = fmaf(d, v[g][6 * b + J].y, acc[g][6 * b + I].y);
        }
    } else {
        const cf e0 = sw_entry<I, J>(P), em = sw_entry_mirror<I, J>(P);
        const cf e = mir ? em : e0;
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g][6 * b + I] = cfma(e, v[g][6 * b + J], acc[g][6 * b + I]);
    }
}

template <int I, int G>
__device__ __forceinline__ void sw_row(const cf P[18], bool mir, int b, const cf v[G][12], cf acc[G][12])
{
    sw_row_term<I, 0, G>(P, mir, b, v, acc);
    sw_row_term<I, 1, G>(P, mir, b, v, acc);
    sw_row_term<I, 2, G>(P, mir, b, v, acc);
    sw_row_term<I, 3, G>(P, mir, b, v, acc);
    sw_row_term<I, 4, G>(P, mir, b, v, acc);
    sw_row_term<I, 5, G>(P, mir, b, v, acc);
}

struct D32 {
    Geom g;
    const cf *links;    // [mu][9][Vphys]
    const cf *clov;     // [2][18][Vphys]
    const char *in;     // right-hand side r at in + r * vbytes
    char *out;
    const char *y, *x;  // CHEB epilogue operands
    int64_t vbytes;
    int nrhs, gamma5;
    float c, s1, s2;    // CHEB: out = s1 (Q in - c y) - s2 x
    float dm[QS_MAX_RHS];   // 4 + m0 per right-hand side
    // device-side overrides (for launches replayed from a CUDA graph): if set, (c, s1, s2)
    // are read from coef[0..2] and 4 + m0 of right-hand side r from dmdev[r]
    const float *coef, *dmdev;
};

template <int MU, int STEP, class S, int G>
__device__ __forceinline__ void hop(const D32 &a, const Site &c, bool mir, int r0, int nr, cf acc[G][12])
{
    int sg;
    const Nb n = nbr_of<MU, STEP>(a.g, c, &sg);
    const int lp = STEP > 0 ? c.p : n.p;
    const bool lcj = STEP > 0 ? mir : n.mir;
    const int64_t V = a.g.Vphys;
    // M = -1/2 sg (forward: W, backward: W^+), W = lcj ? conj(U) : U
    cf U[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) U[k] = __ldg(a.links + (int64_t)(MU * 9 + k) * V + lp);
    const float f = -0.5f * (float)sg;
    const bool neg = STEP > 0 ? lcj : !lcj;
    const float fi = neg ? -f : f;
    cf M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const cf u = STEP > 0 ? U[i * 3 + j] : U[j * 3 + i];
            M[i * 3 + j] = make_float2(f * u.x, fi * u.y);
        }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < nr) {
            cf v[12];
            cf h[2][3], xx[2][3];
            if constexpr (S::kScaled) {
                // the site's scale commutes with the projection: apply it to the 6
                // projected components instead of the 12 loaded ones
                float sc;
                S::ld_raw(a.in + (int64_t)(r0 + g) * a.vbytes, n.s, v, &sc);
                project<MU, (STEP > 0)>(v, h);
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int i = 0; i < 3; ++i) h[q][i] = make_float2(sc * h[q][i].x, sc * h[q][i].y);
            } else {
                S::ld(a.in + (int64_t)(r0 + g) * a.vbytes, n.s, v);
                project<MU, (STEP > 0)>(v, h);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    cf t = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 3; ++j) t = cfma(M[i * 3 + j], h[q][j], t);
                    xx[q][i] = t;
                }
            reconstruct<MU, (STEP > 0)>(acc[g], xx);
        }
    }
}

// block (bx, by): sites [bx * 128 / RL, ...), right-hand sides [by * RL * G, ...)
template <class S, int G, int RL, bool CHEB>
__device__ __forceinline__ void site_kernel(const D32 &a, unsigned bx, unsigned by)
{
    constexpr int SPB = 128 / RL;   // sites per block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rl = RL > 1 ? (lane % RL) : 0;
    const int sl = RL > 1 ? (lane / RL) : lane;
    const int s = (int)bx * SPB + warp * (32 / RL) + sl;
    const int r0 = (int)by * (RL * G) + rl * G;
    if (s >= (int)a.g.Ns || r0 >= a.nrhs) return;
    const int nr = min(G, a.nrhs - r0);
    const Site c = site_of(a.g, s);
    const bool mir = c.x >= a.g.L;

    cf acc[G][12];
    {
        // diagonal part (4 + m0 + A) psi, one chiral block at a time
        cf v[G][12];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < nr) S::ld(a.in + (int64_t)(r0 + g) * a.vbytes, s, v[g]);
            else {
#pragma unroll
                for (int i = 0; i < 12; ++i) v[g][i] = make_float2(0.f, 0.f);
            }
            const float dm = a.dmdev ? __ldg(a.dmdev + (g < nr ? r0 + g : r0)) : a.dm[g < nr ? r0 + g : r0];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[g][i] = make_float2(dm * v[g][i].x, dm * v[g][i].y);
        }
        const int64_t V = a.g.Vphys;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            cf P[18];
#pragma unroll
            for (int q = 0; q < 18; ++q) P[q] = __ldg(a.clov + (int64_t)(b * 18 + q) * V + c.p);
            sw_row<0, G>(P, mir, b, v, acc);
            sw_row<1, G>(P, mir, b, v, acc);
            sw_row<2, G>(P, mir, b, v, acc);
            sw_row<3, G>(P, mir, b, v, acc);
            sw_row<4, G>(P, mir, b, v, acc);
            sw_row<5, G>(P, mir, b, v, acc);
        }
    }
    hop<0, +1, S, G>(a, c, mir, r0, nr, acc);
    hop<0, -1, S, G>(a, c, mir, r0, nr, acc);
    hop<1, +1, S, G>(a, c, mir, r0, nr, acc);
    hop<1, -1, S, G>(a, c, mir, r0, nr, acc);
    hop<2, +1, S, G>(a, c, mir, r0, nr, acc);
    hop<2, -1, S, G>(a, c, mir, r0, nr, acc);
    hop<3, +1, S, G>(a, c, mir, r0, nr, acc);
    hop<3, -1, S, G>(a, c, mir, r0, nr, acc);

#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < nr) {
            if (a.gamma5) {
#pragma unroll
                for (int i = 6; i < 12; ++i) acc[g][i] = cneg(acc[g][i]);
            }
            const int64_t off = (int64_t)(r0 + g) * a.vbytes;
            if (CHEB) {
                cf yv[12], xv[12];
                S::ld(a.y + off, s, yv);
                S::ld(a.x + off, s, xv);
                const float cc = a.coef ? __ldg(a.coef) : a.c;
                const float s1 = a.coef ? __ldg(a.coef + 1) : a.s1;
                const float s2 = a.coef ? __ldg(a.coef + 2) : a.s2;
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    acc[g][i].x = s1 * fmaf(-cc, yv[i].x, acc[g][i].x) - s2 * xv[i].x;
                    acc[g][i].y = s1 * fmaf(-cc, yv[i].y, acc[g][i].y) - s2 * xv[i].y;
                }
            }
            S::st(a.out + off, s, acc[g]);
        }
    }
}

// One-dimensional grid over (site tile, right-hand-side group).  SITE_MAJOR: the groups
// of a site tile are consecutive blocks, so a tile's links and SW terms leave DRAM once
// for all right-hand sides (the time-slice window of all of them must then fit in L2);
// otherwise the groups are outermost (a window of one group only, links re-read per group).
template <class S, int G, int RL, bool CHEB, int MINB, bool SITE_MAJOR>
__global__ void __launch_bounds__(128, MINB) dslash32_kernel(const __grid_constant__ D32 a, unsigned ntile,
                                                             unsigned ngroup)
{
    const unsigned b = blockIdx.x;
    if (SITE_MAJOR) site_kernel<S, G, RL, CHEB>(a, b / ngroup, b % ngroup);
    else site_kernel<S, G, RL, CHEB>(a, b % ntile, b / ntile);
}

// Batched persistent form: work items (lattice i, right-hand-side group, site tile)
// numbered lattice by lattice, right-hand-side groups outermost within a lattice;
// each block takes items w = blockIdx.x, blockIdx.x + gridDim.x, ...
#define QS_B_RL 4
struct D32B {
    int n;
    unsigned off[QS_BATCH_MAX + 1];   // first work item of lattice i; off[n] = all items
    unsigned nbx[QS_BATCH_MAX];       // site tiles of lattice i
    D32 item[QS_BATCH_MAX];
};

static_assert(sizeof(D32B) <= 4096, "batched operator arguments exceed the kernel parameter space");

template <class S>
__global__ void __launch_bounds__(128, 3) dslash32_batch_kernel(const __grid_constant__ D32B b)
{
    for (unsigned w = blockIdx.x; w < b.off[b.n]; w += gridDim.x) {
        int i = 0;
#pragma unroll 1
        while (i + 1 < b.n && w >= b.off[i + 1]) ++i;
        const unsigned local = w - b.off[i];
        site_kernel<S, 1, QS_B_RL, false>(b.item[i], local % b.nbx[i], local / b.nbx[i]);
    }
}

// ---- conversions between tiled storages (per right-hand side and site) -----------
struct StF64Tiled {
    static constexpr int64_t kBytesPerSite = 192;
    __device__ static void ld(const char *__restrict__ base, int s, cf v[12])
    {
        const double2 *b = reinterpret_cast<const double2 *>(base) + ((int64_t)(s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 d = b[c * 16];
            v[c] = make_float2((float)d.x, (float)d.y);
        }
    }
    __device__ static void st(char *__restrict__ base, int s, const cf v[12])
    {
        double2 *b = reinterpret_cast<double2 *>(base) + ((int64_t)(s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) b[c * 16] = make_double2((double)v[c].x, (double)v[c].y);
    }
};

template <class SA, class SB>
__global__ void convert_kernel(const char *__restrict__ in, char *__restrict__ out, int64_t Ns, int k)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Ns * k) return;
    const int r = (int)(i / Ns);
    const int s = (int)(i - (int64_t)r * Ns);
    cf v[12];
    SA::ld(in + (int64_t)r * Ns * SA::kBytesPerSite, s, v);
    SB::st(out + (int64_t)r * Ns * SB::kBytesPerSite, s, v);
}

template <class SA>
cudaError_t convert_from(int to, const void *in, void *out, int64_t Ns, int k, cudaStream_t st)
{
    const unsigned nb = (unsigned)((Ns * k + 255) / 256);
    const char *a = (const char *)in;
    char *b = (char *)out;
    switch (to) {
    case QS_D32_F32_TILED: convert_kernel<SA, StF32Tiled><<<nb, 256, 0, st>>>(a, b, Ns, k); break;
    case QS_D32_F16: convert_kernel<SA, StF16><<<nb, 256, 0, st>>>(a, b, Ns, k); break;
    case QS_D32_BF16: convert_kernel<SA, StBF16><<<nb, 256, 0, st>>>(a, b, Ns, k); break;
    case QS_D32_F64_TILED: convert_kernel<SA, StF64Tiled><<<nb, 256, 0, st>>>(a, b, Ns, k); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- launch ------------------------------------------------------------------
template <class S, int G, int RL, bool CHEB, int MINB, bool SM>
cudaError_t launch(const D32 &a, cudaStream_t st)
{
    constexpr int SPB = 128 / RL;
    const unsigned ntile = (unsigned)((a.g.Ns + SPB - 1) / SPB);
    const unsigned ngroup = (unsigned)((a.nrhs + RL * G - 1) / (RL * G));
    dslash32_kernel<S, G, RL, CHEB, MINB, SM><<<ntile * ngroup, 128, 0, st>>>(a, ntile, ngroup);
    return cudaGetLastError();
}

// variant table per storage: (G, RL, min blocks per SM, block order)
template <class S, bool CHEB>
cudaError_t launch_variant(int v, const D32 &a, cudaStream_t st)
{
    switch (v) {
    case 0: return launch<S, 1, 1, CHEB, 3, false>(a, st);
    case 1: return launch<S, 1, 4, CHEB, 4, false>(a, st);
    case 2: return launch<S, 2, 4, CHEB, 3, false>(a, st);
    case 3: return launch<S, 1, 8, CHEB, 4, false>(a, st);
    case 4: return launch<S, 1, 1, CHEB, 3, true>(a, st);
    case 5: return launch<S, 1, 4, CHEB, 4, true>(a, st);
    case 6: return launch<S, 2, 1, CHEB, 3, true>(a, st);
    default: return launch<S, 2, 4, CHEB, 3, true>(a, st);
    }
}

template <class S>
cudaError_t launch_storage(int v, bool cheb, const D32 &a, cudaStream_t st)
{
    return cheb ? launch_variant<S, true>(v, a, st) : launch_variant<S, false>(v, a, st);
}

template <class S>
cudaError_t batch_launch(const D32B &b, cudaStream_t st)
{
    static int per_sm = 0, nsm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dslash32_batch_kernel<S>, 128, 0);
        if (per_sm < 1) per_sm = 1;
        if (nsm < 1) nsm = 1;
    });
    const unsigned total = b.off[b.n];
    const unsigned grid = total < (unsigned)(per_sm * nsm) ? total : (unsigned)(per_sm * nsm);
    dslash32_batch_kernel<S><<<grid, 128, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

cudaError_t qs_d32_batch_launch(const D32BatchItem *items, int n, int storage, int gamma5, cudaStream_t st)
{
    if (n < 1 || n > QS_BATCH_MAX) return cudaErrorInvalidValue;
    D32B b;
    memset(&b, 0, sizeof(b));
    b.n = n;
    unsigned off = 0;
    for (int i = 0; i < n; ++i) {
        D32 &a = b.item[i];
        const D32BatchItem &it = items[i];
        a.g = it.g;
        a.links = reinterpret_cast<const cf *>(it.links);
        a.clov = reinterpret_cast<const cf *>(it.clov);
        a.in = (const char *)it.in;
        a.out = (char *)it.out;
        a.y = a.x = nullptr;
        a.vbytes = qs_d32_vec_bytes(storage, it.g.Ns);
        a.nrhs = it.nrhs;
        a.gamma5 = gamma5;
        a.c = a.s1 = a.s2 = 0.f;
        a.coef = a.dmdev = nullptr;
        for (int r = 0; r < it.nrhs; ++r) a.dm[r] = (float)(4.0 + it.m0[r]);
        const unsigned spb = 128 / QS_B_RL;
        b.nbx[i] = (unsigned)((it.g.Ns + spb - 1) / spb);
        b.off[i] = off;
        const double items_i = (double)b.nbx[i] * ((it.nrhs + QS_B_RL - 1) / QS_B_RL);
        if (off + items_i > 4e9) return cudaErrorInvalidValue;
        off += (unsigned)items_i;
    }
    b.off[n] = off;
    cudaError_t e;
    switch (storage) {
    case QS_D32_F32_TILED: e = batch_launch<StF32Tiled>(b, st); break;
    case QS_D32_F32_CANON: e = batch_launch<StF32Canon>(b, st); break;
    case QS_D32_F16: e = batch_launch<StF16>(b, st); break;
    case QS_D32_BF16: e = batch_launch<StBF16>(b, st); break;
    default: return cudaErrorInvalidValue;
    }
    qs_note_launches(1);
    return e;
}

int qs_d32_nvariants() { return 8; }

int64_t qs_d32_vec_bytes(int storage, int64_t Ns)
{
    return storage == QS_D32_F16 || storage == QS_D32_BF16 ? Ns * 52 : Ns * 96;
}

cudaError_t qs_d32_launch(const D32Call &c, int variant, cudaStream_t st)
{
    D32 a;
    a.g = c.g;
    a.links = reinterpret_cast<const cf *>(c.links);
    a.clov = reinterpret_cast<const cf *>(c.clov);
    a.in = (const char *)c.in;
    a.out = (char *)c.out;
    a.y = (const char *)c.y;
    a.x = (const char *)c.x;
    a.vbytes = qs_d32_vec_bytes(c.storage, c.g.Ns);
    a.nrhs = c.nrhs;
    a.gamma5 = c.gamma5;
    a.c = (float)c.cheb_c;
    a.s1 = (float)c.cheb_s1;
    a.s2 = (float)c.cheb_s2;
    for (int r = 0; r < c.nrhs; ++r) a.dm[r] = c.m0 ? (float)(4.0 + c.m0[r]) : 0.f;
    a.coef = c.coef_dev;
    a.dmdev = c.dm_dev;
    const bool cheb = c.cheb;
    switch (c.storage) {
    case QS_D32_F32_TILED: return launch_storage<StF32Tiled>(variant, cheb, a, st);
    case QS_D32_F32_CANON: return launch_storage<StF32Canon>(variant, cheb, a, st);
    case QS_D32_F16: return launch_storage<StF16>(variant, cheb, a, st);
    case QS_D32_BF16: return launch_storage<StBF16>(variant, cheb, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t qs_convert_tiled(int from, int to, const void *in, void *out, int64_t Ns, int k, cudaStream_t st)
{
    cudaError_t e;
    switch (from) {
    case QS_D32_F32_TILED: e = convert_from<StF32Tiled>(to, in, out, Ns, k, st); break;
    case QS_D32_F16: e = convert_from<StF16>(to, in, out, Ns, k, st); break;
    case QS_D32_BF16: e = convert_from<StBF16>(to, in, out, Ns, k, st); break;
    case QS_D32_F64_TILED: e = convert_from<StF64Tiled>(to, in, out, Ns, k, st); break;
    default: return cudaErrorInvalidValue;
    }
    qs_note_launches(1);
    return e;
}

cudaError_t qs_q16_from_f64(int storage, const double *in, void *out, int64_t Ns, int k, cudaStream_t st)
{
    return qs_convert_tiled(QS_D32_F64_TILED, storage, in, out, Ns, k, st);
}

cudaError_t qs_f64_from_q16(int storage, const void *in, double *out, int64_t Ns, int k, cudaStream_t st)
{
    return qs_convert_tiled(storage, QS_D32_F64_TILED, in, out, Ns, k, st);
}
