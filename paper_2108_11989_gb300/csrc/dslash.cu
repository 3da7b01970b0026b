// The O(a)-improved Wilson-Dirac operator D and Q = gamma_5 D on the C*-doubled
// lattice (Sec. 2 operator, Sec. 3 doublet and Q) in FP64 arithmetic (the FP32-arithmetic
// form for FP32 and 16-bit storage is dslash32.cu).  One thread per doubled site;
// each thread forms
//   out = (4 + m0) psi + A psi - 1/2 sum_mu [ V (1 - g_mu) psi(x+mu) + V^+ (1 + g_mu) psi(x-mu) ]
// and, for Q, flips the sign of spins 2, 3.  (1 -+ g_mu) has rank 2: in the
// chiral basis g_mu = [[0, e_mu], [e_mu^+, 0]] (e_0 = -1, e_k = -i s_k), so
//   (1 - g_mu) psi = (h, -e_mu^+ h),  h = psi_up - e_mu psi_dn,
//   (1 + g_mu) psi = (h, +e_mu^+ h),  h = psi_up + e_mu psi_dn,
// and only the half spinor h is multiplied by the link.
#include "qs_internal.cuh"
#include "dslash.cuh"
#include "stencil.cuh"

namespace {

template <typename R>
__device__ __forceinline__ void load24(const R *__restrict__ p, R v[24]);
template <>
__device__ __forceinline__ void load24<float>(const float *__restrict__ p, float v[24])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float4 a = __ldg(q + i);
        v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = a.z; v[4 * i + 3] = a.w;
    }
}
template <>
__device__ __forceinline__ void load24<double>(const double *__restrict__ p, double v[24])
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        double2 a = __ldg(q + i);
        v[2 * i] = a.x; v[2 * i + 1] = a.y;
    }
}
template <typename R>
__device__ __forceinline__ void store24(R *__restrict__ p, const R v[24]);
template <>
__device__ __forceinline__ void store24<float>(float *__restrict__ p, const float v[24])
{
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <>
__device__ __forceinline__ void store24<double>(double *__restrict__ p, const double v[24])
{
    double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int i = 0; i < 12; ++i) q[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// Site access in either spinor layout.  Canonical (SOA = false): [site][12][re, im].
// Solver layout (SOA = true): [site / 16][12][site % 16][re, im], so that the 16 or
// 32 threads of a warp handling consecutive sites read each colour-spin component
// as one contiguous 128 B (FP32) or 256 B (FP64) segment.
template <bool SOA, typename R>
__device__ __forceinline__ void ld_site(const R *__restrict__ base, int64_t s, R v[24])
{
    if (!SOA) {
        load24<R>(base + s * 24, v);
    } else {
        typedef typename LinkT<R>::T V2;
        const V2 *b2 = reinterpret_cast<const V2 *>(base) + ((s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            V2 a = __ldg(b2 + c * 16);
            v[2 * c] = a.x;
            v[2 * c + 1] = a.y;
        }
    }
}

template <bool SOA, typename R>
__device__ __forceinline__ void st_site(R *__restrict__ base, int64_t s, const R v[24])
{
    if (!SOA) {
        store24<R>(base + s * 24, v);
    } else {
        typedef typename LinkT<R>::T V2;
        V2 *b2 = reinterpret_cast<V2 *>(base) + ((s >> 4) * 12) * 16 + (s & 15);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            V2 a;
            a.x = v[2 * c];
            a.y = v[2 * c + 1];
            b2[c * 16] = a;
        }
    }
}

template <typename R>
__device__ __forceinline__ C2<R> sp(const R v[24], int s, int c)
{
    return cmk(v[(s * 3 + c) * 2], v[(s * 3 + c) * 2 + 1]);
}

// half spinor h for direction MU, forward (FW = true: 1 - g) or backward (1 + g)
template <int MU, bool FW, typename R>
__device__ __forceinline__ void project(const R v[24], C2<R> h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C2<R> p0 = sp(v, 0, c), p1 = sp(v, 1, c), p2 = sp(v, 2, c), p3 = sp(v, 3, c);
        if (MU == 0) {
            h[0][c] = FW ? p0 + p2 : p0 - p2;
            h[1][c] = FW ? p1 + p3 : p1 - p3;
        } else if (MU == 1) {
            h[0][c] = FW ? p0 + mul_i(p3) : p0 - mul_i(p3);
            h[1][c] = FW ? p1 + mul_i(p2) : p1 - mul_i(p2);
        } else if (MU == 2) {
            h[0][c] = FW ? p0 + p3 : p0 - p3;
            h[1][c] = FW ? p1 - p2 : p1 + p2;
        } else {
            h[0][c] = FW ? p0 + mul_i(p2) : p0 - mul_i(p2);
            h[1][c] = FW ? p1 - mul_i(p3) : p1 + mul_i(p3);
        }
    }
}

// acc += (chi, lower(chi)) with lower = -+ e_mu^+ chi
template <int MU, bool FW, typename R>
__device__ __forceinline__ void reconstruct(C2<R> acc[12], const C2<R> x[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + x[0][c];
        acc[3 + c] = acc[3 + c] + x[1][c];
        C2<R> l2, l3;
        if (MU == 0) {
            l2 = FW ? x[0][c] : cmk(-x[0][c].re, -x[0][c].im);
            l3 = FW ? x[1][c] : cmk(-x[1][c].re, -x[1][c].im);
        } else if (MU == 1) {
            C2<R> a = mul_i(x[1][c]), b = mul_i(x[0][c]);
            l2 = FW ? cmk(-a.re, -a.im) : a;
            l3 = FW ? cmk(-b.re, -b.im) : b;
        } else if (MU == 2) {
            l2 = FW ? cmk(-x[1][c].re, -x[1][c].im) : x[1][c];
            l3 = FW ? x[0][c] : cmk(-x[0][c].re, -x[0][c].im);
        } else {
            C2<R> a = mul_i(x[0][c]), b = mul_i(x[1][c]);
            l2 = FW ? cmk(-a.re, -a.im) : a;
            l3 = FW ? b : cmk(-b.re, -b.im);
        }
        acc[6 + c] = acc[6 + c] + l2;
        acc[9 + c] = acc[9 + c] + l3;
    }
}

template <typename R>
__device__ __forceinline__ void load_link(const typename LinkT<R>::T *__restrict__ links, int64_t Vp, int mu,
                                          int64_t p, C2<R> U[9])
{
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        typename LinkT<R>::T a = __ldg(links + (int64_t)(mu * 9 + k) * Vp + p);
        U[k] = cmk(a.x, a.y);
    }
}

// chi = W h for W = U (conj = false) or U^* (conj = true)
template <typename R>
__device__ __forceinline__ void mul_link(const C2<R> U[9], bool cj, const C2<R> h[2][3], C2<R> x[2][3])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C2<R> r = cmk(R(0), R(0));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                C2<R> u = cj ? conjc(U[a * 3 + b]) : U[a * 3 + b];
                r = r + u * h[s][b];
            }
            x[s][a] = r;
        }
}

// chi = W^+ h for W = U (conj = false) or U^* (conj = true)
template <typename R>
__device__ __forceinline__ void mul_link_dag(const C2<R> U[9], bool cj, const C2<R> h[2][3], C2<R> x[2][3])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C2<R> r = cmk(R(0), R(0));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                C2<R> u = cj ? U[b * 3 + a] : conjc(U[b * 3 + a]);
                r = r + u * h[s][b];
            }
            x[s][a] = r;
        }
}

template <int MU, bool SOA, typename R>
__device__ __forceinline__ void hop_dir(const Geom &g, const typename LinkT<R>::T *__restrict__ links,
                                        const R *__restrict__ in, const Site &c, bool mir, C2<R> acc[12])
{
    C2<R> U[9];
    // forward: V(x, mu) (1 - g_mu) psi(x + mu)
    {
        int sg;
        Nb n = nbr_of<MU, +1>(g, c, &sg);
        R v[24];
        ld_site<SOA, R>(in, n.s, v);
        load_link<R>(links, g.Vphys, MU, c.p, U);
        C2<R> h[2][3], x[2][3];
        project<MU, true, R>(v, h);
        mul_link<R>(U, mir, h, x);
        if (MU == 0 && sg < 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) x[q][cc] = cmk(-x[q][cc].re, -x[q][cc].im);
        }
        reconstruct<MU, true, R>(acc, x);
    }
    // backward: V(x - mu, mu)^+ (1 + g_mu) psi(x - mu)
    {
        int sg;
        Nb n = nbr_of<MU, -1>(g, c, &sg);
        R v[24];
        ld_site<SOA, R>(in, n.s, v);
        load_link<R>(links, g.Vphys, MU, n.p, U);
        C2<R> h[2][3], x[2][3];
        project<MU, false, R>(v, h);
        mul_link_dag<R>(U, n.mir, h, x);
        if (MU == 0 && sg < 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) x[q][cc] = cmk(-x[q][cc].re, -x[q][cc].im);
        }
        reconstruct<MU, false, R>(acc, x);
    }
}

// D (or Q) at doubled site s for right-hand side r: the whole stencil of one site.
template <typename R, bool SOA>
__device__ __forceinline__ void dslash_site(const Geom &g, const typename LinkT<R>::T *__restrict__ links,
                                            const R *__restrict__ clov, const R *__restrict__ in_all,
                                            R *__restrict__ out_all, int gamma5, double m0, int r, int s)
{
    const R *in = in_all + (int64_t)r * g.Ns * 24;
    Site c = site_of(g, s);
    const int p = c.p;
    const bool mir = c.x >= g.L;

    C2<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cmk(R(0), R(0));
    hop_dir<0, SOA, R>(g, links, in, c, mir, acc);
    hop_dir<1, SOA, R>(g, links, in, c, mir, acc);
    hop_dir<2, SOA, R>(g, links, in, c, mir, acc);
    hop_dir<3, SOA, R>(g, links, in, c, mir, acc);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = R(-0.5) * acc[i];

    // diagonal part (4 + m0 + A), one chiral block (spins 2b, 2b+1) at a time.
    // Mirror sites use A' = S conj(A) S, S = s_2 (x) 1, i.e.
    // A'[i][j] = (same spin half ? 1 : -1) * conj(A[i +- 3][j +- 3]).
    R v[24];
    ld_site<SOA, R>(in, s, v);
    const R dm = R(4) + (R)m0;
    const R *cl = clov + p;
    const int64_t V = g.Vphys;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const R *cb = cl + (int64_t)b * 36 * V;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            C2<R> t = dm * cmk(v[(b * 6 + i) * 2], v[(b * 6 + i) * 2 + 1]);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                // element (ii, jj) of the stored block; mirror sites read the
                // spin-swapped element and conjugate it (A' = S conj(A) S)
                const int ii = mir ? (i + 3) % 6 : i, jj = mir ? (j + 3) % 6 : j;
                C2<R> e;
                if (ii == jj) {
                    e = cmk(__ldg(cb + ii * V), R(0));
                } else if (ii > jj) {
                    const int k = 6 + 2 * qs_tri(ii, jj);
                    e = cmk(__ldg(cb + k * V), __ldg(cb + (k + 1) * V));
                } else {
                    const int k = 6 + 2 * qs_tri(jj, ii);
                    e = cmk(__ldg(cb + k * V), -__ldg(cb + (k + 1) * V));
                }
                if (mir) {
                    e = conjc(e);
                    if ((i < 3) != (j < 3)) e = cmk(-e.re, -e.im);
                }
                t = t + e * cmk(v[(b * 6 + j) * 2], v[(b * 6 + j) * 2 + 1]);
            }
            acc[b * 6 + i] = acc[b * 6 + i] + t;
        }
    }
    R o[24];
    const R gs = gamma5 ? R(-1) : R(1);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        R f = i >= 6 ? gs : R(1);
        o[2 * i] = f * acc[i].re;
        o[2 * i + 1] = f * acc[i].im;
    }
    st_site<SOA, R>(out_all + (int64_t)r * g.Ns * 24, s, o);
}

// One thread per (doubled site, right-hand side).  A block handles 128 consecutive
// sites of one right-hand side; the right-hand side runs fastest over consecutive
// blocks, so the blocks of one site tile run together and share the link and
// SW-term loads through L1/L2.  Site coordinates are computed once per thread in
// 32-bit arithmetic; every neighbour and physical index follows by adds and
// compares (no division in the stencil).
template <typename R, int MINB, bool SOA>
__global__ void __launch_bounds__(128, MINB) dslash_kernel(DslashArgs<R> a)
{
    const unsigned b = blockIdx.x;
    const int r = (int)(b % (unsigned)a.nrhs);
    const int s = (int)(b / (unsigned)a.nrhs) * 128 + (int)threadIdx.x;
    if (s >= (int)a.g.Ns) return;
    dslash_site<R, SOA>(a.g, a.links, a.clov, a.in, a.out, a.gamma5, a.m0[r], r, s);
}

// Several lattices (configurations of any volume) in one launch: item i owns the
// blocks [off[i], off[i + 1]), laid out as in dslash_kernel.
template <typename R, bool SOA>
__global__ void __launch_bounds__(128) dslash_batch_kernel(BatchArgs<R> a)
{
    const unsigned b = blockIdx.x;
    int i = 0;
#pragma unroll 1
    while (i + 1 < a.n && b >= a.off[i + 1]) ++i;
    const BatchItem<R> &it = a.item[i];
    const unsigned lb = b - a.off[i];
    const int r = (int)(lb % (unsigned)it.nrhs);
    const int s = (int)(lb / (unsigned)it.nrhs) * 128 + (int)threadIdx.x;
    if (s >= (int)it.g.Ns) return;
    dslash_site<R, SOA>(it.g, it.links, it.clov, it.in, it.out, a.gamma5, it.m0[r], r, s);
}

// The FP64 operator on the sites of one parity only ((t + z + y + x) mod 2 == parity);
// sites of the other parity get zeros.  The even-odd preconditioned operator needs one
// parity of the output of each of its two applications.  Thread j handles the j-th site of
// that parity (a row of 2L sites holds L of each, at x = 2 jx or 2 jx + 1), so the warps
// hold sites of one parity only, and it writes zeros to the other site of its x pair.
__global__ void __launch_bounds__(128) dslash64_parity_kernel(DslashArgs<double> a, int parity)
{
    const unsigned b = blockIdx.x;
    const int r = (int)(b % (unsigned)a.nrhs);
    const int j = (int)(b / (unsigned)a.nrhs) * 128 + (int)threadIdx.x;
    if (j >= (int)(a.g.Ns / 2)) return;
    const int row = j / a.g.L;
    const int jx = j - row * a.g.L;
    const int y = row % a.g.L, z = (row / a.g.L) % a.g.L, t = row / (a.g.L * a.g.L);
    const int x = 2 * jx + ((parity + t + z + y) & 1);
    const int s = row * a.g.L2 + x;
    double2 *o = (double2 *)(a.out + ((int64_t)r * a.g.Ns + (s ^ 1)) * 24);
#pragma unroll
    for (int i = 0; i < 12; ++i) o[i] = make_double2(0.0, 0.0);
    dslash_site<double, false>(a.g, a.links, a.clov, a.in, a.out, a.gamma5, a.m0[r], r, s);
}

}  // namespace

template <typename R, int MINB>
static cudaError_t launch_variant(const DslashArgs<R> &a, int soa, cudaStream_t st)
{
    int64_t nb = ((a.g.Ns + 127) / 128) * a.nrhs;
    if (soa) dslash_kernel<R, MINB, true><<<(unsigned)nb, 128, 0, st>>>(a);
    else dslash_kernel<R, MINB, false><<<(unsigned)nb, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// Launch-bound variants (minimum resident 128-thread blocks per SM); the
// autotuner in capi.cu picks one per (layout, nrhs) by timing.  This kernel serves
// the FP64 operator; FP32 arithmetic runs in dslash32.cu.
template <>
int qs_dslash_nvariants<double>() { return 4; }

template <>
cudaError_t qs_dslash_launch<double>(DslashArgs<double> a, int nrhs, int variant, int soa, cudaStream_t st)
{
    a.nrhs = nrhs;
    switch (variant) {
    case 0: return launch_variant<double, 1>(a, soa, st);
    case 1: return launch_variant<double, 2>(a, soa, st);
    case 2: return launch_variant<double, 3>(a, soa, st);
    default: return launch_variant<double, 4>(a, soa, st);
    }
}

cudaError_t qs_dslash64_parity_launch(const DslashArgs<double> &a, int parity, cudaStream_t st)
{
    const int64_t nb = ((a.g.Ns / 2 + 127) / 128) * a.nrhs;
    dslash64_parity_kernel<<<(unsigned)nb, 128, 0, st>>>(a, parity);
    return cudaGetLastError();
}

// canonical [site][12][re, im] <-> solver [site / 16][12][site % 16][re, im], per vector
__global__ void soa_to_aos_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int64_t Ns)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // canonical complex index
    if (i >= Ns * 12) return;
    int64_t s = i / 12;
    int c = (int)(i % 12);
    out[i] = in[((s >> 4) * 12 + c) * 16 + (s & 15)];
}

cudaError_t qs_soa_to_aos(const double *in, double *out, int64_t Ns, cudaStream_t st)
{
    int64_t n = Ns * 12;
    soa_to_aos_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)in, (double2 *)out, Ns);
    qs_note_launches(1);
    return cudaGetLastError();
}

template <typename R>
cudaError_t qs_dslash_batch_launch(const BatchArgs<R> &a, int soa, cudaStream_t st)
{
    unsigned nb = a.off[a.n];
    if (soa) dslash_batch_kernel<R, true><<<nb, 128, 0, st>>>(a);
    else dslash_batch_kernel<R, false><<<nb, 128, 0, st>>>(a);
    qs_note_launches(1);
    return cudaGetLastError();
}
template cudaError_t qs_dslash_batch_launch<double>(const BatchArgs<double> &, int, cudaStream_t);
