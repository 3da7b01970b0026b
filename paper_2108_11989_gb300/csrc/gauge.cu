// Gauge loading, doubled-lattice links and the SW (clover) term.
//
// Sec. 2: O(a)-improved Wilson fermions with an SU(3) SW term (c_sw) and a U(1)
// SW term (c_sw,U(1)); Sec. 3: C* boundaries, realised on the doubled lattice
// whose mirror half carries the charge-conjugate links U^*, theta -> -theta.
#include "qs_internal.cuh"

#include <math.h>
#include <stdio.h>

namespace {

struct M3 { C2<double> a[9]; };

__device__ inline M3 m3_mul(const M3 &x, const M3 &y)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C2<double> s = cmk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = s + x.a[i * 3 + k] * y.a[k * 3 + j];
            r.a[i * 3 + j] = s;
        }
    return r;
}

__device__ inline M3 m3_dag(const M3 &x)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.a[i * 3 + j] = conjc(x.a[j * 3 + i]);
    return r;
}

// SU(3) link of the doubled lattice at doubled site s (conjugate on the mirror half)
__device__ inline M3 link_d(const Geom &g, const double2 *su3, int64_t s, int mu)
{
    bool mir;
    int64_t p = qs_phys(g, s, &mir);
    const double2 *u = su3 + (p * 4 + mu) * 9;
    M3 r;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 v = u[k];
        r.a[k] = cmk(v.x, mir ? -v.y : v.y);
    }
    return r;
}

__device__ inline double theta_d(const Geom &g, const double *th, int64_t s, int mu)
{
    if (!th) return 0.0;
    bool mir;
    int64_t p = qs_phys(g, s, &mir);
    double v = th[p * 4 + mu];
    return mir ? -v : v;
}

// F_{mu nu}(s) = c_su3 (Q - Q^+)/8 + c_u1 (i/4) sum_leaves sin(phi) 1, with Q the
// four clover leaves at s in the (mu, nu) plane (Sec. 2 SW terms).
__device__ M3 field_strength(const Geom &g, const double2 *su3, const double *th, int64_t s,
                             int mu, int nu, double csu3, double cu1)
{
    int sg;
    int64_t xpm = qs_nbr(g, s, mu, +1, &sg), xmm = qs_nbr(g, s, mu, -1, &sg);
    int64_t xpn = qs_nbr(g, s, nu, +1, &sg), xmn = qs_nbr(g, s, nu, -1, &sg);
    int64_t xmm_pn = qs_nbr(g, xmm, nu, +1, &sg);
    int64_t xmm_mn = qs_nbr(g, xmm, nu, -1, &sg);
    int64_t xmn_pm = qs_nbr(g, xmn, mu, +1, &sg);
    M3 Um = link_d(g, su3, s, mu), Un = link_d(g, su3, s, nu);
    M3 q1 = m3_mul(m3_mul(Um, link_d(g, su3, xpm, nu)), m3_mul(m3_dag(link_d(g, su3, xpn, mu)), m3_dag(Un)));
    M3 Um_mm = link_d(g, su3, xmm, mu), Un_mm = link_d(g, su3, xmm, nu);
    M3 q2 = m3_mul(m3_mul(Un, m3_dag(link_d(g, su3, xmm_pn, mu))), m3_mul(m3_dag(Un_mm), Um_mm));
    M3 q3 = m3_mul(m3_mul(m3_dag(Um_mm), m3_dag(link_d(g, su3, xmm_mn, nu))),
                   m3_mul(link_d(g, su3, xmm_mn, mu), link_d(g, su3, xmn, nu)));
    M3 Un_mn = link_d(g, su3, xmn, nu);
    M3 q4 = m3_mul(m3_mul(m3_dag(Un_mn), link_d(g, su3, xmn, mu)),
                   m3_mul(link_d(g, su3, xmn_pm, nu), m3_dag(Um)));
    M3 F;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            int k = i * 3 + j, kt = j * 3 + i;
            C2<double> q = q1.a[k] + q2.a[k] + q3.a[k] + q4.a[k];
            C2<double> qt = q1.a[kt] + q2.a[kt] + q3.a[kt] + q4.a[kt];
            F.a[k] = (csu3 / 8.0) * (q - conjc(qt));
        }
    if (th && cu1 != 0.0) {
        double a1 = theta_d(g, th, s, mu) + theta_d(g, th, xpm, nu) - theta_d(g, th, xpn, mu) - theta_d(g, th, s, nu);
        double a2 = theta_d(g, th, s, nu) - theta_d(g, th, xmm_pn, mu) - theta_d(g, th, xmm, nu) + theta_d(g, th, xmm, mu);
        double a3 = -theta_d(g, th, xmm, mu) - theta_d(g, th, xmm_mn, nu) + theta_d(g, th, xmm_mn, mu) + theta_d(g, th, xmn, nu);
        double a4 = -theta_d(g, th, xmn, nu) + theta_d(g, th, xmn, mu) + theta_d(g, th, xmn_pm, nu) - theta_d(g, th, s, mu);
        double f = cu1 * 0.25 * (sin(a1) + sin(a2) + sin(a3) + sin(a4));
        for (int i = 0; i < 3; ++i) F.a[i * 4].im += f;
    }
    return F;
}

// One thread per physical site: the two chiral 6x6 blocks of A = (i/4) sum sigma F.
// In the chiral basis sigma_{0k} = diag(s_k, -s_k), sigma_{jk} = -eps_{jkl} diag(s_l, s_l), so
//   A_+- = (i/2) [[B3, B1 - i B2], [B1 + i B2, -B3]],
//   B1 = +-F01 - F23, B2 = +-F02 + F13, B3 = +-F03 - F12   (0 = t, 1 = x, 2 = y, 3 = z).
__global__ void clover_build_kernel(Geom g, const double2 *su3, const double *th, double csu3,
                                    double cu1, double *clov, float2 *clov32)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= g.Vphys) return;
    int64_t s = (p / g.L) * g.L2 + (p % g.L);   // the physical (x < L) doubled site
    M3 F[4][4];
    const int pl[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int q = 0; q < 6; ++q) F[pl[q][0]][pl[q][1]] = field_strength(g, su3, th, s, pl[q][0], pl[q][1], csu3, cu1);
    for (int blk = 0; blk < 2; ++blk) {
        double sg = blk == 0 ? 1.0 : -1.0;
        C2<double> B1[9], B2[9], B3[9];
        for (int k = 0; k < 9; ++k) {
            B1[k] = sg * F[0][1].a[k] - F[2][3].a[k];
            B2[k] = sg * F[0][2].a[k] + F[1][3].a[k];
            B3[k] = sg * F[0][3].a[k] - F[1][2].a[k];
        }
        C2<double> A[6][6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int k = a * 3 + b;
                // (i/2) X
                A[a][b] = 0.5 * mul_i(B3[k]);
                A[a + 3][b + 3] = 0.5 * mul_i(cmk(-B3[k].re, -B3[k].im));
                A[a][b + 3] = 0.5 * mul_i(B1[k] - mul_i(B2[k]));
                A[a + 3][b] = 0.5 * mul_i(B1[k] + mul_i(B2[k]));
            }
        double *dst = clov + (int64_t)blk * 36 * g.Vphys;
        // FP32 copy as pairs [2][18][Vphys]: (A_00, A_11), (A_22, A_33), (A_44, A_55),
        // then the strict-lower entries (re, im) in row order
        float2 *d32 = clov32 + (int64_t)blk * 18 * g.Vphys;
        for (int i = 0; i < 6; ++i) dst[i * g.Vphys + p] = A[i][i].re;
        for (int q = 0; q < 3; ++q)
            d32[q * g.Vphys + p] = make_float2((float)A[2 * q][2 * q].re, (float)A[2 * q + 1][2 * q + 1].re);
        for (int i = 1; i < 6; ++i)
            for (int j = 0; j < i; ++j) {
                int k = 6 + 2 * qs_tri(i, j);
                dst[k * g.Vphys + p] = A[i][j].re;
                dst[(k + 1) * g.Vphys + p] = A[i][j].im;
                d32[(3 + qs_tri(i, j)) * g.Vphys + p] = make_float2((float)A[i][j].re, (float)A[i][j].im);
            }
    }
}

// V = U exp(i theta) into the SoA layout [mu][9][Vphys], FP64 and FP32.
__global__ void pack_links_kernel(Geom g, const double2 *su3, const double *th, double2 *l64, float2 *l32)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= g.Vphys) return;
    for (int mu = 0; mu < 4; ++mu) {
        double c = 1.0, sn = 0.0;
        if (th) sincos(th[p * 4 + mu], &sn, &c);
        for (int k = 0; k < 9; ++k) {
            double2 u = su3[(p * 4 + mu) * 9 + k];
            double2 v = make_double2(u.x * c - u.y * sn, u.x * sn + u.y * c);
            int64_t o = (int64_t)(mu * 9 + k) * g.Vphys + p;
            l64[o] = v;
            l32[o] = make_float2((float)v.x, (float)v.y);
        }
    }
}

// max over physical sites and both chiral blocks of the Frobenius norm of the SW
// term block (an upper bound of its spectral norm); the mirror block S conj(A) S
// has the same norm.  A non-finite SW entry or link anywhere makes the result +inf.
// Positive doubles (and +inf) order like their bit patterns.
__global__ void clover_norm_kernel(Geom g, const double *clov, const double2 *links, unsigned long long *out)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double m = 0;
    if (p < g.Vphys) {
        bool finite = true;
        for (int b = 0; b < 2; ++b) {
            double f = 0;
            for (int i = 0; i < 6; ++i) {
                double d = clov[(int64_t)(b * 36 + i) * g.Vphys + p];
                f += d * d;
            }
            for (int k = 6; k < 36; ++k) {
                double d = clov[(int64_t)(b * 36 + k) * g.Vphys + p];
                f += 2 * d * d;
            }
            finite = finite && isfinite(f);
            m = fmax(m, sqrt(f));
        }
        for (int k = 0; k < 36; ++k) {
            double2 v = links[(int64_t)k * g.Vphys + p];
            finite = finite && isfinite(v.x) && isfinite(v.y);
        }
        if (!finite) m = INFINITY;
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

static void free_gauge(qs_lattice *lat)
{
    cudaFree(lat->links64); cudaFree(lat->links32);
    cudaFree(lat->clov64); cudaFree(lat->clov32);
    lat->links64 = nullptr; lat->links32 = nullptr;
    lat->clov64 = nullptr; lat->clov32 = nullptr;
    lat->gauge_loaded = 0;
}

void qs_free_gauge(qs_lattice *lat) { free_gauge(lat); }

extern "C" int qs_load_gauge(qs_lattice *lat, const double *su3, const double *u1_theta,
                             double csw_su3, double csw_u1)
{
    if (!lat || !su3) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    const Geom &g = lat->g;
    free_gauge(lat);
    size_t nl = (size_t)g.Vphys * 4 * 9;
    double2 *d_su3 = nullptr;
    double *d_th = nullptr;
    int st = QS_OK;
    auto fail = [&](cudaError_t e, const char *w) {
        qs_record_cuda_error(e, w);
        st = e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
    };
    cudaError_t e;
    do {
        if ((e = cudaMalloc(&d_su3, nl * sizeof(double2))) != cudaSuccess) { fail(e, "malloc su3"); break; }
        if (u1_theta && (e = cudaMalloc(&d_th, (size_t)g.Vphys * 4 * sizeof(double))) != cudaSuccess) { fail(e, "malloc theta"); break; }
        if ((e = cudaMalloc(&lat->links64, nl * sizeof(double2))) != cudaSuccess) { fail(e, "malloc links64"); break; }
        if ((e = cudaMalloc(&lat->links32, nl * sizeof(float2))) != cudaSuccess) { fail(e, "malloc links32"); break; }
        if ((e = cudaMalloc(&lat->clov64, (size_t)g.Vphys * 72 * sizeof(double))) != cudaSuccess) { fail(e, "malloc clov64"); break; }
        if ((e = cudaMalloc(&lat->clov32, (size_t)g.Vphys * 36 * sizeof(float2))) != cudaSuccess) { fail(e, "malloc clov32"); break; }
        if ((e = cudaMemcpyAsync(d_su3, su3, nl * sizeof(double2), cudaMemcpyHostToDevice, lat->stream)) != cudaSuccess) { fail(e, "copy su3"); break; }
        if (u1_theta && (e = cudaMemcpyAsync(d_th, u1_theta, (size_t)g.Vphys * 4 * sizeof(double), cudaMemcpyHostToDevice, lat->stream)) != cudaSuccess) { fail(e, "copy theta"); break; }
        int nb = (int)((g.Vphys + 127) / 128);
        clover_build_kernel<<<nb, 128, 0, lat->stream>>>(g, d_su3, d_th, csw_su3, d_th ? csw_u1 : 0.0, lat->clov64, lat->clov32);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "clover_build_kernel"); break; }
        pack_links_kernel<<<nb, 128, 0, lat->stream>>>(g, d_su3, d_th, lat->links64, lat->links32);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "pack_links_kernel"); break; }
        unsigned long long *d_nm = (unsigned long long *)d_th;   // reuse after the builds
        if (!d_nm) {
            if ((e = cudaMalloc(&d_th, sizeof(double))) != cudaSuccess) { fail(e, "malloc norm"); break; }
            d_nm = (unsigned long long *)d_th;
        }
        if ((e = cudaMemsetAsync(d_nm, 0, sizeof(unsigned long long), lat->stream)) != cudaSuccess) { fail(e, "memset"); break; }
        clover_norm_kernel<<<nb, 128, 0, lat->stream>>>(g, lat->clov64, lat->links64, d_nm);
        qs_note_launches(3);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "clover_norm_kernel"); break; }
        unsigned long long hn = 0;
        if ((e = cudaMemcpyAsync(&hn, d_nm, sizeof(hn), cudaMemcpyDeviceToHost, lat->stream)) != cudaSuccess) { fail(e, "copy norm"); break; }
        if ((e = cudaStreamSynchronize(lat->stream)) != cudaSuccess) { fail(e, "load_gauge sync"); break; }
        double dn;
        memcpy(&dn, &hn, sizeof(dn));
        lat->clov_norm = dn;
        if (!isfinite(dn)) st = QS_ENUMERIC;   // NaN / Inf in the gauge field
    } while (0);
    cudaFree(d_su3);
    cudaFree(d_th);
    if (st != QS_OK) {
        free_gauge(lat);
        return st;
    }
    lat->csw_su3 = csw_su3;
    lat->csw_u1 = csw_u1;
    lat->gauge_loaded = 1;
    return QS_OK;
}
