// The antiunitary symmetry of Q on the C*-doubled lattice (Sec. 3): if Q v = lambda v,
// then P v = C T gamma_5 v^* is an eigenvector with the same eigenvalue, orthogonal to v.
// T translates by L along x (quark <-> antiquark half); in the chiral basis
// C gamma_5 = i gamma_0 gamma_2 gamma_5 acts on spin as diag(s2, s2) (s2 the Pauli matrix),
// so (P v)(x) = diag(s2, s2) conj(v(x + L e1)): per colour,
//   out_0 = -i conj(in_1), out_1 = i conj(in_0), out_2 = -i conj(in_3), out_3 = i conj(in_2).
// P commutes with Q and P^2 = -1.
#include "blas.cuh"

namespace {

// one thread per (vector, site, colour); TILED: [site / 16][12][site % 16] double2
template <bool TILED, typename V2 = double2>
__global__ void partner_kernel(const V2 *__restrict__ in, V2 *__restrict__ out, Geom g, int k)
{
    const int64_t n = g.Ns * 3 * k;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int col = (int)(i % 3);
    const int64_t q = i / 3;
    const int r = (int)(q / g.Ns);
    const int64_t s = q - (int64_t)r * g.Ns;
    const int64_t row = s / g.L2;
    const int x = (int)(s - row * g.L2);
    const int64_t sp = row * g.L2 + (x >= g.L ? x - g.L : x + g.L);   // T s
    const V2 *a = in + (int64_t)r * g.Ns * 12;
    V2 *b = out + (int64_t)r * g.Ns * 12;
    auto at = [&](int64_t site, int comp) -> int64_t {
        return TILED ? ((site >> 4) * 12 + comp) * 16 + (site & 15) : site * 12 + comp;
    };
    V2 v[4];
#pragma unroll
    for (int sp_ = 0; sp_ < 4; ++sp_) v[sp_] = a[at(sp, sp_ * 3 + col)];
    V2 o;
    o.x = -v[1].y; o.y = -v[1].x; b[at(s, 0 * 3 + col)] = o;
    o.x = v[0].y;  o.y = v[0].x;  b[at(s, 1 * 3 + col)] = o;
    o.x = -v[3].y; o.y = -v[3].x; b[at(s, 2 * 3 + col)] = o;
    o.x = v[2].y;  o.y = v[2].x;  b[at(s, 3 * 3 + col)] = o;
}

}  // namespace

cudaError_t qs_partner(const double *in, double *out, const Geom &g, int k, int tiled, cudaStream_t st)
{
    const int64_t n = g.Ns * 3 * k;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (tiled) partner_kernel<true><<<nb, 256, 0, st>>>((const double2 *)in, (double2 *)out, g, k);
    else partner_kernel<false><<<nb, 256, 0, st>>>((const double2 *)in, (double2 *)out, g, k);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_partner32(const float *in, float *out, const Geom &g, int k, cudaStream_t st)
{
    const int64_t n = g.Ns * 3 * k;
    const unsigned nb = (unsigned)((n + 255) / 256);
    partner_kernel<true, float2><<<nb, 256, 0, st>>>((const float2 *)in, (float2 *)out, g, k);
    qs_note_launches(1);
    return cudaGetLastError();
}

extern "C" int qs_cstar_partner(qs_lattice *lat, const void *in, void *out, int nrhs, int prec)
{
    if (!lat || !in || !out || nrhs < 1) return QS_EINVAL;
    const int tiled = (prec & QS_LAYOUT_TILED) ? 1 : 0;
    if ((prec & ~QS_LAYOUT_TILED) != QS_F64) return QS_EINVAL;
    const size_t bytes = (size_t)nrhs * lat->g.Ns * 24 * sizeof(double);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return QS_EINVAL;
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    QS_CUDA(qs_partner((const double *)in, (double *)out, lat->g, nrhs, tiled, lat->stream));
    return QS_OK;
}
