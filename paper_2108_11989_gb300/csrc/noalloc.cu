// qs_apply_Q_norm2_noalloc: out = Q(m0) in together with |out_r|^2 for every
// right-hand side, without allocating anything.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// apply the operator, e.g. code running while a CUDA graph is being captured, a
// host callback, a real-time loop with a fixed memory budget, or an embedding
// framework that owns every device allocation.  The operator itself needs no
// scratch; the norm reduction needs partial sums, and here they live in one
// statically sized device array that is part of the library image.
#include "blas.cuh"
#include "dslash.cuh"

#define QS_NOALLOC_MAX_RHS 64

// Partial sums of the norm reduction: QS_RED_BLOCKS per right-hand side.  Every
// slot a call reads is written earlier in the same call, so nothing needs
// clearing; every call (on any handle of the device) shares the array.
static __device__ __align__(256) double qs_noalloc_partials[QS_RED_BLOCKS * QS_NOALLOC_MAX_RHS];

// Device address of the array, looked up once per device with that device current.
static double *g_noalloc_ptr[256];

template <typename R>
static int run(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, double *norm2, double *scratch)
{
    // the variant the autotuner already chose, else a fixed one (timing the
    // variants would create events)
    if (sizeof(R) == 8) {
        DslashArgs<double> d;
        d.g = lat->g;
        d.in = (const double *)in;
        d.out = (double *)out;
        d.gamma5 = 1;
        d.nrhs = nrhs;
        for (int r = 0; r < nrhs; ++r) d.m0[r] = m0;
        d.links = lat->links64;
        d.clov = lat->clov64;
        const int tv = lat->tuned64[0][nrhs];
        QS_CUDA(qs_dslash_launch<double>(d, nrhs, tv > 0 ? tv - 1 : 2, 0, lat->stream));
    } else {
        double m[QS_MAX_RHS];
        for (int r = 0; r < nrhs; ++r) m[r] = m0;
        D32Call c;
        memset(&c, 0, sizeof(c));
        c.g = lat->g;
        c.links = lat->links32;
        c.clov = lat->clov32;
        c.in = in;
        c.out = out;
        c.storage = QS_D32_F32_CANON;
        c.nrhs = nrhs;
        c.gamma5 = 1;
        c.m0 = m;
        const int tv = lat->tuned32[QS_D32_F32_CANON][0][nrhs];
        QS_CUDA(qs_d32_launch(c, tv > 0 ? tv - 1 : 1, lat->stream));
    }
    qs_note_launches(1);
    QS_CUDA(qs_norm2<R>((const R *)out, nrhs, lat->g.Ns * 24, scratch, norm2, lat->stream));
    return QS_OK;
}

extern "C" int qs_apply_Q_norm2_noalloc(qs_lattice *lat, double m0, const void *in, void *out, int nrhs,
                                        int prec, double *norm2)
{
    if (!lat || !in || !out || !norm2 || nrhs < 1) return QS_EINVAL;
    if (nrhs > QS_NOALLOC_MAX_RHS) return QS_EINVAL;   // beyond the static scratch
    if (!lat->gauge_loaded || (prec != QS_F64 && prec != QS_F32)) return QS_EINVAL;
    size_t bytes = (size_t)nrhs * lat->g.Ns * 24 * (prec == QS_F64 ? 8 : 4);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return QS_EINVAL;
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL;
    if (lat->device < 0 || lat->device >= 256) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    if (!g_noalloc_ptr[lat->device]) {
        void *p = nullptr;
        QS_CUDA(cudaGetSymbolAddress(&p, qs_noalloc_partials));
        g_noalloc_ptr[lat->device] = (double *)p;
    }
    double *scratch = g_noalloc_ptr[lat->device];
    if (prec == QS_F64) return run<double>(lat, m0, in, out, nrhs, norm2, scratch);
    return run<float>(lat, m0, in, out, nrhs, norm2, scratch);
}
