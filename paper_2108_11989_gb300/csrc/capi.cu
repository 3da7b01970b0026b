// C-ABI entry points: lattice handles, operator application, status strings.
#include "qs_internal.cuh"
#include "dslash.cuh"

#include <stdio.h>
#include <stdlib.h>

#include <vector>

// Events around operator launches while profiling is on; resolved in batches.
struct ProfState {
    struct Rec {
        cudaEvent_t a, b;
        int prec;
        double bytes;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    qs_profile acc;
    int on;
};

static cudaEvent_t prof_event(ProfState *p)
{
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static int prof_resolve(qs_lattice *lat)
{
    ProfState *p = lat->prof;
    if (!p || p->pending.empty()) return QS_OK;
    QS_CUDA(cudaStreamSynchronize(lat->stream));
    for (auto &r : p->pending) {
        float ms = 0.f;
        QS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        qs_kernel_prof &k = p->acc.dslash[r.prec];
        k.launches += 1;
        k.ms += ms;
        k.bytes += r.bytes;
        p->pool.push_back(r.a);
        p->pool.push_back(r.b);
    }
    p->pending.clear();
    return QS_OK;
}

static void prof_free(qs_lattice *lat)
{
    ProfState *p = lat->prof;
    if (!p) return;
    for (auto &r : p->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->pool) cudaEventDestroy(e);
    delete p;
    lat->prof = nullptr;
}

extern "C" int qs_set_profiling(qs_lattice *lat, int on)
{
    if (!lat) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    if (on) {
        if (!lat->prof) lat->prof = new ProfState();
        QS_TRY(prof_resolve(lat));
        memset(&lat->prof->acc, 0, sizeof(qs_profile));
        lat->prof->on = 1;
    } else if (lat->prof) {
        lat->prof->on = 0;
    }
    return QS_OK;
}

extern "C" int qs_get_profile(qs_lattice *lat, qs_profile *prof)
{
    if (!lat || !prof) return QS_EINVAL;
    memset(prof, 0, sizeof(*prof));
    if (!lat->prof) return QS_OK;
    QS_CUDA(cudaSetDevice(lat->device));
    QS_TRY(prof_resolve(lat));
    *prof = lat->prof->acc;
    return QS_OK;
}

static char g_last_cuda_error[256] = "";
static long long g_launches = 0;

void qs_note_launches(int n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }

extern "C" int64_t qs_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void qs_record_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", where, cudaGetErrorString(e));
}

Geom qs_make_geom(int L, int T, int cstar_mask, int t_anti)
{
    Geom g;
    g.L = L; g.T = T; g.L2 = 2 * L;
    g.cstar_y = (cstar_mask >> 1) & 1;
    g.cstar_z = (cstar_mask >> 2) & 1;
    g.t_anti = t_anti ? 1 : 0;
    g.sy = g.L2;
    g.sz = (int64_t)g.L2 * L;
    g.st = (int64_t)g.L2 * L * L;
    g.Ns = g.st * T;
    g.Vphys = g.Ns / 2;
    return g;
}

void qs_free_gauge(qs_lattice *lat);
void qs_free_workspace(qs_lattice *lat);

extern "C" int qs_create_lattice(const qs_geom *geom, void *stream, qs_lattice **out)
{
    if (!geom || !out) return QS_EINVAL;
    *out = nullptr;
    if (geom->L < 2 || (geom->L & 1) || geom->T < 2 || !(geom->cstar_mask & 1) ||
        geom->cstar_mask < 0 || geom->cstar_mask > 7)
        return QS_EINVAL;
    // the operator indexes sites in 32-bit arithmetic: N_s = 2 L^3 T below 2^30
    if (2.0 * geom->L * geom->L * geom->L * geom->T >= 1073741824.0) return QS_EINVAL;
    int ndev = 0;
    QS_CUDA(cudaGetDeviceCount(&ndev));
    if (geom->device < 0 || geom->device >= ndev) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(geom->device));
    qs_lattice *lat = (qs_lattice *)calloc(1, sizeof(qs_lattice));
    if (!lat) return QS_ENOMEM;
    lat->g = qs_make_geom(geom->L, geom->T, geom->cstar_mask, geom->t_antiperiodic);
    lat->device = geom->device;
    lat->stream = (cudaStream_t)stream;
    *out = lat;
    return QS_OK;
}

extern "C" int qs_destroy_lattice(qs_lattice *lat)
{
    if (!lat) return QS_OK;
    cudaSetDevice(lat->device);
    qs_free_gauge(lat);
    qs_free_workspace(lat);
    prof_free(lat);
    free(lat);
    return QS_OK;
}

extern "C" int64_t qs_n_sites(const qs_lattice *lat) { return lat ? lat->g.Ns : 0; }

template <typename R>
static DslashArgs<R> make_args(qs_lattice *lat, const double *m0, const void *in, void *out, int nrhs,
                               int gamma5);
template <>
DslashArgs<double> make_args<double>(qs_lattice *lat, const double *m0, const void *in, void *out,
                                     int nrhs, int gamma5)
{
    DslashArgs<double> d;
    d.g = lat->g; d.links = lat->links64; d.clov = lat->clov64;
    d.in = (const double *)in; d.out = (double *)out; d.gamma5 = gamma5; d.nrhs = nrhs;
    for (int r = 0; r < nrhs; ++r) d.m0[r] = m0[r];
    return d;
}
template <>
DslashArgs<float> make_args<float>(qs_lattice *lat, const double *m0, const void *in, void *out,
                                   int nrhs, int gamma5)
{
    DslashArgs<float> d;
    d.g = lat->g; d.links = lat->links32; d.clov = lat->clov32;
    d.in = (const float *)in; d.out = (float *)out; d.gamma5 = gamma5; d.nrhs = nrhs;
    for (int r = 0; r < nrhs; ++r) d.m0[r] = m0[r];
    return d;
}

template <typename R>
static int run_typed(qs_lattice *lat, int pi, const double *m0, const void *in, void *out, int nrhs,
                     int gamma5, int soa)
{
    DslashArgs<R> d = make_args<R>(lat, m0, in, out, nrhs, gamma5);
    int &tv = lat->tuned[soa ? 1 : 0][pi][nrhs];
    if (tv == 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        QS_CUDA(cudaStreamIsCapturing(lat->stream, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            tv = 1 + (qs_dslash_nvariants<R>() > 2 ? 2 : 0);   // cannot time inside a capture
        } else {
            cudaEvent_t e0, e1;
            QS_CUDA(cudaEventCreate(&e0));
            QS_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            int bv = 0;
            for (int v = 0; v < qs_dslash_nvariants<R>(); ++v) {
                QS_CUDA(qs_dslash_launch<R>(d, nrhs, v, soa, lat->stream));   // warm-up
                QS_CUDA(cudaEventRecord(e0, lat->stream));
                for (int rep = 0; rep < 3; ++rep) QS_CUDA(qs_dslash_launch<R>(d, nrhs, v, soa, lat->stream));
                QS_CUDA(cudaEventRecord(e1, lat->stream));
                QS_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                QS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; bv = v; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            tv = bv + 1;
        }
    }
    ProfState *pf = (lat->prof && lat->prof->on) ? lat->prof : nullptr;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (pf) {
        if (pf->pending.size() >= 4096) QS_TRY(prof_resolve(lat));
        ea = prof_event(pf);
        eb = prof_event(pf);
        QS_CUDA(cudaEventRecord(ea, lat->stream));
    }
    cudaError_t e = qs_dslash_launch<R>(d, nrhs, tv - 1, soa, lat->stream);
    qs_note_launches(1);
    if (pf) {
        QS_CUDA(cudaEventRecord(eb, lat->stream));
        pf->pending.push_back({ea, eb, pi == 0 ? QS_F64 : QS_F32,
                               (double)lat->g.Ns * (48.0 * nrhs + 72.0) * sizeof(R)});
    }
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "dslash launch");
        return QS_ECUDA;
    }
    return QS_OK;
}

int qs_dslash_run(qs_lattice *lat, int prec, const double *m0, const void *in, void *out, int nrhs,
                  int gamma5, int soa)
{
    if (prec == QS_F64) return run_typed<double>(lat, 0, m0, in, out, nrhs, gamma5, soa);
    if (prec == QS_F32) return run_typed<float>(lat, 1, m0, in, out, nrhs, gamma5, soa);
    return QS_EINVAL;
}

int qs_apply_op(qs_lattice *lat, const double *m0, const void *in, void *out, int nrhs, int prec,
                int gamma5)
{
    if (!lat || !in || !out || nrhs < 1 || nrhs > QS_MAX_RHS) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    const int tiled = (prec & QS_LAYOUT_TILED) ? 1 : 0;
    prec &= ~QS_LAYOUT_TILED;
    if (prec != QS_F64 && prec != QS_F32) return QS_EINVAL;
    size_t bytes = (size_t)nrhs * lat->g.Ns * 24 * (prec == QS_F64 ? 8 : 4);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return QS_EINVAL;      // overlap
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL; // vector loads need 16 B
    QS_CUDA(cudaSetDevice(lat->device));
    return qs_dslash_run(lat, prec, m0, in, out, nrhs, gamma5, tiled);
}

extern "C" int qs_apply_Dw(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int prec)
{
    double m[QS_MAX_RHS];
    if (nrhs < 1 || nrhs > QS_MAX_RHS) return QS_EINVAL;
    for (int r = 0; r < nrhs; ++r) m[r] = m0;
    return qs_apply_op(lat, m, in, out, nrhs, prec, 0);
}

extern "C" int qs_apply_Q(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int prec)
{
    double m[QS_MAX_RHS];
    if (nrhs < 1 || nrhs > QS_MAX_RHS) return QS_EINVAL;
    for (int r = 0; r < nrhs; ++r) m[r] = m0;
    return qs_apply_op(lat, m, in, out, nrhs, prec, 1);
}

extern "C" const char *qs_strerror(int status)
{
    switch (status) {
    case QS_OK: return "ok";
    case QS_EINVAL: return "invalid argument";
    case QS_ENOMEM: return "device allocation failed";
    case QS_ECUDA: return "CUDA runtime error";
    case QS_ENOCONV: return "iteration cap reached before the tolerance";
    case QS_ETIMEOUT: return "bounded device wait gave up";
    case QS_ENUMERIC: return "NaN or Inf in a reduction";
    case QS_EUNDECIDED: return "|lambda| at the target mass is below its certified accuracy";
    default: return "unknown status";
    }
}

extern "C" const char *qs_last_cuda_error(void) { return g_last_cuda_error; }

template <typename R>
static int batch_typed(const qs_batch_item *items, int n, int tiled, cudaStream_t st)
{
    BatchArgs<R> a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.gamma5 = 1;
    unsigned off = 0;
    for (int i = 0; i < n; ++i) {
        qs_lattice *lat = items[i].lat;
        BatchItem<R> &it = a.item[i];
        it.g = lat->g;
        if (sizeof(R) == 8) {
            it.links = (const typename LinkT<R>::T *)lat->links64;
            it.clov = (const R *)lat->clov64;
        } else {
            it.links = (const typename LinkT<R>::T *)lat->links32;
            it.clov = (const R *)lat->clov32;
        }
        it.in = (const R *)items[i].in;
        it.out = (R *)items[i].out;
        it.nrhs = items[i].nrhs;
        for (int r = 0; r < it.nrhs; ++r) it.m0[r] = items[i].m0[r];
        a.off[i] = off;
        double nb = (double)((lat->g.Ns + 127) / 128) * it.nrhs;
        if (off + nb > 2147483647.0) return QS_EINVAL;
        off += (unsigned)nb;
    }
    a.off[n] = off;
    cudaError_t e = qs_dslash_batch_launch<R>(a, tiled, st);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "batched dslash launch");
        return QS_ECUDA;
    }
    return QS_OK;
}

extern "C" int qs_apply_Q_batch(const qs_batch_item *items, int n, int prec, void *stream)
{
    if (!items || n < 1 || n > QS_BATCH_MAX) return QS_EINVAL;
    const int tiled = (prec & QS_LAYOUT_TILED) ? 1 : 0;
    prec &= ~QS_LAYOUT_TILED;
    if (prec != QS_F64 && prec != QS_F32) return QS_EINVAL;
    const size_t rs = prec == QS_F64 ? 8 : 4;
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        const qs_batch_item &it = items[i];
        if (!it.lat || !it.in || !it.out || !it.m0 || it.nrhs < 1 || it.nrhs > QS_BATCH_RHS) return QS_EINVAL;
        if (!it.lat->gauge_loaded) return QS_EINVAL;
        if (dev >= 0 && it.lat->device != dev) return QS_EINVAL;
        dev = it.lat->device;
        size_t bytes = (size_t)it.nrhs * it.lat->g.Ns * 24 * rs;
        const char *a = (const char *)it.in, *b = (const char *)it.out;
        if (a < b + bytes && b < a + bytes) return QS_EINVAL;
        if (((uintptr_t)it.in | (uintptr_t)it.out) & 15) return QS_EINVAL;
    }
    QS_CUDA(cudaSetDevice(dev));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == QS_F64) return batch_typed<double>(items, n, tiled, st);
    return batch_typed<float>(items, n, tiled, st);
}
