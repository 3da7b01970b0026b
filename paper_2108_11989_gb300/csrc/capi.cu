// C-ABI entry points: lattice handles, operator application, status strings.
#include "qs_internal.cuh"
#include "dslash.cuh"

#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

// Events around operator launches while profiling is on; resolved in batches.
struct ProfState {
    struct Rec {
        cudaEvent_t a, b;
        int prec;
        double bytes;
        int launches;
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
        k.launches += r.launches;
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

static thread_local char g_last_cuda_error[256] = "";
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

static DslashArgs<double> make_args64(qs_lattice *lat, const double *m0, const void *in, void *out, int nrhs,
                                      int gamma5)
{
    DslashArgs<double> d;
    d.g = lat->g; d.links = lat->links64; d.clov = lat->clov64;
    d.in = (const double *)in; d.out = (double *)out; d.gamma5 = gamma5; d.nrhs = nrhs;
    for (int r = 0; r < nrhs; ++r) d.m0[r] = m0[r];
    return d;
}

// ---- launch-variant autotuner -------------------------------------------------
// Each operator form (kernel, storage, epilogue, nrhs) on each lattice shape is timed
// once over all its launch variants (tile shape: right-hand sides per thread and per
// warp, registers per thread) with CUDA events on the handle's stream; the fastest is
// kept in the handle and in a process-wide table.  If QS_TUNE_CACHE names a file, the
// table is read from it at the first use and every new choice is appended to it, so
// later processes on the same GPU model skip the timing.
namespace {
struct TuneCache {
    std::map<std::string, int> m;
    bool loaded = false;
    std::string path;
};
TuneCache &tune_cache()
{
    static TuneCache c;
    return c;
}
std::mutex g_tune_mu;

std::string tune_key(const qs_lattice *lat, const char *kernel, int storage, int cheb, int nrhs)
{
    cudaDeviceProp p;
    char buf[512];
    const char *gpu = cudaGetDeviceProperties(&p, lat->device) == cudaSuccess ? p.name : "gpu";
    snprintf(buf, sizeof(buf), "%s|%s|%d|%d|%d|%dx%d", gpu, kernel, storage, cheb, nrhs, lat->g.L, lat->g.T);
    for (char *c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

int tune_lookup(const std::string &key)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneCache &c = tune_cache();
    if (!c.loaded) {
        c.loaded = true;
        const char *e = getenv("QS_TUNE_CACHE");
        if (e && *e) {
            c.path = e;
            FILE *f = fopen(e, "r");
            if (f) {
                char k[512];
                int v;
                while (fscanf(f, "%511s %d", k, &v) == 2) c.m[k] = v;
                fclose(f);
            }
        }
    }
    auto it = c.m.find(key);
    return it == c.m.end() ? -1 : it->second;
}

void tune_store(const std::string &key, int v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneCache &c = tune_cache();
    c.m[key] = v;
    if (!c.path.empty()) {
        FILE *f = fopen(c.path.c_str(), "a");
        if (f) {
            fprintf(f, "%s %d\n", key.c_str(), v);
            fclose(f);
        }
    }
}

// time `nv` variants of `launch(v)` on the stream; returns the fastest (0-based)
template <typename F>
int time_variants(qs_lattice *lat, int nv, F launch, int *status)
{
    *status = QS_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        *status = QS_ECUDA;
        return 0;
    }
    float best = 1e30f;
    int bv = 0;
    for (int v = 0; v < nv && *status == QS_OK; ++v) {
        cudaError_t e = launch(v);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, lat->stream);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = launch(v);
        if (e == cudaSuccess) e = cudaEventRecord(e1, lat->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            qs_record_cuda_error(e, "autotune");
            *status = QS_ECUDA;
        } else if (ms < best) {
            best = ms;
            bv = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return bv;
}

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}
}  // namespace

// ---- profiling records -----------------------------------------------------------
static int prof_begin(qs_lattice *lat, cudaEvent_t *ea, cudaEvent_t *eb)
{
    ProfState *pf = (lat->prof && lat->prof->on && !capturing(lat->stream)) ? lat->prof : nullptr;
    *ea = *eb = nullptr;
    if (!pf) return QS_OK;
    if (pf->pending.size() >= 4096) QS_TRY(prof_resolve(lat));
    *ea = prof_event(pf);
    *eb = prof_event(pf);
    QS_CUDA(cudaEventRecord(*ea, lat->stream));
    return QS_OK;
}

static int prof_end(qs_lattice *lat, cudaEvent_t ea, cudaEvent_t eb, int prec, double bytes)
{
    if (!ea) return QS_OK;
    QS_CUDA(cudaEventRecord(eb, lat->stream));
    lat->prof->pending.push_back({ea, eb, prec, bytes, 1});
    return QS_OK;
}

int qs_prof_begin(qs_lattice *lat, cudaEvent_t *ea, cudaEvent_t *eb) { return prof_begin(lat, ea, eb); }

int qs_prof_end(qs_lattice *lat, cudaEvent_t ea, cudaEvent_t eb, int prec, double bytes, int launches)
{
    if (!ea) return QS_OK;
    QS_CUDA(cudaEventRecord(eb, lat->stream));
    lat->prof->pending.push_back({ea, eb, prec, bytes, launches});
    return QS_OK;
}

static int run64(qs_lattice *lat, const double *m0, const void *in, void *out, int nrhs, int gamma5, int soa)
{
    DslashArgs<double> d = make_args64(lat, m0, in, out, nrhs, gamma5);
    int &tv = lat->tuned64[soa ? 1 : 0][nrhs];
    if (tv == 0) {
        const std::string key = tune_key(lat, "dslash64", soa, 0, nrhs);
        int v = tune_lookup(key);
        if (v < 0 || v >= qs_dslash_nvariants<double>()) {
            if (capturing(lat->stream)) {
                v = 2;   // no timing inside a capture: a fixed variant
            } else {
                int st = QS_OK;
                v = time_variants(lat, qs_dslash_nvariants<double>(),
                                  [&](int q) { return qs_dslash_launch<double>(d, nrhs, q, soa, lat->stream); }, &st);
                if (st != QS_OK) return st;
                tune_store(key, v);
            }
        }
        tv = v + 1;
    }
    cudaEvent_t ea, eb;
    QS_TRY(prof_begin(lat, &ea, &eb));
    cudaError_t e = qs_dslash_launch<double>(d, nrhs, tv - 1, soa, lat->stream);
    qs_note_launches(1);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "dslash launch");
        return QS_ECUDA;
    }
    return prof_end(lat, ea, eb, QS_F64, (double)lat->g.Ns * (48.0 * nrhs + 72.0) * 8);
}

static int prec_of_storage(int storage)
{
    return storage == QS_D32_F16 ? QS_F16 : storage == QS_D32_BF16 ? QS_BF16 : QS_F32;
}

int qs_d32_run(qs_lattice *lat, int storage, const double *m0, const void *in, void *out, int nrhs, int gamma5,
               const void *cheb_y, const void *cheb_x, double cheb_c, double cheb_s1, double cheb_s2,
               const float *coef_dev, const float *dm_dev)
{
    D32Call c;
    c.coef_dev = coef_dev;
    c.dm_dev = dm_dev;
    c.g = lat->g;
    c.links = lat->links32;
    c.clov = lat->clov32;
    c.in = in;
    c.out = out;
    c.y = cheb_y;
    c.x = cheb_x;
    c.storage = storage;
    c.nrhs = nrhs;
    c.gamma5 = gamma5;
    c.cheb = cheb_y != nullptr;
    c.cheb_c = cheb_c;
    c.cheb_s1 = cheb_s1;
    c.cheb_s2 = cheb_s2;
    c.m0 = m0;
    int &tv = lat->tuned32[storage][c.cheb][nrhs];
    if (tv == 0) {
        const std::string key = tune_key(lat, "dslash32", storage, c.cheb, nrhs);
        int v = tune_lookup(key);
        if (v < 0 || v >= qs_d32_nvariants()) {
            if (capturing(lat->stream)) {
                v = 1;   // no timing inside a capture: a fixed variant
            } else {
                // timing writes `out` only (in, y and x are read): harmless to the caller
                int st = QS_OK;
                v = time_variants(lat, qs_d32_nvariants(), [&](int q) { return qs_d32_launch(c, q, lat->stream); }, &st);
                if (st != QS_OK) return st;
                tune_store(key, v);
                if (getenv("QS_VERBOSE")) fprintf(stderr, "[qstar] autotune %s -> variant %d\n", key.c_str(), v);
            }
        }
        tv = v + 1;
    }
    cudaEvent_t ea, eb;
    QS_TRY(prof_begin(lat, &ea, &eb));
    cudaError_t e = qs_d32_launch(c, tv - 1, lat->stream);
    qs_note_launches(1);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "dslash32 launch");
        return QS_ECUDA;
    }
    // algorithmic bytes: per doubled site, each right-hand side's spinor in and out
    // (plus y and x for the Chebyshev epilogue), and once per launch 36 link + 36 SW
    // FP32 reals (each physical link and SW block serves the site and its mirror)
    const double vs = (double)qs_d32_vec_bytes(storage, 1);
    const double bytes = (double)lat->g.Ns * (vs * (c.cheb ? 4 : 2) * nrhs + 72.0 * 4);
    return prof_end(lat, ea, eb, prec_of_storage(storage), bytes);
}

int qs_dslash_run(qs_lattice *lat, int prec, const double *m0, const void *in, void *out, int nrhs,
                  int gamma5, int soa)
{
    if (prec == QS_F64) return run64(lat, m0, in, out, nrhs, gamma5, soa);
    if (prec == QS_F32) return qs_d32_run(lat, soa ? QS_D32_F32_TILED : QS_D32_F32_CANON, m0, in, out, nrhs, gamma5);
    if (prec == QS_F16 && soa) return qs_d32_run(lat, QS_D32_F16, m0, in, out, nrhs, gamma5);
    if (prec == QS_BF16 && soa) return qs_d32_run(lat, QS_D32_BF16, m0, in, out, nrhs, gamma5);
    return QS_EINVAL;
}

// bytes of one right-hand side of the given precision and layout (0: not supported)
static size_t vec_bytes(const qs_lattice *lat, int prec, int tiled)
{
    switch (prec) {
    case QS_F64: return (size_t)lat->g.Ns * 24 * 8;
    case QS_F32: return (size_t)lat->g.Ns * 24 * 4;
    case QS_F16:
    case QS_BF16: return tiled ? (size_t)qs_d32_vec_bytes(QS_D32_F16, lat->g.Ns) : 0;
    default: return 0;
    }
}

int qs_apply_op(qs_lattice *lat, const double *m0, const void *in, void *out, int nrhs, int prec,
                int gamma5)
{
    if (!lat || !in || !out || nrhs < 1 || nrhs > QS_MAX_RHS) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    const int tiled = (prec & QS_LAYOUT_TILED) ? 1 : 0;
    prec &= ~QS_LAYOUT_TILED;
    const size_t vb = vec_bytes(lat, prec, tiled);
    if (!vb) return QS_EINVAL;
    size_t bytes = (size_t)nrhs * vb;
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return QS_EINVAL;      // overlap
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL; // vector loads need 16 B
    QS_CUDA(cudaSetDevice(lat->device));
    return qs_dslash_run(lat, prec, m0, in, out, nrhs, gamma5, tiled);
}

static int storage_of_prec(int prec)
{
    switch (prec) {
    case QS_F64: return QS_D32_F64_TILED;
    case QS_F32: return QS_D32_F32_TILED;
    case QS_F16: return QS_D32_F16;
    case QS_BF16: return QS_D32_BF16;
    default: return -1;
    }
}

extern "C" int qs_convert_spinors(qs_lattice *lat, const void *in, int in_prec, void *out, int out_prec, int nrhs)
{
    if (!lat || !in || !out || nrhs < 1) return QS_EINVAL;
    const int a = storage_of_prec(in_prec & ~QS_LAYOUT_TILED), b = storage_of_prec(out_prec & ~QS_LAYOUT_TILED);
    if (a < 0 || b < 0 || a == b) return QS_EINVAL;
    const size_t na = (size_t)nrhs * vec_bytes(lat, in_prec & ~QS_LAYOUT_TILED, 1);
    const size_t nb = (size_t)nrhs * vec_bytes(lat, out_prec & ~QS_LAYOUT_TILED, 1);
    const char *x = (const char *)in, *y = (const char *)out;
    if (x < y + nb && y < x + na) return QS_EINVAL;
    if (((uintptr_t)in | (uintptr_t)out) & 15) return QS_EINVAL;
    QS_CUDA(cudaSetDevice(lat->device));
    QS_CUDA(qs_convert_tiled(a, b, in, out, lat->g.Ns, nrhs, lat->stream));
    return QS_OK;
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

static int batch64(const qs_batch_item *items, int n, int tiled, cudaStream_t st)
{
    BatchArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.gamma5 = 1;
    unsigned off = 0;
    for (int i = 0; i < n; ++i) {
        qs_lattice *lat = items[i].lat;
        BatchItem<double> &it = a.item[i];
        it.g = lat->g;
        it.links = lat->links64;
        it.clov = lat->clov64;
        it.in = (const double *)items[i].in;
        it.out = (double *)items[i].out;
        it.nrhs = items[i].nrhs;
        for (int r = 0; r < it.nrhs; ++r) it.m0[r] = items[i].m0[r];
        a.off[i] = off;
        double nb = (double)((lat->g.Ns + 127) / 128) * it.nrhs;
        if (off + nb > 2147483647.0) return QS_EINVAL;
        off += (unsigned)nb;
    }
    a.off[n] = off;
    cudaError_t e = qs_dslash_batch_launch<double>(a, tiled, st);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "batched dslash launch");
        return QS_ECUDA;
    }
    return QS_OK;
}

static int batch32(const qs_batch_item *items, int n, int storage, cudaStream_t st)
{
    D32BatchItem b[QS_BATCH_MAX];
    for (int i = 0; i < n; ++i) {
        qs_lattice *lat = items[i].lat;
        b[i].g = lat->g;
        b[i].links = lat->links32;
        b[i].clov = lat->clov32;
        b[i].in = items[i].in;
        b[i].out = items[i].out;
        b[i].nrhs = items[i].nrhs;
        for (int r = 0; r < items[i].nrhs; ++r) b[i].m0[r] = items[i].m0[r];
    }
    cudaError_t e = qs_d32_batch_launch(b, n, storage, 1, st);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "batched dslash32 launch");
        return QS_ECUDA;
    }
    return QS_OK;
}

extern "C" int qs_apply_Q_batch(const qs_batch_item *items, int n, int prec, void *stream)
{
    if (!items || n < 1 || n > QS_BATCH_MAX) return QS_EINVAL;
    const int tiled = (prec & QS_LAYOUT_TILED) ? 1 : 0;
    prec &= ~QS_LAYOUT_TILED;
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        const qs_batch_item &it = items[i];
        if (!it.lat || !it.in || !it.out || !it.m0 || it.nrhs < 1 || it.nrhs > QS_BATCH_RHS) return QS_EINVAL;
        if (!it.lat->gauge_loaded) return QS_EINVAL;
        if (dev >= 0 && it.lat->device != dev) return QS_EINVAL;
        dev = it.lat->device;
        const size_t vb = vec_bytes(it.lat, prec, tiled);
        if (!vb) return QS_EINVAL;
        size_t bytes = (size_t)it.nrhs * vb;
        const char *a = (const char *)it.in, *b = (const char *)it.out;
        if (a < b + bytes && b < a + bytes) return QS_EINVAL;
        if (((uintptr_t)it.in | (uintptr_t)it.out) & 15) return QS_EINVAL;
    }
    QS_CUDA(cudaSetDevice(dev));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == QS_F64) return batch64(items, n, tiled, st);
    if (prec == QS_F32) return batch32(items, n, tiled ? QS_D32_F32_TILED : QS_D32_F32_CANON, st);
    return batch32(items, n, prec == QS_F16 ? QS_D32_F16 : QS_D32_BF16, st);
}
