// Low modes of Q(m0) and the Pfaffian sign by the mass flow (Sec. 3).
//
// lowmodes: block subspace iteration, Rayleigh-Ritz of the FP64 Q.
//   * filter pass: Y = C_d(Q^2) V with the scaled Chebyshev recurrence on the
//     interval [theta_k^2, b] (b >= lambda_max(Q^2)), FP32 storage and arithmetic;
//   * refinement pass: one power step with Q^-2 (the operator Sec. 3 names),
//     W = Q^-2 V by CG on Q^2 with FP32 inner iterations and FP64 defect
//     correction, started from V Theta^-2;
//   * orthonormalisation: column scaling + Cholesky-QR twice, FP64;
//   * Rayleigh-Ritz: H = V^H Q V, Jacobi, rotate V and QV, residuals in FP64.
#include "blas.cuh"
#include "dslash.cuh"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>

#include <algorithm>
#include <vector>

// A captured Chebyshev filter (2 d operator launches on fixed buffers, coefficients
// and masses read from device tables), replayed with cudaGraphLaunch.
struct FilterGraph {
    int kf, d, storage;
    const void *links, *clov;   // the gauge field the launches were captured with
    cudaGraphExec_t exec;
    void *res;                  // the buffer holding the filtered block after a replay
};
#define QS_GRAPH_MAX_DEG 511
#define QS_NGRAPH 6

struct Workspace {
    FilterGraph fg[QS_NGRAPH];
    int nfg;
    float *coef_dev, *coef_host;   // [3 * QS_GRAPH_MAX_DEG + 64]: (c, s1, s2) per step, then 4 + m0
    int k;
    int64_t nr;
    double *blk64[6];     // FP64 blocks [k][nr]
    float *blk32[5];      // FP32 blocks [k][nr]: filter (captured buffers 0-3) and CG work
    float *f32b[3];       // FP32 basis of the filter stage: V, QV and a rotation target
    int iv, iq, it3;      // which of f32b holds V, QV and the scratch
    double *part;         // reduction partials
    double2 *G, *Rinv, *Hm, *Ym;
    double *ds;           // device scalars, S_NSLOT slots of 64
    int *di;              // device ints, 64 + 8
    double *hp;           // pinned host mirror of ds (S_NSLOT x 64)
    int *hi;              // pinned host ints (64 + 8)
    int have_V;
    int pinv;             // the span of blk64[0] is closed under the C* partner map
    int64_t f32_count, f64_count, cg_count;
};

#define DS(ws, slot) ((ws)->ds + 64 * (slot))
static float *V32(Workspace *w);
static float *QV32(Workspace *w);
static float *T32(Workspace *w);
enum { S_TMP = 0, S_THETA = 1, S_COEF = 2, S_RR = 3, S_RR0 = 4, S_PAP = 5, S_BETA = 6, S_ONES = 7, S_RN = 8,
       S_DOT = 9 /* two slots */, S_VN = 11, S_NSLOT = 12 };

static void ws_free(Workspace *w)
{
    if (!w) return;
    for (int i = 0; i < w->nfg; ++i) cudaGraphExecDestroy(w->fg[i].exec);
    cudaFree(w->coef_dev);
    cudaFreeHost(w->coef_host);
    for (int i = 0; i < 6; ++i) cudaFree(w->blk64[i]);
    for (int i = 0; i < 5; ++i) cudaFree(w->blk32[i]);
    for (int i = 0; i < 3; ++i) cudaFree(w->f32b[i]);
    cudaFree(w->part); cudaFree(w->G); cudaFree(w->Rinv); cudaFree(w->Hm); cudaFree(w->Ym);
    cudaFree(w->ds); cudaFree(w->di);
    cudaFreeHost(w->hp); cudaFreeHost(w->hi);
    free(w);
}

void qs_free_workspace(qs_lattice *lat)
{
    ws_free(lat->ws);
    lat->ws = nullptr;
}

#define CK(call)                                                           \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) {                                           \
            qs_record_cuda_error(_e, #call);                               \
            return _e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA; \
        }                                                                  \
    } while (0)

static int ws_alloc(qs_lattice *lat, Workspace *w, int k)
{
    w->k = k;
    w->nr = lat->g.Ns * 24;
    size_t n64 = (size_t)k * w->nr * sizeof(double), n32 = (size_t)k * w->nr * sizeof(float);
    for (int i = 0; i < 6; ++i) CK(cudaMalloc(&w->blk64[i], n64));
    for (int i = 0; i < 5; ++i) CK(cudaMalloc(&w->blk32[i], n32));
    for (int i = 0; i < 3; ++i) CK(cudaMalloc(&w->f32b[i], n32));
    w->iv = 0; w->iq = 1; w->it3 = 2;
    CK(cudaMalloc(&w->part, (size_t)QS_RED_BLOCKS * 2 * 64 * 64 * sizeof(double)));
    CK(cudaMalloc(&w->G, 64 * 64 * sizeof(double2)));
    CK(cudaMalloc(&w->Rinv, 64 * 64 * sizeof(double2)));
    CK(cudaMalloc(&w->Hm, 64 * 64 * sizeof(double2)));
    CK(cudaMalloc(&w->Ym, 64 * 64 * sizeof(double2)));
    CK(cudaMalloc(&w->ds, S_NSLOT * 64 * sizeof(double)));
    CK(cudaMalloc(&w->di, 72 * sizeof(int)));
    CK(cudaMallocHost(&w->hp, S_NSLOT * 64 * sizeof(double)));
    CK(cudaMallocHost(&w->hi, 72 * sizeof(int)));
    CK(cudaMalloc(&w->coef_dev, (3 * QS_GRAPH_MAX_DEG + 64) * sizeof(float)));
    CK(cudaMallocHost(&w->coef_host, (3 * QS_GRAPH_MAX_DEG + 64) * sizeof(float)));
    CK(cudaMemsetAsync(w->di, 0, 72 * sizeof(int), lat->stream));
    for (int i = 0; i < 64; ++i) w->hp[i] = 1.0;
    CK(cudaMemcpyAsync(DS(w, S_ONES), w->hp, 64 * sizeof(double), cudaMemcpyHostToDevice, lat->stream));
    CK(cudaStreamSynchronize(lat->stream));
    w->have_V = 0;
    return QS_OK;
}

// the handle's workspace for block size k: allocated all at once, or not at all
static int ws_get(qs_lattice *lat, int k, Workspace **out)
{
    Workspace *w = lat->ws;
    if (w && w->k == k) { *out = w; return QS_OK; }
    qs_free_workspace(lat);
    w = (Workspace *)calloc(1, sizeof(Workspace));
    if (!w) return QS_ENOMEM;
    int st = ws_alloc(lat, w, k);
    if (st != QS_OK) {
        ws_free(w);
        return st;
    }
    lat->ws = w;
    *out = w;
    return QS_OK;
}

// ---- operator helpers ---------------------------------------------------------
static int opQ(qs_lattice *lat, Workspace *w, int prec, double m0, const void *in, void *out, int k)
{
    double m[QS_MAX_RHS];
    for (int r = 0; r < k; ++r) m[r] = m0;
    if (prec == QS_F32) w->f32_count += k; else w->f64_count += k;
    return qs_dslash_run(lat, prec, m, in, out, k, 1, 1);   // solver layout
}

static int opQ2(qs_lattice *lat, Workspace *w, int prec, double m0, const void *in, void *tmp, void *out, int k)
{
    QS_TRY(opQ(lat, w, prec, m0, in, tmp, k));
    return opQ(lat, w, prec, m0, tmp, out, k);
}

static int sync_read(qs_lattice *lat, Workspace *w, int slot, int n)
{
    CK(cudaMemcpyAsync(w->hp + 64 * slot, DS(w, slot), n * sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
    CK(cudaMemcpyAsync(w->hi, w->di, 72 * sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
    CK(cudaStreamSynchronize(lat->stream));
    return QS_OK;
}

// column scaling + Cholesky-QR twice: X becomes orthonormal (tmp is clobbered)
// glow: FP32 products in the Gram matrices; rlow: FP32 products in the rotations (the
// filter stage, where the block is far from converged and FP32 rounding is far below
// its residuals).  Rounding in a rotation perturbs the vectors themselves (by ~1e-7,
// an absolute residual floor of ~1e-7 ||Q||), rounding in a Gram matrix only the
// coefficients of the next rotation.
static int orthonormalize(qs_lattice *lat, Workspace *w, double *X, double *tmp, int k, int glow, int rlow)
{
    cudaStream_t st = lat->stream;
    CK(qs_norm2<double>(X, k, w->nr, w->part, DS(w, S_TMP), st));
    CK(qs_map_scalars(DS(w, S_TMP), DS(w, S_COEF), k, 0, st));
    CK(qs_scale_cols(X, DS(w, S_COEF), k, w->nr, st));
    for (int pass = 0; pass < 2; ++pass) {
        double *src = pass == 0 ? X : tmp, *dst = pass == 0 ? tmp : X;
        CK(qs_gram(src, k, src, k, w->nr, w->part, w->G, st, glow));
        CK(qs_chol_rinv(w->G, k, w->Rinv, w->di + 64 + pass, st));
        CK(qs_rotate(src, k, w->Rinv, k, w->nr, dst, st, rlow));
    }
    return QS_OK;
}

// Rayleigh-Ritz on the orthonormal block V = blk64[0].
// * mu: Ritz values of Q^2 (H2 = (QV)^H QV); only the largest is used, as the lower
//   edge of the next filter interval.
// * theta: Ritz values of Q over the whole block (H = V^H Q V), V <- V Y, QV <- QV Y,
//   residuals r = ||Q v - theta v|| (some eigenvalue of Q lies within r of theta).
// The low |lambda| of the indefinite Q are interior eigenvalues, where Ritz values can
// be spurious (+lambda and -lambda contaminations averaging to a small theta, with a
// large r).  The pairs are therefore ordered by <v, Q^2 v> = theta^2 + r^2, which is
// close to lambda^2 for a genuine pair and large for a spurious one.
// Ritz values and residual bounds read back from the pinned mirror (slots S_THETA, S_TMP
// = r^2, S_RN = Q^2 Ritz values) into rz, pairs ordered by theta^2 + r^2
static int finish_ritz(Workspace *w, int k, Ritz *rz)
{
    if (w->hi[64] || w->hi[65]) return QS_ENUMERIC;   // Cholesky-QR broke down
    if (w->hi[66] || w->hi[67]) return QS_ENOCONV;    // Jacobi hit its sweep cap
    double th[64], rs[64], key[64];
    rz->mu_max = 0;
    for (int i = 0; i < k; ++i) {
        th[i] = w->hp[64 * S_THETA + i];
        double r2 = w->hp[64 * S_TMP + i];
        rs[i] = sqrt(r2 > 0 ? r2 : 0);
        key[i] = th[i] * th[i] + rs[i] * rs[i];
        rz->mu_max = std::max(rz->mu_max, fabs(w->hp[64 * S_RN + i]));
        rz->theta_dev[i] = th[i];
        rz->res_dev[i] = rs[i];
        rz->col[i] = i;
        if (!isfinite(th[i]) || !isfinite(rs[i])) return QS_ENUMERIC;
    }
    std::stable_sort(rz->col, rz->col + k, [&](int a, int b) { return key[a] < key[b]; });
    for (int i = 0; i < k; ++i) {
        rz->theta[i] = th[rz->col[i]];
        rz->res[i] = rs[rz->col[i]];
    }
    return QS_OK;
}

// prec: operator precision (FP32 while far from convergence, FP64 otherwise).
// glow: FP32 products in the Gram matrices (then the block is orthonormal only to ~1e-7
// and every residual is divided by ||v||); the rotations use FP32 products only with
// the FP32 operator.  Some eigenvalue of Q lies within ||Q v - theta v|| / ||v|| of
// theta for any theta and v, so the returned bounds hold whatever the rounding of H.
static int rayleigh_ritz(qs_lattice *lat, Workspace *w, double m0, int k, Ritz *rz, int prec, int glow)
{
    cudaStream_t st = lat->stream;
    if (prec == QS_F64) {
        QS_TRY(opQ(lat, w, QS_F64, m0, w->blk64[0], w->blk64[1], k));
    } else {
        CK(qs_d2f(w->blk64[0], w->blk32[0], nullptr, k, w->nr, st));
        QS_TRY(opQ(lat, w, QS_F32, m0, w->blk32[0], w->blk32[1], k));
        CK(qs_f2d(w->blk32[1], w->blk64[1], k, w->nr, st));
    }
    const int rlow = prec == QS_F32;
    glow = glow || rlow;
    // the Q^2 Ritz values only place the filter interval: FP32 products always
    CK(qs_gram(w->blk64[1], k, w->blk64[1], k, w->nr, w->part, w->Hm, st, 1));
    CK(qs_herm_eig(w->Hm, k, DS(w, S_RN), w->Ym, w->di + 66, st));
    CK(qs_gram(w->blk64[0], k, w->blk64[1], k, w->nr, w->part, w->Hm, st, glow));
    CK(qs_herm_eig(w->Hm, k, DS(w, S_THETA), w->Ym, w->di + 67, st));
    CK(qs_rotate(w->blk64[0], k, w->Ym, k, w->nr, w->blk64[2], st, rlow));
    CK(qs_rotate(w->blk64[1], k, w->Ym, k, w->nr, w->blk64[3], st, rlow));
    std::swap(w->blk64[0], w->blk64[2]);
    std::swap(w->blk64[1], w->blk64[3]);
    const bool scale = glow && prec == QS_F64;
    if (scale) CK(qs_norm2<double>(w->blk64[0], k, w->nr, w->part, DS(w, S_VN), st));
    CK(qs_resid2(w->blk64[1], w->blk64[0], DS(w, S_THETA), k, w->nr, w->part, DS(w, S_TMP), st));
    CK(cudaMemcpyAsync(w->hp + 64 * S_THETA, DS(w, S_THETA), k * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w->hp + 64 * S_RN, DS(w, S_RN), k * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (scale) CK(cudaMemcpyAsync(w->hp + 64 * S_VN, DS(w, S_VN), k * sizeof(double), cudaMemcpyDeviceToHost, st));
    QS_TRY(sync_read(lat, w, S_TMP, k));
    if (scale)
        for (int i = 0; i < k; ++i) {
            const double vn = w->hp[64 * S_VN + i];
            w->hp[64 * S_TMP + i] = vn > 0 ? w->hp[64 * S_TMP + i] / vn : INFINITY;
        }
    return finish_ritz(w, k, rz);
}

// Chebyshev filter of degree d on Q^2 over [a, b] with FP32 arithmetic: blk32[0] (in)
// -> result in *res (one of blk32), scaled three-term recurrence (values at 0 kept
// O(1)).  Each degree is two operator launches: T = Q Y, then the second one computes
// Y_new = s1 (Q T - c Y) - s2 Y_old in its epilogue.  storage: QS_D32_F32_TILED, or a
// 16-bit storage whose vectors (52 B per site) live in the same FP32 blocks.
// ---- the filter stage on FP32 blocks ---------------------------------------------
// While the block is far from converged (relative residuals above ~1e-3) the basis, its
// image under Q, the Gram matrices and the rotations stay in FP32 (f32b): no FP64
// traffic and no FP64 <-> FP32 conversions, which run on GB300's slow FP64 pipe.
static float *V32(Workspace *w) { return w->f32b[w->iv]; }
static float *QV32(Workspace *w) { return w->f32b[w->iq]; }
static float *T32(Workspace *w) { return w->f32b[w->it3]; }

// copy k columns (vectors of nr reals of `bytes` each) src[sel[i]] -> dst[i]
static int gather_raw(qs_lattice *lat, const void *src, const int *sel, int h, void *dst, size_t vbytes)
{
    for (int i = 0; i < h; ++i)
        CK(cudaMemcpyAsync((char *)dst + (size_t)i * vbytes, (const char *)src + (size_t)sel[i] * vbytes, vbytes,
                           cudaMemcpyDeviceToDevice, lat->stream));
    return QS_OK;
}

static int orthonormalize32(qs_lattice *lat, Workspace *w, int k)
{
    cudaStream_t st = lat->stream;
    CK(qs_norm2<float>(V32(w), k, w->nr, w->part, DS(w, S_TMP), st));
    CK(qs_map_scalars(DS(w, S_TMP), DS(w, S_COEF), k, 0, st));
    CK(qs_scale_cols<float>(V32(w), DS(w, S_COEF), k, w->nr, st));
    for (int pass = 0; pass < 2; ++pass) {
        CK(qs_gram32(V32(w), k, V32(w), k, w->nr, w->part, w->G, st));
        CK(qs_chol_rinv(w->G, k, w->Rinv, w->di + 64 + pass, st));
        CK(qs_rotate32(V32(w), k, w->Rinv, k, w->nr, T32(w), st));
        std::swap(w->iv, w->it3);
    }
    return QS_OK;
}

// the Rayleigh-Ritz of rayleigh_ritz() with the FP32 operator on the FP32 basis
static int rayleigh_ritz32(qs_lattice *lat, Workspace *w, double m0, int k, Ritz *rz)
{
    cudaStream_t st = lat->stream;
    QS_TRY(opQ(lat, w, QS_F32, m0, V32(w), QV32(w), k));
    CK(qs_gram32(QV32(w), k, QV32(w), k, w->nr, w->part, w->Hm, st));
    CK(qs_herm_eig(w->Hm, k, DS(w, S_RN), w->Ym, w->di + 66, st));
    CK(qs_gram32(V32(w), k, QV32(w), k, w->nr, w->part, w->Hm, st));
    CK(qs_herm_eig(w->Hm, k, DS(w, S_THETA), w->Ym, w->di + 67, st));
    CK(qs_rotate32(V32(w), k, w->Ym, k, w->nr, T32(w), st));
    std::swap(w->iv, w->it3);
    CK(qs_rotate32(QV32(w), k, w->Ym, k, w->nr, T32(w), st));
    std::swap(w->iq, w->it3);
    CK(qs_resid2<float>(QV32(w), V32(w), DS(w, S_THETA), k, w->nr, w->part, DS(w, S_TMP), st));
    CK(cudaMemcpyAsync(w->hp + 64 * S_THETA, DS(w, S_THETA), k * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w->hp + 64 * S_RN, DS(w, S_RN), k * sizeof(double), cudaMemcpyDeviceToHost, st));
    QS_TRY(sync_read(lat, w, S_TMP, k));
    return finish_ritz(w, k, rz);
}

// the launches of one filter, in order: step i (0-based) is T = Q Y_i, then
// Y_{i+1} = s1_i (Q T - c Y_i) - s2_i Y_{i-1}; returns the result buffer.  With coef_dev the
// coefficients of step i and the masses are read from the device tables.
static int cheb_launches(qs_lattice *lat, Workspace *w, const double *m, int k, int d, int storage,
                         const double *cf, const float *coef_dev, const float *dm_dev, void **res)
{
    void *X = w->blk32[0], *Y = w->blk32[1], *Yn = w->blk32[2], *T = w->blk32[3];
    for (int i = 0; i < d; ++i) {
        void *in = i == 0 ? X : Y, *yv = i == 0 ? X : Y, *xv = X, *out = i == 0 ? Y : Yn;
        QS_TRY(qs_d32_run(lat, storage, m, in, T, k, 1, nullptr, nullptr, 0, 0, 0, nullptr, dm_dev));
        QS_TRY(qs_d32_run(lat, storage, m, T, out, k, 1, yv, xv, cf[3 * i], cf[3 * i + 1], cf[3 * i + 2],
                          coef_dev ? coef_dev + 3 * i : nullptr, dm_dev));
        if (i > 0) {
            void *tmp = X; X = Y; Y = Yn; Yn = tmp;
        }
    }
    *res = Y;
    return QS_OK;
}

static bool use_graphs()
{
    static const bool on = [] {
        const char *e = getenv("QS_NO_GRAPHS");
        return !(e && atoi(e));
    }();
    return on;
}

// Chebyshev filter of degree d on Q^2 over [a, b] with FP32 arithmetic: blk32[0] (in)
// -> result in *res (one of blk32), scaled three-term recurrence (values at 0 kept
// O(1)).  Each degree is two operator launches: T = Q Y, then the second one computes
// Y_new = s1 (Q T - c Y) - s2 Y_old in its epilogue.  storage: QS_D32_F32_TILED, or a
// 16-bit storage whose vectors (52 B per site) live in the same FP32 blocks.  On a
// handle with its own stream the 2 d launches are captured once per (k, d, storage) as
// a CUDA graph and replayed; only the coefficient table changes between replays.
static int cheb_filter(qs_lattice *lat, Workspace *w, double m0, int k, int d, double a, double b, int storage,
                       void **res)
{
    cudaStream_t st = lat->stream;
    double m[QS_MAX_RHS];
    for (int r = 0; r < k; ++r) m[r] = m0;
    double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma1 = e / (0.0 - c);
    double sigma = sigma1, g = 2.0 / sigma1;
    std::vector<double> cf(3 * (size_t)d);
    cf[0] = c; cf[1] = sigma1 / e; cf[2] = 0.0;
    for (int i = 1; i < d; ++i) {
        double s2 = 1.0 / (g - sigma);
        cf[3 * i] = c;
        cf[3 * i + 1] = 2.0 * s2 / e;
        cf[3 * i + 2] = sigma * s2;
        sigma = s2;
    }
    w->f32_count += 2 * (int64_t)k * d;
    const bool tuned = lat->tuned32[storage][0][k] && lat->tuned32[storage][1][k];
    if (!(use_graphs() && st != nullptr && d <= QS_GRAPH_MAX_DEG && tuned))
        return cheb_launches(lat, w, m, k, d, storage, cf.data(), nullptr, nullptr, res);
    FilterGraph *fgp = nullptr;
    for (int i = 0; i < w->nfg; ++i) {
        FilterGraph &f = w->fg[i];
        if (f.kf == k && f.d == d && f.storage == storage && f.links == lat->links32 && f.clov == lat->clov32)
            fgp = &f;
    }
    if (!fgp) {
        if (w->nfg == QS_NGRAPH) {   // drop the oldest
            cudaGraphExecDestroy(w->fg[0].exec);
            memmove(&w->fg[0], &w->fg[1], (QS_NGRAPH - 1) * sizeof(FilterGraph));
            --w->nfg;
        }
        FilterGraph f;
        f.kf = k; f.d = d; f.storage = storage;
        f.links = lat->links32; f.clov = lat->clov32;
        const int64_t n0 = qs_kernel_launches();
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int s = cheb_launches(lat, w, m, k, d, storage, cf.data(), w->coef_dev, w->coef_dev + 3 * QS_GRAPH_MAX_DEG,
                              &f.res);
        cudaGraph_t graph = nullptr;
        cudaError_t e1 = cudaStreamEndCapture(st, &graph);
        qs_note_launches((int)(n0 - qs_kernel_launches()));   // counted at replay instead
        if (s != QS_OK) { if (graph) cudaGraphDestroy(graph); return s; }
        CK(e1);
        cudaError_t e2 = cudaGraphInstantiate(&f.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e2);
        w->fg[w->nfg++] = f;
        fgp = &w->fg[w->nfg - 1];
    }
    float *hc = w->coef_host;
    for (int i = 0; i < 3 * d; ++i) hc[i] = (float)cf[i];
    for (int r = 0; r < k; ++r) hc[3 * QS_GRAPH_MAX_DEG + r] = (float)(4.0 + m0);
    CK(cudaMemcpyAsync(w->coef_dev, hc, 3 * (size_t)d * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->coef_dev + 3 * QS_GRAPH_MAX_DEG, hc + 3 * QS_GRAPH_MAX_DEG, k * sizeof(float),
                       cudaMemcpyHostToDevice, st));
    cudaEvent_t ea, eb;
    QS_TRY(qs_prof_begin(lat, &ea, &eb));
    CK(cudaGraphLaunch(fgp->exec, st));
    qs_note_launches(2 * d);
    const double vs = (double)qs_d32_vec_bytes(storage, 1);
    const double bytes = (double)lat->g.Ns * d * (vs * 6 * k + 2 * 72.0 * 4);
    const int prec = storage == QS_D32_F16 ? QS_F16 : storage == QS_D32_BF16 ? QS_BF16 : QS_F32;
    QS_TRY(qs_prof_end(lat, ea, eb, prec, bytes, 2 * d));
    *res = fgp->res;
    return QS_OK;
}

// The same filter in FP64 on blk64[0] (V, kept) with blk64[1..5] as work blocks;
// the filtered block ends in blk64[0] (plain FP64 form of the solver).
static int cheb_filter64(qs_lattice *lat, Workspace *w, double m0, int k, int d, double a, double b)
{
    cudaStream_t st = lat->stream;
    double *X = w->blk64[1], *Y = w->blk64[2], *Yn = w->blk64[3], *T = w->blk64[4], *AY = w->blk64[5];
    int64_t n = (int64_t)k * w->nr;
    CK(cudaMemcpyAsync(X, w->blk64[0], n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma1 = e / (0.0 - c);
    double sigma = sigma1, g = 2.0 / sigma1;
    QS_TRY(opQ2(lat, w, QS_F64, m0, X, T, AY, k));
    CK(qs_cheb_step<double>(Y, AY, X, X, c, sigma1 / e, 0.0, n, st));
    for (int i = 2; i <= d; ++i) {
        double s2 = 1.0 / (g - sigma);
        QS_TRY(opQ2(lat, w, QS_F64, m0, Y, T, AY, k));
        CK(qs_cheb_step<double>(Yn, AY, Y, X, c, 2.0 * s2 / e, sigma * s2, n, st));
        double *tmp = X; X = Y; Y = Yn; Yn = tmp;
        sigma = s2;
    }
    CK(cudaMemcpyAsync(w->blk64[0], Y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return QS_OK;
}

// FP32 CG on Q^2 for k right-hand sides in r (overwritten); solution in x.
static int cg_f32(qs_lattice *lat, Workspace *w, double m0, int k, float *x, float *r, float *p, float *t,
                  float *ap, double tol, int maxit, int *iters)
{
    cudaStream_t st = lat->stream;
    CgScalars s;
    s.rr = DS(w, S_RR); s.rr0 = DS(w, S_RR0); s.pap = DS(w, S_PAP); s.beta = DS(w, S_BETA);
    s.active = w->di;
    size_t bytes = (size_t)k * w->nr * sizeof(float);
    CK(cudaMemsetAsync(x, 0, bytes, st));
    CK(cudaMemcpyAsync(p, r, bytes, cudaMemcpyDeviceToDevice, st));
    CK(qs_norm2<float>(r, k, w->nr, w->part, DS(w, S_TMP), st));
    CK(qs_cg_init(s, DS(w, S_TMP), k, st));
    int it;
    for (it = 1; it <= maxit; ++it) {
        QS_TRY(opQ(lat, w, QS_F32, m0, p, t, k));
        QS_TRY(opQ(lat, w, QS_F32, m0, t, ap, k));
        CK(qs_norm2<float>(t, k, w->nr, w->part, s.pap, st));        // <p, Q^2 p> = |Q p|^2
        CK(qs_cg_update(x, r, p, ap, s, k, w->nr, w->part, st));
        CK(qs_cg_finalize(s, tol * tol, k, w->part, w->di + 70, st));
        CK(qs_cg_pupdate(p, r, s, k, w->nr, st));
        if (it % 16 == 0 || it == maxit) {
            CK(cudaMemcpyAsync(w->hi + 70, w->di + 70, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (w->hi[70] == 0) break;
        }
    }
    w->cg_count += it;
    *iters = it;
    return QS_OK;
}

static int verbose()
{
    static const int v = [] {
        const char *e = getenv("QS_VERBOSE");
        return e ? atoi(e) : 0;
    }();
    return v;
}

// X (initial guess in, solution out) of Q^2 X = B for orthonormal B, by FP32 CG
// inner solves and FP64 residuals; stops when every ||B - Q^2 X|| <= tol.
static int solve_q2_mixed(qs_lattice *lat, Workspace *w, double m0, int k, const double *B, double *X,
                          double *T1, double *T2, double tol)
{
    cudaStream_t st = lat->stream;
    for (int outer = 0; outer < 40; ++outer) {
        QS_TRY(opQ2(lat, w, QS_F64, m0, X, T1, T2, k));
        CK(qs_axpby<double>(1.0, B, -1.0, T2, (int64_t)k * w->nr, st));       // T2 = B - Q^2 X
        CK(qs_norm2<double>(T2, k, w->nr, w->part, DS(w, S_RN), st));
        QS_TRY(sync_read(lat, w, S_RN, k));
        double rmax = 0;
        for (int i = 0; i < k; ++i) rmax = std::max(rmax, sqrt(w->hp[64 * S_RN + i]));
        if (verbose() > 1) fprintf(stderr, "[qstar]   solve outer %d max|r| %.3e (target %.3e)\n", outer, rmax, tol);
        if (rmax <= tol) return QS_OK;
        CK(qs_map_scalars(DS(w, S_RN), DS(w, S_COEF), k, 0, st));             // 1 / |r|
        CK(qs_d2f(T2, w->blk32[0], DS(w, S_COEF), k, w->nr, st));
        double tin = std::max(2e-6, std::min(0.1, 0.3 * tol / rmax));
        int its = 0;
        QS_TRY(cg_f32(lat, w, m0, k, w->blk32[1], w->blk32[0], w->blk32[2], w->blk32[3], w->blk32[4], tin,
                      20000, &its));
        if (verbose() > 1) fprintf(stderr, "[qstar]   inner CG %d iterations (tol %.2e)\n", its, tin);
        CK(qs_map_scalars(DS(w, S_RN), DS(w, S_COEF), k, 1, st));             // |r|
        CK(qs_axpy_f2d(X, w->blk32[1], DS(w, S_COEF), k, w->nr, st));
    }
    return QS_ENOCONV;
}

// k / 2 representatives of the block V = blk64[0] (device columns, written to sel)
// whose span together with their C* partners P v is (as nearly as possible) the span of
// V.  Candidates are taken in Ritz order (rz->col).  M = V^H P V (FP32 products) gives the
// coordinates in V of the projection of every partner; a candidate is kept only if it has
// a component of norm^2 > 1/2 outside span{v_s, P v_s} of those kept so far (Gram-Schmidt
// in the k coordinates), so the two members of a degenerate pair are never both picked.
static int pick_representatives(qs_lattice *lat, Workspace *w, const Ritz *rz, int k, int *sel, bool fp32)
{
    const int h = k / 2;
    cudaStream_t st = lat->stream;
    if (fp32) {
        CK(qs_partner32(V32(w), T32(w), lat->g, k, st));
        CK(qs_gram32(V32(w), k, T32(w), k, w->nr, w->part, w->G, st));
    } else {
        CK(qs_partner(w->blk64[0], w->blk64[3], lat->g, k, 1, st));
        CK(qs_gram(w->blk64[0], k, w->blk64[3], k, w->nr, w->part, w->G, st, 1));
    }
    static thread_local double2 M[64 * 64];
    CK(cudaMemcpyAsync(M, w->G, (size_t)k * k * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<std::vector<double2>> basis;
    auto residual = [&](std::vector<double2> x) {
        for (const auto &b : basis) {
            double cr = 0, ci = 0;   // <b, x>
            for (int j = 0; j < k; ++j) {
                cr += b[j].x * x[j].x + b[j].y * x[j].y;
                ci += b[j].x * x[j].y - b[j].y * x[j].x;
            }
            for (int j = 0; j < k; ++j) {
                x[j].x -= cr * b[j].x - ci * b[j].y;
                x[j].y -= cr * b[j].y + ci * b[j].x;
            }
        }
        return x;
    };
    auto norm2 = [&](const std::vector<double2> &x) {
        double n = 0;
        for (int j = 0; j < k; ++j) n += x[j].x * x[j].x + x[j].y * x[j].y;
        return n;
    };
    int n = 0;
    bool used[64] = {false};
    for (int i = 0; i < k && n < h; ++i) {
        const int c = rz->col[i];
        std::vector<double2> e(k, make_double2(0, 0));
        e[c] = make_double2(1, 0);
        std::vector<double2> r = residual(e);
        double nr2 = norm2(r);
        if (nr2 <= 0.5) continue;
        sel[n++] = c;
        used[c] = true;
        for (int j = 0; j < k; ++j) { r[j].x /= sqrt(nr2); r[j].y /= sqrt(nr2); }
        basis.push_back(r);
        std::vector<double2> m(k);
        for (int j = 0; j < k; ++j) m[j] = M[j * k + c];   // P v_c = sum_j v_j M[j][c]
        std::vector<double2> rm = residual(m);
        double nm2 = norm2(rm);
        if (nm2 > 1e-6) {
            for (int j = 0; j < k; ++j) { rm[j].x /= sqrt(nm2); rm[j].y /= sqrt(nm2); }
            basis.push_back(rm);
        }
    }
    for (int i = 0; i < k && n < h; ++i)   // only if the span is far from closed under P
        if (!used[rz->col[i]]) { sel[n++] = rz->col[i]; used[rz->col[i]] = true; }
    return QS_OK;
}

// blk64[dst][0..h) = blk64[0][sel[i]] (scaled by coef[sel[i]] if coef != NULL)
static int gather_columns(qs_lattice *lat, Workspace *w, const int *sel, int h, double *dst, const double *coef)
{
    for (int i = 0; i < h; ++i)
        CK(cudaMemcpyAsync(dst + (size_t)i * w->nr, w->blk64[0] + (size_t)sel[i] * w->nr, w->nr * sizeof(double),
                           cudaMemcpyDeviceToDevice, lat->stream));
    if (coef) {
        double c[64];
        for (int i = 0; i < h; ++i) c[i] = coef[sel[i]];
        CK(cudaMemcpyAsync(DS(w, S_COEF), c, h * sizeof(double), cudaMemcpyHostToDevice, lat->stream));
        CK(qs_scale_cols(dst, DS(w, S_COEF), h, w->nr, lat->stream));
    }
    return QS_OK;
}

static double now_s()
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

extern "C" void qs_eig_default_opts(qs_eig_opts *o)
{
    if (!o) return;
    o->k = 16;
    o->nwant = 4;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->cheb_degree = 24;
    o->warm_start = 1;
    o->seed = 1;
    o->precision = QS_F32;
    o->pairing = 1;
}


int qs_lowmodes_impl(qs_lattice *lat, double m0, const qs_eig_opts *o, Ritz *rz, int *conv, qs_eig_stats *stats)
{
    int k = o->k;
    Workspace *w;
    QS_TRY(ws_get(lat, k, &w));
    cudaStream_t st = lat->stream;
    double t0 = now_s();
    int64_t f32_0 = w->f32_count, f64_0 = w->f64_count, cg_0 = w->cg_count;
    if (!(o->warm_start && w->have_V)) {
        CK(qs_fill_gauss(w->blk64[0], (int64_t)k * w->nr, o->seed * 0x9E3779B97F4A7C15ULL + 17, st));
        w->pinv = 0;
    }
    w->have_V = 0;
    const bool plain = o->precision == QS_F64;
    const bool pair = !plain && o->pairing && k >= 4;
    // Gram products in FP32 also in the FP64-operator stages when the requested accuracy
    // allows it (with the FP64 operator their rounding is ~1e-7 relative to the
    // eigenvalue scale); rotations stay FP64 there
    const int glow = (!plain && o->tol >= 1e-6) ? 1 : 0;
    // in32: the current basis is the FP32 one (filter stage of the mixed forms); else blk64[0]
    bool in32 = false;
    auto to32 = [&]() -> int {          // FP64 basis -> FP32 basis
        CK(qs_d2f(w->blk64[0], V32(w), nullptr, k, w->nr, st));
        in32 = true;
        return QS_OK;
    };
    auto to64 = [&]() -> int {          // FP32 basis -> FP64 basis
        if (in32) CK(qs_f2d(V32(w), w->blk64[0], k, w->nr, st));
        in32 = false;
        return QS_OK;
    };
    auto rr32 = [&]() -> int {          // FP32 orthonormalisation + Rayleigh-Ritz
        QS_TRY(orthonormalize32(lat, w, k));
        return rayleigh_ritz32(lat, w, m0, k, rz);
    };
    if (plain) {
        QS_TRY(orthonormalize(lat, w, w->blk64[0], w->blk64[2], k, 0, 0));
        QS_TRY(rayleigh_ritz(lat, w, m0, k, rz, QS_F64, 0));
    } else {
        QS_TRY(to32());
        QS_TRY(rr32());
    }
    // b >= lambda_max(Q^2): ||Q|| = ||D|| <= max_x ||4 + m0 + A(x)|| + ||hopping||,
    // ||hopping|| <= 4 (each direction is a partial isometry pair of norm 1)
    double qn = fabs(4.0 + m0) + lat->clov_norm + 4.0;
    double b = qn * qn;
    // Relative residual with an absolute floor: a pair with r <= atol counts as converged
    // whatever its theta, so an exact zero mode (|lambda| below any relative accuracy)
    // still ends the iteration, with |theta| - r <= 0 telling the caller it is undecided.
    const double atol = 1e-13 * qn;
    const double theta_floor = atol / o->tol;
    auto rel = [&](int i) { return rz->res[i] / std::max(fabs(rz->theta[i]), theta_floor); };
    int it = 0, nf = 0, nref = 0;
    *conv = 0;
    double prev_worst = 1e300;
    int stall = 0, fstall = 0, restarts = 0;
    int last_prec = plain ? QS_F64 : QS_F32;
    for (it = 0; it < o->max_iter; ++it) {
        double worst = 0;
        for (int i = 0; i < o->nwant; ++i) worst = std::max(worst, rel(i));
        // Filter while it makes progress and the block is far from converged; then
        // power steps with Q^-2, whose rate (lambda_i / lambda_{k+1})^2 does not
        // depend on how small lambda_bar is.  The FP32 filter cannot improve a block
        // below ~1e-5 relative residual, so only a stagnating refinement hands back.
        bool refine = (worst < 1e-3 || fstall >= 2) && !(stall >= 3 && worst > 1e-5);
        if (plain) refine = false;   // plain FP64 form: filter passes only
        if (stall >= 3 && fstall >= 2 && restarts < 3) {
            // both stages stagnate (typically a warm start from a distant mass): keep the
            // converged pairs, moved to the front so Cholesky-QR preserves them, and
            // refill the rest of the block with random vectors
            QS_TRY(to64());
            int nconv = 0;
            double2 P[64 * 64];
            for (int i = 0; i < k * k; ++i) P[i] = make_double2(0, 0);
            for (int i = 0; i < k; ++i)
                if (rel(i) <= o->tol) P[rz->col[i] * k + nconv++] = make_double2(1, 0);
            for (int i = 0, j = nconv; i < k; ++i)
                if (!(rel(i) <= o->tol)) P[rz->col[i] * k + j++] = make_double2(1, 0);
            CK(cudaMemcpyAsync(w->Ym, P, k * k * sizeof(double2), cudaMemcpyHostToDevice, st));
            CK(qs_rotate(w->blk64[0], k, w->Ym, k, w->nr, w->blk64[2], st));
            std::swap(w->blk64[0], w->blk64[2]);
            CK(qs_fill_gauss(w->blk64[0] + (size_t)nconv * w->nr, (int64_t)(k - nconv) * w->nr,
                             o->seed * 0x2545F4914F6CDD1DULL + 977 * (restarts + 1), st));
            w->pinv = 0;
            if (plain) {
                QS_TRY(orthonormalize(lat, w, w->blk64[0], w->blk64[2], k, 0, 0));
                QS_TRY(rayleigh_ritz(lat, w, m0, k, rz, QS_F64, 0));
            } else {
                QS_TRY(to32());
                QS_TRY(rr32());
            }
            last_prec = plain ? QS_F64 : QS_F32;
            stall = fstall = 0;
            prev_worst = 1e300;
            ++restarts;
            if (verbose()) fprintf(stderr, "[qstar] m0=%.6f restart keeping %d converged pairs\n", m0, nconv);
            continue;
        }
        if (verbose())
            fprintf(stderr, "[qstar] m0=%.6f pass %d worst_rel_res=%.3e theta0=%.6e res0=%.3e theta_k=%.4e b=%.3e next=%s\n",
                    m0, it, worst, rz->theta[0], rz->res[0], rz->theta[k - 1], b,
                    worst <= o->tol ? "done" : (refine ? "refine" : "filter"));
        if (worst <= o->tol) {
            if (last_prec == QS_F64) { *conv = 1; break; }
            // confirm with the FP64 operator (and an FP64-orthonormal block) before accepting
            QS_TRY(to64());
            QS_TRY(orthonormalize(lat, w, w->blk64[0], w->blk64[2], k, glow, 0));
            QS_TRY(rayleigh_ritz(lat, w, m0, k, rz, QS_F64, glow));
            last_prec = QS_F64;
            continue;
        }
        bool paired = false;
        if (!refine) {
            // Chebyshev filter on [a, b], a = largest Q^2 Ritz value of the block
            double a = rz->mu_max;
            if (a >= 0.5 * b || it == 0) a = std::min(a, 0.05 * b);
            if (plain) {
                QS_TRY(cheb_filter64(lat, w, m0, k, std::max(2, o->cheb_degree), a, b));
            } else {
                if (!in32) QS_TRY(to32());
                const int storage = o->precision == QS_F16 ? QS_D32_F16
                                  : o->precision == QS_BF16 ? QS_D32_BF16 : QS_D32_F32_TILED;
                // C* pairing: filter k / 2 representatives, their partners complete the
                // block (the filter is a polynomial in Q^2, which commutes with P)
                // (a random start block is first filtered whole: its Ritz vectors are not yet
                // close to pairs)
                const bool pp = pair && (w->pinv || nf + nref > 0);
                const int kf = pp ? k / 2 : k;
                const size_t vb32 = w->nr * sizeof(float);
                const float *src = V32(w);
                if (pp) {
                    int sel[32];
                    QS_TRY(pick_representatives(lat, w, rz, k, sel, true));
                    QS_TRY(gather_raw(lat, V32(w), sel, kf, T32(w), vb32));
                    src = T32(w);
                }
                if (storage == QS_D32_F32_TILED)
                    CK(cudaMemcpyAsync(w->blk32[0], src, kf * vb32, cudaMemcpyDeviceToDevice, st));
                else
                    CK(qs_convert_tiled(QS_D32_F32_TILED, storage, src, w->blk32[0], lat->g.Ns, kf, st));
                void *Y = nullptr;
                QS_TRY(cheb_filter(lat, w, m0, kf, std::max(2, o->cheb_degree), a, b, storage, &Y));
                if (storage == QS_D32_F32_TILED)
                    CK(cudaMemcpyAsync(V32(w), Y, kf * vb32, cudaMemcpyDeviceToDevice, st));
                else
                    CK(qs_convert_tiled(storage, QS_D32_F32_TILED, Y, V32(w), lat->g.Ns, kf, st));
                if (pp) {
                    CK(qs_partner32(V32(w), V32(w) + (size_t)kf * w->nr, lat->g, kf, st));
                    w->pinv = 1;
                    paired = true;
                }
            }
            ++nf;
        } else {
            // power step with Q^-2: X = Q^-2 V, started from V_i / <v_i, Q^2 v_i>
            // (<v, Q^2 v> = theta^2 + r^2 for each Ritz vector)
            QS_TRY(to64());
            double inv[64];
            for (int i = 0; i < k; ++i) {   // device column order
                double q2 = rz->theta_dev[i] * rz->theta_dev[i] + rz->res_dev[i] * rz->res_dev[i];
                inv[i] = q2 > 0 ? 1.0 / q2 : 0.0;
            }
            // solve accuracy tied to the absolute residual the target needs
            double tsol = std::max(1e-13, std::min(1e-2, 0.05 * worst * fabs(rz->theta[0])));
            if (pair && (w->pinv || nf + nref > 0)) {
                // Q^-2 commutes with P: solve for k / 2 representatives, partners complete
                const int h = k / 2;
                int sel[32];
                QS_TRY(pick_representatives(lat, w, rz, k, sel, false));
                QS_TRY(gather_columns(lat, w, sel, h, w->blk64[3], nullptr));
                QS_TRY(gather_columns(lat, w, sel, h, w->blk64[2], inv));
                int s = solve_q2_mixed(lat, w, m0, h, w->blk64[3], w->blk64[2], w->blk64[4], w->blk64[5], tsol);
                if (s != QS_OK && s != QS_ENOCONV) return s;
                CK(qs_partner(w->blk64[2], w->blk64[2] + (size_t)h * w->nr, lat->g, h, 1, st));
                w->pinv = 1;
                paired = true;
            } else {
                CK(cudaMemcpyAsync(DS(w, S_COEF), inv, k * sizeof(double), cudaMemcpyHostToDevice, st));
                CK(qs_scaled_copy(w->blk64[2], w->blk64[0], DS(w, S_COEF), k, w->nr, st));
                int s = solve_q2_mixed(lat, w, m0, k, w->blk64[0], w->blk64[2], w->blk64[4], w->blk64[5], tsol);
                if (s != QS_OK && s != QS_ENOCONV) return s;
            }
            std::swap(w->blk64[0], w->blk64[2]);
            ++nref;
        }
        // FP32 operator, Gram and rotation while the block is far from converged (its
        // residuals are then far above FP32 rounding); FP64 from the refinement on
        last_prec = (plain || refine || worst < 1e-3) ? QS_F64 : QS_F32;
        int rr;
        if (last_prec == QS_F32) {
            if (!in32) QS_TRY(to32());
            rr = rr32();
        } else {
            QS_TRY(to64());
            QS_TRY(orthonormalize(lat, w, w->blk64[0], w->blk64[2], k, plain ? 0 : glow, 0));
            rr = rayleigh_ritz(lat, w, m0, k, rz, QS_F64, plain ? 0 : glow);
        }
        if (rr == QS_ENUMERIC && paired) {
            // the completed block was (numerically) rank deficient: replace the partner half
            // by random vectors and orthonormalise again
            QS_TRY(to64());
            CK(qs_fill_gauss(w->blk64[0] + (size_t)(k / 2) * w->nr, (int64_t)(k - k / 2) * w->nr,
                             o->seed * 0x5851F42D4C957F2DULL + 31 * (it + 1), st));
            w->pinv = 0;
            CK(cudaMemsetAsync(w->di + 64, 0, 2 * sizeof(int), st));
            if (last_prec == QS_F32) {
                QS_TRY(to32());
                rr = rr32();
            } else {
                QS_TRY(orthonormalize(lat, w, w->blk64[0], w->blk64[2], k, glow, 0));
                rr = rayleigh_ritz(lat, w, m0, k, rz, QS_F64, glow);
            }
        }
        QS_TRY(rr);
        double nw = 0;
        for (int i = 0; i < o->nwant; ++i) nw = std::max(nw, rel(i));
        if (refine) { if (nw > 0.97 * prev_worst) ++stall; else stall = 0; }
        else { if (nw > 0.9 * prev_worst) ++fstall; else fstall = 0; }
        prev_worst = nw;
    }
    QS_TRY(to64());   // the FP64 block is the result (and the next warm start)
    w->have_V = 1;
    if (stats) {
        stats->iterations = it;
        stats->filter_passes = nf;
        stats->refine_passes = nref;
        stats->dslash_f32 = w->f32_count - f32_0;
        stats->dslash_f64 = w->f64_count - f64_0;
        stats->cg_iterations = w->cg_count - cg_0;
        stats->seconds = now_s() - t0;
    }
    return QS_OK;
}

extern "C" int qs_lowmodes_at_mass(qs_lattice *lat, double m0, const qs_eig_opts *opts, double *evals,
                                   double *resid, void *evecs, qs_eig_stats *stats)
{
    if (!lat || !evals || !resid) return QS_EINVAL;
    if (!lat->gauge_loaded) return QS_EINVAL;
    qs_eig_opts o;
    if (opts) o = *opts; else qs_eig_default_opts(&o);
    if (o.k < 2 || o.k > 64 || (o.k & 1) || o.nwant < 1 || o.nwant > o.k || !(o.tol > 0) || o.max_iter < 0 ||
        o.cheb_degree < 2 || o.precision < QS_F64 || o.precision > QS_BF16)
        return QS_EINVAL;
    if (12 * lat->g.Ns < o.k) return QS_EINVAL;
    CK(cudaSetDevice(lat->device));
    Ritz rz;
    int conv = 0;
    QS_TRY(qs_lowmodes_impl(lat, m0, &o, &rz, &conv, stats));
    for (int i = 0; i < o.k; ++i) { evals[i] = rz.theta[i]; resid[i] = rz.res[i]; }
    if (evecs) {   // Ritz vectors in the order of the returned values, canonical layout
        const size_t nr = lat->ws->nr;
        for (int i = 0; i < o.k; ++i)
            CK(qs_soa_to_aos(lat->ws->blk64[0] + (size_t)rz.col[i] * nr, (double *)evecs + (size_t)i * nr,
                             lat->g.Ns, lat->stream));
        CK(cudaStreamSynchronize(lat->stream));
    }
    return conv ? QS_OK : QS_ENOCONV;
}
