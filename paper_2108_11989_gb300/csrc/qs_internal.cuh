// Internal definitions of the qstar library (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include "../../include/qstar.h"

// ---------------------------------------------------------------------------
// error plumbing: no call aborts; CUDA errors become QS_ECUDA
// ---------------------------------------------------------------------------
void qs_record_cuda_error(cudaError_t e, const char *where);

#define QS_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) {                                             \
            qs_record_cuda_error(_e, #call);                                 \
            return _e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;   \
        }                                                                    \
    } while (0)

#define QS_TRY(expr)                    \
    do {                                \
        int _s = (expr);                \
        if (_s != QS_OK) return _s;     \
    } while (0)

// ---------------------------------------------------------------------------
// geometry of the doubled lattice (T x L x L x 2L), see include/qstar.h
// ---------------------------------------------------------------------------
struct Geom {
    int L, T, L2;          // L2 = 2L
    int cstar_y, cstar_z;  // C* in y / z (x always)
    int t_anti;
    int64_t Ns, Vphys;     // doubled sites, physical sites
    int64_t sy, sz, st;    // strides of y, z, t in the doubled site index
};

struct qs_lattice {
    Geom g;
    int device;
    cudaStream_t stream;
    int gauge_loaded;
    double csw_su3, csw_u1;
    double clov_norm;      // max over sites of ||A(x)||_F (bounds ||A(x)||)
    // V = U exp(i theta) on the physical lattice, SoA [mu][9][Vphys] complex
    double2 *links64;
    float2 *links32;
    // SW term A on the physical lattice (two packed 6x6 Hermitian blocks); the mirror
    // site's blocks are derived on the fly.  FP64: [72][Vphys] reals (per block 6 real
    // diagonals, then 15 strict-lower (re, im)); FP32: [2][18][Vphys] pairs (per block
    // 3 pairs of diagonals, then the 15 strict-lower entries)
    double *clov64;
    float2 *clov32;
    // autotuned launch variant + 1 (0: not tuned): FP64 operator per [layout][nrhs],
    // FP32-arithmetic operator per [storage][Chebyshev epilogue][nrhs]
    int tuned64[2][65];
    int tuned32[4][2][65];
    // solver workspace (allocated on first use, see solver.cu)
    struct Workspace *ws;
    // kernel profiling state (capi.cu), NULL when off
    struct ProfState *prof;
};

// neighbour of doubled site s in direction mu, step +1/-1; *sgn = fermion bc factor
__host__ __device__ inline int64_t qs_nbr(const Geom &g, int64_t s, int mu, int step, int *sgn)
{
    int x = (int)(s % g.L2);
    int64_t r = s / g.L2;
    int y = (int)(r % g.L);
    r /= g.L;
    int z = (int)(r % g.L);
    int t = (int)(r / g.L);
    *sgn = 1;
    switch (mu) {
    case 0: {
        int tn = t + step;
        if (tn < 0 || tn >= g.T) {
            tn = (tn + g.T) % g.T;
            if (g.t_anti) *sgn = -1;
        }
        return s + (int64_t)(tn - t) * g.st;
    }
    case 1: {
        int xn = (x + step + g.L2) % g.L2;
        return s + (xn - x);
    }
    case 2: {
        int yn = y + step;
        int xn = x;
        if (yn < 0 || yn >= g.L) {
            yn = (yn + g.L) % g.L;
            if (g.cstar_y) xn = (x + g.L) % g.L2;
        }
        return s + (int64_t)(yn - y) * g.sy + (xn - x);
    }
    default: {
        int zn = z + step;
        int xn = x;
        if (zn < 0 || zn >= g.L) {
            zn = (zn + g.L) % g.L;
            if (g.cstar_z) xn = (x + g.L) % g.L2;
        }
        return s + (int64_t)(zn - z) * g.sz + (xn - x);
    }
    }
}

// physical site of doubled site s, and whether s is on the mirror (antiquark) half
__host__ __device__ inline int64_t qs_phys(const Geom &g, int64_t s, bool *mirror)
{
    int x = (int)(s % g.L2);
    *mirror = x >= g.L;
    return (s / g.L2) * g.L + (x >= g.L ? x - g.L : x);
}

// ---------------------------------------------------------------------------
// small complex helpers (R = float or double)
// ---------------------------------------------------------------------------
template <typename R> struct C2 { R re, im; };

template <typename R> __host__ __device__ inline C2<R> cmk(R a, R b) { C2<R> c; c.re = a; c.im = b; return c; }
template <typename R> __host__ __device__ inline C2<R> operator+(C2<R> a, C2<R> b) { return cmk(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ inline C2<R> operator-(C2<R> a, C2<R> b) { return cmk(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ inline C2<R> operator*(C2<R> a, C2<R> b)
{
    return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ inline C2<R> operator*(R a, C2<R> b) { return cmk(a * b.re, a * b.im); }
template <typename R> __host__ __device__ inline C2<R> conjc(C2<R> a) { return cmk(a.re, -a.im); }
// multiply by i
template <typename R> __host__ __device__ inline C2<R> mul_i(C2<R> a) { return cmk(-a.im, a.re); }
// a * conj(b)
template <typename R> __host__ __device__ inline C2<R> mul_cj(C2<R> a, C2<R> b)
{
    return cmk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
// conj(a) * b
template <typename R> __host__ __device__ inline C2<R> cj_mul(C2<R> a, C2<R> b)
{
    return cmk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}

// packed Hermitian 6x6: 6 real diagonals then 15 complex strict-lower entries
// (i > j) in row order; index of (i, j) is i (i - 1) / 2 + j
__host__ __device__ inline int qs_tri(int i, int j) { return i * (i - 1) / 2 + j; }

Geom qs_make_geom(int L, int T, int cstar_mask, int t_anti);

// process-wide count of kernel launches made by the library
void qs_note_launches(int n);

// operator launch with the handle's autotuned variant (capi.cu).  prec: QS_F64, QS_F32,
// QS_F16, QS_BF16 (the 16-bit ones in the tiled layout only); soa: tiled layout
int qs_dslash_run(qs_lattice *lat, int prec, const double *m0, const void *in, void *out, int nrhs,
                  int gamma5, int soa);
// FP32-arithmetic operator for a storage QS_D32_*, optionally with the Chebyshev
// epilogue out = s1 (Q in - c y) - s2 x (cheb_y != NULL)
int qs_d32_run(qs_lattice *lat, int storage, const double *m0, const void *in, void *out, int nrhs, int gamma5,
               const void *cheb_y = nullptr, const void *cheb_x = nullptr, double cheb_c = 0,
               double cheb_s1 = 0, double cheb_s2 = 0, const float *coef_dev = nullptr,
               const float *dm_dev = nullptr);
// record one profiling interval covering `launches` operator launches (graph replays)
int qs_prof_begin(qs_lattice *lat, cudaEvent_t *ea, cudaEvent_t *eb);
int qs_prof_end(qs_lattice *lat, cudaEvent_t ea, cudaEvent_t eb, int prec, double bytes, int launches);
