// Launch interface of the Dslash kernels (internal).
#pragma once
#include "qs_internal.cuh"

#define QS_MAX_RHS 64

template <typename R> struct LinkT;
template <> struct LinkT<double> { typedef double2 T; };
template <> struct LinkT<float> { typedef float2 T; };

template <typename R>
struct DslashArgs {
    Geom g;
    const typename LinkT<R>::T *links;   // [mu][9][Vphys]
    const R *clov;                        // [72][Vphys]
    const R *in;                          // [nrhs][Ns][24]
    R *out;
    int gamma5;                           // 1: Q = gamma_5 D
    int nrhs;                             // right-hand sides in this launch
    double m0[QS_MAX_RHS];                // bare mass per right-hand side
};

// batched form: up to QS_BATCH_MAX lattices, up to QS_BATCH_RHS right-hand sides each
#define QS_BATCH_MAX 8
#define QS_BATCH_RHS 16
template <typename R>
struct BatchItem {
    Geom g;
    const typename LinkT<R>::T *links;
    const R *clov;
    const R *in;
    R *out;
    int nrhs;
    double m0[QS_BATCH_RHS];
};
template <typename R>
struct BatchArgs {
    int n, gamma5;
    unsigned off[QS_BATCH_MAX + 1];   // first block of each item, off[n] = total blocks
    BatchItem<R> item[QS_BATCH_MAX];
};
template <typename R>
cudaError_t qs_dslash_batch_launch(const BatchArgs<R> &a, int soa, cudaStream_t st);

// out = D in (or Q in) for nrhs vectors with launch variant `variant`
// (0 .. qs_dslash_nvariants<R>() - 1); in and out must not overlap.
// soa = 1: the solver's site-tiled spinor layout [site / 16][12][site % 16][re, im]
template <typename R>
cudaError_t qs_dslash_launch(DslashArgs<R> a, int nrhs, int variant, int soa, cudaStream_t st);
template <typename R>
int qs_dslash_nvariants();


// ---- FP32-arithmetic operator (dslash32.cu) for FP32 and 16-bit storage ------
enum { QS_D32_F32_TILED = 0, QS_D32_F32_CANON = 1, QS_D32_F16 = 2, QS_D32_BF16 = 3,
       QS_D32_F64_TILED = 4 /* conversions only */ };

struct D32Call {
    Geom g;
    const float2 *links;   // [mu][9][Vphys] FP32
    const float2 *clov;    // [2][18][Vphys] FP32 pairs (packed SW blocks)
    const void *in;        // nrhs vectors, vector r at in + r * qs_d32_vec_bytes(storage, Ns)
    void *out;
    const void *y, *x;     // cheb = 1: out = s1 (Q in - c y) - s2 x
    int storage, nrhs, gamma5, cheb;
    double cheb_c, cheb_s1, cheb_s2;
    const double *m0;      // host, nrhs masses (ignored where dm_dev is set)
    const float *coef_dev; // NULL, or device (c, s1, s2) of the Chebyshev epilogue
    const float *dm_dev;   // NULL, or device 4 + m0 per right-hand side
};
int qs_d32_nvariants();
int64_t qs_d32_vec_bytes(int storage, int64_t Ns);
cudaError_t qs_d32_launch(const D32Call &c, int variant, cudaStream_t st);
// k vectors from one tiled storage to another (QS_D32_F32_TILED, _F16, _BF16, _F64_TILED)
cudaError_t qs_convert_tiled(int from, int to, const void *in, void *out, int64_t Ns, int k, cudaStream_t st);
// FP64 solver-layout block of k vectors <-> 16-bit scaled storage
cudaError_t qs_q16_from_f64(int storage, const double *in, void *out, int64_t Ns, int k, cudaStream_t st);
cudaError_t qs_f64_from_q16(int storage, const void *in, double *out, int64_t Ns, int k, cudaStream_t st);
// Batched persistent form: up to QS_BATCH_MAX lattices of any volume, one launch; the
// blocks loop over (lattice, right-hand-side group, site tile) work items.
struct D32BatchItem {
    Geom g;
    const float2 *links, *clov;
    const void *in;
    void *out;
    int nrhs;
    double m0[QS_BATCH_RHS];
};
cudaError_t qs_d32_batch_launch(const D32BatchItem *items, int n, int storage, int gamma5, cudaStream_t st);

// one vector from the solver layout to the canonical layout (FP64)
cudaError_t qs_soa_to_aos(const double *in, double *out, int64_t Ns, cudaStream_t st);
