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

// Picks (and caches in the handle) the fastest variant for this precision and
// nrhs by timing each once on the handle's stream, then launches it.
int qs_dslash_run(qs_lattice *lat, int prec, const double *m0, const void *in, void *out,
                  int nrhs, int gamma5, int soa = 0);

// one vector from the solver layout to the canonical layout (FP64)
cudaError_t qs_soa_to_aos(const double *in, double *out, int64_t Ns, cudaStream_t st);
