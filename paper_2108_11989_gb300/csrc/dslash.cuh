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
    double m0[QS_MAX_RHS];                // bare mass per right-hand side
};

// out = D in (or Q in) for nrhs vectors; in and out must not overlap.
template <typename R>
cudaError_t qs_dslash_launch(DslashArgs<R> a, int nrhs, cudaStream_t st);
