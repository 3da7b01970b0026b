// Internal entry points of the even-odd preconditioned operator (Sec. 4), shared by the
// W_eo / D_hat code and the mass reweighting.
#pragma once
#include "dslash.cuh"
#include "qs_internal.cuh"

// the FP64 operator on the output sites of one parity ((t + z + y + x) mod 2), zeros on the
// others; canonical layout (dslash.cu)
cudaError_t qs_dslash64_parity_launch(const DslashArgs<double> &a, int parity, cudaStream_t st);

// D_hat = D_ee - D_eo (D_oo)^-1 D_oe (gamma5 = 1: Q_hat = gamma_5 D_hat) of nrhs FP64 vectors
// in the canonical layout; odd-site entries of in are ignored, those of out set to zero.
// Asynchronous on the lattice's stream; work: 3 * nrhs * N_s * 24 doubles; in may equal out.
// inv: NULL (the odd-site blocks are solved on the fly) or the inverses from
// qs_clover_inverse_odd at the same m0.
int qs_dhat_run(qs_lattice *lat, double m0, const double *in, double *out, int nrhs, int gamma5, double *work,
                const double2 *inv = nullptr);

// inv = (4 + m0 + A)^-1 on the odd physical sites, [2][6][6][V_phys / 2] complex, the odd
// physical site p at index p / 2 (asynchronous)
int qs_clover_inverse_odd(qs_lattice *lat, double m0, double2 *inv);

// out = in on the even sites, 0 on the odd ones (nrhs FP64 vectors, asynchronous)
int qs_even_mask(qs_lattice *lat, const double *in, double *out, int nrhs);

// out = scale (D_oo)^-1 in on the odd sites (inverses from qs_clover_inverse_odd), 0 on the
// even sites (asynchronous; in and out must not overlap)
int qs_oo_inverse_apply(qs_lattice *lat, const double2 *inv, const double *in, double *out, int nrhs, double scale);

// out = D in on the output sites of one parity, 0 on the others (FP64, asynchronous)
int qs_dslash64_parity(qs_lattice *lat, double m0, const double *in, double *out, int nrhs, int parity);
