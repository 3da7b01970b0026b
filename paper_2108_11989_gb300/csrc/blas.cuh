// Vector and block kernels of the eigensolver and the CG (internal).
#pragma once
#include "qs_internal.cuh"

#define QS_RED_BLOCKS 608      // partial sums per vector (4 x 152 SMs)
#define QS_RED_THREADS 256

// v has k vectors of nr reals each ([k][nr]); out[r] = sum over vector r of v^2 (FP64)
template <typename R>
cudaError_t qs_norm2(const R *v, int k, int64_t nr, double *part, double *out, cudaStream_t st);
// out[r] = <a_r, b_r> (complex, conj on a), out as [k][2]
template <typename R>
cudaError_t qs_dot(const R *a, const R *b, int k, int64_t nr, double *part, double *out, cudaStream_t st);
// out[r] = || a_r - theta[r] b_r ||^2 (FP64 or FP32 vectors, FP64 sum, theta on device)
template <typename R>
cudaError_t qs_resid2(const R *a, const R *b, const double *theta, int k, int64_t nr,
                      double *part, double *out, cudaStream_t st);
// G[i][j] = <A_i, B_j>, i < ka, j < kb, complex row-major [ka][kb] (FP64 vectors);
// lowp: products and per-chunk sums in FP32, chunk sums accumulated in FP64
cudaError_t qs_gram(const double *A, int ka, const double *B, int kb, int64_t nr, double *part,
                    double2 *G, cudaStream_t st, int lowp = 0);
// V_j = sum_i W_i C[i][j], j < kc (C complex row-major [ka][kc]); V must not alias W;
// lowp: the k-term sums in FP32
cudaError_t qs_rotate(const double *W, int ka, const double2 *C, int kc, int64_t nr, double *V,
                      cudaStream_t st, int lowp = 0);
// the Gram matrix and the rotation on FP32 blocks (FP32 products, FP64 Gram totals)
cudaError_t qs_gram32(const float *A, int ka, const float *B, int kb, int64_t nr, double *part, double2 *G,
                      cudaStream_t st);
cudaError_t qs_rotate32(const float *W, int ka, const double2 *C, int kc, int64_t nr, float *V, cudaStream_t st);
// y_r = (float)(x_r * scale[r])  (scale on device, may be NULL for 1)
cudaError_t qs_d2f(const double *x, float *y, const double *scale, int k, int64_t nr, cudaStream_t st);
// y_r = (double) x_r
cudaError_t qs_f2d(const float *x, double *y, int k, int64_t nr, cudaStream_t st);
// x_r += coef[r] * (double) e_r  (coef on device)
cudaError_t qs_axpy_f2d(double *x, const float *e, const double *coef, int k, int64_t nr, cudaStream_t st);
// ynew = s1 * (ay - c * y) - s2 * x   (all vectors of the block)
template <typename R>
cudaError_t qs_cheb_step(R *ynew, const R *ay, const R *y, const R *x, double c, double s1, double s2,
                         int64_t n, cudaStream_t st);
// y = a * x + b * y over n reals
template <typename R>
cudaError_t qs_axpby(double a, const R *x, double b, R *y, int64_t n, cudaStream_t st);
// x_r *= scale[r] (device)
template <typename R>
cudaError_t qs_scale_cols(R *x, const double *scale, int k, int64_t nr, cudaStream_t st);
// Gaussian entries from a counter-based hash of (seed, index)
cudaError_t qs_fill_gauss(double *x, int64_t n, uint64_t seed, cudaStream_t st);
// x_r = b_r * coef[r] (coef on device)
cudaError_t qs_scaled_copy(double *x, const double *b, const double *coef, int k, int64_t nr, cudaStream_t st);
// out[r] = 1 / sqrt(in[r]) (0 stays 0), or theta^-2 style maps, on device
cudaError_t qs_map_scalars(const double *in, double *out, int k, int mode, cudaStream_t st);
// C* partner map P v = C T gamma_5 v^* of k FP64 or FP32 vectors (partner.cu); in != out
cudaError_t qs_partner(const double *in, double *out, const Geom &g, int k, int tiled, cudaStream_t st);
cudaError_t qs_partner32(const float *in, float *out, const Geom &g, int k, cudaStream_t st);
// single-CTA dense kernels (k <= 64)
cudaError_t qs_chol_rinv(const double2 *G, int k, double2 *Rinv, int *info, cudaStream_t st);
cudaError_t qs_herm_eig(const double2 *H, int k, double *evals, double2 *Y, int *info, cudaStream_t st);

// CG helpers (FP32 vectors, per-rhs scalars on device)
struct CgScalars {
    double *rr, *rr0, *pap, *beta;
    int *active;
};
cudaError_t qs_cg_update(float *x, float *r, const float *p, const float *ap, CgScalars s, int k, int64_t nr,
                         double *part, cudaStream_t st);
cudaError_t qs_cg_finalize(CgScalars s, double tol2, int k, double *part, int *nactive, cudaStream_t st);
cudaError_t qs_cg_pupdate(float *p, const float *r, CgScalars s, int k, int64_t nr, cudaStream_t st);
cudaError_t qs_cg_init(CgScalars s, const double *rr, int k, cudaStream_t st);

// Ritz values (sorted by |theta|) and residual norms of the current block
// Ritz pairs ordered by <v, Q^2 v> = theta^2 + r^2; col[i] is the device column of
// pair i; theta_dev / res_dev are in device column order.
struct Ritz {
    double theta[64], res[64];
    double theta_dev[64], res_dev[64];
    int col[64];
    double mu_max;   // largest Q^2 Ritz value of the block
};
int qs_lowmodes_impl(qs_lattice *lat, double m0, const qs_eig_opts *o, Ritz *rz, int *conv, qs_eig_stats *stats);
