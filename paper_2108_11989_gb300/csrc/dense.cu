// Small dense FP64 kernels (k <= 64), one thread block each: Cholesky factor
// and its inverse for the Cholesky-QR orthogonalisation, and a cyclic Jacobi
// eigensolver for the Rayleigh-Ritz matrix.  Complex matrices are row-major
// double2 [k][k].
#include "blas.cuh"

#include <mutex>

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// G = R^H R with R upper triangular; Rinv = R^-1 (upper).  info = 1 if G is not
// numerically positive definite.
__global__ void chol_rinv_kernel(const double2 *G, int k, double2 *Rinv, int *info)
{
    extern __shared__ double2 sm[];
    double2 *R = sm;            // [k][k]
    __shared__ int bad;
    int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int i = t; i < k * k; i += blockDim.x) R[i] = make_double2(0, 0);
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (t == 0) {
            double d = G[j * k + j].x;
            for (int i = 0; i < j; ++i) d -= R[i * k + j].x * R[i * k + j].x + R[i * k + j].y * R[i * k + j].y;
            if (!(d > 0) || !isfinite(d)) { bad = 1; d = 1.0; }
            R[j * k + j] = make_double2(sqrt(d), 0);
        }
        __syncthreads();
        double rjj = R[j * k + j].x;
        for (int l = j + 1 + t; l < k; l += blockDim.x) {
            double2 s = G[j * k + l];
            for (int i = 0; i < j; ++i) s = csub(s, cmul(cconj(R[i * k + j]), R[i * k + l]));
            R[j * k + l] = cscale(1.0 / rjj, s);
        }
        __syncthreads();
    }
    // back substitution, one column of the inverse per thread
    for (int c = t; c < k; c += blockDim.x) {
        for (int i = k - 1; i >= 0; --i) {
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int l = i + 1; l <= c; ++l) s = csub(s, cmul(R[i * k + l], Rinv[l * k + c]));
            Rinv[i * k + c] = i > c ? make_double2(0, 0) : cscale(1.0 / R[i * k + i].x, s);
        }
    }
    __syncthreads();
    if (t == 0) *info = bad;
}

// Jacobi eigensolver for a Hermitian H: H = Y diag(ev) Y^H; eigenpairs returned in
// order of increasing |ev|.  Parallel ordering (Brent and Luk's round-robin): a sweep
// is k - 1 rounds, each round rotates k / 2 disjoint pivot pairs at once (a tournament
// schedule in which every pair (p, q) meets exactly once per sweep).  Rotation for
// pivot (p, q), h_pq = c u (|u| = 1): with D = diag(1, conj u) the 2x2 block becomes real
// symmetric [[a, c], [c, b]], diagonalised by [[cs, sn], [-sn, cs]], t = sn / cs the
// smaller root of t^2 + 2 tau t - 1 = 0, tau = (b - a) / (2 c).  J = D [[cs, sn], [-sn, cs]].
// Disjoint rotations commute, so all column updates of a round are applied together,
// then all row updates.  k must be even.
__device__ __forceinline__ int rr_player(int j, int r, int k)
{
    return j == 0 ? 0 : ((j - 1 + r) % (k - 1)) + 1;
}

__global__ void jacobi_kernel(const double2 *Hin, int k, double *ev, double2 *Yout, int *info)
{
    extern __shared__ double2 sm[];
    double2 *H = sm;              // [k][k]
    double2 *Y = sm + k * k;      // [k][k]
    __shared__ double s_cs[32], s_sn[32];
    __shared__ double2 s_u[32];
    __shared__ int s_p[32], s_q[32], s_skip[32];
    __shared__ double red[2][8];
    __shared__ int perm[64];
    const int t = threadIdx.x, nt = blockDim.x, half = k / 2;
    for (int i = t; i < k * k; i += nt) {
        H[i] = Hin[i];
        Y[i] = make_double2((i / k) == (i % k) ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    // symmetrise exactly (H is Hermitian up to rounding)
    for (int i = t; i < k * k; i += nt) {
        int r = i / k, c = i % k;
        if (r < c) {
            double2 a = H[r * k + c], b = H[c * k + r];
            double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            H[r * k + c] = m;
            H[c * k + r] = cconj(m);
        } else if (r == c) {
            H[i].y = 0;
        }
    }
    __syncthreads();
    int sweep;
    for (sweep = 0; sweep < 40; ++sweep) {
        double o = 0, s = 0;
        for (int i = t; i < k * k; i += nt) {
            double m2 = H[i].x * H[i].x + H[i].y * H[i].y;
            s += m2;
            if (i / k != i % k) o += m2;
        }
        for (int d = 16; d > 0; d >>= 1) {
            o += __shfl_xor_sync(0xffffffffu, o, d);
            s += __shfl_xor_sync(0xffffffffu, s, d);
        }
        if ((t & 31) == 0) { red[0][t >> 5] = o; red[1][t >> 5] = s; }
        __syncthreads();
        double off = 0, tot = 0;
        for (int w = 0; w < (nt >> 5); ++w) { off += red[0][w]; tot += red[1][w]; }
        __syncthreads();
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int r = 0; r < k - 1; ++r) {
            if (t < half) {
                int p = rr_player(t, r, k), q = rr_player(k - 1 - t, r, k);
                if (p > q) { int x = p; p = q; q = x; }
                s_p[t] = p;
                s_q[t] = q;
                double2 h = H[p * k + q];
                double c = sqrt(h.x * h.x + h.y * h.y);
                double a = H[p * k + p].x, b = H[q * k + q].x;
                if (c <= 1e-300 || c <= 1e-18 * (fabs(a) + fabs(b))) {
                    s_skip[t] = 1;
                } else {
                    s_skip[t] = 0;
                    s_u[t] = make_double2(h.x / c, h.y / c);
                    double tau = (b - a) / (2.0 * c);
                    double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    double cs = 1.0 / sqrt(1.0 + tt * tt);
                    s_cs[t] = cs;
                    s_sn[t] = tt * cs;
                }
            }
            __syncthreads();
            // columns: H J and Y J, J = [[cs, sn], [-ub sn, ub cs]] on (p, q)
            for (int w = t; w < half * k; w += nt) {
                const int i = w / k, l = w % k;
                if (s_skip[i]) continue;
                const int p = s_p[i], q = s_q[i];
                const double cs = s_cs[i], sn = s_sn[i];
                const double2 ub = cconj(s_u[i]);
                double2 hp = H[l * k + p], hq = H[l * k + q];
                H[l * k + p] = csub(cscale(cs, hp), cscale(sn, cmul(ub, hq)));
                H[l * k + q] = cadd(cscale(sn, hp), cscale(cs, cmul(ub, hq)));
                double2 yp = Y[l * k + p], yq = Y[l * k + q];
                Y[l * k + p] = csub(cscale(cs, yp), cscale(sn, cmul(ub, yq)));
                Y[l * k + q] = cadd(cscale(sn, yp), cscale(cs, cmul(ub, yq)));
            }
            __syncthreads();
            // rows: J^H H, rows p' = cs p - u sn q, q' = sn p + u cs q
            for (int w = t; w < half * k; w += nt) {
                const int i = w / k, l = w % k;
                if (s_skip[i]) continue;
                const int p = s_p[i], q = s_q[i];
                const double cs = s_cs[i], sn = s_sn[i];
                const double2 u = s_u[i];
                double2 hp = H[p * k + l], hq = H[q * k + l];
                H[p * k + l] = csub(cscale(cs, hp), cscale(sn, cmul(u, hq)));
                H[q * k + l] = cadd(cscale(sn, hp), cscale(cs, cmul(u, hq)));
            }
            __syncthreads();
            if (t < half && !s_skip[t]) {
                const int p = s_p[t], q = s_q[t];
                H[p * k + q] = make_double2(0, 0);
                H[q * k + p] = make_double2(0, 0);
                H[p * k + p].y = 0;
                H[q * k + q].y = 0;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        for (int i = 0; i < k; ++i) perm[i] = i;
        for (int i = 0; i < k; ++i)          // selection sort by |ev|, stable on ties
            for (int j = i + 1; j < k; ++j)
                if (fabs(H[perm[j] * k + perm[j]].x) < fabs(H[perm[i] * k + perm[i]].x)) {
                    int s2 = perm[i]; perm[i] = perm[j]; perm[j] = s2;
                }
        *info = sweep >= 40 ? 1 : 0;
    }
    __syncthreads();
    for (int i = t; i < k; i += nt) ev[i] = H[perm[i] * k + perm[i]].x;
    for (int i = t; i < k * k; i += nt) {
        int r = i / k, c = i % k;
        Yout[r * k + c] = Y[r * k + perm[c]];
    }
}

}  // namespace

cudaError_t qs_chol_rinv(const double2 *G, int k, double2 *Rinv, int *info, cudaStream_t st)
{
    if (k > 64) return cudaErrorInvalidValue;
    chol_rinv_kernel<<<1, 64, k * k * sizeof(double2), st>>>(G, k, Rinv, info);
    qs_note_launches(1);
    return cudaGetLastError();
}

cudaError_t qs_herm_eig(const double2 *H, int k, double *evals, double2 *Y, int *info, cudaStream_t st)
{
    if (k > 64) return cudaErrorInvalidValue;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 16);
    });
    if (k & 1) return cudaErrorInvalidValue;   // the round-robin ordering pairs all indices
    jacobi_kernel<<<1, 256, 2 * k * k * sizeof(double2), st>>>(H, k, evals, Y, info);
    qs_note_launches(1);
    return cudaGetLastError();
}
