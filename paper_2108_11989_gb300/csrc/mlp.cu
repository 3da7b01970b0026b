// Step-proposal network of the learned form of the sign flow: a 3-layer
// perceptron in FP32 (in -> hidden -> hidden -> out, ReLU), trained on the GPU by
// the kernels below (forward, backward, loss, Adam).  The paper itself steps with
// m <- m + c lambda_bar (Sec. 3); a proposal of this network is used only where the
// flow's no-crossing certificate (eq. derivativebound) accepts it.
//
// Parameters are one FP32 array [W1 (h x in), b1, W2 (h x h), b2, W3 (out x h), b3].
// Loss over B rows, targets T (column 0 regression, columns 1.. labels):
//   L = (1/B) sum_b [ (Y_b0 - T_b0)^2 / 2 + sum_{j>=1} (softplus(Y_bj) - T_bj Y_bj) ].
#include "qs_internal.cuh"

#include <stdlib.h>

struct qs_mlp {
    int ni, nh, no, maxB, device;
    cudaStream_t stream;
    size_t np, off[7];
    float *P, *G, *M, *V;
    float *Z1, *A1, *Z2, *A2, *Y, *dY, *dA, *rowloss, *loss;
    int t;
};

namespace {

#define TS 16
// C[m][n] (+)= sum_k A[m*sam + k*sak] * B[k*sbk + n*sbn] (+ bias[n]); C row-major, ld = ldc
__global__ void gemm_kernel(int M, int N, int K, const float *__restrict__ A, long sam, long sak,
                            const float *__restrict__ B, long sbk, long sbn, float *__restrict__ C, int ldc,
                            const float *__restrict__ bias)
{
    __shared__ float as[TS][TS + 1], bs[TS][TS + 1];
    int m = blockIdx.y * TS + threadIdx.y, n = blockIdx.x * TS + threadIdx.x;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TS) {
        int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        as[threadIdx.y][threadIdx.x] = (m < M && ka < K) ? A[m * sam + ka * sak] : 0.f;
        bs[threadIdx.y][threadIdx.x] = (kb < K && n < N) ? B[kb * sbk + n * sbn] : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TS; ++kk) acc = fmaf(as[threadIdx.y][kk], bs[kk][threadIdx.x], acc);
        __syncthreads();
    }
    if (m < M && n < N) C[(long)m * ldc + n] = acc + (bias ? bias[n] : 0.f);
}

__global__ void relu_fwd(const float *__restrict__ Z, float *__restrict__ A, long n)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) A[i] = fmaxf(Z[i], 0.f);
}

__global__ void relu_bwd(float *__restrict__ dA, const float *__restrict__ Z, long n)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n && !(Z[i] > 0.f)) dA[i] = 0.f;
}

// out[c] = sum_r X[r][c] (fixed order per column)
__global__ void colsum(const float *__restrict__ X, int R, int Cn, float *__restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Cn) return;
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += X[(long)r * Cn + c];
    out[c] = s;
}

__global__ void loss_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, int B, int no,
                                 float *__restrict__ dY, float *__restrict__ rowloss)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *y = Y + (long)b * no, *t = T + (long)b * no;
    float *d = dY + (long)b * no;
    float r = y[0] - t[0];
    float l = 0.5f * r * r;
    d[0] = r / B;
    for (int j = 1; j < no; ++j) {
        float z = y[j];
        float sp = z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        l += sp - t[j] * z;
        d[j] = (1.f / (1.f + expf(-z)) - t[j]) / B;
    }
    rowloss[b] = l;
}

__global__ void mean_kernel(const float *__restrict__ x, int n, float *__restrict__ out)
{
    __shared__ float sh[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / n;
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = G[i];
    float m = b1 * M[i] + (1.f - b1) * g;
    float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

inline unsigned nblk(long n) { return (unsigned)((n + 255) / 256); }

cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float *A, long sam, long sak, const float *B,
                 long sbk, long sbn, float *C, int ldc, const float *bias)
{
    dim3 blk(TS, TS), grd((N + TS - 1) / TS, (M + TS - 1) / TS);
    gemm_kernel<<<grd, blk, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias);
    qs_note_launches(1);
    return cudaGetLastError();
}

int forward(qs_mlp *n, const float *X, int B)
{
    const int ni = n->ni, nh = n->nh, no = n->no;
    float *W1 = n->P + n->off[0], *b1 = n->P + n->off[1], *W2 = n->P + n->off[2], *b2 = n->P + n->off[3];
    float *W3 = n->P + n->off[4], *b3 = n->P + n->off[5];
    cudaStream_t st = n->stream;
    QS_CUDA(gemm(st, B, nh, ni, X, ni, 1, W1, 1, ni, n->Z1, nh, b1));
    relu_fwd<<<nblk((long)B * nh), 256, 0, st>>>(n->Z1, n->A1, (long)B * nh);
    QS_CUDA(gemm(st, B, nh, nh, n->A1, nh, 1, W2, 1, nh, n->Z2, nh, b2));
    relu_fwd<<<nblk((long)B * nh), 256, 0, st>>>(n->Z2, n->A2, (long)B * nh);
    QS_CUDA(gemm(st, B, no, nh, n->A2, nh, 1, W3, 1, nh, n->Y, no, b3));
    qs_note_launches(2);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
}

}  // namespace

extern "C" int qs_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void *stream, qs_mlp **out)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 2 || max_batch < 1) return QS_EINVAL;
    if ((long)max_batch * (n_hidden > n_out ? n_hidden : n_out) > (1L << 28)) return QS_EINVAL;
    *out = nullptr;
    qs_mlp *n = (qs_mlp *)calloc(1, sizeof(qs_mlp));
    if (!n) return QS_ENOMEM;
    QS_CUDA(cudaGetDevice(&n->device));
    n->ni = n_in; n->nh = n_hidden; n->no = n_out; n->maxB = max_batch;
    n->stream = (cudaStream_t)stream;
    size_t sz[6] = {(size_t)n_hidden * n_in, (size_t)n_hidden, (size_t)n_hidden * n_hidden, (size_t)n_hidden,
                    (size_t)n_out * n_hidden, (size_t)n_out};
    n->off[0] = 0;
    for (int i = 0; i < 6; ++i) n->off[i + 1] = n->off[i] + sz[i];
    n->np = n->off[6];
    size_t hb = (size_t)max_batch * n_hidden, ob = (size_t)max_batch * n_out;
    cudaError_t e = cudaSuccess;
    float **bufs[] = {&n->P, &n->G, &n->M, &n->V};
    for (float **b : bufs) if (e == cudaSuccess) e = cudaMalloc(b, n->np * sizeof(float));
    float **acts[] = {&n->Z1, &n->A1, &n->Z2, &n->A2, &n->dA};
    for (float **b : acts) if (e == cudaSuccess) e = cudaMalloc(b, hb * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->Y, ob * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->dY, ob * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->rowloss, (size_t)max_batch * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(n->P, 0, n->np * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->M, 0, n->np * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->V, 0, n->np * sizeof(float), n->stream);
    if (e != cudaSuccess) {
        qs_record_cuda_error(e, "qs_mlp_create");
        qs_mlp_destroy(n);
        return e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
    }
    *out = n;
    return QS_OK;
}

extern "C" int qs_mlp_destroy(qs_mlp *n)
{
    if (!n) return QS_OK;
    float *all[] = {n->P, n->G, n->M, n->V, n->Z1, n->A1, n->Z2, n->A2, n->dA, n->Y, n->dY, n->rowloss, n->loss};
    for (float *p : all) cudaFree(p);
    free(n);
    return QS_OK;
}

extern "C" int64_t qs_mlp_n_params(const qs_mlp *n) { return n ? (int64_t)n->np : 0; }

cudaStream_t qs_mlp_stream(const qs_mlp *n) { return n->stream; }

extern "C" int qs_mlp_set_params(qs_mlp *n, const float *host)
{
    if (!n || !host) return QS_EINVAL;
    QS_CUDA(cudaMemcpyAsync(n->P, host, n->np * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    QS_CUDA(cudaMemsetAsync(n->M, 0, n->np * sizeof(float), n->stream));
    QS_CUDA(cudaMemsetAsync(n->V, 0, n->np * sizeof(float), n->stream));
    QS_CUDA(cudaStreamSynchronize(n->stream));
    n->t = 0;
    return QS_OK;
}

extern "C" int qs_mlp_get_params(qs_mlp *n, float *host)
{
    if (!n || !host) return QS_EINVAL;
    QS_CUDA(cudaMemcpyAsync(host, n->P, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    QS_CUDA(cudaStreamSynchronize(n->stream));
    return QS_OK;
}

extern "C" int qs_mlp_get_grads(qs_mlp *n, float *host)
{
    if (!n || !host) return QS_EINVAL;
    QS_CUDA(cudaMemcpyAsync(host, n->G, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    QS_CUDA(cudaStreamSynchronize(n->stream));
    return QS_OK;
}

extern "C" int qs_mlp_forward(qs_mlp *n, const float *X, int B, float *Y)
{
    if (!n || !X || !Y || B < 1 || B > n->maxB) return QS_EINVAL;
    QS_TRY(forward(n, X, B));
    QS_CUDA(cudaMemcpyAsync(Y, n->Y, (size_t)B * n->no * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    return QS_OK;
}

extern "C" int qs_mlp_train_step(qs_mlp *n, const float *X, const float *T, int B, float lr, float *loss)
{
    if (!n || !X || !T || B < 1 || B > n->maxB || !(lr > 0)) return QS_EINVAL;
    const int ni = n->ni, nh = n->nh, no = n->no;
    cudaStream_t st = n->stream;
    QS_TRY(forward(n, X, B));
    float *W2 = n->P + n->off[2], *W3 = n->P + n->off[4];
    float *gW1 = n->G + n->off[0], *gb1 = n->G + n->off[1], *gW2 = n->G + n->off[2], *gb2 = n->G + n->off[3];
    float *gW3 = n->G + n->off[4], *gb3 = n->G + n->off[5];
    loss_grad_kernel<<<nblk(B), 256, 0, st>>>(n->Y, T, B, no, n->dY, n->rowloss);
    mean_kernel<<<1, 256, 0, st>>>(n->rowloss, B, n->loss);
    // layer 3: dW3 = dY^T A2, db3 = sum dY, dA2 = dY W3
    QS_CUDA(gemm(st, no, nh, B, n->dY, 1, no, n->A2, nh, 1, gW3, nh, nullptr));
    colsum<<<nblk(no), 256, 0, st>>>(n->dY, B, no, gb3);
    QS_CUDA(gemm(st, B, nh, no, n->dY, no, 1, W3, nh, 1, n->dA, nh, nullptr));
    relu_bwd<<<nblk((long)B * nh), 256, 0, st>>>(n->dA, n->Z2, (long)B * nh);     // dZ2
    // layer 2: dW2 = dZ2^T A1, db2 = sum dZ2, dA1 = dZ2 W2 (into A2's buffer, no longer needed)
    QS_CUDA(gemm(st, nh, nh, B, n->dA, 1, nh, n->A1, nh, 1, gW2, nh, nullptr));
    colsum<<<nblk(nh), 256, 0, st>>>(n->dA, B, nh, gb2);
    QS_CUDA(gemm(st, B, nh, nh, n->dA, nh, 1, W2, nh, 1, n->A2, nh, nullptr));
    relu_bwd<<<nblk((long)B * nh), 256, 0, st>>>(n->A2, n->Z1, (long)B * nh);     // dZ1
    // layer 1: dW1 = dZ1^T X, db1 = sum dZ1
    QS_CUDA(gemm(st, nh, ni, B, n->A2, 1, nh, X, ni, 1, gW1, ni, nullptr));
    colsum<<<nblk(nh), 256, 0, st>>>(n->A2, B, nh, gb1);
    n->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    adam_kernel<<<nblk((long)n->np), 256, 0, st>>>(n->P, n->G, n->M, n->V, (long)n->np, lr, b1, b2, 1e-8f,
                                                  1.f - powf(b1, (float)n->t), 1.f - powf(b2, (float)n->t));
    qs_note_launches(8);
    QS_CUDA(cudaGetLastError());
    if (loss) {
        QS_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        QS_CUDA(cudaStreamSynchronize(st));
    }
    return QS_OK;
}
