// Learned cost model of the tile picker: a 12-64-64-64-2 ReLU MLP (FP32).
//
// The paper explores tile sizes exhaustively (Sec. 5.1.5); the engine also
// learns the autotuner's records so a tile shape can be picked without
// timing every candidate.  All arithmetic of training and inference runs in
// these kernels:
//   forward   y = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4
//   gradient  of L = (1/B) sum_b sum_o 0.5 (y_bo - t_bo)^2, per-CTA partial
//             sums reduced in a fixed order (deterministic)
//   Adam      m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
//             p -= lr (m / (1-b1^s)) / (sqrt(v / (1-b2^s)) + eps)
//   argmin    of one output column (the pick)
// Parameters are one flat array: W1 (64x12), b1, W2 (64x64), b2, W3, b3,
// W4 (2x64), b4; weights are (out, in) row-major.
#include "kernels.h"

namespace pcot {
namespace mlp {

constexpr int NIN = 12, NH = 64, NOUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NOUT * NH;
constexpr int NPARAM = OFF_B4 + NOUT;  // 9282
constexpr int SB = 32;                 // samples per CTA
constexpr int THREADS = 256;

namespace {

struct Smem {
    float p[NPARAM];
    float h0[SB][NIN];
    float h1[SB][NH];
    float h2[SB][NH];
    float h3[SB][NH];
    float y[SB][NOUT];
};

// out[s][j] = b[j] + sum_i W[j][i] in[s][i] (optionally relu), i ascending.
template <int IN, int OUT, bool RELU>
__device__ __forceinline__ void dense(const float* W, const float* b, const float (*in)[IN], float (*out)[OUT],
                                      int ns) {
    for (int k = threadIdx.x; k < ns * OUT; k += blockDim.x) {
        const int s = k / OUT, j = k - s * OUT;
        float acc = b[j];
        const float* w = W + j * IN;
#pragma unroll 4
        for (int i = 0; i < IN; ++i) acc = __fmaf_rn(w[i], in[s][i], acc);
        out[s][j] = RELU ? fmaxf(acc, 0.f) : acc;
    }
}

__device__ void load_and_forward(Smem& S, const float* __restrict__ P, const float* __restrict__ X, int s0, int ns) {
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) S.p[i] = P[i];
    for (int i = threadIdx.x; i < ns * NIN; i += blockDim.x) S.h0[i / NIN][i % NIN] = X[(size_t)s0 * NIN + i];
    __syncthreads();
    dense<NIN, NH, true>(S.p + OFF_W1, S.p + OFF_B1, S.h0, S.h1, ns);
    __syncthreads();
    dense<NH, NH, true>(S.p + OFF_W2, S.p + OFF_B2, S.h1, S.h2, ns);
    __syncthreads();
    dense<NH, NH, true>(S.p + OFF_W3, S.p + OFF_B3, S.h2, S.h3, ns);
    __syncthreads();
    dense<NH, NOUT, false>(S.p + OFF_W4, S.p + OFF_B4, S.h3, S.y, ns);
    __syncthreads();
}

__global__ void __launch_bounds__(THREADS) forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                          int B, float* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& S = *reinterpret_cast<Smem*>(raw);
    const int s0 = blockIdx.x * SB;
    const int ns = min(SB, B - s0);
    load_and_forward(S, P, X, s0, ns);
    for (int i = threadIdx.x; i < ns * NOUT; i += blockDim.x) Y[(size_t)s0 * NOUT + i] = S.y[i / NOUT][i % NOUT];
}

// Weight and bias gradients of one dense layer from this CTA's samples:
// gW[j][i] = sum_s d[s][j] in[s][i], gb[j] = sum_s d[s][j]  (s ascending).
template <int IN, int OUT>
__device__ __forceinline__ void layer_grad(const float (*d)[OUT], const float (*in)[IN], float* gW, float* gb,
                                           int ns) {
    for (int k = threadIdx.x; k < OUT * IN; k += blockDim.x) {
        const int j = k / IN, i = k - j * IN;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = __fmaf_rn(d[s][j], in[s][i], acc);
        gW[k] = acc;
    }
    for (int j = threadIdx.x; j < OUT; j += blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += d[s][j];
        gb[j] = acc;
    }
}

// din[s][i] = (sum_j d[s][j] W[j][i]) * (h[s][i] > 0)  (j ascending).
template <int IN, int OUT>
__device__ __forceinline__ void back_through(const float* W, const float (*d)[OUT], const float (*h)[IN],
                                             float (*din)[IN], int ns) {
    for (int k = threadIdx.x; k < ns * IN; k += blockDim.x) {
        const int s = k / IN, i = k - s * IN;
        float acc = 0.f;
        for (int j = 0; j < OUT; ++j) acc = __fmaf_rn(d[s][j], W[j * IN + i], acc);
        din[s][i] = h[s][i] > 0.f ? acc : 0.f;
    }
}

__global__ void __launch_bounds__(THREADS) grad_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                       const float* __restrict__ Tg, int B,
                                                       float* __restrict__ partial, float* __restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& S = *reinterpret_cast<Smem*>(raw);
    __shared__ float dy[SB][NOUT];
    __shared__ float red[THREADS];
    const int s0 = blockIdx.x * SB;
    const int ns = min(SB, B - s0);
    load_and_forward(S, P, X, s0, ns);
    float l = 0.f;
    for (int i = threadIdx.x; i < ns * NOUT; i += blockDim.x) {
        const int s = i / NOUT, o = i % NOUT;
        const float e = S.y[s][o] - Tg[(size_t)(s0 + s) * NOUT + o];
        dy[s][o] = e / (float)B;
        l += 0.5f * e * e;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
    float* g = partial + (size_t)blockIdx.x * NPARAM;
    // Layer 4, then back into h3 (reuse h-buffers for the deltas).
    layer_grad<NH, NOUT>(dy, S.h3, g + OFF_W4, g + OFF_B4, ns);
    __syncthreads();
    // dz3 = (dy W4) * (h3 > 0)
    __shared__ float dz[SB][NH];
    back_through<NH, NOUT>(S.p + OFF_W4, dy, S.h3, dz, ns);
    __syncthreads();
    layer_grad<NH, NH>(dz, S.h2, g + OFF_W3, g + OFF_B3, ns);
    __syncthreads();
    // dz2 = (dz3 W3) * (h2 > 0) -> into h3 (h3 no longer needed)
    back_through<NH, NH>(S.p + OFF_W3, dz, S.h2, S.h3, ns);
    __syncthreads();
    layer_grad<NH, NH>(S.h3, S.h1, g + OFF_W2, g + OFF_B2, ns);
    __syncthreads();
    // dz1 = (dz2 W2) * (h1 > 0) -> into dz
    back_through<NH, NH>(S.p + OFF_W2, S.h3, S.h1, dz, ns);
    __syncthreads();
    layer_grad<NIN, NH>(dz, S.h0, g + OFF_W1, g + OFF_B1, ns);
}

// grad[i] = sum over CTAs c (ascending) of partial[c][i]; loss likewise.
__global__ void reduce_kernel(const float* __restrict__ partial, int nct, float* __restrict__ grad,
                              const float* __restrict__ lpart, float* __restrict__ loss, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) {
        float acc = 0.f;
        for (int c = 0; c < nct; ++c) acc += partial[(size_t)c * NPARAM + i];
        grad[i] = acc;
    }
    if (i == 0 && loss) {
        float acc = 0.f;
        for (int c = 0; c < nct; ++c) acc += lpart[c];
        *loss = acc / (float)B;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void argmin_kernel(const float* __restrict__ y, int n, int stride, int col, int* __restrict__ out) {
    __shared__ float bv[256];
    __shared__ int bi[256];
    float best = 3.4e38f;
    int idx = -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float v = y[(size_t)i * stride + col];
        if (v < best || (v == best && i < idx)) {
            best = v;
            idx = i;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const float o = bv[threadIdx.x + w];
            const int oi = bi[threadIdx.x + w];
            if (oi >= 0 && (o < bv[threadIdx.x] || (o == bv[threadIdx.x] && (bi[threadIdx.x] < 0 || oi < bi[threadIdx.x])))) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = bi[0];
}

}  // namespace

int param_count() { return NPARAM; }

size_t scratch_bytes(int B) {
    const int nct = (B + SB - 1) / SB;
    return (size_t)nct * NPARAM * sizeof(float) + (size_t)nct * sizeof(float) + 256;
}

cudaError_t forward(const float* P, const float* X, int B, float* Y, cudaStream_t s) {
    const int nct = (B + SB - 1) / SB;
    const size_t sm = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    forward_kernel<<<nct, THREADS, sm, s>>>(P, X, B, Y);
    return cudaGetLastError();
}

cudaError_t grad(const float* P, const float* X, const float* Tg, int B, float* G, float* loss, void* scratch,
                 cudaStream_t s) {
    const int nct = (B + SB - 1) / SB;
    float* partial = (float*)scratch;
    float* lpart = partial + (size_t)nct * NPARAM;
    const size_t sm = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    grad_kernel<<<nct, THREADS, sm, s>>>(P, X, Tg, B, partial, lpart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(partial, nct, G, lpart, loss, B);
    return cudaGetLastError();
}

cudaError_t adam(float* P, const float* G, float* M, float* V, int n, int step, float lr, float b1, float b2,
                 float eps, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, G, M, V, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t argmin(const float* Y, int n, int stride, int col, int* out, cudaStream_t s) {
    argmin_kernel<<<1, 256, 0, s>>>(Y, n, stride, col, out);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace pcot
