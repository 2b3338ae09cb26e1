// kernels_mlp.cu -- the proposal network of the learned subQUBO selection
// (an addition to IC-D2S's Algorithm 4 subset choice): per-variable features,
// the 6-64-64-1 score network (BF16 weights, FP32 arithmetic), its training by
// backpropagation of a weighted binary cross-entropy with a deterministic
// gradient reduction, Adam, and the improvement log that supplies the labels.
//
//  k_gmax       one CTA per replica: max_j |g_j|.
//  k_features   one thread per (replica, variable): the six features
//               f = (x, g/(max|g|+1), T/alpha, C/c, H/(t+1), eta_hat/2^16).
//  k_score      one thread per row: the network in float with one fused
//               multiply-add per product in a fixed order (units and inputs
//               ascending), so the selection decision is reproducible.
//  k_mlp_grad   128 rows per CTA: forward into shared memory, then the
//               gradient of the mean loss summed over the CTA's rows in row
//               order; one partial gradient per CTA.
//  k_mlp_reduce sums the partial gradients in CTA order (deterministic) and
//               applies Adam to the float32 master weights, re-rounding the
//               BF16 copy.
//  k_log        appends an improvement-log entry (features of the replica
//               that produced the new best, label = best_x XOR previous best).
//
// Why CUDA cores and not the tensor cores: the network is 8 960 FLOPs per
// row; at 32 replicas x 10 000 variables a score pass is ~3 GFLOP (tens of
// microseconds on the FP32 pipes), and rounding the activations to BF16/TF32
// for tcgen05 would move the scores by ~1e-3 relative -- the tolerance the
// scores are held to -- and would change the ranking the selection takes.
#include <cuda_bf16.h>

#include "common.cuh"

namespace icd2s {

namespace {

constexpr int kRowsPerCta = 128;
constexpr int kHS = 65;  // padded row stride of the activation tiles (bank-conflict free)
constexpr int kFS = 7;   // padded row stride of the feature tile

__device__ __forceinline__ float softplus(float v) { return fmaxf(v, 0.f) + log1pf(expf(-fabsf(v))); }
__device__ __forceinline__ float sigmoid(float v) { return 1.f / (1.f + expf(-v)); }

__device__ __forceinline__ void load_weights(const __nv_bfloat16* __restrict__ Wb, float* w)
{
    for (int q = threadIdx.x; q < kNPar; q += blockDim.x) w[q] = __bfloat162float(Wb[q]);
}

// Float score of one row (see the header comment): W in shared memory.
__device__ __forceinline__ float score_row(const float* __restrict__ w, const float f[6])
{
    float h1[64];
#pragma unroll
    for (int o = 0; o < 64; ++o) {
        float a = w[kOffB1 + o];
#pragma unroll
        for (int k = 0; k < 6; ++k) a = __fmaf_rn(w[kOffW1 + o * 6 + k], f[k], a);
        h1[o] = a > 0.f ? a : 0.f;
    }
    float s = w[kOffB3];
#pragma unroll 1
    for (int o = 0; o < 64; ++o) {
        const float* w2 = w + kOffW2 + o * 64;
        float a = w[kOffB2 + o];
#pragma unroll
        for (int k = 0; k < 64; ++k) a = __fmaf_rn(w2[k], h1[k], a);
        const float h2 = a > 0.f ? a : 0.f;
        s = __fmaf_rn(w[kOffW3 + o], h2, s);
    }
    return s;
}

__device__ __forceinline__ int block_max_int(int v, int* red)
{
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0;
        w = __reduce_max_sync(0xffffffffu, w);
        if (threadIdx.x == 0) red[32] = w;
    }
    __syncthreads();
    return red[32];
}

}  // namespace

// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_gmax(const int32_t* __restrict__ G, int n, int ld, int32_t* gmax)
{
    __shared__ int red[33];
    const int p = blockIdx.x;
    int m = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) m = max(m, abs(G[(size_t)p * ld + j]));
    m = block_max_int(m, red);
    if (threadIdx.x == 0) gmax[p] = m;
}

__global__ __launch_bounds__(256) void k_features(Dev d, int t_arg, const int32_t* iter_dev, int alpha, int c,
                                                  const int32_t* __restrict__ gmax)
{
    const int p = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.ld) return;
    const int t = iter_dev ? *iter_dev : t_arg;
    const size_t e = (size_t)p * d.ld + j;
    float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (j < d.n) {
        f[0] = (float)d.X[e];
        f[1] = __fdiv_rn((float)d.G[e], (float)(gmax[p] + 1));
        f[2] = alpha > 0 ? __fdiv_rn((float)d.T[e], (float)alpha) : 0.f;
        f[3] = __fdiv_rn((float)d.C[e], (float)c);
        f[4] = __fdiv_rn((float)d.H[e], (float)(t + 1));
        f[5] = __fdiv_rn((float)d.etahat[j], 65536.f);
    }
    float2* out = reinterpret_cast<float2*>(d.F + e * 6);
    out[0] = make_float2(f[0], f[1]);
    out[1] = make_float2(f[2], f[3]);
    out[2] = make_float2(f[4], f[5]);
}

__global__ __launch_bounds__(256) void k_score(const float* __restrict__ F, long long rows,
                                               const __nv_bfloat16* __restrict__ Wb, float* __restrict__ out)
{
    __shared__ __align__(16) float w[kNParPad];
    load_weights(Wb, w);
    __syncthreads();
    // one row per thread: with a row loop the compiler keeps the loop-invariant
    // shared weights in registers and spills
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float2* fr = reinterpret_cast<const float2*>(F + r * 6);
    const float2 a = fr[0], b = fr[1], c = fr[2];
    const float f[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
    out[r] = score_row(w, f);
}

// ---------------------------------------------------------------------------
// Row r of the step's batch: all rows in order when the batch covers them,
// otherwise a Philox draw (counter (r, TAG_TRAIN << 24, step, 0)) modulo rows.
__device__ __forceinline__ long long batch_row(long long r, long long rows, long long batch, uint32_t step, uint32_t k0,
                                               uint32_t k1)
{
    if (batch >= rows) return r;
    const u32x4 v = philox10((uint32_t)r, kTagTrain << 24, step, 0u, k0, k1);
    const unsigned long long u = ((unsigned long long)v.v[1] << 32) | v.v[0];
    return (long long)(u % (unsigned long long)rows);
}

__global__ __launch_bounds__(kRowsPerCta) void k_mlp_grad(const float* __restrict__ F, const uint8_t* __restrict__ y,
                                                          long long rows, long long batch, uint32_t step, uint32_t k0,
                                                          uint32_t k1, const __nv_bfloat16* __restrict__ Wb,
                                                          float pos_weight, float* __restrict__ partial)
{
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                                  // [kNParPad]
    float* H1 = w + kNParPad;                       // [128][kHS]: h1, later dL/da1
    float* H2 = H1 + kRowsPerCta * kHS;             // [128][kHS]: h2, later dL/da2
    float* Fs = H2 + kRowsPerCta * kHS;             // [128][kFS]
    float* DS = Fs + kRowsPerCta * kFS;             // [128] dL/ds
    float* LS = DS + kRowsPerCta;                   // [128] loss terms
    const int tid = threadIdx.x;
    const long long nb = batch < rows ? batch : rows;
    const long long r0 = (long long)blockIdx.x * kRowsPerCta;
    load_weights(Wb, w);
    __syncthreads();

    // forward, one row per thread
    {
        const long long r = r0 + tid;
        const bool valid = r < nb;
        float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float yv = 0.f;
        if (valid) {
            const long long row = batch_row(r, rows, batch, step, k0, k1);
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = F[row * 6 + k];
            yv = y[row] ? 1.f : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) Fs[tid * kFS + k] = f[k];
        float h1[64];
#pragma unroll
        for (int o = 0; o < 64; ++o) {
            float a = w[kOffB1 + o];
#pragma unroll
            for (int k = 0; k < 6; ++k) a = __fmaf_rn(w[kOffW1 + o * 6 + k], f[k], a);
            h1[o] = a > 0.f ? a : 0.f;
            H1[tid * kHS + o] = h1[o];
        }
        float s = w[kOffB3];
#pragma unroll 1
        for (int o = 0; o < 64; ++o) {
            float a = w[kOffB2 + o];
#pragma unroll
            for (int k = 0; k < 64; ++k) a = __fmaf_rn(w[kOffW2 + o * 64 + k], h1[k], a);
            const float h2 = a > 0.f ? a : 0.f;
            H2[tid * kHS + o] = h2;
            s = __fmaf_rn(w[kOffW3 + o], h2, s);
        }
        const float sg = sigmoid(s);
        DS[tid] = valid ? (pos_weight * yv * (sg - 1.f) + (1.f - yv) * sg) / (float)nb : 0.f;
        LS[tid] = valid ? pos_weight * yv * softplus(-s) + (1.f - yv) * softplus(s) : 0.f;
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * kPartStride;
    // w3 and b3
    if (tid < 64) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerCta; ++r) g = __fmaf_rn(DS[r], H2[r * kHS + tid], g);
        out[kOffW3 + tid] = g;
    } else if (tid == 64) {
        float g = 0.f, l = 0.f;
        for (int r = 0; r < kRowsPerCta; ++r) { g += DS[r]; l += LS[r]; }
        out[kOffB3] = g;
        out[kNPar] = l / (float)nb;
    }
    __syncthreads();
    // dL/da2 in place of h2 (own row)
    {
        const float ds = DS[tid];
#pragma unroll 8
        for (int o = 0; o < 64; ++o) {
            const float h2 = H2[tid * kHS + o];
            H2[tid * kHS + o] = h2 > 0.f ? ds * w[kOffW3 + o] : 0.f;
        }
    }
    __syncthreads();
    // W2 (4096) and b2 (64): output q = o * 64 + k, rows in order
    for (int q = tid; q < 64 * 64 + 64; q += kRowsPerCta) {
        float g = 0.f;
        if (q < 4096) {
            const int o = q >> 6, k = q & 63;
            for (int r = 0; r < kRowsPerCta; ++r) g = __fmaf_rn(H2[r * kHS + o], H1[r * kHS + k], g);
            out[kOffW2 + q] = g;
        } else {
            const int o = q - 4096;
            for (int r = 0; r < kRowsPerCta; ++r) g += H2[r * kHS + o];
            out[kOffB2 + o] = g;
        }
    }
    __syncthreads();
    // dL/da1 in place of h1 (own row): (sum_o dL/da2_o W2_ok) [a1_k > 0]
    {
        float d2[64];
#pragma unroll
        for (int o = 0; o < 64; ++o) d2[o] = H2[tid * kHS + o];
#pragma unroll 1
        for (int k = 0; k < 64; ++k) {
            float a = 0.f;
#pragma unroll
            for (int o = 0; o < 64; ++o) a = __fmaf_rn(d2[o], w[kOffW2 + o * 64 + k], a);
            const float h1 = H1[tid * kHS + k];
            H1[tid * kHS + k] = h1 > 0.f ? a : 0.f;
        }
    }
    __syncthreads();
    // W1 (384) and b1 (64)
    for (int q = tid; q < 64 * 6 + 64; q += kRowsPerCta) {
        float g = 0.f;
        if (q < 384) {
            const int o = q / 6, k = q % 6;
            for (int r = 0; r < kRowsPerCta; ++r) g = __fmaf_rn(H1[r * kHS + o], Fs[r * kFS + k], g);
            out[kOffW1 + q] = g;
        } else {
            const int o = q - 384;
            for (int r = 0; r < kRowsPerCta; ++r) g += H1[r * kHS + o];
            out[kOffB1 + o] = g;
        }
    }
}

// ---------------------------------------------------------------------------
// The same partial gradient with its three 64-wide contractions on the tensor
// cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation): the layer-2
// forward A2 = H1 W2^T, the weight gradient dW2 = dA2^T H1 and the backward
// dA1 = dA2 W2, per CTA of 128 rows (warp w: rows 32 w .. 32 w + 31, or
// output rows 16 w .. of dW2).  The activations h1 and dA2 are rounded to
// BF16 for the products (the weights already are BF16); layer 1, the losses
// and the column sums (b1, b2, w3, b3, W1) stay in FP32 on the CUDA cores,
// summed over the rows in order.  Deterministic: the summation order of every
// output is fixed.
// ---------------------------------------------------------------------------
namespace {

constexpr int kTS = 72;    // row stride (bf16) of the 64-wide operand tiles
constexpr int kTT = 136;   // row stride (bf16) of the transposed 128-wide tiles

// D += A B: A 16 x 16 (row-major), B 16 x 8 (column-major), BF16 -> FP32
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// acc[mt][nt] += A[r0 + 16 mt ..][k] B[k][16 nt ..] over k < K: A row-major with
// stride lda, B stored by columns (column n contiguous in k) with stride ldb
template <int MT, int K>
__device__ __forceinline__ void warp_gemm_n64(float (&acc)[MT][8][4], const __nv_bfloat16* A, int lda, int r0,
                                              const __nv_bfloat16* Bc, int ldb)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const __nv_bfloat16* ar = A + (size_t)(r0 + 16 * mt + g) * lda + k0 + 2 * t;
            a[mt][0] = ld_pair(ar);
            a[mt][1] = ld_pair(ar + 8 * lda);
            a[mt][2] = ld_pair(ar + 8);
            a[mt][3] = ld_pair(ar + 8 * lda + 8);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* br = Bc + (size_t)(8 * nt + g) * ldb + k0 + 2 * t;
            const uint32_t b0 = ld_pair(br), b1 = ld_pair(br + 8);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) mma_bf16_16816(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
        }
    }
}

}  // namespace

__global__ __launch_bounds__(kRowsPerCta) void k_mlp_grad_tc(const float* __restrict__ F,
                                                             const uint8_t* __restrict__ y, long long rows,
                                                             long long batch, uint32_t step, uint32_t k0, uint32_t k1,
                                                             const __nv_bfloat16* __restrict__ Wb, float pos_weight,
                                                             float* __restrict__ partial)
{
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                                          // [kNParPad] FP32 copy of the BF16 weights
    float* Fs = w + kNParPad;                               // [128][kFS]
    float* DS = Fs + kRowsPerCta * kFS;                     // [128] dL/ds
    float* LS = DS + kRowsPerCta;                           // [128] loss terms
    float* X2 = LS + kRowsPerCta;                           // [128][kHS] h2, later dL/da1 (FP32)
    __nv_bfloat16* H1b = reinterpret_cast<__nv_bfloat16*>(X2 + kRowsPerCta * kHS);  // [128][kTS] h1
    __nv_bfloat16* H1t = H1b + kRowsPerCta * kTS;           // [64][kTT] h1^T
    __nv_bfloat16* W2b = H1t + 64 * kTT;                    // [64][kTS] W2 (row o: weights into unit o)
    __nv_bfloat16* W2t = W2b + 64 * kTS;                    // [64][kTS] W2^T
    __nv_bfloat16* D2b = W2t + 64 * kTS;                    // [128][kTS] dL/da2
    __nv_bfloat16* D2t = D2b + kRowsPerCta * kTS;           // [64][kTT] dL/da2^T
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const long long nb = batch < rows ? batch : rows;
    const long long r0 = (long long)blockIdx.x * kRowsPerCta;
    load_weights(Wb, w);
    for (int q = tid; q < 64 * 64; q += kRowsPerCta) {
        const int o = q >> 6, k = q & 63;
        W2b[o * kTS + k] = Wb[kOffW2 + q];
        W2t[k * kTS + o] = Wb[kOffW2 + q];
    }
    __syncthreads();

    // layer 1 (FP32), one row per thread
    float yv = 0.f;
    const bool valid = r0 + tid < nb;
    {
        float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const long long row = batch_row(r0 + tid, rows, batch, step, k0, k1);
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = F[row * 6 + k];
            yv = y[row] ? 1.f : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) Fs[tid * kFS + k] = f[k];
#pragma unroll 8
        for (int o = 0; o < 64; ++o) {
            float a = w[kOffB1 + o];
#pragma unroll
            for (int k = 0; k < 6; ++k) a = __fmaf_rn(w[kOffW1 + o * 6 + k], f[k], a);
            const __nv_bfloat16 h = __float2bfloat16_rn(a > 0.f ? a : 0.f);
            H1b[tid * kTS + o] = h;
            H1t[o * kTT + tid] = h;
        }
    }
    __syncthreads();

    // layer 2 forward on the tensor cores: rows 32 warp .. + 31, all 64 units
    {
        float acc[2][8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
        warp_gemm_n64<2, 64>(acc, H1b, kTS, 32 * warp, W2b, kTS);
        // h2 = relu(a2 + b2) into X2; the row's score s = b3 + sum_o w3_o h2_o
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {           // rows g and g + 8 of the tile
                const int r = 32 * warp + 16 * mt + g + 8 * hf;
                float part = 0.f;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int o = 8 * nt + 2 * t + e;
                        const float a = acc[mt][nt][2 * hf + e] + w[kOffB2 + o];
                        const float h2 = a > 0.f ? a : 0.f;
                        X2[r * kHS + o] = h2;
                        part = __fmaf_rn(w[kOffW3 + o], h2, part);
                    }
                // the row's 64 products: 4 threads x 16, added in a fixed tree
                part += __shfl_xor_sync(0xffffffffu, part, 1);
                part += __shfl_xor_sync(0xffffffffu, part, 2);
                if (t == 0) DS[r] = part;   // the score without b3, for the owner thread below
            }
    }
    __syncthreads();
    {
        const float s = w[kOffB3] + DS[tid];
        const float sg = sigmoid(s);
        DS[tid] = valid ? (pos_weight * yv * (sg - 1.f) + (1.f - yv) * sg) / (float)nb : 0.f;
        LS[tid] = valid ? pos_weight * yv * softplus(-s) + (1.f - yv) * softplus(s) : 0.f;
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * kPartStride;
    // w3, b2, b3 (FP32, rows in order); dL/da2 = ds w3 [h2 > 0] as BF16 tiles
    if (tid < 64) {
        float gsum = 0.f, bsum = 0.f;
        const float w3 = w[kOffW3 + tid];
        for (int r = 0; r < kRowsPerCta; ++r) {
            const float h2 = X2[r * kHS + tid];
            gsum = __fmaf_rn(DS[r], h2, gsum);
            bsum += h2 > 0.f ? DS[r] * w3 : 0.f;
        }
        out[kOffW3 + tid] = gsum;
        out[kOffB2 + tid] = bsum;
    } else if (tid == 64) {
        float gsum = 0.f, l = 0.f;
        for (int r = 0; r < kRowsPerCta; ++r) { gsum += DS[r]; l += LS[r]; }
        out[kOffB3] = gsum;
        out[kNPar] = l / (float)nb;
    }
    {
        const float ds = DS[tid];
#pragma unroll 8
        for (int o = 0; o < 64; ++o) {
            const float d2 = X2[tid * kHS + o] > 0.f ? ds * w[kOffW3 + o] : 0.f;
            const __nv_bfloat16 b = __float2bfloat16_rn(d2);
            D2b[tid * kTS + o] = b;
            D2t[o * kTT + tid] = b;
        }
    }
    __syncthreads();
    // dW2 = dA2^T H1 on the tensor cores: output rows 16 warp .. + 15
    {
        float acc[1][8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[0][nt][e] = 0.f;
        warp_gemm_n64<1, kRowsPerCta>(acc, D2t, kTT, 16 * warp, H1t, kTT);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int o0 = 16 * warp + g, k = 8 * nt + 2 * t;
            out[kOffW2 + o0 * 64 + k] = acc[0][nt][0];
            out[kOffW2 + o0 * 64 + k + 1] = acc[0][nt][1];
            out[kOffW2 + (o0 + 8) * 64 + k] = acc[0][nt][2];
            out[kOffW2 + (o0 + 8) * 64 + k + 1] = acc[0][nt][3];
        }
    }
    // dA1 = dA2 W2 on the tensor cores, masked by h1 > 0, into X2 (FP32)
    {
        float acc[2][8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
        warp_gemm_n64<2, 64>(acc, D2b, kTS, 32 * warp, W2t, kTS);
        __syncthreads();   // every thread has read X2 (the h2 values) above
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = 32 * warp + 16 * mt + g + 8 * (e >> 1), k = 8 * nt + 2 * t + (e & 1);
                    X2[r * kHS + k] = __bfloat162float(H1b[r * kTS + k]) > 0.f ? acc[mt][nt][e] : 0.f;
                }
    }
    __syncthreads();
    // W1 (384) and b1 (64), FP32, rows in order
    for (int q = tid; q < 64 * 6 + 64; q += kRowsPerCta) {
        float gsum = 0.f;
        if (q < 384) {
            const int o = q / 6, k = q % 6;
            for (int r = 0; r < kRowsPerCta; ++r) gsum = __fmaf_rn(X2[r * kHS + o], Fs[r * kFS + k], gsum);
            out[kOffW1 + q] = gsum;
        } else {
            const int o = q - 384;
            for (int r = 0; r < kRowsPerCta; ++r) gsum += X2[r * kHS + o];
            out[kOffB1 + o] = gsum;
        }
    }
}

// Sums the partial gradients (and losses) of `blocks` CTAs in CTA order; then
// optionally Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr (m / bc1) / (sqrt(v / bc2) + eps), with bc1/bc2 the bias corrections.
__global__ __launch_bounds__(256) void k_mlp_reduce(const float* __restrict__ partial, int blocks, float* grad_out,
                                                    float* loss_out, float* master, float* mom, float* vel,
                                                    __nv_bfloat16* Wb, int adam, float lr, float b1, float b2,
                                                    float eps, float bc1, float bc2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > kNPar) return;
    float g = 0.f;
    for (int b = 0; b < blocks; ++b) g += partial[(size_t)b * kPartStride + q];
    if (q == kNPar) {
        if (loss_out) *loss_out = g;
        return;
    }
    if (grad_out) grad_out[q] = g;
    if (!adam) return;
    const float m = b1 * mom[q] + (1.f - b1) * g;
    const float v = b2 * vel[q] + (1.f - b2) * g * g;
    mom[q] = m;
    vel[q] = v;
    const float wq = master[q] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    master[q] = wq;
    Wb[q] = __float2bfloat16_rn(wq);
}

__global__ void k_round_bf16(const float* __restrict__ master, __nv_bfloat16* Wb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kNPar) Wb[q] = __float2bfloat16_rn(master[q]);
}

// ---------------------------------------------------------------------------
// flags[4] = improved during the iteration just finished, flags[3] = replica
// whose row was last copied into best_x, flags[5] = log slot of this entry.
__global__ __launch_bounds__(256) void k_log(const float* __restrict__ F, int n, int ld, const uint8_t* __restrict__ best_x,
                                             uint8_t* prev_x, const int32_t* __restrict__ flags, float* LF,
                                             uint8_t* LY, int32_t* lrep)
{
    if (!flags[4]) return;
    const int p = flags[3], slot = flags[5];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) lrep[slot] = p;
    if (j >= n) return;
    const float* src = F + ((size_t)p * ld + j) * 6;
    float* dst = LF + ((size_t)slot * n + j) * 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = src[k];
    const uint8_t b = best_x[j];
    LY[(size_t)slot * n + j] = b ^ prev_x[j];
    prev_x[j] = b;
}

// ---------------------------------------------------------------------------
cudaError_t launch_features(const Dev& d, int t, const int32_t* iter_dev, int alpha, int c, int32_t* gmax,
                            cudaStream_t s)
{
    k_gmax<<<d.R, 256, 0, s>>>(d.G, d.n, d.ld, gmax);
    dim3 grid((d.ld + 255) / 256, d.R);
    k_features<<<grid, 256, 0, s>>>(d, t, iter_dev, alpha, c, gmax);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_score(const float* F, long long rows, const void* Wb, float* out, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    const long long grid = (rows + 255) / 256;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_score<<<(unsigned)grid, 256, 0, s>>>(F, rows, reinterpret_cast<const __nv_bfloat16*>(Wb), out);
    note_launch(1);
    return cudaGetLastError();
}

size_t mlp_partial_floats(long long batch) { return (size_t)((batch + kRowsPerCta - 1) / kRowsPerCta) * kPartStride; }

cudaError_t launch_mlp_grad(const float* F, const uint8_t* y, long long rows, long long batch, uint32_t step,
                            uint32_t k0, uint32_t k1, const void* Wb, float pos_weight, float* partial,
                            float* grad_out, float* loss_out, float* master, float* mom, float* vel, void* Wb_out,
                            int adam, float lr, float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s,
                            bool tensor_cores)
{
    const long long nb = batch < rows ? batch : rows;
    const int blocks = (int)((nb + kRowsPerCta - 1) / kRowsPerCta);
    if (tensor_cores) {
        const size_t smem = sizeof(float) * ((size_t)kNParPad + kRowsPerCta * kFS + 2 * kRowsPerCta +
                                             kRowsPerCta * kHS) +
                            sizeof(__nv_bfloat16) * (2 * (size_t)kRowsPerCta * kTS + 2 * 64 * kTT + 2 * 64 * kTS);
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mlp_grad_tc<<<blocks, kRowsPerCta, smem, s>>>(F, y, rows, batch, step, k0, k1,
                                                        reinterpret_cast<const __nv_bfloat16*>(Wb), pos_weight,
                                                        partial);
    } else {
        const size_t smem =
            sizeof(float) * ((size_t)kNParPad + 2 * kRowsPerCta * kHS + kRowsPerCta * kFS + 2 * kRowsPerCta);
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mlp_grad<<<blocks, kRowsPerCta, smem, s>>>(F, y, rows, batch, step, k0, k1,
                                                     reinterpret_cast<const __nv_bfloat16*>(Wb), pos_weight, partial);
    }
    k_mlp_reduce<<<(kNPar + 1 + 255) / 256, 256, 0, s>>>(partial, blocks, grad_out, loss_out, master, mom, vel,
                                                        reinterpret_cast<__nv_bfloat16*>(Wb_out), adam, lr, b1, b2,
                                                        eps, bc1, bc2);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_round_bf16(const float* master, void* Wb, cudaStream_t s)
{
    k_round_bf16<<<(kNPar + 255) / 256, 256, 0, s>>>(master, reinterpret_cast<__nv_bfloat16*>(Wb));
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_log(const Dev& d, uint8_t* prev_x, float* LF, uint8_t* LY, int32_t* lrep, cudaStream_t s)
{
    k_log<<<(d.n + 255) / 256, 256, 0, s>>>(d.F, d.n, d.ld, d.best_x, prev_x, d.flags, LF, LY, lrep);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
