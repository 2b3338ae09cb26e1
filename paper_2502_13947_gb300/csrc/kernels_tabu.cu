// kernels_tabu.cu -- Tabu search (Algorithm 1, Section 2.4) on every replica.
//
// One CTA per replica.  Thread t owns the W groups of 4 consecutive
// variables j = 4 (t + w NT) + {0..3}; their gains g_j and tabu memory C_j
// live in registers for the whole search.  One iteration is:
//   1. every thread knows the chosen move (i, g_i, x_i) from the previous
//      block-wide arg-min;
//   2. it streams its 4W bytes of row i of Q (coalesced 4-byte loads; the row
//      index is only known after the arg-min, so there is nothing to
//      prefetch -- the rows stay hot in L2) and applies
//      g_j += 2 Q_ij (1 - 2 x_i)(1 - 2 x_j) for j != i, g_i = -g_i,
//      C_i += c, then C_j -= 1 where positive;
//   3. it takes the arg-min of g over its non-tabu variables, the warp takes
//      the arg-min with two redux.sync (gain, then index), and one
//      __syncthreads publishes the per-warp minima; every thread reduces
//      those itself, so the loop has exactly one barrier.
// Ties go to the lowest index, exactly as a scan in index order would.
// The objective OV is tracked in int64 by every thread (uniform).  The move
// log (uint16 per iteration) stays in shared memory; after the last
// iteration the moves made after the best visit are undone in one pass:
// variables moved an odd number of times flip back, and their rows of Q
// correct the gains (x_min is reconstructed without copying x on every
// improvement).
#include <climits>

#include "common.cuh"

namespace icd2s {

namespace {

__device__ __forceinline__ void warp_argmin(int g, unsigned jx, int& wg, unsigned& wjx)
{
    wg = __reduce_min_sync(0xffffffffu, g);
    wjx = __reduce_min_sync(0xffffffffu, g == wg ? jx : 0xffffffffu);
}

__device__ __forceinline__ unsigned long long pack_key(int g, unsigned jx)
{
    return ((unsigned long long)((unsigned)g ^ 0x80000000u) << 32) | jx;
}

}  // namespace

template <int W>
__global__ __launch_bounds__(1024) void k_tabu(Dev d, int alpha, int c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* wkeys = reinterpret_cast<unsigned long long*>(smem);         // [2][32]
    int* nF = reinterpret_cast<int*>(smem + 512);                                     // [1]
    int32_t* Ts = reinterpret_cast<int32_t*>(smem + 528);                             // [ld]
    uint32_t* undo = reinterpret_cast<uint32_t*>(smem + 528 + 4 * (size_t)d.ld);      // [ld / 32]
    uint16_t* mlog = reinterpret_cast<uint16_t*>(smem + 528 + 4 * (size_t)d.ld + d.ld / 8);  // [alpha]

    const int p = blockIdx.x;
    const int NT = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int n = d.n, ld = d.ld;
    const int8_t* __restrict__ Q = d.Q;
    uint8_t* xrow = d.X + (size_t)p * ld;
    int32_t* grow = d.G + (size_t)p * ld;

    for (int j = tid; j < ld; j += NT) Ts[j] = 0;
    for (int j = tid; j < ld / 32; j += NT) undo[j] = 0;
    if (tid == 0) *nF = 0;

    int g[W][4], C[W][4];
    unsigned xb = 0;  // bit 4w+b = x of the owned variable
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int j0 = 4 * (tid + w * NT);
        if (j0 < ld) {
            const int4 gv = *reinterpret_cast<const int4*>(grow + j0);
            const uint32_t xv = *reinterpret_cast<const uint32_t*>(xrow + j0);
            g[w][0] = gv.x; g[w][1] = gv.y; g[w][2] = gv.z; g[w][3] = gv.w;
#pragma unroll
            for (int b = 0; b < 4; ++b) xb |= ((xv >> (8 * b)) & 1u) << (4 * w + b);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) g[w][b] = 0;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) C[w][b] = 0;
    }

    // arg-min over the owned non-tabu variables, then the warp's, published to slot `slot`
    auto local_argmin = [&](int slot) {
        int bg = INT_MAX;
        unsigned bjx = 0xffffffffu;
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = 4 * (tid + w * NT) + b;
                if (j < n && C[w][b] <= 0 && g[w][b] < bg) {
                    bg = g[w][b];
                    bjx = ((unsigned)j << 1) | ((xb >> (4 * w + b)) & 1u);
                }
            }
        int wg; unsigned wjx;
        warp_argmin(bg, bjx, wg, wjx);
        if (lane == 0) wkeys[slot * 32 + warp] = pack_key(wg, wjx);
    };
    auto block_argmin = [&](int slot) -> unsigned long long {
        const unsigned long long k = lane < NW ? wkeys[slot * 32 + lane] : ~0ull;
        const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)(k >> 32));
        const unsigned lo = __reduce_min_sync(0xffffffffu, (unsigned)(k >> 32) == hi ? (unsigned)k : 0xffffffffu);
        return ((unsigned long long)hi << 32) | lo;
    };

    __syncthreads();  // shared-memory clears visible
    local_argmin(0);
    __syncthreads();
    unsigned long long key = block_argmin(0);

    long long OV = d.E[p], OVmin = OV;
    int best_it = -1;

    for (int it = 0; it < alpha; ++it) {
        const int gi = (int)((unsigned)(key >> 32) ^ 0x80000000u);
        const unsigned jx = (unsigned)key;
        const int i = (int)(jx >> 1);
        const int si = 1 - 2 * (int)(jx & 1u);
        const int8_t* row = Q + (size_t)i * ld;
        int q[W][4];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int j0 = 4 * (tid + w * NT);
            const int v = j0 < ld ? __ldg(reinterpret_cast<const int*>(row + j0)) : 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) q[w][b] = (int)(int8_t)(v >> (8 * b));
        }
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = 4 * (tid + w * NT) + b;
                const int sj = 1 - 2 * (int)((xb >> (4 * w + b)) & 1u);
                if (j == i) {
                    g[w][b] = -g[w][b];
                    xb ^= 1u << (4 * w + b);
                    C[w][b] += c;
                } else {
                    g[w][b] += 2 * q[w][b] * si * sj;
                }
                C[w][b] = C[w][b] > 0 ? C[w][b] - 1 : C[w][b];
            }
        OV += gi;
        if (OV < OVmin) { OVmin = OV; best_it = it; }
        if (tid == 0) { Ts[i] += 1; mlog[it] = (uint16_t)i; }
        const int slot = (it + 1) & 1;
        local_argmin(slot);
        __syncthreads();
        key = block_argmin(slot);
    }

    // toggle counts out; parity of the moves made after the best visit
    int32_t* Tout = d.T + (size_t)p * ld;
    for (int j = tid; j < ld; j += NT) Tout[j] = Ts[j];
    for (int e = best_it + 1 + tid; e < alpha; e += NT) {
        const int i = mlog[e];
        atomicXor(&undo[i >> 5], 1u << (i & 31));
    }
    __syncthreads();
    int32_t* flist = Ts;  // reuse: T has been written out
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = 4 * (tid + w * NT) + b;
            if (j < n && ((undo[j >> 5] >> (j & 31)) & 1u)) {
                const int slot = atomicAdd(nF, 1);
                flist[slot] = j | (int)(((xb >> (4 * w + b)) & 1u) << 31);
            }
        }
    __syncthreads();
    const int F = *nF;
    int acc[W][4];
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[w][b] = 0;
    for (int e = 0; e < F; ++e) {
        const int v = flist[e];
        const int i = v & 0x7fffffff;
        const int di = v < 0 ? -1 : 1;  // 1 - 2 x_i before the flip back
        const int8_t* row = Q + (size_t)i * ld;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int j0 = 4 * (tid + w * NT);
            const int rv = j0 < ld ? __ldg(reinterpret_cast<const int*>(row + j0)) : 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (j0 + b != i) acc[w][b] += di * (int)(int8_t)(rv >> (8 * b));
        }
    }
    int32_t* Cout = d.C + (size_t)p * ld;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int j0 = 4 * (tid + w * NT);
        if (j0 >= ld) continue;
        int gv[4], cv[4];
        uint32_t xv = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + b;
            int xj = (int)((xb >> (4 * w + b)) & 1u);
            int gj = 0;
            if (j < n) {
                const int dj = d.diag[j];
                const int h = ((1 - 2 * xj) * g[w][b] - dj) / 2 + acc[w][b];
                xj ^= (int)((undo[j >> 5] >> (j & 31)) & 1u);
                gj = (1 - 2 * xj) * (dj + 2 * h);
            } else {
                xj = 0;
            }
            gv[b] = gj;
            cv[b] = C[w][b];
            xv |= (uint32_t)xj << (8 * b);
        }
        *reinterpret_cast<int4*>(grow + j0) = make_int4(gv[0], gv[1], gv[2], gv[3]);
        *reinterpret_cast<int4*>(Cout + j0) = make_int4(cv[0], cv[1], cv[2], cv[3]);
        *reinterpret_cast<uint32_t*>(xrow + j0) = xv;
    }
    if (tid == 0) d.E[p] = OVmin;
}

size_t tabu_smem_bytes(int n, int alpha)
{
    const int ld = round_up(n, kLdAlign);
    return 528 + 4 * (size_t)ld + (size_t)ld / 8 + 2 * (size_t)alpha + 16;
}

template <int W>
static cudaError_t launch_tabu_w(const Dev& d, int alpha, int c, cudaStream_t s)
{
    int nt = (d.n + 4 * W - 1) / (4 * W);
    nt = (nt + 31) / 32 * 32;
    if (nt > 1024) return cudaErrorInvalidConfiguration;
    const size_t sm = tabu_smem_bytes(d.n, alpha);
    cudaError_t e = cudaFuncSetAttribute(k_tabu<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_tabu<W><<<d.R, nt, sm, s>>>(d, alpha, c);
    note_launch(1);
    return cudaGetLastError();
}

// w_words: 4-variable groups per thread (1..4); 0 picks the smallest that fits 1024 threads.
cudaError_t launch_tabu(const Dev& d, int alpha, int c, int w_words, cudaStream_t s)
{
    if (w_words <= 0) {
        w_words = 1;
        while (w_words < 4 && (d.n + 4 * w_words - 1) / (4 * w_words) > 1024) ++w_words;
    }
    switch (w_words) {
        case 1: return launch_tabu_w<1>(d, alpha, c, s);
        case 2: return launch_tabu_w<2>(d, alpha, c, s);
        case 3: return launch_tabu_w<3>(d, alpha, c, s);
        case 4: return launch_tabu_w<4>(d, alpha, c, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace icd2s
