// kernels_update.cu -- write-back of accepted flips into the solutions,
// their exact int32 gains and int64 energies.
//
// For a set F of variables flipped together (old values x_i, d_i = 1 - 2 x_i):
//   h_j  <- h_j + sum_{i in F, i != j} Q_ij d_i         (off-diagonal field)
//   x_j  <- x_j xor [j in F]
//   g_j  <- (1 - 2 x_j)(Q_jj + 2 h_j)
//   E    <- E + (1/2) sum_{i in F} (g_i(old) - g_i(new))
// The last identity follows from applying the flips one after the other:
// the energy change is sum_{i in F} g_i + 2 sum_{pairs {i,i'} in F} Q_ii' d_i d_i',
// and g_i(new) = -g_i(old) - 2 sum_{i' in F, i' != i} Q_ii' d_i d_i'.
// h is recovered from the tracked gain as h_j = ((1 - 2 x_j) g_j - Q_jj) / 2.
//
// k_apply: grid (ld / 1024, R), 256 threads, each thread owns 4 consecutive
// columns j of one replica.  The replica's flip list is staged in shared
// memory in chunks; for every listed row i the thread streams the 4 bytes
// Q[i][j..j+3] (coalesced 1 KiB per CTA per row -- Q is symmetric, so the
// row is the column).  Per-CTA energy terms go to an int64 accumulator; the
// last CTA of the replica (ticket counter) folds it into E and resets the
// list, the accumulator and the counter, so the next producer starts clean.
#include "common.cuh"

namespace icd2s {

constexpr int kApplyThreads = 256;
constexpr int kApplyTile = 4 * kApplyThreads;  // columns per CTA
constexpr int kApplyChunk = 2048;              // list entries staged per pass

__global__ __launch_bounds__(kApplyThreads) void k_apply(Dev d)
{
    __shared__ int32_t sl[kApplyChunk];
    __shared__ uint32_t tileflip[kApplyTile / 32];
    __shared__ long long red[kApplyThreads / 32];
    const int p = blockIdx.y, tid = threadIdx.x;
    const int ld = d.ld, n = d.n;
    const int cnt = min(d.FCNT[p], ld);  // a list never exceeds n entries
    if (cnt == 0) return;  // nothing to apply for this replica (counters are already clear)
    const int tile0 = blockIdx.x * kApplyTile;
    const int j0 = tile0 + 4 * tid;
    const int32_t* fl = d.FL + (size_t)p * ld;
    if (tid < kApplyTile / 32) tileflip[tid] = 0;
    int acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    for (int c0 = 0; c0 < cnt; c0 += kApplyChunk) {
        const int cn = min(kApplyChunk, cnt - c0);
        __syncthreads();
        for (int e = tid; e < cn; e += kApplyThreads) {
            const int v = fl[c0 + e];
            sl[e] = v;
            const int i = v & 0x7fffffff;
            if (i >= tile0 && i < tile0 + kApplyTile)
                atomicOr(&tileflip[(i - tile0) >> 5], 1u << ((i - tile0) & 31));
        }
        __syncthreads();
        if (j0 < ld) {
            int e = 0;
            for (; e + 4 <= cn; e += 4) {
                int rv[4], di[4], ii[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int v = sl[e + u];
                    ii[u] = v & 0x7fffffff;
                    di[u] = v < 0 ? -1 : 1;
                    rv[u] = __ldg(reinterpret_cast<const int*>(d.Q + (size_t)ii[u] * ld + j0));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = rv[u], dd = di[u], i = ii[u];
                    acc0 += (j0 + 0 != i) ? dd * (int)(int8_t)(r) : 0;
                    acc1 += (j0 + 1 != i) ? dd * (int)(int8_t)(r >> 8) : 0;
                    acc2 += (j0 + 2 != i) ? dd * (int)(int8_t)(r >> 16) : 0;
                    acc3 += (j0 + 3 != i) ? dd * (int)(int8_t)(r >> 24) : 0;
                }
            }
            for (; e < cn; ++e) {
                const int v = sl[e];
                const int i = v & 0x7fffffff, dd = v < 0 ? -1 : 1;
                const int r = __ldg(reinterpret_cast<const int*>(d.Q + (size_t)i * ld + j0));
                acc0 += (j0 + 0 != i) ? dd * (int)(int8_t)(r) : 0;
                acc1 += (j0 + 1 != i) ? dd * (int)(int8_t)(r >> 8) : 0;
                acc2 += (j0 + 2 != i) ? dd * (int)(int8_t)(r >> 16) : 0;
                acc3 += (j0 + 3 != i) ? dd * (int)(int8_t)(r >> 24) : 0;
            }
        }
    }
    long long dpart = 0;
    if (j0 < ld) {
        uint8_t* xrow = d.X + (size_t)p * ld;
        int32_t* grow = d.G + (size_t)p * ld;
        const int4 gv = *reinterpret_cast<const int4*>(grow + j0);
        const uint32_t xv = *reinterpret_cast<const uint32_t*>(xrow + j0);
        const int gin[4] = {gv.x, gv.y, gv.z, gv.w};
        const int acc[4] = {acc0, acc1, acc2, acc3};
        int gout[4];
        uint32_t xo = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + b;
            int xj = (int)((xv >> (8 * b)) & 1u);
            if (j < n) {
                const int dj = d.diag[j];
                const int h = ((1 - 2 * xj) * gin[b] - dj) / 2 + acc[b];
                const int fl_j = (int)((tileflip[(j - tile0) >> 5] >> ((j - tile0) & 31)) & 1u);
                xj ^= fl_j;
                gout[b] = (1 - 2 * xj) * (dj + 2 * h);
                if (fl_j) dpart += (long long)gin[b] - gout[b];
            } else {
                gout[b] = 0;
                xj = 0;
            }
            xo |= (uint32_t)xj << (8 * b);
        }
        *reinterpret_cast<int4*>(grow + j0) = make_int4(gout[0], gout[1], gout[2], gout[3]);
        *reinterpret_cast<uint32_t*>(xrow + j0) = xo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dpart += __shfl_xor_sync(0xffffffffu, dpart, o);
    if ((tid & 31) == 0) red[tid >> 5] = dpart;
    __syncthreads();
    if (tid == 0) {
        long long tot = 0;
        for (int w = 0; w < kApplyThreads / 32; ++w) tot += red[w];
        if (tot != 0) atomicAdd(&d.DEACC[p], (unsigned long long)tot);
        __threadfence();
        const unsigned ticket = atomicAdd(&d.DONE[p], 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            const long long sum = (long long)atomicExch(&d.DEACC[p], 0ull);
            d.E[p] += sum / 2;
            d.DONE[p] = 0;
            d.FCNT[p] = 0;
        }
    }
}

cudaError_t launch_apply(const Dev& d, cudaStream_t s)
{
    dim3 grid((d.ld + kApplyTile - 1) / kApplyTile, d.R);
    k_apply<<<grid, kApplyThreads, 0, s>>>(d);
    note_launch(1);
    return cudaGetLastError();
}

// mask [R][ldm] (0/1) -> flip lists (index | old x << 31), one CTA per replica
__global__ __launch_bounds__(256) void k_compact_mask(Dev d, const uint8_t* __restrict__ mask, int ldm)
{
    const int p = blockIdx.x, lane = threadIdx.x & 31;
    const uint8_t* mrow = mask + (size_t)p * ldm;
    const uint8_t* xrow = d.X + (size_t)p * d.ld;
    int32_t* fl = d.FL + (size_t)p * d.ld;
    for (int j0 = 0; j0 < d.n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool f = j < d.n && mrow[j] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&d.FCNT[p], __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        if (f && pos < d.ld) fl[pos] = j | (int)((unsigned)xrow[j] << 31);
    }
}

cudaError_t launch_compact_mask(const Dev& d, const uint8_t* mask, int ldm, cudaStream_t s)
{
    k_compact_mask<<<d.R, 256, 0, s>>>(d, mask, ldm);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
