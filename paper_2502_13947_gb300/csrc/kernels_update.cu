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
// k_apply: grid (ld / 2048, R, S), 128 threads; each thread owns 16
// consecutive columns j of one replica (4 columns and 256 threads when the
// caller's buffers are only 4-byte aligned).  The replica's flip list is staged in
// shared memory in chunks; for every listed row i the thread streams the 16
// bytes Q[i][j..j+15] (coalesced 2 KiB per CTA per row -- Q is symmetric, so
// the row is the column), sixteen rows in flight per thread.  Long lists are
// split over up to S CTAs per column tile (at least kMinRows rows each, so
// the HBM stream has enough loads in flight): CTA z stores its partial sums
// to the plane ACC[z][p][j], and the last of them (a per-tile ticket) adds
// the other planes to its own and finishes the tile.  A short list is done by
// one CTA per tile.  Per-tile energy terms go to an int64 accumulator; the last tile
// of the replica (ticket counter) folds it into E and resets the list, the
// accumulator and the counters, so the next producer starts clean.
#include "common.cuh"

namespace icd2s {

// Two shapes: 16 columns per thread (16-byte loads; rows and solution rows
// 16-byte aligned, ld % 16 == 0 -- every state the library allocates) and 4
// columns per thread (4-byte loads; ld % 4 == 0, for caller-owned buffers).
template <int COLS> struct ApplyShape {
    static constexpr int threads = COLS == 16 ? 128 : 256;
    static constexpr int tile = COLS * threads;  // columns per CTA
};
constexpr int kApplyChunk = 2048;  // list entries staged per pass
constexpr int kMinRows = 64;       // rows per CTA before a list is split

template <int COLS> struct RowLoad;
template <> struct RowLoad<16> {
    static __device__ __forceinline__ void get(const int8_t* p, unsigned (&w)[4])
    {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
};
template <> struct RowLoad<4> {
    static __device__ __forceinline__ void get(const int8_t* p, unsigned (&w)[1])
    {
        w[0] = __ldg(reinterpret_cast<const unsigned*>(p));
    }
};

// acc[c] += d_i Q[i][j0 + c] over the staged rows, 16 rows in flight per
// thread; the diagonal term Q_jj d_j that a flipped j adds to its own sum is
// taken out when the tile is finished.
template <int COLS>
__device__ __forceinline__ void accumulate_rows(const Dev& d, const int32_t* sl, int cn, int j0, int (&acc)[COLS])
{
    const int ld = d.ld;
    int e = 0;
    for (; e + 16 <= cn; e += 16) {
        unsigned rv[16][COLS / 4];
        int di[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int v = sl[e + u];
            di[u] = v < 0 ? -1 : 1;
            RowLoad<COLS>::get(d.Q + (size_t)(v & 0x7fffffff) * ld + j0, rv[u]);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < COLS; ++c) acc[c] += di[u] * (int)(int8_t)(rv[u][c >> 2] >> (8 * (c & 3)));
    }
    for (; e < cn; ++e) {
        const int v = sl[e];
        const int dd = v < 0 ? -1 : 1;
        unsigned w[COLS / 4];
        RowLoad<COLS>::get(d.Q + (size_t)(v & 0x7fffffff) * ld + j0, w);
#pragma unroll
        for (int c = 0; c < COLS; ++c) acc[c] += dd * (int)(int8_t)(w[c >> 2] >> (8 * (c & 3)));
    }
}

template <int COLS>
__global__ __launch_bounds__(ApplyShape<COLS>::threads) void k_apply(Dev d)
{
    constexpr int kApplyThreads = ApplyShape<COLS>::threads, kApplyTile = ApplyShape<COLS>::tile;
    constexpr int kApplyCols = COLS;
    __shared__ int32_t sl[kApplyChunk];
    __shared__ uint32_t tileflip[kApplyTile / 32];
    __shared__ long long red[kApplyThreads / 32];
    __shared__ int s_last;
    const int p = blockIdx.y, tid = threadIdx.x;
    const int ld = d.ld, n = d.n;
    const int cnt = min(d.FCNT[p], ld);  // a list never exceeds n entries
    if (cnt == 0) return;  // nothing to apply for this replica (counters are already clear)
    const int S = (d.ACC && gridDim.z > 1) ? (int)gridDim.z : 1;
    const int used = min(S, (cnt + kMinRows - 1) / kMinRows);
    const int z = blockIdx.z;
    if (z >= used) return;
    const int lo = (int)((long long)cnt * z / used), hi = (int)((long long)cnt * (z + 1) / used);
    const int tile0 = blockIdx.x * kApplyTile;
    const int j0 = tile0 + kApplyCols * tid;  // ld % COLS == 0: j0 < ld implies j0 + COLS <= ld
    const int32_t* fl = d.FL + (size_t)p * ld;
    int acc[kApplyCols];
#pragma unroll
    for (int c = 0; c < kApplyCols; ++c) acc[c] = 0;
    for (int c0 = lo; c0 < hi; c0 += kApplyChunk) {
        const int cn = min(kApplyChunk, hi - c0);
        __syncthreads();
        for (int e = tid; e < cn; e += kApplyThreads) sl[e] = fl[c0 + e];
        __syncthreads();
        if (j0 < ld) accumulate_rows(d, sl, cn, j0, acc);
    }
    if (used > 1) {  // partial sums to ACC[z]; the tile's last CTA adds them up
        const size_t plane = (size_t)d.R * ld;
        int32_t* mine = d.ACC + (size_t)z * plane + (size_t)p * ld + j0;
        if (j0 < ld) {
#pragma unroll
            for (int c4 = 0; c4 < COLS / 4; ++c4)
                reinterpret_cast<int4*>(mine)[c4] = make_int4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2],
                                                              acc[4 * c4 + 3]);
        }
        __threadfence();
        __syncthreads();
        unsigned* tt = d.TT + (size_t)p * gridDim.x + blockIdx.x;
        if (tid == 0) s_last = atomicAdd(tt, 1u) == (unsigned)(used - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        if (j0 < ld) {
            for (int z2 = 0; z2 < used; ++z2) {
                if (z2 == z) continue;
                const int4* other = reinterpret_cast<const int4*>(d.ACC + (size_t)z2 * plane + (size_t)p * ld + j0);
#pragma unroll
                for (int c4 = 0; c4 < COLS / 4; ++c4) {
                    const int4 v = __ldcg(other + c4);
                    acc[4 * c4] += v.x; acc[4 * c4 + 1] += v.y; acc[4 * c4 + 2] += v.z; acc[4 * c4 + 3] += v.w;
                }
            }
        }
        if (tid == 0) *tt = 0u;  // every CTA of the tile has arrived
    }
    // the flips that fall in this tile (the whole list)
    for (int w = tid; w < kApplyTile / 32; w += kApplyThreads) tileflip[w] = 0;
    __syncthreads();
    for (int e = tid; e < cnt; e += kApplyThreads) {
        const int i = fl[e] & 0x7fffffff;
        if (i >= tile0 && i < tile0 + kApplyTile) atomicOr(&tileflip[(i - tile0) >> 5], 1u << ((i - tile0) & 31));
    }
    __syncthreads();
    long long dpart = 0;
    if (j0 < ld) {
        uint8_t* xrow = d.X + (size_t)p * ld;
        int32_t* grow = d.G + (size_t)p * ld;
        unsigned xw[COLS / 4], xo[COLS / 4];
        if constexpr (COLS == 16) {
            const uint4 xv4 = *reinterpret_cast<const uint4*>(xrow + j0);
            xw[0] = xv4.x; xw[1] = xv4.y; xw[2] = xv4.z; xw[3] = xv4.w;
        } else {
            xw[0] = *reinterpret_cast<const unsigned*>(xrow + j0);
        }
#pragma unroll
        for (int c4 = 0; c4 < COLS / 4; ++c4) xo[c4] = 0u;
        const unsigned fbits = (tileflip[(j0 - tile0) >> 5] >> ((j0 - tile0) & 31)) & ((1u << COLS) - 1u);
#pragma unroll
        for (int c4 = 0; c4 < kApplyCols / 4; ++c4) {
            const int4 gv = *reinterpret_cast<const int4*>(grow + j0 + 4 * c4);
            const int gin[4] = {gv.x, gv.y, gv.z, gv.w};
            int gout[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = 4 * c4 + b, j = j0 + c;
                int xj = (int)((xw[c4] >> (8 * b)) & 1u);
                if (j < n) {
                    const int dj = d.diag[j];
                    const int fl_j = (int)((fbits >> c) & 1u);
                    const int h = ((1 - 2 * xj) * gin[b] - dj) / 2 + acc[c] - (fl_j ? (1 - 2 * xj) * dj : 0);
                    xj ^= fl_j;
                    gout[b] = (1 - 2 * xj) * (dj + 2 * h);
                    if (fl_j) dpart += (long long)gin[b] - gout[b];
                } else {  // columns past n: left as they are (padding of caller-owned rows)
                    gout[b] = gin[b];
                    xj = (int)((xw[c4] >> (8 * b)) & 0xffu);
                }
                xo[c4] |= (unsigned)xj << (8 * b);
            }
            *reinterpret_cast<int4*>(grow + j0 + 4 * c4) = make_int4(gout[0], gout[1], gout[2], gout[3]);
        }
        if constexpr (COLS == 16)
            *reinterpret_cast<uint4*>(xrow + j0) = make_uint4(xo[0], xo[1], xo[2], xo[3]);
        else
            *reinterpret_cast<unsigned*>(xrow + j0) = xo[0];
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
    const bool wide = d.ld % 16 == 0 && ((uintptr_t)d.Q % 16) == 0 && ((uintptr_t)d.X % 16) == 0;
    if (wide) {
        const int tiles = (d.ld + ApplyShape<16>::tile - 1) / ApplyShape<16>::tile;
        const int S = (d.ACC && d.TT && d.apply_splits > 1) ? d.apply_splits : 1;
        k_apply<16><<<dim3(tiles, d.R, S), ApplyShape<16>::threads, 0, s>>>(d);
    } else {  // caller-owned buffers with 4-byte alignment: no splitting
        Dev d4 = d;
        d4.ACC = nullptr;
        d4.TT = nullptr;
        const int tiles = (d.ld + ApplyShape<4>::tile - 1) / ApplyShape<4>::tile;
        k_apply<4><<<dim3(tiles, d.R, 1), ApplyShape<4>::threads, 0, s>>>(d4);
    }
    note_launch(1);
    return cudaGetLastError();
}

// Splits giving about 6 CTAs per SM when every tile of every replica has a
// long list (16-column shape; measured best of 4, 6, 8 and 12 on the
// n = 16 384 write-back).
int apply_splits_for(int ld, int R)
{
    const long long base = (long long)apply_tiles(ld) * R;
    const long long want = 6LL * device_sm_count();
    long long S = (want + base - 1) / base;
    return (int)(S < 1 ? 1 : (S > 16 ? 16 : S));
}

int apply_tiles(int ld) { return (ld + ApplyShape<16>::tile - 1) / ApplyShape<16>::tile; }

// mask [R][ldm] (0/1) -> flip lists (index | old x << 31).  Grid
// (ceil(n / 4096), R): each thread tests 16 columns (coalesced byte loads),
// a block-wide scan orders the CTA's flips and one atomic per CTA reserves
// their slots in the replica's list (the order of a list is immaterial).
constexpr int kCompactThreads = 256, kCompactPer = 16;

__global__ __launch_bounds__(kCompactThreads) void k_compact_mask(Dev d, const uint8_t* __restrict__ mask, int ldm)
{
    __shared__ int wsum[kCompactThreads / 32];
    __shared__ int s_base;
    const int p = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base_j = blockIdx.x * kCompactThreads * kCompactPer;
    const uint8_t* mrow = mask + (size_t)p * ldm;
    const uint8_t* xrow = d.X + (size_t)p * d.ld;
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k) {
        const int j = base_j + k * kCompactThreads + tid;
        bits |= (unsigned)(j < d.n && mrow[j] != 0) << k;
    }
    const int c = __popc(bits);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) { const int v = wsum[w]; wsum[w] = tot; tot += v; }
        s_base = tot ? atomicAdd(&d.FCNT[p], tot) : 0;
    }
    __syncthreads();
    int pos = s_base + wsum[warp] + incl - c;
    int32_t* fl = d.FL + (size_t)p * d.ld;
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k)
        if ((bits >> k) & 1u) {
            const int j = base_j + k * kCompactThreads + tid;
            if (pos < d.ld) fl[pos] = j | (int)((unsigned)xrow[j] << 31);
            ++pos;
        }
}

cudaError_t launch_compact_mask(const Dev& d, const uint8_t* mask, int ldm, cudaStream_t s)
{
    const int per = kCompactThreads * kCompactPer;
    dim3 grid((d.n + per - 1) / per, d.R);
    k_compact_mask<<<grid, kCompactThreads, 0, s>>>(d, mask, ldm);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
