// kernels_exact.cu -- exact Ising machine for small subQUBOs (m <= 24): the
// "precise solution" of a subQUBO (Section 3) by trying all 2^m assignments.
//
// One CTA of 128 walkers per subQUBO.  Q' = Q[S, S] (diagonal stored as 0)
// is staged in shared memory, one 32-byte row per position.  The 2^m
// assignments are walked in Gray-code order t -> y = t xor (t >> 1), split
// into L = min(128, 2^m) contiguous ranges of 2^k codes (k = m - log2 L), one
// per walker.  A walker
// first moves from the current assignment to the first code of its range
// (flipping the differing positions one by one), then steps through its
// range: step u flips position ctz(u) -- the same position in every lane,
// because each range starts at a multiple of 2^k -- so all walkers read the
// same row of Q' (a shared-memory broadcast).  Walkers keep the sign-free field
// h_a = (1 - 2 y_a) l_a of every position (l_a the gain): a flip of b changes
// the objective by l_b and adds 2 Q'_ab (1 - 2 y_b) to every h_a (24
// multiply-adds; padding rows and columns are 0).  Each walker keeps its best
// (objective, y) pair; the CTA takes the minimum of (objective, y as the
// integer sum_a y_a 2^a), which fixes the choice among equal objectives.
// The gains of the current assignment are the global gains (Eq. 4's bias
// makes the subQUBO's local gain equal the global one), read from G.
//
// Output as for the annealer: the positions that change, as a 0/1 mask or
// appended to the replica's flip list, and the objective change.
#include <climits>

#include "common.cuh"

namespace icd2s {

constexpr int kExactMaxM = 24;
constexpr int kExactRow = 32;  // bytes per staged row
constexpr int kExactThreads = 128;  // walkers per subQUBO (one CTA each)
constexpr int kExactLog = 7;        // log2 kExactThreads

__global__ __launch_bounds__(kExactThreads) void k_exact(Dev d, AnnealArgs a)
{
    __shared__ __align__(16) int8_t qs[kExactMaxM * kExactRow];
    __shared__ long long wbest[kExactThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = a.group_stride > 0 ? (int)blockIdx.x * a.group_stride + a.group_k : (int)blockIdx.x;
    const int p = s / a.per_replica;
    const int* S = nullptr;
    int m;
    int bbase = a.block_base;
    if (a.idx) {
        const int b0 = a.off[s];
        m = a.off[s + 1] - b0;
        S = a.idx + b0;
    } else {
        m = a.block_m;
        bbase += (s - p * a.per_replica) * a.block_m;  // block s mod per_replica of the group
    }
    const int ld = d.ld;
    auto var = [&](int r) { return S ? __ldg(S + r) : bbase + r; };

    // stage Q' with a zero diagonal and zero padding
    for (int e = tid; e < kExactMaxM * kExactRow; e += kExactThreads) {
        const int r = e / kExactRow, c = e % kExactRow;
        int8_t v = 0;
        if (r < m && c < m && r != c) v = d.Q[(size_t)var(r) * ld + var(c)];
        qs[e] = v;
    }
    __syncthreads();

    // current assignment x0 and the sign-free fields at x0 (every lane)
    const int32_t* grow = d.G + (size_t)p * ld;
    const uint8_t* xrow = d.X + (size_t)p * ld;
    unsigned x0 = 0;
    int h[kExactMaxM];
#pragma unroll
    for (int c = 0; c < kExactMaxM; ++c) {
        int xv = 0, g = 0;
        if (c < m) {
            const int j = var(c);
            xv = xrow[j];
            g = grow[j];
        }
        x0 |= (unsigned)xv << c;
        h[c] = xv ? -g : g;
    }
    // flip of position b: objective change, fields, assignment; `hb` is h[b]
    auto flip_with = [&](int b, int hb, unsigned& y, int& f) {
        const int sb = ((y >> b) & 1u) ? -1 : 1;
        f += sb * hb;
        const uint32_t* row = reinterpret_cast<const uint32_t*>(qs + b * kExactRow);
        const int s2 = 2 * sb;
#pragma unroll
        for (int w = 0; w < kExactMaxM / 4; ++w) {
            const uint32_t v = row[w];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[4 * w + q] += s2 * (int)(int8_t)(v >> (8 * q));
        }
        y ^= 1u << b;
    };
    auto flip = [&](int b, unsigned& y, int& f) {  // b not known at compile time
        int hb = 0;
#pragma unroll
        for (int c = 0; c < kExactMaxM; ++c) hb = c == b ? h[c] : hb;
        flip_with(b, hb, y, f);
    };
    // key of (objective, y) ordered lexicographically (0 <= y < 2^24)
    auto keyof = [](int f, unsigned y) { return (long long)f * 4294967296LL + (long long)y; };

    const int lg = m < kExactLog ? m : kExactLog;  // log2 of the walkers in use
    const int k = m - lg;                          // Gray-code bits each walker covers
    const bool active = tid < (1 << lg);
    unsigned y = x0;
    int f = 0;                                     // objective relative to x0
    long long best = LLONG_MAX;
    if (active) {
        const unsigned t0 = (unsigned)tid << k;
        const unsigned y0 = t0 ^ (t0 >> 1);
        unsigned diff = y0 ^ x0;
        while (diff) {
            const int b = __ffs(diff) - 1;
            diff &= diff - 1u;
            flip(b, y, f);
        }
        best = keyof(f, y);
        const unsigned steps = 1u << k;
        if (k < 4) {
            for (unsigned u = 1; u < steps; ++u) {
                flip(__ffs(u) - 1, y, f);
                const long long key = keyof(f, y);
                best = key < best ? key : best;
            }
        } else {
            // blocks of 16 codes: inside a block the flipped positions are
            // ctz(1..15) = 0 1 0 2 0 1 0 3 0 1 0 2 0 1 0 (known at compile
            // time); the block boundary u0 flips position ctz(u0) >= 4
            for (unsigned u0 = 0; u0 < steps; u0 += 16) {
                if (u0) {
                    flip(__ffs(u0) - 1, y, f);
                    const long long key = keyof(f, y);
                    best = key < best ? key : best;
                }
#pragma unroll
                for (int v = 1; v < 16; ++v) {
                    const int b = (v & 1) ? 0 : (v & 2) ? 1 : (v & 4) ? 2 : 3;
                    flip_with(b, h[b], y, f);
                    const long long key = keyof(f, y);
                    best = key < best ? key : best;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int w = 1; w < kExactThreads / 32; ++w) best = wbest[w] < best ? wbest[w] : best;
    const unsigned ybest = (unsigned)((unsigned long long)best & 0xffffffffull);
    const int fbest = (int)((best - (long long)ybest) / 4294967296LL);
    const unsigned changed = (ybest ^ x0) & ((m >= 32) ? 0xffffffffu : ((1u << m) - 1u));

    // output: positions r with bit r of `changed`, lane r handles position r (m <= 24 < 32)
    const bool mine = lane < m && ((changed >> lane) & 1u);
    if (a.mask) {
        if (mine) a.mask[(size_t)p * a.ldm + var(lane)] = 1;
    } else {
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        const int total = __popc(bal);
        int base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(&d.FCNT[p], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (mine) {
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            if (pos < ld) d.FL[(size_t)p * ld + pos] = var(lane) | (int)(((x0 >> lane) & 1u) << 31);
        }
    }
    if (lane == 0 && a.dE) a.dE[s] = fbest;
}

cudaError_t launch_exact(const Dev& d, const AnnealArgs& a, cudaStream_t s)
{
    if (a.count <= 0) return cudaSuccess;
    if (a.m_max > kExactMaxM) return cudaErrorInvalidValue;
    k_exact<<<a.count, kExactThreads, 0, s>>>(d, a);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
