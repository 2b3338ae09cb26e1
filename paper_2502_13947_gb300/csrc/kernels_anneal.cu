// kernels_anneal.cu -- the emulated Ising machine (Eq. 4, Algorithm 4).
//
// One warp per subQUBO S (m <= 32 P variables, ascending indices).  Lane l
// owns the P consecutive positions b = l P .. l P + P - 1.
//
// Gather (Eq. 4): Q' = Q[S, S] is staged as int8 in shared memory (m rows of
// 32 P bytes).  The boundary bias b_i = sum_{j not in S} 2 Q_ij x_j is never
// formed explicitly: the local gain of position a in the biased subQUBO,
// (1 - 2 x_a)(Q_aa + b_a + 2 sum_{c in S, c != a} Q_ac x_c), equals the global
// gain g_a, which the solution set already tracks exactly; so the gains of S
// are read straight from G.
//
// Anneal: sweeps k = 0..K-1 visit positions 0..m-1 in order; attempt (k, b)
// draws u = Philox(ctr = (k / 4, (TAG_ANNEAL << 24) | b, slot, iter)).word[k mod 4]
// and accepts iff l_b <= 0 or l_b * BETA[k] < NLOG[u >> 20].  A sweep is run
// as a sequence of "first accept" rounds: every lane tests all of its
// positions at or after the current one against the current gains, a ballot
// finds the first accepted position, that flip is applied (each lane
// updates its gains from one P-byte row segment of Q'), and the scan resumes
// just after it.  Positions before the first accept would have been tested
// with exactly these gains by a one-at-a-time sweep, so the trajectory is
// identical to the sequential one; a sweep costs (accepts + 1) rounds
// instead of m dependent steps.  Each lane draws one Philox block per owned
// position every 4 sweeps, so no random words are wasted or exchanged.
//
// Output: the changed positions, either as a 0/1 mask [R][ldm] or appended
// to the replica's flip list (index | old x << 31) for k_apply; and the
// subQUBO energy change (sum of the accepted gains).
#include "common.cuh"

namespace icd2s {

template <int P>
struct RowSeg;  // P bytes of a shared-memory row as one load
template <> struct RowSeg<1> { using T = uint8_t; };
template <> struct RowSeg<2> { using T = uint16_t; };
template <> struct RowSeg<4> { using T = uint32_t; };
template <> struct RowSeg<8> { using T = unsigned long long; };

template <int P>
__global__ __launch_bounds__(128) void k_anneal(Dev d, AnnealArgs a)
{
    constexpr int MC = 32 * P;  // row length (bytes) of the staged Q'
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int s = blockIdx.x * wpb + wib;
    if (s >= a.count) return;  // whole warp leaves; no block-level barriers below
    int8_t* Qs = reinterpret_cast<int8_t*>(smem) + (size_t)wib * MC * MC;

    const int p = s / a.per_replica;
    const int* S = nullptr;
    int m;
    if (a.idx) {
        const int b0 = a.off[s];
        m = a.off[s + 1] - b0;
        S = a.idx + b0;
    } else {
        m = a.block_m;
    }
    const int ld = d.ld;

    int col[P];
    bool valid[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int b = lane * P + q;
        valid[q] = b < m;
        col[q] = valid[q] ? (S ? __ldg(S + b) : a.block_base + b) : 0;
    }
    // gather Q[S, S]
    for (int r = 0; r < m; ++r) {
        const int ir = S ? __ldg(S + r) : a.block_base + r;
        const int8_t* row = d.Q + (size_t)ir * ld;
        typename RowSeg<P>::T packed = 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const uint8_t v = valid[q] ? (uint8_t)__ldg(row + col[q]) : (uint8_t)0;
            packed |= (typename RowSeg<P>::T)v << (8 * q);
        }
        *reinterpret_cast<typename RowSeg<P>::T*>(Qs + (size_t)r * MC + lane * P) = packed;
    }
    __syncwarp();

    int l[P];
    unsigned xb = 0;
    const int32_t* grow = d.G + (size_t)p * ld;
    const uint8_t* xrow = d.X + (size_t)p * ld;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        l[q] = valid[q] ? grow[col[q]] : 0;
        xb |= (valid[q] ? (unsigned)xrow[col[q]] : 0u) << q;
    }
    const unsigned x0 = xb;
    const uint32_t slot = a.slot_base + (uint32_t)s;
    long long dE = 0;

    for (int k4 = 0; k4 < a.sweeps; k4 += 4) {
        uint32_t thr[4][P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            if (valid[q]) {
                const u32x4 u = philox10((uint32_t)(k4 >> 2), (kTagAnneal << 24) | (uint32_t)(lane * P + q), slot,
                                         a.iter, d.k0, d.k1);
#pragma unroll
                for (int r = 0; r < 4; ++r) thr[r][q] = __ldg(a.nlog + (u.v[r] >> 20));
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) thr[r][q] = 0;
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = k4 + r;
            if (k >= a.sweeps) break;
            const unsigned long long bk = __ldg(a.beta + k);
            int start = 0;
            while (true) {
                int fq = P;
#pragma unroll
                for (int q = P - 1; q >= 0; --q) {
                    const int b = lane * P + q;
                    const bool acc = valid[q] && b >= start &&
                                     (l[q] <= 0 || (unsigned long long)(unsigned)l[q] * bk < thr[r][q]);
                    fq = acc ? q : fq;
                }
                const unsigned any = __ballot_sync(0xffffffffu, fq < P);
                if (any == 0u) break;
                const int L = __ffs(any) - 1;
                const int v = __shfl_sync(0xffffffffu, fq | (int)(((xb >> (fq & 31)) & 1u) << 8), L);
                const int qs = v & 0xff;
                const int si = 1 - 2 * (v >> 8);
                const int bsel = L * P + qs;
                const typename RowSeg<P>::T seg =
                    *reinterpret_cast<const typename RowSeg<P>::T*>(Qs + (size_t)bsel * MC + lane * P);
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const bool is_i = (lane == L) && (q == qs);
                    const int qv = (int)(int8_t)(uint8_t)(seg >> (8 * q));
                    const int sq = 1 - 2 * (int)((xb >> q) & 1u);
                    if (is_i) { dE += l[q]; l[q] = -l[q]; }
                    else l[q] += 2 * qv * si * sq;
                }
                if (lane == L) xb ^= 1u << qs;
                start = bsel + 1;
            }
        }
    }

    const unsigned changed = xb ^ x0;
    if (a.mask) {
#pragma unroll
        for (int q = 0; q < P; ++q)
            if (valid[q] && ((changed >> q) & 1u)) a.mask[(size_t)p * a.ldm + col[q]] = 1;
    } else {
        const int cnt = __popc(changed);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(&d.FCNT[p], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        int pos = base + incl - cnt;
        int32_t* fl = d.FL + (size_t)p * ld;
#pragma unroll
        for (int q = 0; q < P; ++q)
            if ((changed >> q) & 1u) {
                if (pos < ld) fl[pos] = col[q] | (int)(((x0 >> q) & 1u) << 31);  // a list never exceeds n entries
                ++pos;
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(0xffffffffu, dE, o);
    if (lane == 0) {
        if (a.dE) a.dE[s] = dE;
        if (a.attempts_acc) atomicAdd(reinterpret_cast<unsigned long long*>(a.attempts_acc),
                                      (unsigned long long)a.sweeps * (unsigned long long)m);
    }
}

template <int P>
static cudaError_t launch_anneal_p(const Dev& d, const AnnealArgs& a, int wpb, cudaStream_t s)
{
    constexpr int MC = 32 * P;
    const size_t sm = (size_t)wpb * MC * MC;
    cudaError_t e = cudaFuncSetAttribute(k_anneal<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = (a.count + wpb - 1) / wpb;
    k_anneal<P><<<blocks, 32 * wpb, sm, s>>>(d, a);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_anneal(const Dev& d, const AnnealArgs& a, cudaStream_t s)
{
    if (a.count <= 0) return cudaSuccess;
    const int m = a.m_max;
    if (m <= 32) return launch_anneal_p<1>(d, a, 2, s);
    if (m <= 64) return launch_anneal_p<2>(d, a, 2, s);
    if (m <= 128) return launch_anneal_p<4>(d, a, 2, s);
    if (m <= 256) return launch_anneal_p<8>(d, a, 1, s);
    return cudaErrorInvalidValue;
}

}  // namespace icd2s
