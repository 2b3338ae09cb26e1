// kernels_tabu.cu -- Tabu search (Algorithm 1, Section 2.4) on every replica.
//
// One CTA per replica.  Thread t owns the W groups of 4 consecutive
// variables j = 4 (t + w NT) + {0..3}.  Per owned variable it keeps, in
// registers for the whole search:
//   gf_j = (1 - 2 x_j) g_j   the gain with the variable's sign folded in, so a
//                            move i only adds 2 Q_ij (1 - 2 x_i) to it (one
//                            multiply-add per variable) and the moved variable
//                            keeps its value (g_i -> -g_i and x_i -> 1 - x_i);
//   fa_j                     the first iteration at which j may move again:
//                            C_j <= 0 at iteration t  <=>  t >= fa_j, with
//                            fa_i = t + c when i moves at iteration t (C_i += c
//                            and the same-iteration decrement leave c - 1).
// One iteration is:
//   1. every thread knows the chosen move (g_i, i, x_i) from the previous
//      block-wide arg-min;
//   2. it streams its 4W bytes of row i of Q (coalesced 4-byte loads; the row
//      index is only known after the arg-min, so there is nothing to
//      prefetch -- rows stay hot in L1/L2) and applies the update; while the
//      row is in flight, the owner of i flips it and takes the update's term
//      2 (1 - 2 x_i) Q_ii off its gain in advance (Q_jj of the owned variables
//      is held in a register), and thread 0 logs the move;
//   3. it takes the arg-min over its free variables as the minimum of 32-bit
//      keys (g + 2^26) << 5 | local index (the local index orders a thread's
//      variables by j), the warp takes the arg-min with two redux.sync (gain,
//      then global index), and one __syncthreads publishes the per-warp
//      minima; every thread reduces those itself, so the loop has exactly one
//      barrier.
// Ties go to the lowest index, exactly as a scan in index order would.
// Compact keys (CK): when every gain of the instance is known to satisfy
// |g| < 2^(31 - sh) - 1 with sh = 1 + (bits of n), the whole move fits one
// 32-bit key (g + 2^(31 - sh)) << sh | j << 1 | x_j, so the warp and the block
// each take their arg-min with a single redux.sync and the key carries x_i.
// The bound max_j max(|Q_jj - 2 N_j|, |Q_jj + 2 P_j|) (P_j, N_j: the positive
// and negative off-diagonal sums of column j in magnitude) holds for every x
// and is attained, so it is computed once per instance.
// Parity labels (PK), where that bound is one bit too wide: g_j is congruent
// to Q_jj mod 2 for every x, so the gain field's lowest bit already names the
// parity class of the variable, and within a class the rank r of j (in index
// order) identifies it.  The search then runs on Q relabeled with the n0
// even-diagonal variables first (label L = r, or n0 + r for the odd class) and
// the key (g + 2^(31 - sh)) << sh | r << 1 | x_j needs sh - 1 = bits of the
// larger class instead of bits of n.  Key order is still (g, j): equal gains
// share a class, where ranks follow j.  The state is gathered through the
// labels at the start and scattered back at the end.
// Each variable's update is one dp4a of the row word with the byte
// 2 (1 - 2 x_i) in the variable's lane.  Signed rows (SR, on request; not for
// Q with an entry -128): the rows (1 - 2x) Q_i interleaved, row 2i + x, so the
// move (i, x_i) reads row 2i + x_i (the key's low bits) and the byte is 2.
// The objective OV is tracked in int64 by thread 0, which also keeps the
// move log and publishes the best visit at the end; the toggle counts are
// counted from the move log after the search.  The move log (uint16 per
// iteration) stays in shared memory; after the last iteration the moves
// made after the best visit are undone in one pass: variables moved an odd
// number of times flip back, and their rows of Q correct the gains (x_min is
// reconstructed without copying x on every improvement).  The tabu memory
// returned is C_j = max(0, fa_j - alpha).
//
// Cluster split (G = 2 or 4 CTAs per replica, when replicas are fewer than
// the SMs): CTA r of the replica's cluster owns the slice [r S, r S + S) of
// the variables (S a multiple of 128) and reads only that slice of each moved
// row.  Per move it takes its slice's arg-min key as above, then thread 0
// writes the key into slot [move parity][r] of every other CTA of the cluster
// (st.async into distributed shared memory, completing bytes on that CTA's
// per-parity mbarrier) and every thread waits, with a bounded try_wait, for
// the G - 1 keys of its peers; the minimum over the G keys is the move, the
// same in every CTA.  Two parity slots let a CTA run one move ahead of a
// slower peer without overwriting a key that peer has not read.  (A relaxed
// store of the key with a sequence number, polled by the receiver, measured
// slower.)  With
// aspiration each CTA also sends the arg-min over all variables, so the
// all-tabu fallback needs no extra exchange.  A timed-out wait raises
// flags[6]; the barrier of the next move (a block-wide OR) ends the search in
// every thread of the CTA at once, the peers' waits then time out as well,
// and the clusters meet at a final cluster barrier before any CTA leaves.
// Every CTA keeps the objective, the best visit and the move log itself;
// toggle counts, undo pass and the outputs are written per slice.  Keys are
// exchanged as 64 bits (compact keys zero-extended, wide keys as gain half
// and index half), so the unsigned minimum orders them as the block
// reductions do.
#include <climits>
#include <type_traits>

#include "common.cuh"

namespace icd2s {

namespace {

constexpr unsigned kKeyBias = 1u << 26;  // |g| <= 128 + 256 (n - 1) < 2^22, so g + bias < 2^27
constexpr int kKeyShift = 5;             // local index 4 w + b < 32 (W <= 8); (g + bias) << 5 < 2^32
// shared-memory layout: warp keys [0, 1024), flip count, best visit, exchange
// barriers [2] and keys [2][4][2], then the toggle counts [ld], undo and x bitmaps [ld / 32]
// each, and the move log [alpha]
constexpr int kSmNF = 1024, kSmBest = 1032, kSmBar = 1040, kSmKeys = 1056, kSmTs = 1280;

__device__ __forceinline__ unsigned long long pack_key(unsigned hi, unsigned lo)
{
    return ((unsigned long long)hi << 32) | lo;
}

template <int S>
using slot_t = std::integral_constant<int, S>;

// ---- distributed shared memory exchange of the cluster split ----
constexpr int kClusterWaitLimit = 1 << 24;  // try_wait polls before a wait gives up (and about 1 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the address of this CTA's shared-memory location `addr` in cluster CTA `rank`
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init_cta(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 8 bytes into a peer's shared memory, counted on the peer's mbarrier
__device__ __forceinline__ void st_async_b64(uint32_t raddr, unsigned long long v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr), "l"(v),
                 "r"(rbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase `parity` of `bar`: false if it never completes
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < kClusterWaitLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if ((i & 1023) == 1023) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 1000000000ull) break;
        }
    }
    return false;
}

}  // namespace

// ASP: the aspiration criterion (reading S4): a tabu variable is also a
// candidate when its move would beat the best objective visited so far, i.e.
// g < OVmin - OV, which in key units is (key >> shift) < OVmin - OV + bias.
// G: CTAs per replica (a thread-block cluster of G; 1 = no cluster); each owns
// `slice` variables (a multiple of 128; G slice >= ld).
template <int W, int MAXT, bool ASP, bool CK, bool SR, int G, bool PK = false>
__global__ __launch_bounds__(MAXT) void k_tabu(Dev d, int alpha, int c, int sh, int slice)
{
    static_assert(4 * W <= (1 << kKeyShift), "the local index must fit the key");
    static_assert(!PK || (CK && G == 1 && !SR), "parity labels: compact keys, one CTA per replica, plain rows");
    extern __shared__ __align__(16) unsigned char smem[];
    // warp keys of the arg-min: wide keys [2][32] (+0), and with the cluster split
    // and aspiration the unmasked ones [2][32] (+512); compact keys [2][32] (+0)
    // and the unmasked ones [2][32] (+256)
    unsigned long long* wkeys = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* wkeysU = wkeys + 64;
    unsigned* wkeys32 = reinterpret_cast<unsigned*>(smem);
    int* nF = reinterpret_cast<int*>(smem + kSmNF);
    // G > 1: per-parity mbarriers of the key exchange and the peers' keys [2][G][2]
    // (move parity, rank): the arg-min key (CK: zero-extended) and, with
    // aspiration, the unmasked one
    const uint32_t cbar0 = smem_addr(smem + kSmBar), ckey0 = smem_addr(smem + kSmKeys);
    const unsigned long long* ckeys = reinterpret_cast<const unsigned long long*>(smem + kSmKeys);
    int32_t* Ts = reinterpret_cast<int32_t*>(smem + kSmTs);                            // [ld]
    uint32_t* undo = reinterpret_cast<uint32_t*>(smem + kSmTs + 4 * (size_t)d.ld);    // [ld / 32]
    uint32_t* xe = undo + d.ld / 32;                                                  // [ld / 32] (G > 1)
    const int p = G > 1 ? (int)(blockIdx.x / G) : (int)blockIdx.x;
    const int rank = G > 1 ? (int)cluster_ctarank() : 0;
    // [alpha]: in shared memory, or in global memory (d.TL) when a long search does not fit
    // (there rank 0 writes it and every CTA of the cluster reads it after the search)
    uint16_t* mlog = d.TL ? d.TL + (size_t)p * (size_t)d.tl_cap
                          : reinterpret_cast<uint16_t*>(smem + kSmTs + 4 * (size_t)d.ld + 2 * (d.ld / 8));
    const bool log_writer = G == 1 || !d.TL || rank == 0;

    const int NT = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = d.n, ld = d.ld;
    const int lo = G > 1 ? rank * slice : 0;                 // owned variables [lo, hi)
    const int hi = G > 1 ? min(lo + slice, ld) : ld;
    const int8_t* __restrict__ Q = PK ? d.Qpk : d.Q;   // PK: rows and columns in label order
    const int32_t* __restrict__ lab = d.pk_perm;        // PK: label -> variable
    const unsigned n0 = PK ? (unsigned)d.pk_n0 : 0u;
    const int8_t* __restrict__ Q2 = d.Q2;  // SR: row 2i + x = (1 - 2x) Q_i
    uint8_t* xrow = d.X + (size_t)p * ld;
    int32_t* grow = d.G + (size_t)p * ld;

    for (int j = tid; j < ld; j += NT) Ts[j] = 0;
    for (int j = tid; j < 2 * (ld / 32); j += NT) undo[j] = 0;   // undo and xe
    for (int j = tid; j < 128; j += NT) wkeys[j] = ~0ull;  // slots of absent warps read as "no candidate"
    if (tid == 0) *nF = 0;
    if constexpr (G > 1) {
        if (tid == 0) {
            mbar_init_cta(cbar0, 1);
            mbar_init_cta(cbar0 + 8, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }

    int gf[W][4], fa[W][4];
    // 2^shift (1 - 2 x_j) mod 2^32: the key is gf * s32 + kc, one multiply-add
    unsigned s32[W][4];
    // CK: kc = bias << sh | j << 1 | x_j (PK: the rank r in place of j); otherwise
    // the constant bias << 5 | local index
    unsigned kc[W][4];
    const unsigned cbias = CK ? 1u << (31 - sh) : kKeyBias;
    const unsigned imask = CK ? (1u << (sh - 1)) - 1u : 0u;  // CK: the index field (2^(sh-1) > n; PK: > each class)
    unsigned xb = 0;  // bit 4w+b = x of the owned variable
    uint32_t dq[W];   // byte b of dq[w] = Q_jj of the owned variable 4w+b (the moved variable's own term)
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int j0 = lo + 4 * (tid + w * NT);
        int gv[4] = {0, 0, 0, 0};
        uint32_t xv = 0;
        dq[w] = 0u;
        if (j0 < hi) {
            if constexpr (PK) {  // gathered through the labels (padding: 0)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (j0 + b < n) {
                        const int v = lab[j0 + b];
                        gv[b] = grow[v];
                        xv |= (uint32_t)(xrow[v] & 1u) << (8 * b);
                    }
            } else {
                const int4 g4 = *reinterpret_cast<const int4*>(grow + j0);
                xv = *reinterpret_cast<const uint32_t*>(xrow + j0);
                gv[0] = g4.x; gv[1] = g4.y; gv[2] = g4.z; gv[3] = g4.w;
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const unsigned xj = (xv >> (8 * b)) & 1u;
            xb |= xj << (4 * w + b);
            gf[w][b] = xj ? -gv[b] : gv[b];
            const unsigned one = CK ? 1u << sh : 1u << kKeyShift;
            s32[w][b] = xj ? 0u - one : one;
            unsigned jk = (unsigned)(j0 + b);  // the key's index: j, or (PK) the rank in the class
            if constexpr (PK) jk = jk >= (unsigned)n ? imask : (jk >= n0 ? jk - n0 : jk);
            kc[w][b] = CK ? (cbias << sh) | (jk << 1) | xj : (kKeyBias << kKeyShift) | (unsigned)(4 * w + b);
            fa[w][b] = (j0 + b < n && j0 < hi) ? 0 : INT_MAX;  // padding never becomes free
            if (j0 + b < n && j0 < hi) dq[w] |= (uint32_t)(uint8_t)(int8_t)d.diag[PK ? lab[j0 + b] : j0 + b] << (8 * b);
        }
    }

    // a warp's arg-min of the thread minima tk, published to slot `slot` (of the
    // unmasked keys when `unmasked`)
    auto publish = [&](unsigned tk, int slot, bool unmasked) {
        if constexpr (CK) {
            const unsigned wk = __reduce_min_sync(0xffffffffu, tk);
            if (lane == 0) wkeys32[(unmasked ? 2 + slot : slot) * 32 + warp] = wk;
        } else {
            const unsigned wg = __reduce_min_sync(0xffffffffu, tk >> kKeyShift);
            const unsigned k = tk & ((1u << kKeyShift) - 1u);
            const unsigned j = (unsigned)lo + 4u * (unsigned)(tid + (int)(k >> 2) * NT) + (k & 3u);
            const unsigned cand =
                (tk != 0xffffffffu && (tk >> kKeyShift) == wg) ? ((j << 1) | ((xb >> k) & 1u)) : 0xffffffffu;
            const unsigned wj = __reduce_min_sync(0xffffffffu, cand);
            if (lane == 0) (unmasked ? wkeysU : wkeys)[slot * 32 + warp] = pack_key(wg, wj);
        }
    };
    // the warp's arg-min over free variables at iteration `itn`, published to slot `slot`
    // (G > 1 with aspiration: also the arg-min over every variable)
    auto warp_argmin = [&](int itn, int slot, unsigned ulim) {
        unsigned tk = 0xffffffffu, tu = 0xffffffffu;
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                // ((g + bias) << shift) | low bits with g = (1 - 2x) gf, one multiply-add modulo 2^32
                const unsigned key = (unsigned)gf[w][b] * s32[w][b] + kc[w][b];
                const bool ok = itn >= fa[w][b] || (ASP && (key >> (CK ? sh : kKeyShift)) < ulim);
                tk = ok ? min(tk, key) : tk;
                if constexpr (G > 1 && ASP) tu = fa[w][b] != INT_MAX ? min(tu, key) : tu;
            }
        publish(tk, slot, false);
        if constexpr (G > 1 && ASP) publish(tu, slot, true);
    };
    // the block's arg-min key (CK: zero-extended; otherwise gain half, index half)
    auto block_argmin = [&](int slot, bool unmasked = false) -> unsigned long long {
        if constexpr (CK) return __reduce_min_sync(0xffffffffu, wkeys32[(unmasked ? 2 + slot : slot) * 32 + lane]);
        const unsigned long long k = (unmasked ? wkeysU : wkeys)[slot * 32 + lane];
        const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)(k >> 32));
        const unsigned lo = __reduce_min_sync(0xffffffffu, (unsigned)(k >> 32) == hi ? (unsigned)k : 0xffffffffu);
        return pack_key(hi, lo);
    };

    // G > 1: remote addresses of this CTA's key slot and of the exchange barrier
    // in every other CTA of the cluster (thread 0 sends)
    uint32_t rkey[2][G > 1 ? G - 1 : 1], rbar[2][G > 1 ? G - 1 : 1];
    if constexpr (G > 1) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
#pragma unroll
            for (int q = 0; q < G - 1; ++q) {
                const uint32_t peer = (uint32_t)((rank + 1 + q) % G);
                rkey[sl][q] = map_to_rank(ckey0 + 16u * (uint32_t)(sl * G + rank), peer);
                rbar[sl][q] = map_to_rank(cbar0 + 8u * (uint32_t)sl, peer);
            }
    }
    uint32_t xph[2] = {0u, 0u};  // phase parity of each exchange barrier
    bool tmo = false;            // this thread's exchange wait timed out
    // G > 1: the cluster-wide move from this CTA's key (and, with aspiration,
    // its arg-min over every variable); slot = the move's parity.  A key with
    // an all-ones index half names no candidate.
    auto exchange = [&](unsigned long long mine, unsigned long long mine_all, int slot) -> unsigned long long {
        if constexpr (G > 1) {
            const uint32_t bar = cbar0 + 8u * (uint32_t)slot;
            if (tid == 0) {
                mbar_arrive_expect(bar, (ASP ? 16u : 8u) * (G - 1));
#pragma unroll
                for (int q = 0; q < G - 1; ++q) {
                    const uint32_t rk = slot ? rkey[1][q] : rkey[0][q], rb = slot ? rbar[1][q] : rbar[0][q];
                    st_async_b64(rk, mine, rb);
                    if constexpr (ASP) st_async_b64(rk + 8u, mine_all, rb);
                }
            }
            const bool ok = mbar_wait_bounded(bar, xph[slot]);
            xph[slot] ^= 1u;
            unsigned long long km = mine, ka = mine_all;
            if (!ok) {
                tmo = true;
                atomicExch(&d.flags[6], 1);
            } else {
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (q == rank) continue;
                    km = min(km, ckeys[2 * (slot * G + q)]);
                    if constexpr (ASP) ka = min(ka, ckeys[2 * (slot * G + q) + 1]);
                }
            }
            // aspiration: with every variable tabu and none aspirated, the unmasked
            // arg-min (reading S6)
            return (ASP && (unsigned)km == 0xffffffffu) ? ka : km;
        } else {
            return mine;
        }
    };

    long long OV = d.E[p], OVmin = OV;
    int best_it = -1;
    // aspiration limit in key units: clamp(OVmin - OV + bias, 0, 2 bias)
    auto asp_limit = [&]() -> unsigned {
        const long long v = OVmin - OV + (long long)cbias;
        return v <= 0 ? 0u : (v >= 2LL * cbias ? 2u * cbias : (unsigned)v);
    };

    if constexpr (G > 1) cluster_barrier();  // every CTA's exchange barriers exist before any key is sent
    __syncthreads();  // shared-memory clears visible
    warp_argmin(0, 0, ASP ? asp_limit() : 0u);
    __syncthreads();
    unsigned long long key = block_argmin(0);
    if constexpr (G > 1) {
        if (alpha > 0) key = exchange(key, ASP ? block_argmin(0, true) : ~0ull, 0);
    }

    bool stop = false;
    // Iteration `it`: apply the chosen move, publish the next arg-min to slot
    // SLOT = (it + 1) & 1 (a compile-time constant: the loop runs two moves per
    // trip), and read it back.
    auto move = [&](int it, auto slot_c) {
        constexpr int slot = decltype(slot_c)::value;
        // the chosen move: index and value (CK: no candidate is the key ~0,
        // whose index field 2^(sh-1) - 1 >= n; otherwise its index half is ~0)
        unsigned jx = CK ? (unsigned)key & (2u * imask + 1u) : (unsigned)key;
        if constexpr (PK) {
            // the label: the rank, plus n0 for the odd class (the gain's parity,
            // bit sh of the key); no candidate (all ones) gives imask + n0 >= n
            const unsigned L = (((unsigned)key >> 1) & imask) + (((unsigned)key >> sh) & 1u) * n0;
            jx = (L << 1) | ((unsigned)key & 1u);
        }
        // Without aspiration at most c - 1 <= n - 1 variables are tabu, so a
        // move always exists; the clamp only keeps the row read in bounds.
        // (With the cluster split the fallback key always names a variable.)
        if constexpr (!ASP || G > 1) jx = min(jx, 2u * (unsigned)n - 1u);
        const int i = (int)(jx >> 1);
        if constexpr (ASP && G == 1) {
            if (i >= n) {  // no move at all: stop, uniformly
                if (tid == 0) d.flags[2] = 1;
                alpha = it;
                stop = true;
                return;
            }
        }
        const int si2 = (jx & 1u) ? -2 : 2;       // 2 (1 - 2 x_i)
        const int8_t* row = SR ? Q2 + (size_t)jx * ld : Q + (size_t)i * ld;
        int rv[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int j0 = lo + 4 * (tid + w * NT);
            rv[w] = j0 < hi ? __ldg(reinterpret_cast<const int*>(row + j0)) : 0;
        }
        // the moved variable keeps its folded gain (the update below adds
        // 2 (1 - 2 x_i) Q_ii to it, taken off here from the diagonal held in a
        // register, so that this runs while the row is in flight), flips, and
        // becomes tabu (owned by this CTA only if it lies in the slice)
        const int rel = (G == 1 || (i >= lo && i < hi)) ? ((i - lo) >> 2) - tid : -1;
        const int bi = i & 3;
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (rel == w * NT) {
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (b == bi) {
                        gf[w][b] -= (int)(int8_t)(dq[w] >> (8 * b)) * si2;
                        xb ^= 1u << (4 * w + b);
                        s32[w][b] = 0u - s32[w][b];
                        if (CK) kc[w][b] ^= 1u;
                        // C += c: free again c iterations after the later of now and the
                        // iteration it was to become free (a tabu move, by aspiration)
                        fa[w][b] = max(fa[w][b], it) + c;
                    }
            }
        // the objective, best visit and move log: one thread (the objective in
        // every thread with aspiration, whose limit needs it)
        auto objective = [&]() {
            const int gi = CK ? (int)((unsigned)key >> sh) - (int)cbias : (int)(unsigned)(key >> 32) - (int)kKeyBias;
            OV += gi;
            if (OV < OVmin) { OVmin = OV; best_it = it; }
        };
        if constexpr (ASP) {
            objective();
            if (tid == 0 && log_writer) mlog[it] = (uint16_t)i;
        } else if (tid == 0) {
            objective();
            if (log_writer) mlog[it] = (uint16_t)i;
        }
        // + 2 (1 - 2 x_i) Q_ij: one dp4a per variable with the byte 2 (1 - 2 x_i)
        // in the variable's lane (the masks depend on the move only, so they are
        // warp-uniform; signed rows already carry the sign)
        if constexpr (!CK || ASP) {
            // a warp-uniform branch on the move's sign, so the byte masks are
            // immediates (measured faster for the wide keys and with aspiration,
            // slower for the compact keys without it)
            if (SR || !(jx & 1u)) {
#pragma unroll
                for (int w = 0; w < W; ++w)
#pragma unroll
                    for (int b = 0; b < 4; ++b) gf[w][b] = __dp4a(rv[w], (int)(0x02u << (8 * b)), gf[w][b]);
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w)
#pragma unroll
                    for (int b = 0; b < 4; ++b) gf[w][b] = __dp4a(rv[w], (int)(0xFEu << (8 * b)), gf[w][b]);
            }
        } else {
            unsigned msk[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) msk[b] = (SR || !(jx & 1u) ? 0x02u : 0xFEu) << (8 * b);
#pragma unroll
            for (int w = 0; w < W; ++w)
#pragma unroll
                for (int b = 0; b < 4; ++b) gf[w][b] = __dp4a(rv[w], (int)msk[b], gf[w][b]);
        }
        warp_argmin(it + 1, slot, ASP ? asp_limit() : 0u);
        if constexpr (G > 1) {
            // one barrier per move, which also makes an exchange time-out end the
            // search in every thread of the CTA at once
            if (__syncthreads_or(tmo)) {
                alpha = it + 1;
                stop = true;
                return;
            }
            key = block_argmin(slot);
            if (it + 1 < alpha)  // the key after the last move is not used: no exchange
                key = exchange(key, ASP ? block_argmin(slot, true) : ~0ull, slot);
            return;
        } else {
            __syncthreads();
        }
        key = block_argmin(slot);
        if constexpr (ASP) {
            // A variable moved again while tabu keeps c more iterations of tabu
            // memory, so every move can be tabu and none aspirated: then the
            // unmasked arg-min (reading S6).  No warp had a candidate iff the
            // block's key (its index half without CK) is all ones.  key is uniform.
            if ((unsigned)key == 0xffffffffu && it + 1 < alpha) {
                __syncthreads();                      // every thread has read this slot
                warp_argmin(INT_MAX - 1, slot, 0u);   // every real variable (padding stays out)
                __syncthreads();
                key = block_argmin(slot);
            }
        }
    };
    int it = 0;
    for (; it + 1 < alpha; it += 2) {
        move(it, slot_t<1>{});
        if ((ASP || G > 1) && stop) break;
        move(it + 1, slot_t<0>{});
        if ((ASP || G > 1) && stop) break;
    }
    if (!stop && it < alpha) move(it, slot_t<1>{});

    // every exchange has landed (no CTA writes into another's shared memory any
    // more) and rank 0's global move log is visible to the cluster
    if constexpr (G > 1) cluster_barrier();
    // toggle counts from the move log; parity of the moves made after the best visit
    int* s_best = reinterpret_cast<int*>(smem + kSmBest);
    if (tid == 0) *s_best = best_it;
    __syncthreads();  // the move log is complete
    for (int e = tid; e < alpha; e += NT) atomicAdd(&Ts[mlog[e]], 1);
    best_it = *s_best;
    for (int e = best_it + 1 + tid; e < alpha; e += NT) {
        const int i = mlog[e];
        atomicXor(&undo[i >> 5], 1u << (i & 31));
    }
    __syncthreads();
    if constexpr (G > 1) {
        // x at the end of the search of every variable to flip back (also those
        // of the other slices): the initial x and the parity of its toggles
        for (int j = tid; j < n; j += NT)
            if ((undo[j >> 5] >> (j & 31)) & 1u)
                atomicOr(&xe[j >> 5], ((uint32_t)(xrow[j] ^ Ts[j]) & 1u) << (j & 31));
        __syncthreads();
    }
    int32_t* Tout = d.T + (size_t)p * ld;
    for (int j = lo + tid; j < hi; j += NT) Tout[PK && j < n ? lab[j] : j] = Ts[j];
    __syncthreads();  // T has been read out before the flip list reuses it
    int32_t* flist = Ts;
    if constexpr (G > 1) {
        for (int j = tid; j < n; j += NT)
            if ((undo[j >> 5] >> (j & 31)) & 1u) {
                const int slot = atomicAdd(nF, 1);
                flist[slot] = j | (int)(((xe[j >> 5] >> (j & 31)) & 1u) << 31);
            }
    } else {
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
    }
    __syncthreads();
    // G > 1: every CTA has read the initial x of the whole row before any writes its slice
    if constexpr (G > 1) cluster_barrier();
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
            const int j0 = lo + 4 * (tid + w * NT);
            const int r4 = j0 < hi ? __ldg(reinterpret_cast<const int*>(row + j0)) : 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (j0 + b != i) acc[w][b] += di * (int)(int8_t)(r4 >> (8 * b));
        }
    }
    int32_t* Cout = d.C + (size_t)p * ld;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int j0 = lo + 4 * (tid + w * NT);
        if (j0 >= hi) continue;
        int gv[4], cv[4];
        uint32_t xv = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + b;
            int xj = (int)((xb >> (4 * w + b)) & 1u);
            int gj = 0, cj = 0;
            if (j < n) {
                const int dj = d.diag[PK ? lab[j] : j];
                const int h = (gf[w][b] - dj) / 2 + acc[w][b];   // (1 - 2x) g = Q_jj + 2 h
                xj ^= (int)((undo[j >> 5] >> (j & 31)) & 1u);
                gj = (1 - 2 * xj) * (dj + 2 * h);
                cj = fa[w][b] > alpha ? fa[w][b] - alpha : 0;
            } else {
                xj = 0;
            }
            gv[b] = gj;
            cv[b] = cj;
            xv |= (uint32_t)xj << (8 * b);
        }
        if constexpr (PK) {  // scattered back through the labels
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int v = j0 + b < n ? lab[j0 + b] : j0 + b;
                grow[v] = gv[b];
                Cout[v] = cv[b];
                xrow[v] = (uint8_t)(xv >> (8 * b));
            }
        } else {
            *reinterpret_cast<int4*>(grow + j0) = make_int4(gv[0], gv[1], gv[2], gv[3]);
            *reinterpret_cast<int4*>(Cout + j0) = make_int4(cv[0], cv[1], cv[2], cv[3]);
            *reinterpret_cast<uint32_t*>(xrow + j0) = xv;
        }
    }
    if (tid == 0 && rank == 0) d.E[p] = OVmin;
}

// (the cluster split's x bitmap beside the undo bitmap is counted for every
// shape, so that whether the move log fits does not depend on the split)
size_t tabu_smem_bytes(int n, int alpha)
{
    const int ld = round_up(n, kLdAlign);
    return kSmTs + 4 * (size_t)ld + 2 * ((size_t)ld / 8) + 2 * (size_t)alpha + 16;
}

bool tabu_log_in_smem(int n, int alpha) { return tabu_smem_bytes(n, alpha) <= kTabuSmemLimit; }

// Variables per CTA of a G-CTA split: a multiple of 128 covering n.
int tabu_slice(int n, int G)
{
    return G <= 1 ? round_up(n, kLdAlign) : round_up((n + G - 1) / G, kLdAlign);
}

template <int W, int MAXT, bool ASP, bool CK, bool SR, int G, bool PK = false>
static cudaError_t launch_tabu_w(const Dev& d, int alpha, int c, int sh, cudaStream_t s)
{
    const int slice = tabu_slice(d.n, G);
    int nt = ((G > 1 ? slice : d.n) + 4 * W - 1) / (4 * W);
    nt = (nt + 31) / 32 * 32;
    if (nt > MAXT) return cudaErrorInvalidConfiguration;
    const bool in_smem = tabu_log_in_smem(d.n, alpha);
    if (!in_smem && (!d.TL || d.tl_cap < alpha)) return cudaErrorInvalidValue;
    const size_t sm = tabu_smem_bytes(d.n, in_smem ? alpha : 0);
    auto kern = k_tabu<W, MAXT, ASP, CK, SR, G, PK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // as little shared memory as the block needs: the rest of the SM's 256 KB
    // is L1, which holds the recently moved rows of Q
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxL1);
    if (e != cudaSuccess) return e;
    Dev dd = d;
    if (in_smem) dd.TL = nullptr;  // the move log stays in shared memory
    if constexpr (G == 1) {
        kern<<<d.R, nt, sm, s>>>(dd, alpha, c, sh, slice);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(d.R * G), 1, 1);
        cfg.blockDim = dim3((unsigned)nt, 1, 1);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        // the CTAs of a cluster on different SMs: each brings its own issue slots
        at[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
        at[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicySpread;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        e = cudaLaunchKernelEx(&cfg, kern, dd, alpha, c, sh, slice);
        if (e != cudaSuccess) return e;
    }
    note_launch(1);
    return cudaGetLastError();
}

// One kernel shape: picks the build for aspiration, compact keys (sh > 0; only
// where CKOK; sh < 0: compact keys on parity labels, shift -sh, one CTA per
// replica, plain rows) and signed rows; G CTAs per replica.
template <int W, int MAXT, bool CKOK, int G>
static cudaError_t launch_shape(const Dev& d, int alpha, int c, int sh, bool asp, bool sr, cudaStream_t s)
{
    if constexpr (CKOK && G == 1) {
        if (sh < 0) {
            if (asp) return launch_tabu_w<W, MAXT, true, true, false, 1, true>(d, alpha, c, -sh, s);
            return launch_tabu_w<W, MAXT, false, true, false, 1, true>(d, alpha, c, -sh, s);
        }
    }
    if (sh < 0) sh = 0;   // (other shapes: the wide keys)
    if constexpr (CKOK) {
        if (sh) {
            if (asp) return sr ? launch_tabu_w<W, MAXT, true, true, true, G>(d, alpha, c, sh, s)
                               : launch_tabu_w<W, MAXT, true, true, false, G>(d, alpha, c, sh, s);
            return sr ? launch_tabu_w<W, MAXT, false, true, true, G>(d, alpha, c, sh, s)
                      : launch_tabu_w<W, MAXT, false, true, false, G>(d, alpha, c, sh, s);
        }
    }
    if (asp) return sr ? launch_tabu_w<W, MAXT, true, false, true, G>(d, alpha, c, 0, s)
                       : launch_tabu_w<W, MAXT, true, false, false, G>(d, alpha, c, 0, s);
    return sr ? launch_tabu_w<W, MAXT, false, false, true, G>(d, alpha, c, 0, s)
              : launch_tabu_w<W, MAXT, false, false, false, G>(d, alpha, c, 0, s);
}

// Variants of the Tabu kernel: 4-variable groups per thread W and the block
// size they are compiled for (fewer, wider threads cut the per-move
// reduction and barrier work; the block must still cover n).
struct TabuVariant { int W, maxt; };
static const TabuVariant kTabuVariants[] = {{1, 1024}, {2, 1024}, {3, 1024}, {4, 1024}, {4, 256}, {8, 256}};
constexpr int kNumTabuVariants = sizeof(kTabuVariants) / sizeof(kTabuVariants[0]);

bool tabu_variant_fits(int variant, int n, int G)
{
    if (variant < 0 || variant >= kNumTabuVariants) return false;
    if (G > 1 && (variant == 2 || variant == 3)) return false;  // built for one CTA per replica only
    const TabuVariant v = kTabuVariants[variant];
    const int cover = G > 1 ? tabu_slice(n, G) : n;
    return (cover + 4 * v.W - 1) / (4 * v.W) <= v.maxt;
}

int tabu_num_variants() { return kNumTabuVariants; }

// The default: the narrowest 1024-thread variant that covers n (the search
// is latency-bound and more threads per replica measured faster: at
// n = 2500, 640 threads 5.9 ms vs 160 threads 7.9 ms per 12 500 moves).
int tabu_default_variant(int n, int G)
{
    for (int v = 0; v < 4; ++v)
        if (tabu_variant_fits(v, n, G)) return v;
    return -1;
}

int tabu_key_shift(int n, long long gain_bound)
{
    int ib = 0;
    while ((1 << ib) <= n) ++ib;   // 2^ib > n: the index field never reads as a variable when all ones
    const int sh = ib + 1;
    return sh <= 30 && gain_bound + 1 < (1LL << (31 - sh)) ? sh : 0;
}

// The same for the keys on parity labels: the index field holds the rank in
// the larger parity class.
int tabu_key_shift_pk(int n_even, int n_odd, long long gain_bound)
{
    const int m = n_even > n_odd ? n_even : n_odd;
    int ib = 0;
    while ((1 << ib) <= m) ++ib;
    const int sh = ib + 1;
    return sh <= 30 && gain_bound + 1 < (1LL << (31 - sh)) ? sh : 0;
}

// CTAs per replica when the caller leaves it open.  The exchange through
// distributed shared memory costs about as much per move as the work a split
// saves up to n of several thousand (GB300, z = 32: n = 2500 one CTA 3.6 ms, two
// 5.7, four 5.8; n = 5000: 13.5, 16.4, 14.5; n = 10 000: 8.6, 8.7, 7.9 ms per
// search), so the split is the default only for large instances whose
// replicas leave three quarters of the SMs idle.
int tabu_default_cluster(int n, int R, int sm_count)
{
    return ((long long)R * 4 <= sm_count && n >= 8192) ? 4 : 1;
}

// variant: index into kTabuVariants; < 0 picks the default.  Compact keys are
// used when the instance's gain bound allows them, unless wide_keys is set.
// rows: 0 or 1 = plain rows (each variable's update is one dp4a with the move's
// sign in its byte lane; measured as fast as or faster than signed rows from
// n = 1000 to 13 001), 2 = signed rows where the state has them.
// cluster: CTAs per replica (1, 2, 4; 0 = tabu_default_cluster).
cudaError_t launch_tabu(const Dev& d, int alpha, int c, int variant, cudaStream_t s, bool aspiration, bool wide_keys,
                        int rows, int cluster)
{
    int sh = wide_keys ? 0 : tabu_key_shift(d.n, d.gain_bound);
    int G = cluster == 0 ? tabu_default_cluster(d.n, d.R, device_sm_count()) : cluster;
    if (G != 1 && G != 2 && G != 4) return cudaErrorInvalidValue;
    // a default split gives way to a kernel shape chosen for one CTA per replica
    if (cluster == 0 && variant >= 0 && !tabu_variant_fits(variant, d.n, G)) G = 1;
    if (variant < 0) variant = tabu_default_variant(d.n, G);
    if (!tabu_variant_fits(variant, d.n, G)) return cudaErrorInvalidConfiguration;
    // a gain bound one bit too wide for the compact keys: the parity labels, where the
    // instance has them (one CTA per replica)
    if (!wide_keys && sh == 0 && G == 1 && d.Qpk) sh = -tabu_key_shift_pk(d.pk_n0, d.n - d.pk_n0, d.gain_bound);
    const bool sr = d.Q2 != nullptr && rows == 2;
    // the 1024-thread shapes with 12 and 16 variables per thread would spill the
    // per-variable key constants: they keep the wide keys (and one CTA per replica)
    if (G == 2) {
        switch (variant) {
            case 0: return launch_shape<1, 1024, true, 2>(d, alpha, c, sh, aspiration, sr, s);
            case 1: return launch_shape<2, 1024, true, 2>(d, alpha, c, sh, aspiration, sr, s);
            case 4: return launch_shape<4, 256, true, 2>(d, alpha, c, sh, aspiration, sr, s);
            case 5: return launch_shape<8, 256, true, 2>(d, alpha, c, sh, aspiration, sr, s);
            default: return cudaErrorInvalidConfiguration;
        }
    }
    if (G == 4) {
        switch (variant) {
            case 0: return launch_shape<1, 1024, true, 4>(d, alpha, c, sh, aspiration, sr, s);
            case 1: return launch_shape<2, 1024, true, 4>(d, alpha, c, sh, aspiration, sr, s);
            case 4: return launch_shape<4, 256, true, 4>(d, alpha, c, sh, aspiration, sr, s);
            case 5: return launch_shape<8, 256, true, 4>(d, alpha, c, sh, aspiration, sr, s);
            default: return cudaErrorInvalidConfiguration;
        }
    }
    switch (variant) {
        case 0: return launch_shape<1, 1024, true, 1>(d, alpha, c, sh, aspiration, sr, s);
        case 1: return launch_shape<2, 1024, true, 1>(d, alpha, c, sh, aspiration, sr, s);
        case 2: return launch_shape<3, 1024, false, 1>(d, alpha, c, sh, aspiration, sr, s);
        case 3: return launch_shape<4, 1024, false, 1>(d, alpha, c, sh, aspiration, sr, s);
        case 4: return launch_shape<4, 256, true, 1>(d, alpha, c, sh, aspiration, sr, s);
        case 5: return launch_shape<8, 256, true, 1>(d, alpha, c, sh, aspiration, sr, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace icd2s
