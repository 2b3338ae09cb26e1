// kernels_anneal.cu -- the emulated Ising machine (Eq. 4, Algorithm 4).
//
// One warp per subQUBO S (m <= 32 P variables, ascending indices).  Lane l
// owns the P positions b = l + 32 q (q = 0..P-1), so the sweep order
// (position-major) is q-major across lanes: the first accepted position is
// found from P ballots without any shuffle.
//
// Gather (Eq. 4): Q' = Q[S, S] is staged as int8 in shared memory in a
// permuted layout, Qs[r][l P + q] = Q'[r][l + 32 q], so that the P entries a
// lane needs from row r are one contiguous P-byte load; the diagonal is
// stored as 0, so the row update of a flip leaves the flipped position alone.
// The boundary bias b_i = sum_{j not in S} 2 Q_ij x_j is never formed
// explicitly: the local gain of position a in the biased subQUBO,
// (1 - 2 x_a)(Q_aa + b_a + 2 sum_{c in S, c != a} Q_ac x_c), equals the global
// gain g_a, which the solution set already tracks exactly; so the gains of S
// are read straight from G.
//
// Anneal: sweeps k = 0..K-1 visit positions 0..m-1 in order; attempt (k, b)
// draws u = Philox(ctr = (k / 4, (TAG_ANNEAL << 24) | b, slot, iter)).word[k mod 4]
// and accepts iff l_b <= 0 or l_b * BETA[k] < NLOG[u >> 20].  For integer
// gains this is l_b <= LIM[k][u >> 20] with LIM[k][j] = floor((NLOG[j] - 1) /
// BETA[k]) (0 when NLOG[j] = 0, unbounded when BETA[k] = 0): a per-schedule
// table built once on the device (k_limtab), so an attempt costs one
// L1-resident load and one compare.  Each lane draws one Philox block per
// owned position every 4 sweeps, so no random words are wasted or exchanged.
//
// Rounds (one form of a sweep; the others are at anneal_one, whose per-sweep
// choice picks between them).  In a round every lane tests its unvisited
// positions against the current gains (P ballots).  For m <= 128 the warp
// also knows which positions are coupled (Q'_ab != 0; one bit mask per owned
// position, built from ballots during the gather): a tentative decision is
// final unless the position is coupled to an earlier tentatively accepted
// one, so the round ends at the first such position and every accept before
// it is applied -- those accepts are pairwise uncoupled, hence the gains each
// of them and every rejected position saw are exactly the gains of a
// one-at-a-time sweep.  For m > 128 a round ends at the first accept.  A
// sweep of a sparse subQUBO thus costs far fewer rounds than accepts; the
// trajectory is the sequential one bit for bit either way.
//
// Lanes keep the sign-free field h_b = (1 - 2 x_b) l_b: a flip of a adds
// 2 Q'_ab (1 - 2 x_a) to every h_b (one multiply-add with a warp-uniform
// factor, two rows per step so the shared-memory loads overlap) and only
// negates the sign of a itself.
//
// Output: the changed positions, either as a 0/1 mask [R][ldm] or appended
// to the replica's flip list (index | old x << 31) for k_apply; and the
// subQUBO energy change (sum of the accepted gains).
#include <climits>

#include "common.cuh"

namespace icd2s {

template <int P>
struct RowSeg;  // P bytes of a shared-memory row as one load
template <> struct RowSeg<1> { using T = uint8_t; };
template <> struct RowSeg<2> { using T = uint16_t; };
template <> struct RowSeg<4> { using T = uint32_t; };
template <> struct RowSeg<8> { using T = unsigned long long; };

// Largest gain accepted by the test l * beta < thr (see above).
__device__ __forceinline__ int accept_limit(uint32_t thr, uint32_t beta)
{
    if (thr == 0u) return 0;        // no positive gain passes
    if (beta == 0u) return INT_MAX; // every gain passes
    return (int)((thr - 1u) / beta);
}

// Anneals subQUBO s with the calling warp; Qs is the warp's (32 P)^2-byte
// shared-memory tile.  Warp-synchronous: no block-level barriers.
// SEQ: 0 = rounds (multi-accept for P <= 4, first accept for P = 8);
// 1 = position by position; 2 = position by position with the next
// position's decision taken for both outcomes of the current one; 3 = per
// sweep, rounds or by position (as 2), whichever the
// previous sweep's accepts predict cheaper.
template <int P, int SEQ>
__device__ __forceinline__ void anneal_one(const Dev& d, const AnnealArgs& a, int s, int lane, int8_t* Qs)
{
    using Seg = typename RowSeg<P>::T;
    constexpr int MC = 32 * P;  // row length (bytes) of the staged Q'
    uint32_t iter = a.iter_dev ? (uint32_t)*a.iter_dev : a.iter;

    const int p = s / a.per_replica;
    const int* S = nullptr;
    int m;
    int bbase = a.block_base;
    uint32_t slot = a.slot_base + (uint32_t)s;
    if (a.idx) {
        const int b0 = a.off[s];
        m = a.off[s + 1] - b0;
        S = a.idx + b0;
    } else {
        // contiguous blocks: block k = s mod per_replica of the launch's group for
        // replica p starts k blocks after block_base and counts as iteration iter + k
        // of Call_IM_Solution_Set; its random stream is the replica's (slot p)
        m = a.block_m;
        const int k = s - p * a.per_replica;
        bbase += k * a.block_m;
        iter += (uint32_t)k;
        slot = a.slot_base + (uint32_t)p;
    }
    const int ld = d.ld;

    int col[P];
    bool valid[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int b = lane + 32 * q;
        valid[q] = b < m;
        col[q] = valid[q] ? (S ? __ldg(S + b) : bbase + b) : 0;
    }
    // gather Q[S, S] into the permuted layout, diagonal as 0; for P <= 4 also
    // the coupling masks of the owned positions: bit L of nz[q][q2] is set
    // iff Q'[lane + 32 q][L + 32 q2] != 0 (ballots over the row's columns,
    // kept by the row's owner)
    constexpr bool kSparse = P <= 4;
    unsigned nz[kSparse ? P : 1][kSparse ? P : 1];
#pragma unroll
    for (int q = 0; q < (kSparse ? P : 1); ++q)
#pragma unroll
        for (int q2 = 0; q2 < (kSparse ? P : 1); ++q2) nz[q][q2] = 0u;
#pragma unroll 4
    for (int r = 0; r < m; ++r) {
        const int ir = S ? __ldg(S + r) : bbase + r;
        const int8_t* row = d.Q + (size_t)ir * ld;
        Seg packed = 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const bool take = valid[q] && (lane + 32 * q != r);
            const uint8_t v = take ? (uint8_t)__ldg(row + col[q]) : (uint8_t)0;
            packed |= (Seg)v << (8 * q);
        }
        *reinterpret_cast<Seg*>(Qs + (size_t)r * MC + lane * P) = packed;
        if constexpr (kSparse) {
            const bool owner = lane == (r & 31);
#pragma unroll
            for (int q2 = 0; q2 < P; ++q2) {
                const unsigned bm = __ballot_sync(0xffffffffu, ((packed >> (8 * q2)) & 0xff) != 0);
#pragma unroll
                for (int q = 0; q < P; ++q) nz[q][q2] = (owner && (r >> 5) == q) ? bm : nz[q][q2];
            }
        }
    }
    __syncwarp();

    // Owned positions keep the sign-free field h = (1 - 2x) l (l the gain) and
    // the sign sg = 1 - 2x, so l = sg h.  A flip of position a changes the
    // field of every other position b by 2 Q'_ab (1 - 2 x_a) -- one
    // multiply-add per owned position with a warp-uniform factor -- and leaves
    // its own field alone (Q'_aa is stored as 0); the flipped position only
    // changes its sign.
    int h[P], sg[P];
    unsigned X[P];         // warp-uniform: bit lane of X[q] = x at position lane + 32 q
    const int32_t* grow = d.G + (size_t)p * ld;
    const uint8_t* xrow = d.X + (size_t)p * ld;
    unsigned x0 = 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int xv = valid[q] ? (int)xrow[col[q]] : 0;
        sg[q] = 1 - 2 * xv;
        h[q] = valid[q] ? sg[q] * grow[col[q]] : 0;
        x0 |= (unsigned)xv << q;
        X[q] = __ballot_sync(0xffffffffu, xv != 0);
    }
    // The anneal's energy change comes at the end from the gains alone: for the
    // set F of positions whose value changed, E(x') - E(x) = (1/2) sum_{i in F}
    // (g_i(x) - g_i(x')) (flip them one after the other), so no step of a sweep
    // tracks it.  g0 = the gains at the start.
    int g0[P];
#pragma unroll
    for (int q = 0; q < P; ++q) g0[q] = sg[q] * h[q];

    // acceptance limits of 4 consecutive sweeps: Philox block k4/4 of every owned
    // position, looked up in the schedule's table (issued one block ahead, so
    // the table loads overlap the previous block's sweeps)
    auto load_limits = [&](int k4, int (&out)[4][P]) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const u32x4 u = philox10((uint32_t)(k4 >> 2), (kTagAnneal << 24) | (uint32_t)(lane + 32 * q), slot,
                                     iter, d.k0, d.k1);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = k4 + r < a.sweeps ? k4 + r : a.sweeps - 1;
                out[r][q] = valid[q] ? __ldg(a.limtab + (size_t)k * 4096 + (u.v[r] >> 20)) : INT_MIN;
            }
        }
    };
    // field updates of the flips of the positions in the warp-uniform mask A
    // of column block qf (all before their sign changes), two rows at a time
    // so that the shared-memory loads overlap
    auto apply_fields = [&](unsigned A, int qf) {
        while (A) {
            const int L1 = __ffs(A) - 1;
            A &= A - 1u;
            const bool two = A != 0u;
            const int L2 = two ? __ffs(A) - 1 : L1;
            A = two ? (A & (A - 1u)) : A;
            const Seg s1 = *reinterpret_cast<const Seg*>(Qs + (size_t)(L1 + 32 * qf) * MC + lane * P);
            const Seg s2 = *reinterpret_cast<const Seg*>(Qs + (size_t)(L2 + 32 * qf) * MC + lane * P);
            const int f1 = ((X[qf] >> L1) & 1u) ? -2 : 2;
            const int f2 = two ? (((X[qf] >> L2) & 1u) ? -2 : 2) : 0;
#pragma unroll
            for (int q = 0; q < P; ++q)
                h[q] += f1 * (int)(int8_t)(uint8_t)(s1 >> (8 * q)) + f2 * (int)(int8_t)(uint8_t)(s2 >> (8 * q));
        }
    };
    // sign changes (and accepted gains) of the flipped positions in A[q]
    auto flip_signs = [&](const unsigned (&A)[P]) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const bool f = (A[q] >> lane) & 1u;
            sg[q] = f ? -sg[q] : sg[q];
            X[q] ^= A[q];
        }
    };
    // One sweep, position by position in order: the owner's test against the
    // current gain decides (one ballot), and every lane adds the flipped
    // row's entries (zero factor when rejected), so there is no branch.  Row
    // b's segment is loaded one position ahead.
    auto sweep_seq = [&](const int (&lim)[P]) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            if (32 * q >= m) break;
            const int8_t* base = Qs + (size_t)(32 * q) * MC + lane * P;
            Seg rn = *reinterpret_cast<const Seg*>(base);
            bool t = sg[q] * h[q] <= lim[q];  // the decision input of position 32 q
            // x of position 32 q + L only changes at step L, so the block-start
            // values give every step's factor; the flips of the block are
            // collected apart and applied to X at its end (no chain through X)
            const unsigned xs = X[q];
            unsigned fl = 0u;
#pragma unroll(P <= 4 ? 32 : 8)
            for (int L = 0; L < 32; ++L) {
                // positions past m (checked every 8) are harmless: their test
                // fails (limit INT_MIN) and their tile rows are in bounds
                if ((L & 7) == 0 && 32 * q + L >= m) break;
                const Seg rb = rn;
                if (L < 31) rn = *reinterpret_cast<const Seg*>(base + (size_t)(L + 1) * MC);
                const int fx = ((xs >> L) & 1u) ? -2 : 2;  // 2 (1 - 2 x_b)
                // the simple form on request, otherwise both outcomes (measured faster
                // at every size once a step no longer tracks the energy)
                if constexpr (SEQ == 1) {
                    const bool acc = (__ballot_sync(0xffffffffu, t) >> L) & 1u;
                    const int f = acc ? fx : 0;
#pragma unroll
                    for (int q2 = 0; q2 < P; ++q2) h[q2] += f * (int)(int8_t)(uint8_t)(rb >> (8 * q2));
                    // a flipped position's sign changes at the end of the block: its
                    // test is not read again in this block
                    fl |= (unsigned)acc << L;
                    t = sg[q] * h[q] <= lim[q];
                } else {
                    // fields if b flips, and the next position's test for either outcome
                    int hp[P];
#pragma unroll
                    for (int q2 = 0; q2 < P; ++q2) hp[q2] = h[q2] + fx * (int)(int8_t)(uint8_t)(rb >> (8 * q2));
                    // (rejected, the state and so every lane's test stay as they are:
                    // up to 64 positions the test is kept, beyond it is taken again --
                    // each measured the faster there)
                    const bool tA = sg[q] * hp[q] <= lim[q];
                    const bool tR = P <= 2 ? t : sg[q] * h[q] <= lim[q];
                    const bool acc = (__ballot_sync(0xffffffffu, t) >> L) & 1u;
#pragma unroll
                    for (int q2 = 0; q2 < P; ++q2) h[q2] = acc ? hp[q2] : h[q2];
                    fl |= (unsigned)acc << L;
                    t = acc ? tA : tR;
                }
            }
            sg[q] = ((fl >> lane) & 1u) ? -sg[q] : sg[q];
            X[q] ^= fl;
        }
    };

    // One sweep in rounds (see above); returns the number of rounds.
    auto sweep_rounds = [&](const int (&lim)[P]) -> int {
        unsigned M[P];  // lanes whose position q has not been visited in this sweep
#pragma unroll
        for (int q = 0; q < P; ++q) M[q] = 0xffffffffu;
        int rounds = 0;
        if constexpr (kSparse) {
            // Rounds of several accepts: the tentative decisions of all
            // unvisited positions are taken against the current gains; a
            // position's decision is final unless it is coupled to an
            // earlier tentatively accepted position (whose flip would
            // change its gain).  The first such position ends the round:
            // the accepts before it are pairwise uncoupled, so applying
            // them in any order gives exactly the gains a one-at-a-time
            // sweep sees.
            const unsigned below = (1u << lane) - 1u;
            while (true) {
                ++rounds;
                unsigned B[P], any = 0u;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    B[q] = __ballot_sync(0xffffffffu, sg[q] * h[q] <= lim[q]) & M[q];
                    any |= B[q];
                }
                if (!any) break;
                unsigned Cf[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    unsigned c = nz[q][q] & B[q] & below;
#pragma unroll
                    for (int q2 = 0; q2 < q; ++q2) c |= nz[q][q2] & B[q2];
                    Cf[q] = __ballot_sync(0xffffffffu, c != 0u) & M[q];
                }
                int qc = P, Lc = 0;
#pragma unroll
                for (int q = P - 1; q >= 0; --q)
                    if (Cf[q]) { qc = q; Lc = __ffs(Cf[q]) - 1; }
                unsigned A[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    A[q] = q < qc ? B[q] : (q == qc ? (B[q] & ((1u << Lc) - 1u)) : 0u);
                    apply_fields(A[q], q);
                }
                flip_signs(A);
                if (qc == P) break;  // every remaining decision was final
#pragma unroll
                for (int q = 0; q < P; ++q)
                    M[q] = q < qc ? 0u : (q == qc ? (M[q] & (0xffffffffu << Lc)) : M[q]);
            }
        } else {
            // one accept per round: the first accepted unvisited position
            while (true) {
                ++rounds;
                unsigned B[P];
#pragma unroll
                for (int q = 0; q < P; ++q) B[q] = __ballot_sync(0xffffffffu, sg[q] * h[q] <= lim[q]) & M[q];
                int qs = -1;
                unsigned bq = 0u;
#pragma unroll
                for (int q = P - 1; q >= 0; --q)
                    if (B[q]) { qs = q; bq = B[q]; }
                if (qs < 0) break;
                const int L = __ffs(bq) - 1;
                unsigned A[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    A[q] = q == qs ? (1u << L) : 0u;
                    if (q == qs) apply_fields(A[q], q);
                }
                flip_signs(A);
#pragma unroll
                for (int q = 0; q < P; ++q)
                    M[q] = q < qs ? 0u : (q == qs ? (M[q] & (0xfffffffeu << L)) : M[q]);
            }
        }
        return rounds;
    };

    if constexpr (SEQ != 0) {
        // the limits of sweep k + 1 are loaded while sweep k runs; a Philox
        // block of each owned position covers 4 sweeps
        u32x4 ub[P];
        auto philox_block = [&](int k) {
#pragma unroll
            for (int q = 0; q < P; ++q)
                ub[q] = philox10((uint32_t)(k >> 2), (kTagAnneal << 24) | (uint32_t)(lane + 32 * q), slot, iter,
                                 d.k0, d.k1);
        };
        auto limits_of = [&](int k, int (&out)[P]) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int w = k & 3;
                const uint32_t u = w == 0 ? ub[q].v[0] : (w == 1 ? ub[q].v[1] : (w == 2 ? ub[q].v[2] : ub[q].v[3]));
                out[q] = valid[q] ? __ldg(a.limtab + (size_t)k * 4096 + (u >> 20)) : INT_MIN;
            }
        };
        // SEQ 3 picks the scheme per sweep from the previous sweep's accepts:
        // a round costs about as much as 7 positions of the by-position sweep,
        // and the last rounds sweep gives the rounds per accept.  Both schemes
        // give the same trajectory, so the choice only changes the time.
        int a_prev = m, r_last = 1, a_last = kSparse ? 3 : 1;
        int limN[P];
        philox_block(0);
        limits_of(0, limN);
#pragma unroll 1
        for (int k = 0; k < a.sweeps; ++k) {
            int lim[P];
#pragma unroll
            for (int q = 0; q < P; ++q) lim[q] = limN[q];
            if (k + 1 < a.sweeps) {
                if (((k + 1) & 3) == 0) philox_block(k + 1);
                limits_of(k + 1, limN);
            }
            if constexpr (SEQ == 3) {
                unsigned Xs[P];
#pragma unroll
                for (int q = 0; q < P; ++q) Xs[q] = X[q];
                const bool rounds_now = 7 * (r_last * a_prev + a_last) < m * a_last;
                int r = 0;
                if (rounds_now) r = sweep_rounds(lim);
                else sweep_seq(lim);
                int acc = 0;
#pragma unroll
                for (int q = 0; q < P; ++q) acc += __popc(X[q] ^ Xs[q]);
                a_prev = acc;
                if (rounds_now && acc > 0) { r_last = r; a_last = acc; }
            } else {
                sweep_seq(lim);
            }
        }
    } else {
        int limA[4][P];
        load_limits(0, limA);
        for (int k4 = 0; k4 < a.sweeps; k4 += 4) {
            int limB[4][P];
            if (k4 + 4 < a.sweeps) load_limits(k4 + 4, limB);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (k4 + r >= a.sweeps) break;
                sweep_rounds(limA[r]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < P; ++q) limA[r][q] = limB[r][q];
        }
    }

    unsigned changed = 0;
#pragma unroll
    for (int q = 0; q < P; ++q) changed |= (unsigned)(valid[q] && (((X[q] >> lane) & 1u) != ((x0 >> q) & 1u))) << q;
    if (a.mask) {
#pragma unroll
        for (int q = 0; q < P; ++q)
            if ((changed >> q) & 1u) a.mask[(size_t)p * a.ldm + col[q]] = 1;
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
    long long dEl = 0;  // twice the energy change
#pragma unroll
    for (int q = 0; q < P; ++q)
        if ((changed >> q) & 1u) dEl += (long long)g0[q] - (long long)(sg[q] * h[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dEl += __shfl_xor_sync(0xffffffffu, dEl, o);
    if (lane == 0) {
        if (a.dE) a.dE[s] = dEl / 2;
        if (a.attempts_acc) atomicAdd(reinterpret_cast<unsigned long long*>(a.attempts_acc),
                                      (unsigned long long)a.sweeps * (unsigned long long)m);
    }
}

// One warp per subQUBO, subQUBO s = CTA * warps + warp (sizes up to 32 P).
template <int P, int SEQ>
__global__ __launch_bounds__(128) void k_anneal(Dev d, AnnealArgs a)
{
    constexpr int MC = 32 * P;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int s = blockIdx.x * wpb + wib;
    if (s >= a.count) return;  // whole warp leaves; no block-level barriers below
    const int se = a.group_stride > 0 ? s * a.group_stride + a.group_k : s;
    anneal_one<P, SEQ>(d, a, se, lane, reinterpret_cast<int8_t*>(smem) + (size_t)wib * MC * MC);
}

// Persistent batch of subQUBOs of uneven size: every warp takes the next
// subQUBO from a device queue in largest-first order (a.order, sizes
// descending, built by k_sizes) and anneals it with the narrowest lane layout
// that fits its size.  The queue is one counter; no warp ever waits on
// another, and each subQUBO's result does not depend on which warp runs it.
template <int PMAX, int SEQ>
__global__ __launch_bounds__(128) void k_anneal_queue(Dev d, AnnealArgs a)
{
    constexpr int MC = 32 * PMAX;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int8_t* Qs = reinterpret_cast<int8_t*>(smem) + (size_t)wib * MC * MC;
    while (true) {
        int next = 0;
        if (lane == 0) next = atomicAdd(a.queue, 1);
        next = __shfl_sync(0xffffffffu, next, 0);
        if (next >= a.count) break;
        const int s = a.order[next];
        const int m = a.off[s + 1] - a.off[s];
        if (m <= 32) anneal_one<1, SEQ>(d, a, s, lane, Qs);
        else if (m <= 64) { if constexpr (PMAX >= 2) anneal_one<2, SEQ>(d, a, s, lane, Qs); }
        else if (m <= 128) { if constexpr (PMAX >= 4) anneal_one<4, SEQ>(d, a, s, lane, Qs); }
        else { if constexpr (PMAX >= 8) anneal_one<8, SEQ>(d, a, s, lane, Qs); }
        __syncwarp();  // the tile is reused by the next subQUBO
    }
}

// LIM[k][j] for the whole schedule: the largest gain that attempt (k, j) accepts.
__global__ void k_limtab(const uint32_t* __restrict__ beta, int sweeps, const uint32_t* __restrict__ nlog,
                         int* __restrict__ lim)
{
    const size_t total = (size_t)sweeps * 4096;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
        lim[e] = accept_limit(nlog[e & 4095], beta[e >> 12]);
}

cudaError_t launch_limtab(const uint32_t* beta, int sweeps, const uint32_t* nlog, int* lim, cudaStream_t s)
{
    const size_t total = (size_t)sweeps * 4096;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_limtab<<<blocks, 256, 0, s>>>(beta, sweeps, nlog, lim);
    note_launch(1);
    return cudaGetLastError();
}

template <int P, int SEQ>
static cudaError_t launch_anneal_p(const Dev& d, const AnnealArgs& a, int wpb, cudaStream_t s)
{
    constexpr int MC = 32 * P;
    const size_t sm = (size_t)wpb * MC * MC;
    cudaError_t e = cudaFuncSetAttribute(k_anneal<P, SEQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = (a.count + wpb - 1) / wpb;
    k_anneal<P, SEQ><<<blocks, 32 * wpb, sm, s>>>(d, a);
    note_launch(1);
    return cudaGetLastError();
}

// Persistent launch: as many warps as fit on the GPU at once (by shared
// memory), never more than there are subQUBOs.
template <int PMAX, int SEQ>
static cudaError_t launch_anneal_queue(const Dev& d, const AnnealArgs& a, int wpb, cudaStream_t s)
{
    constexpr int MC = 32 * PMAX;
    const size_t per_warp = (size_t)MC * MC;
    const size_t sm = (size_t)wpb * per_warp;
    cudaError_t e = cudaFuncSetAttribute(k_anneal_queue<PMAX, SEQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int ctas_per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, k_anneal_queue<PMAX, SEQ>, 32 * wpb, sm);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    int blocks = device_sm_count() * ctas_per_sm;
    const int need = (a.count + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    k_anneal_queue<PMAX, SEQ><<<blocks, 32 * wpb, sm, s>>>(d, a);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_anneal(const Dev& d, const AnnealArgs& a, cudaStream_t s)
{
    if (a.count <= 0) return cudaSuccess;
    const int m = a.m_max;
    // warps (subQUBOs) per CTA: shared memory is 1 KiB / 4 KiB / 16 KiB / 64 KiB per warp
    int wpb = a.warps_per_cta;
    if (wpb <= 0) wpb = m <= 128 ? 2 : 1;
    if (m > 128 && wpb > 3) wpb = 3;
    if (wpb > 4) wpb = 4;
    const int seq = a.scheme == 0 ? 3 : a.scheme - 1;
#define ICD2S_ANNEAL_SEQ(SQ)                                           \
    if (a.queue) {                                                     \
        if (m <= 32) return launch_anneal_queue<1, SQ>(d, a, wpb, s);  \
        if (m <= 64) return launch_anneal_queue<2, SQ>(d, a, wpb, s);  \
        if (m <= 128) return launch_anneal_queue<4, SQ>(d, a, wpb, s); \
        if (m <= 256) return launch_anneal_queue<8, SQ>(d, a, wpb, s); \
        return cudaErrorInvalidValue;                                  \
    }                                                                  \
    if (m <= 32) return launch_anneal_p<1, SQ>(d, a, wpb, s);          \
    if (m <= 64) return launch_anneal_p<2, SQ>(d, a, wpb, s);          \
    if (m <= 128) return launch_anneal_p<4, SQ>(d, a, wpb, s);         \
    if (m <= 256) return launch_anneal_p<8, SQ>(d, a, wpb, s);         \
    return cudaErrorInvalidValue;
    switch (seq) {
        case 0: { ICD2S_ANNEAL_SEQ(0) }
        case 1: { ICD2S_ANNEAL_SEQ(1) }
        case 2: { ICD2S_ANNEAL_SEQ(2) }
        default: { ICD2S_ANNEAL_SEQ(3) }
    }
#undef ICD2S_ANNEAL_SEQ
}

}  // namespace icd2s
