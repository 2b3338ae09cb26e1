// common.cuh -- internal declarations of the IC-D2S sm_103a library.
//
// Device layouts (all row-major, rows padded to LD = round_up(n, 128) bytes /
// elements so that every row starts 16-byte aligned and vector loads never
// need a tail case; padding entries are zero and never selected):
//   Q      int8  [n][LD]       the QUBO matrix (Eq. 1)
//   diag   int32 [LD]          Q_ii
//   etahat int32 [LD]          eta_j / max eta in Q16 (Eq. 6)
//   X      uint8 [R][LD]       solutions (replicas)
//   G      int32 [R][LD]       1-flip gains g_i = (1-2x_i)(Q_ii + 2 sum_{j!=i} Q_ij x_j)
//   E      int64 [R]           energies (Eq. 1)
//   T, C   int32 [R][LD]       Tabu toggle counts and final tabu memory (Algorithm 1)
//   A      int32 [R][LD]       aggregated control parameter (Algorithm 3, Q16)
//   order  int32 [R][LD]       variables ranked by (A desc, index asc)
//   sel    uint8 [R][LD]       1 where the variable is in S' (last selection)
//   FL     int32 [R][LD]       flip lists: index | (old x << 31), FCNT[R] entries
//   ACC    int32 [S][R][LD]    partial sums of a split write-back (one plane per split)
//   H      int32 [R][LD]       selection hit counts (Ising-machine calls that included j)
//   F      float [R][LD][6]    features of the learned selection at selection time
//   score  float [R][LD]       proposal-network scores
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace icd2s {

constexpr int kLdAlign = 128;
constexpr int kMaxN = 16384;
constexpr int kMaxM = 256;
constexpr int kMaxReplicas = 4096;
constexpr int kMaxSweeps = 16384;   // the acceptance-limit table is sweeps x 4096 int32

constexpr uint32_t kTagInit = 1u, kTagAnneal = 2u, kTagMut = 3u, kTagSize = 4u, kTagMlpInit = 5u, kTagTrain = 6u,
                   kTagRank = 7u;

// Proposal network 6-64-64-1: flat parameters W1[64][6], b1[64], W2[64][64],
// b2[64], w3[64], b3 (row o of W1/W2 = weights into hidden unit o).
constexpr int kOffW1 = 0, kOffB1 = 384, kOffW2 = 448, kOffB2 = 4544, kOffW3 = 4608, kOffB3 = 4672;
constexpr int kNPar = 4673;
constexpr int kNParPad = 4676;     // float4-aligned shared copy
constexpr int kPartStride = 4680;  // per-CTA partial gradient + loss

inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): the two Philox
// multipliers act on words 0 and 2; the high halves are mixed with words 1/3
// and the round key; the key advances by the two Weyl increments per round.
struct u32x4 { uint32_t v[4]; };

__host__ __device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#if defined(__CUDA_ARCH__)
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
#else
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0, m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
        const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
#endif
        const uint32_t t0 = hi1 ^ c1 ^ k0, t2 = hi0 ^ c3 ^ k1;
        c0 = t0; c1 = lo1; c2 = t2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    u32x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Device view of one problem + solution set, passed by value to kernels.
struct Dev {
    const int8_t* Q;       // [n][ld]
    const int32_t* diag;   // [ld]
    const int32_t* etahat; // [ld]
    int n, ld, R;
    uint8_t* X; int32_t* G; int64_t* E;
    int32_t* T; int32_t* C;
    int32_t* gamma; int32_t* A; int32_t* delta; int32_t* order; uint8_t* sel;
    int32_t* FL; int32_t* FCNT; unsigned long long* DEACC; unsigned int* DONE;
    uint8_t* best_x; int64_t* best_E; int32_t* flags; // flags[0] improved, [1] stale, [2] error,
                                                       // [3] last best replica, [4] improved in the
                                                       // finished iteration, [5] its log slot,
                                                       // [6] a Tabu cluster exchange timed out,
                                                       // [7] stamp of the last best update
    int32_t* H; float* F; float* score;
    int32_t* ACC; unsigned* TT; int apply_splits;     // split write-back: partial sums, tile tickets
    uint32_t k0, k1; // Philox key = seed halves
    long long gain_bound;  // max over j and x of |g_j| (the Tabu keys' width depends on it)
    const int8_t* Q2;      // [2n][ld] signed rows: row 2i + x = (1 - 2x) Q_i (null unless asked for)
    // Q on parity labels for the Tabu keys (null unless the instance needs them):
    // Qpk[L][M] = Q[pk_perm[L]][pk_perm[M]], the pk_n0 variables with an even Q_jj
    // first, each class in index order
    const int8_t* Qpk; const int32_t* pk_perm; int pk_n0;
    uint16_t* TL; long long tl_cap;  // Tabu move logs [R][tl_cap] for searches whose log exceeds shared memory
    // replica sharding: these R replicas are replicas p0 .. p0 + R - 1 of a set of
    // z_total (every random stream is keyed by the global replica index; gamma is
    // taken over all z_total replicas)
    int p0, z_total;
};

// Counts kernel launches (process-wide, for reporting).
void note_launch(int kernels);

// Sets the calling thread's icd2s_last_error() message.
void set_error_message(const char* msg);

// ---- launchers (each returns cudaGetLastError() of its launch) ----
// eta_max[0] receives max_j eta_j (eta_j = sum_i |Q_ij|), eta_max[1] the
// number of entries equal to -128; gain_max (zeroed by the caller) the largest
// |g_j| over all j and x.
cudaError_t launch_prepare(const int8_t* Q, int n, int ld, int32_t* eta, int32_t* etahat, int32_t* diag,
                           int* mismatches, int* eta_max, int* gain_max, cudaStream_t s);
// Qpk[L][M] = Q[perm[L]][perm[M]] for L, M < n; padding columns 0.
cudaError_t launch_relabel(const int8_t* Q, const int32_t* perm, int n, int ld, int8_t* Qpk, cudaStream_t s);
// Q2[2i + x][j] = (1 - 2x) Q[i][j] (Q without -128 entries; padding columns 0).
cudaError_t launch_signed_rows(const int8_t* Q, int n, int ld, int8_t* Q2, cudaStream_t s);
cudaError_t launch_init_x(const Dev& d, cudaStream_t s);
cudaError_t launch_recompute(const Dev& d, const uint8_t* X, int ldx, int R, int32_t* G, int64_t* E,
                             cudaStream_t s);  // gains + energies of X (padded rows)
cudaError_t launch_pad_rows(const uint8_t* src, int n, int rows, uint8_t* dst, int ld, cudaStream_t s);
// variant: kernel shape (< 0: default); aspiration: Tabu with the aspiration criterion.
// wide_keys: the two-reduction keys even where the compact ones apply;
// rows: 0 = the default choice of plain or signed rows, 1 = plain rows (the sign
// applied per variable), 2 = signed rows where d.Q2 exists.
// cluster: CTAs per replica, 1, 2 or 4 (a thread-block cluster splitting the
// variables; compact keys only, else one CTA), 0 = tabu_default_cluster.
cudaError_t launch_tabu(const Dev& d, int alpha, int c, int variant, cudaStream_t s, bool aspiration = false,
                        bool wide_keys = false, int rows = 0, int cluster = 1);
// Shift of the compact Tabu keys for n and the instance's gain bound (0: they do not apply).
int tabu_key_shift(int n, long long gain_bound);
// The shift of the compact keys on parity labels (0: they do not apply either).
int tabu_key_shift_pk(int n_even, int n_odd, long long gain_bound);
size_t tabu_smem_bytes(int n, int alpha);
constexpr size_t kTabuSmemLimit = 227 * 1024;
// false: the Tabu move log of alpha moves goes to global memory (Dev::TL, tl_cap >= alpha)
bool tabu_log_in_smem(int n, int alpha);
int tabu_slice(int n, int G);
int tabu_default_cluster(int n, int R, int sm_count);
// gamma (Eq. 8) from column counts: counts[j] = sum over all d.z_total replicas of
// x_pj (null: the counts of this state's own replicas, whose d.R must then be
// d.z_total)
cudaError_t launch_gamma(const Dev& d, const int32_t* counts, cudaStream_t s);
// counts[j] = sum over this state's replicas of x_pj (j < n)
cudaError_t launch_colsum(const Dev& d, int32_t* counts, cudaStream_t s);
// Iteration context read by the kernels of a captured outer iteration (a CUDA
// graph replays the same launches, so the iteration number and the mutation
// rate come from device memory): iter_dev[0] = t, rates[t] = the rate.  When
// iter_dev is null the kernels use their `iter` / `rate` arguments.
// p0: global index of replica 0 (the sizes are drawn per global replica)
cudaError_t launch_sizes(int R, int K, int m_min, int m_max, uint32_t k0, uint32_t k1, uint32_t iter,
                         const int32_t* iter_dev, int32_t* off, int32_t* order, int32_t* queue, cudaStream_t s,
                         int p0 = 0);
// mode: 0 rank S' by A; 1 by d.score; 2 by d.score on even replicas.  Hit
// counts d.H are incremented for S' when count_hits.
// ablation 2 (No_SM): A is replaced by the random key Philox(ctr = (j / 4, 7 << 24, p, t)) >> 1.
cudaError_t launch_select(const Dev& d, int64_t w1, int64_t w2, int64_t w3, int K, const int32_t* off,
                          int32_t* idx, int mode, bool count_hits, cudaStream_t s, uint32_t iter = 0,
                          const int32_t* iter_dev = nullptr, int ablation = 0);
// half: every candidate flips with probability 1/2 (No_SM) instead of the normalised A.
cudaError_t launch_mutate(const Dev& d, int K, const int32_t* off, double rate, uint32_t iter,
                          const int32_t* iter_dev, const double* rates, uint8_t* mask, int ldm, cudaStream_t s,
                          bool half = false);
struct AnnealArgs {
    const int32_t* idx; const int32_t* off; int count; int per_replica;
    int block_m; int block_base;          // idx == nullptr: contiguous block [base, base+m)
    const int* limtab; int sweeps; uint32_t iter; uint32_t slot_base;   // limtab: [sweeps][4096]
    uint8_t* mask; int ldm;               // mask output (nullptr: flip lists FL/FCNT)
    int64_t* dE; int64_t* attempts_acc;   // optional outputs
    int m_max;
    int warps_per_cta;                    // 0: default
    const int32_t* iter_dev;              // non-null: the iteration number is read from here
    int32_t* queue;                       // non-null: persistent kernel, subQUBOs taken in `order`
    const int32_t* order;
    int group_stride, group_k;            // group_stride > 0: launch subQUBO s is s * group_stride + group_k
                                          // (one group of every replica, Gauss-Seidel order)
    int scheme;                           // sweep scheme: 0 default (4), 1 rounds, 2 by position, 3 by
                                          // position with both outcomes of the next test, 4 per sweep 1 or
                                          // by position
};
int device_sm_count();
bool tabu_variant_fits(int variant, int n, int G = 1);
int tabu_num_variants();
int tabu_default_variant(int n, int G = 1);
cudaError_t launch_anneal(const Dev& d, const AnnealArgs& a, cudaStream_t s);
cudaError_t launch_exact(const Dev& d, const AnnealArgs& a, cudaStream_t s);  // exact IM, m <= 24
cudaError_t launch_limtab(const uint32_t* beta, int sweeps, const uint32_t* nlog, int* lim, cudaStream_t s);
cudaError_t launch_compact_mask(const Dev& d, const uint8_t* mask, int ldm, cudaStream_t s);
cudaError_t launch_apply(const Dev& d, cudaStream_t s);
int apply_splits_for(int ld, int R);   // CTAs per column tile for long flip lists
int apply_tiles(int ld);
// log_ctl (iteration end only, may be null): {entries written, capacity} of the improvement log.
// stamp: when this update happens (3 t + phase + 1 inside iteration t, 0
// outside one; with iter_dev the t comes from *iter_dev); flags[7] keeps the
// stamp of the update that last set the best, which orders equal energies of
// different replica shards by the time they were reached.
cudaError_t launch_best(const Dev& d, int64_t* trace_slot, int iter_end, int32_t* iter_dev, cudaStream_t s,
                        int32_t* log_ctl = nullptr, int phase = -1, int t = 0);
cudaError_t launch_set_iter(int32_t* iter_dev, int t, cudaStream_t s);
// dense refresh on the tensor cores (kernels_refresh.cu)
cudaError_t launch_to_bf16(const void* src, bool is_signed, size_t count, void* dst, cudaStream_t s);
// H[R][ld] += Q X^T (BF16 copies of Q and X), persistent over the SMs: bn
// replicas and rows (128 / 256) of Q per tile, ctas persistent CTAs (0: one
// per SM); every pipeline wait bounded by wait_ns, after which err is raised;
// skip_loads: fault injection for tests (the producer issues no loads)
cudaError_t launch_refresh_mma(const void* Qb, const void* Xb, int n, int R, int ld, int32_t* H, int* err, int bn,
                               int ctas, int rows, unsigned long long wait_ns, int skip_loads, cudaStream_t s);
// the same with Q read as int8 bytes and converted to BF16 in shared memory
// (one tile and K split per CTA: splits K splits, 0 = a single wave)
cudaError_t launch_refresh_i8(const void* Q8, const void* Xb, int n, int R, int ld, int32_t* H, int* err, int bn,
                              int splits, unsigned long long wait_ns, int skip_loads, cudaStream_t s);
cudaError_t launch_finish_gains(const int32_t* diag, int n, int ld, const uint8_t* X, int32_t* G, int64_t* E, int R,
                                cudaStream_t s);
// learned selection (kernels_mlp.cu)
cudaError_t launch_features(const Dev& d, int t, const int32_t* iter_dev, int alpha, int c, int32_t* gmax,
                            cudaStream_t s);
cudaError_t launch_score(const float* F, long long rows, const void* Wb, float* out, cudaStream_t s);
size_t mlp_partial_floats(long long batch);
cudaError_t launch_mlp_grad(const float* F, const uint8_t* y, long long rows, long long batch, uint32_t step,
                            uint32_t k0, uint32_t k1, const void* Wb, float pos_weight, float* partial,
                            float* grad_out, float* loss_out, float* master, float* mom, float* vel, void* Wb_out,
                            int adam, float lr, float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s,
                            bool tensor_cores = false);
cudaError_t launch_round_bf16(const float* master, void* Wb, cudaStream_t s);
cudaError_t launch_log(const Dev& d, uint8_t* prev_x, float* LF, uint8_t* LY, int32_t* lrep, cudaStream_t s);
cudaError_t launch_compare(const int32_t* G1, const int64_t* E1, const int32_t* G2, const int64_t* E2, int n, int ld,
                           int R, int* mismatches, cudaStream_t s);

}  // namespace icd2s
