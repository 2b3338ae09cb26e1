// kernels_state.cu -- initial solutions, exact gain/energy recompute,
// Deviation_Extraction (gamma, Eq. 8) and best-solution tracking.
#include <climits>

#include "common.cuh"

namespace icd2s {

// ---------------------------------------------------------------------------
// Generate_Initial_Solution_Set (Algorithm 2): x[p][j] is bit (j mod 32) of
// word ((j / 32) mod 4) of Philox(ctr = (j / 128, TAG_INIT << 24, p, 0)), p
// the global replica index (p0 + the local one).
// One thread per (replica, 128 variables); padding bytes are written as 0.
// ---------------------------------------------------------------------------
__global__ void k_init_x(uint8_t* X, int n, int ld, int R, int p0, uint32_t k0, uint32_t k1)
{
    const int blocks = ld / 128;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= R * blocks) return;
    const int p = gid / blocks, b = gid % blocks;
    const u32x4 w = philox10((uint32_t)b, kTagInit << 24, (uint32_t)(p0 + p), 0u, k0, k1);
    uint8_t* row = X + (size_t)p * ld + (size_t)b * 128;
#pragma unroll
    for (int v = 0; v < 8; ++v) {   // 8 x 16 bytes
        uint32_t packed[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t word = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int jj = v * 16 + q * 4 + t;            // 0..127
                const int j = b * 128 + jj;
                const uint32_t bit = (w.v[(jj >> 5) & 3] >> (jj & 31)) & 1u;
                word |= (j < n ? bit : 0u) << (8 * t);
            }
            packed[q] = word;
        }
        *reinterpret_cast<uint4*>(row + v * 16) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
}

cudaError_t launch_init_x(const Dev& d, cudaStream_t s)
{
    const int total = d.R * (d.ld / 128);
    k_init_x<<<(total + 127) / 128, 128, 0, s>>>(d.X, d.n, d.ld, d.R, d.p0, d.k0, d.k1);
    note_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// H[p][j] = sum_k Q[j][k] x[p][k]  (int8 x {0,1}, exact int32) with dp4a on
// 64 x 64 output tiles; the k loop walks 64-byte chunks staged in shared
// memory.  Rows are padded with zeros to ld, so no tail handling in k.  With
// few tiles the k range is split over gridDim.z CTAs whose partial sums are
// added into H (zeroed first) with integer atomics: exact in any order.
// ---------------------------------------------------------------------------
constexpr int kGT = 64;          // tile edge (rows j and replicas p)
constexpr int kGK = 64;          // bytes of k per stage
constexpr int kGS = kGK / 4 + 1; // row stride in ints (padding against bank conflicts)

__global__ __launch_bounds__(256) void k_hgemm(const int8_t* __restrict__ Q, int n, int ld,
                                               const uint8_t* __restrict__ X, int ldx, int R,
                                               int32_t* __restrict__ H, int ldh)
{
    __shared__ int Qs[kGT * kGS];
    __shared__ int Xs[kGT * kGS];
    const int t = threadIdx.x;
    const int j0 = blockIdx.x * kGT, p0 = blockIdx.y * kGT;
    const int tj = t % 16, tp = t / 16;
    int acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    const int lr = t / 4, lseg = (t % 4) * 16;  // loader: row, byte offset within the chunk
    const int chunks = ld / kGK, ks = (int)gridDim.z;
    const int kb = (int)((long long)chunks * blockIdx.z / ks) * kGK, ke = (int)((long long)chunks * (blockIdx.z + 1) / ks) * kGK;
    for (int k0 = kb; k0 < ke; k0 += kGK) {
        uint4 qv = make_uint4(0, 0, 0, 0), xv = make_uint4(0, 0, 0, 0);
        if (j0 + lr < n) qv = __ldg(reinterpret_cast<const uint4*>(Q + (size_t)(j0 + lr) * ld + k0 + lseg));
        if (p0 + lr < R) xv = *reinterpret_cast<const uint4*>(X + (size_t)(p0 + lr) * ldx + k0 + lseg);
        __syncthreads();
        int* qd = Qs + lr * kGS + lseg / 4;
        int* xd = Xs + lr * kGS + lseg / 4;
        qd[0] = (int)qv.x; qd[1] = (int)qv.y; qd[2] = (int)qv.z; qd[3] = (int)qv.w;
        xd[0] = (int)xv.x; xd[1] = (int)xv.y; xd[2] = (int)xv.z; xd[3] = (int)xv.w;
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kGK / 4; ++kk) {
            int qa[4], xb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) qa[a] = Qs[(tj * 4 + a) * kGS + kk];
#pragma unroll
            for (int b = 0; b < 4; ++b) xb[b] = Xs[(tp * 4 + b) * kGS + kk];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = __dp4a(qa[a], xb[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int p = p0 + tp * 4 + b;
        if (p >= R) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int j = j0 + tj * 4 + a;
            if (j < n) {
                if (ks == 1) H[(size_t)p * ldh + j] = acc[a][b];
                else atomicAdd(&H[(size_t)p * ldh + j], acc[a][b]);
            }
        }
    }
}

// In place: H (incl. diagonal) -> g, and E = sum_j x_j (Q_jj + h_j).
__global__ __launch_bounds__(256) void k_finish_gains(const int32_t* __restrict__ diag, int n, int ld,
                                                      const uint8_t* __restrict__ X, int ldx,
                                                      int32_t* G, int64_t* E)
{
    const int p = blockIdx.x;
    const uint8_t* x = X + (size_t)p * ldx;
    int32_t* g = G + (size_t)p * ld;
    long long e = 0;
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        if (j >= n) { g[j] = 0; continue; }
        const int xj = x[j], dj = diag[j];
        const int h = g[j] - dj * xj;                    // off-diagonal field
        g[j] = (1 - 2 * xj) * (dj + 2 * h);
        e += (long long)xj * (dj + h);
    }
    __shared__ long long red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        e = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (threadIdx.x == 0) E[p] = e;
    }
}

cudaError_t launch_recompute(const Dev& d, const uint8_t* X, int ldx, int R, int32_t* G, int64_t* E,
                             cudaStream_t s)
{
    dim3 grid((d.n + kGT - 1) / kGT, (R + kGT - 1) / kGT);
    // k splits so that about two CTAs per SM run, each over at least 4 chunks of k
    const int tiles = (int)(grid.x * grid.y), chunks = d.ld / kGK;
    int ks = (2 * device_sm_count() + tiles - 1) / tiles;
    if (ks > chunks / 4) ks = chunks / 4;
    if (ks < 1) ks = 1;
    grid.z = (unsigned)ks;
    cudaError_t e;
    if (ks > 1 && (e = cudaMemsetAsync(G, 0, sizeof(int32_t) * (size_t)R * d.ld, s)) != cudaSuccess) return e;
    k_hgemm<<<grid, 256, 0, s>>>(d.Q, d.n, d.ld, X, ldx, R, G, d.ld);
    note_launch(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish_gains<<<R, 256, 0, s>>>(d.diag, d.n, d.ld, X, ldx, G, E);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_finish_gains(const int32_t* diag, int n, int ld, const uint8_t* X, int32_t* G, int64_t* E, int R,
                                cudaStream_t s)
{
    k_finish_gains<<<R, 256, 0, s>>>(diag, n, ld, X, ld, G, E);
    note_launch(1);
    return cudaGetLastError();
}

// dense [rows][n] -> padded [rows][ld] (zero padding)
__global__ void k_pad_rows(const uint8_t* __restrict__ src, int n, int rows, uint8_t* __restrict__ dst, int ld)
{
    const size_t total = (size_t)rows * ld;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / ld, c = i % ld;
        dst[i] = c < (size_t)n ? src[r * n + c] : (uint8_t)0;
    }
}

cudaError_t launch_pad_rows(const uint8_t* src, int n, int rows, uint8_t* dst, int ld, cudaStream_t s)
{
    const size_t total = (size_t)rows * ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_pad_rows<<<blocks, 256, 0, s>>>(src, n, rows, dst, ld);
    note_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deviation_Extraction (Eq. 8): gamma_j = 1 - |sum_p x_pj - z/2| / (z/2)
//                                       = (z - |2 sum_p x_pj - z|) / z, Q16 floor,
// the sum over all z replicas: this state's own (counts == null), or the
// column counts of every replica shard added up by the caller.
// ---------------------------------------------------------------------------
__global__ void k_gamma(const uint8_t* __restrict__ X, int n, int ld, int R, const int32_t* __restrict__ counts,
                        int z, int32_t* __restrict__ gamma)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ld) return;
    if (j >= n) { gamma[j] = 0; return; }
    int col = 0;
    if (counts) {
        col = counts[j];
    } else {
        for (int p = 0; p < R; ++p) col += X[(size_t)p * ld + j];
    }
    const int dev = abs(2 * col - z);
    gamma[j] = (int32_t)(((long long)(z - dev) * 65536) / z);
}

cudaError_t launch_gamma(const Dev& d, const int32_t* counts, cudaStream_t s)
{
    k_gamma<<<(d.ld + 255) / 256, 256, 0, s>>>(d.X, d.n, d.ld, d.R, counts, counts ? d.z_total : d.R, d.gamma);
    note_launch(1);
    return cudaGetLastError();
}

// column counts of this state's replicas (the shard's part of Eq. 8's sum)
__global__ void k_colsum(const uint8_t* __restrict__ X, int n, int ld, int R, int32_t* __restrict__ counts)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int col = 0;
    for (int p = 0; p < R; ++p) col += X[(size_t)p * ld + j];
    counts[j] = col;
}

cudaError_t launch_colsum(const Dev& d, int32_t* counts, cudaStream_t s)
{
    k_colsum<<<(d.ld + 255) / 256, 256, 0, s>>>(d.X, d.n, d.ld, d.R, counts);
    note_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Best solution over the replicas (strictly lower energy; lowest replica on
// ties), optional trace of all energies, and the per-iteration stale counter
// used by the termination rule (Section 3: stop after a number of
// consecutive iterations without a new best).
// flags[0] = improved during this iteration, flags[1] = stale iterations,
// flags[3] = replica last copied into best_x, flags[4] = flags[0] of the
// iteration just ended, flags[5] = its improvement-log slot.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_best(const uint8_t* __restrict__ X, int ld, const int64_t* __restrict__ E,
                                              int R, uint8_t* best_x, int64_t* best_E, int32_t* flags,
                                              int64_t* trace_slot, int iter_end, int32_t* iter_dev,
                                              int32_t* log_ctl, int phase, int t_arg)
{
    __shared__ long long sE[8];
    __shared__ int sP[8];
    __shared__ int s_win;
    long long me = LLONG_MAX;
    int mp = 0x7fffffff;
    for (int p = threadIdx.x; p < R; p += blockDim.x) {
        const long long e = E[p];
        if (trace_slot) trace_slot[p] = e;
        if (e < me || (e == me && p < mp)) { me = e; mp = p; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long oe = __shfl_xor_sync(0xffffffffu, me, o);
        const int op = __shfl_xor_sync(0xffffffffu, mp, o);
        if (oe < me || (oe == me && op < mp)) { me = oe; mp = op; }
    }
    if ((threadIdx.x & 31) == 0) { sE[threadIdx.x >> 5] = me; sP[threadIdx.x >> 5] = mp; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sE[w] < me || (sE[w] == me && sP[w] < mp)) { me = sE[w]; mp = sP[w]; }
        const long long cur = *best_E;
        s_win = (me < cur) ? mp : -1;
        if (s_win >= 0) {
            *best_E = me; flags[0] = 1; flags[3] = mp;
            flags[7] = phase < 0 ? 0 : 3 * (iter_dev ? *iter_dev : t_arg) + phase + 1;
        }
    }
    __syncthreads();
    const int win = s_win;
    if (win >= 0)
        for (int j = threadIdx.x * 16; j < ld; j += blockDim.x * 16)
            *reinterpret_cast<uint4*>(best_x + j) = *reinterpret_cast<const uint4*>(X + (size_t)win * ld + j);
    if (threadIdx.x == 0 && iter_end) {
        if (trace_slot) trace_slot[R] = *best_E;
        flags[1] = flags[0] ? 0 : flags[1] + 1;
        flags[4] = flags[0];
        if (log_ctl && flags[0]) {  // slot of the improvement-log entry (ring buffer)
            flags[5] = log_ctl[0] % log_ctl[1];
            log_ctl[0] += 1;
        }
        flags[0] = 0;
        if (iter_dev) *iter_dev += 1;  // the next replay of a captured iteration is t + 1
    }
}

cudaError_t launch_best(const Dev& d, int64_t* trace_slot, int iter_end, int32_t* iter_dev, cudaStream_t s,
                        int32_t* log_ctl, int phase, int t)
{
    k_best<<<1, 256, 0, s>>>(d.X, d.ld, d.E, d.R, d.best_x, d.best_E, d.flags, trace_slot, iter_end, iter_dev,
                             log_ctl, phase, t);
    note_launch(1);
    return cudaGetLastError();
}

__global__ void k_set_iter(int32_t* iter_dev, int t) { *iter_dev = t; }

cudaError_t launch_set_iter(int32_t* iter_dev, int t, cudaStream_t s)
{
    k_set_iter<<<1, 1, 0, s>>>(iter_dev, t);
    note_launch(1);
    return cudaGetLastError();
}

int device_sm_count()
{
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// Per-instance preparation.  k_symcheck compares 32 x 32 tiles of Q with the
// transposed tiles (counts mismatches); k_eta forms eta_j = sum_i |Q_ij|
// (Eq. 6), the diagonal and the column's largest gain over all x (one thread
// per column, coalesced across j): with P_j / N_j the sums of the positive /
// negative off-diagonal entries' magnitudes, Q_jj + 2 sum_{i != j} Q_ij x_i
// ranges over [Q_jj - 2 N_j, Q_jj + 2 P_j], so max |g_j| = max(|Q_jj - 2 N_j|,
// |Q_jj + 2 P_j|), attained; k_etahat normalises eta by its maximum (Q16, floor).
// ---------------------------------------------------------------------------
__global__ void k_symcheck(const int8_t* __restrict__ Q, int n, int ld, int* mismatches)
{
    __shared__ int8_t A[32][33], B[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    if (bi > bj) return;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = threadIdx.x;
        A[r][c] = (bi + r < n && bj + c < n) ? Q[(size_t)(bi + r) * ld + bj + c] : 0;
        B[r][c] = (bj + r < n && bi + c < n) ? Q[(size_t)(bj + r) * ld + bi + c] : 0;
    }
    __syncthreads();
    int bad = 0;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) bad += A[r][threadIdx.x] != B[threadIdx.x][r];
    bad = __reduce_add_sync(0xffffffffu, (unsigned)bad);
    if (threadIdx.x == 0 && bad) atomicAdd(mismatches, bad);
}

__global__ void k_eta(const int8_t* __restrict__ Q, int n, int ld, int32_t* eta, int32_t* diag, int* n128,
                      int* gmax)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ld) return;
    if (j >= n) { eta[j] = 0; diag[j] = 0; return; }
    int s = 0, m = 0, pos = 0, neg = 0;
    for (int i = 0; i < n; ++i) {
        const int v = Q[(size_t)i * ld + j];
        s += abs(v);
        m += v == -128;
        if (i != j) {
            pos += v > 0 ? v : 0;
            neg += v < 0 ? -v : 0;
        }
    }
    eta[j] = s;
    const int qjj = Q[(size_t)j * ld + j];
    diag[j] = qjj;
    if (m) atomicAdd(n128, m);
    atomicMax(gmax, max(abs(qjj - 2 * neg), abs(qjj + 2 * pos)));
}

__global__ __launch_bounds__(1024) void k_etahat(const int32_t* __restrict__ eta, int n, int ld, int32_t* etahat,
                                                 int* eta_max)
{
    __shared__ int red[32];
    int mx = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = max(mx, eta[j]);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    if (threadIdx.x == 0) *eta_max = mx;
    for (int j = threadIdx.x; j < ld; j += blockDim.x)
        etahat[j] = (j < n && mx > 0) ? (int32_t)(((long long)eta[j] * 65536) / mx) : 0;
}

// Signed row pairs for the Tabu search: one thread per 16 bytes of a row of Q
// writes them to rows 2i and 2i + 1 (bytewise negation; no entry is -128).
__global__ void k_signed_rows(const int8_t* __restrict__ Q, int n, int ld, int8_t* __restrict__ Q2)
{
    const size_t chunks = (size_t)n * (ld / 16);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= chunks) return;
    const size_t i = t / (ld / 16), c = t % (ld / 16);
    const uint4 v = *reinterpret_cast<const uint4*>(Q + i * ld + 16 * c);
    uint32_t w[4] = {v.x, v.y, v.z, v.w}, m[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t r = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) r |= (uint32_t)(uint8_t)(-(int8_t)(w[k] >> (8 * b))) << (8 * b);
        m[k] = r;
    }
    *reinterpret_cast<uint4*>(Q2 + (2 * i) * ld + 16 * c) = v;
    *reinterpret_cast<uint4*>(Q2 + (2 * i + 1) * ld + 16 * c) = make_uint4(m[0], m[1], m[2], m[3]);
}

// One CTA per row of the relabeled matrix; the label table is read through L1.
__global__ void k_relabel(const int8_t* __restrict__ Q, const int32_t* __restrict__ perm, int n, int ld,
                          int8_t* __restrict__ Qpk)
{
    const int L = blockIdx.x;
    const int8_t* src = Q + (size_t)perm[L] * ld;
    int8_t* dst = Qpk + (size_t)L * ld;
    for (int M = threadIdx.x; M < ld; M += blockDim.x) dst[M] = M < n ? src[perm[M]] : (int8_t)0;
}

cudaError_t launch_relabel(const int8_t* Q, const int32_t* perm, int n, int ld, int8_t* Qpk, cudaStream_t s)
{
    k_relabel<<<n, 256, 0, s>>>(Q, perm, n, ld, Qpk);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_signed_rows(const int8_t* Q, int n, int ld, int8_t* Q2, cudaStream_t s)
{
    const size_t chunks = (size_t)n * (ld / 16);
    k_signed_rows<<<(unsigned)((chunks + 255) / 256), 256, 0, s>>>(Q, n, ld, Q2);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const int8_t* Q, int n, int ld, int32_t* eta, int32_t* etahat, int32_t* diag,
                           int* mismatches, int* eta_max, int* gain_max, cudaStream_t s)
{
    const int tiles = (n + 31) / 32;
    k_symcheck<<<dim3(tiles, tiles), dim3(32, 8), 0, s>>>(Q, n, ld, mismatches);
    note_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_eta<<<(ld + 255) / 256, 256, 0, s>>>(Q, n, ld, eta, diag, eta_max + 1, gain_max);
    note_launch(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_etahat<<<1, 1024, 0, s>>>(eta, n, ld, etahat, eta_max);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
