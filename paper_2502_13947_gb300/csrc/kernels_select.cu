// kernels_select.cu -- control parameters, subQUBO selection and the
// mutation operator (Section 3).
//
//  k_sizes   uneven subQUBO sizes m_k = m_min + (Philox(k, TAG_SIZE, p, iter) mod span)
//            and their exclusive prefix (group offsets), one CTA.
//  k_select  one CTA per replica: Delta (Eq. 7) from the Tabu toggle counts,
//            A = w1 eta + w2 gamma - w3 Delta (Algorithm 3, Q16, floor), a
//            bitonic sort of the 64-bit keys (A desc, index asc) in shared
//            memory, the S' mask, and a second bitonic sort of the first
//            sum(m_k) ranks by (group, index) so that every group comes out
//            in ascending index order (Algorithm 4's subset choice).  In the
//            learned mode S' comes from a third sort by the network's score;
//            the selection hit counts H are incremented for S'.
//  k_mutate  one CTA per replica: the first L = floor((n - |S'|) r) ranked
//            variables outside S' are candidates; candidate i flips iff its
//            Philox word is below floor((A_i - A_min)(2^32 - 1)/(A_max - A_min)).
//            Flips go to the replica's flip list for k_apply.
#include <climits>

#include "common.cuh"

namespace icd2s {

namespace {

__device__ __forceinline__ long long floor_div_65536(long long v)
{
    return v >= 0 ? v / 65536 : -((-v + 65535) / 65536);
}

__device__ void bitonic_sort(unsigned long long* s, int N)
{
    const int NT = blockDim.x;
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += NT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = s[i], b = s[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { s[i] = b; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
}

__device__ __forceinline__ int block_reduce_max(int v, int* red)
{
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : INT_MIN;
        w = __reduce_max_sync(0xffffffffu, w);
        if (threadIdx.x == 0) red[32] = w;
    }
    __syncthreads();
    const int r = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int block_reduce_min(int v, int* red)
{
    return -block_reduce_max(-v, red);  // |A| < 2^30, negation is safe
}

__host__ __device__ inline int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Also writes, when `order` is given, the subQUBOs in largest-first order
// (a counting sort by size; the order among equal sizes is immaterial) for
// the persistent anneal kernel, and resets its queue counter.
__global__ __launch_bounds__(1024) void k_sizes(int R, int K, int m_min, int m_max, uint32_t k0, uint32_t k1,
                                                uint32_t iter_arg, const int32_t* iter_dev, int32_t* off,
                                                int32_t* order, int32_t* queue, int p0)
{
    __shared__ int part[1024];
    __shared__ int start[kMaxM + 2];
    const uint32_t iter = iter_dev ? (uint32_t)*iter_dev : iter_arg;
    const int total = R * K;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int chunk = (total + NT - 1) / NT;
    const int lo = tid * chunk, hi = min(total, lo + chunk);
    const uint32_t span = (uint32_t)(m_max - m_min + 1);
    auto size_of = [&](int s) -> int {
        if (m_max == m_min) return m_min;
        const int p = p0 + s / K, k = s % K;   // the global replica
        const u32x4 w = philox10((uint32_t)k, kTagSize << 24, (uint32_t)p, iter, k0, k1);
        return m_min + (int)(w.v[0] % span);
    };
    int sum = 0;
    for (int s = lo; s < hi; ++s) sum += size_of(s);
    part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int t = 0; t < NT; ++t) { const int v = part[t]; part[t] = run; run += v; }
    }
    __syncthreads();
    int run = part[tid];
    for (int s = lo; s < hi; ++s) { off[s] = run; run += size_of(s); }
    if (hi == total && lo < hi) off[total] = run;
    if (total == 0 && tid == 0) off[0] = 0;
    if (!order) return;
    for (int m = tid; m < kMaxM + 2; m += NT) start[m] = 0;
    __syncthreads();
    for (int s = lo; s < hi; ++s) atomicAdd(&start[size_of(s)], 1);
    __syncthreads();
    if (tid == 0) {  // sizes descending: start[m] = number of subQUBOs larger than m
        int acc = 0;
        for (int m = kMaxM; m >= 0; --m) { const int v = start[m]; start[m] = acc; acc += v; }
        *queue = 0;
    }
    __syncthreads();
    for (int s = lo; s < hi; ++s) order[atomicAdd(&start[size_of(s)], 1)] = s;
}

cudaError_t launch_sizes(int R, int K, int m_min, int m_max, uint32_t k0, uint32_t k1, uint32_t iter,
                         const int32_t* iter_dev, int32_t* off, int32_t* order, int32_t* queue, cudaStream_t s,
                         int p0)
{
    k_sizes<<<1, 1024, 0, s>>>(R, K, m_min, m_max, k0, k1, iter, iter_dev, off, order, queue, p0);
    note_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ __launch_bounds__(1024) void k_select(Dev d, int64_t w1, int64_t w2, int64_t w3, int K,
                                                 const int32_t* __restrict__ off, int32_t* __restrict__ idx, int mode,
                                                 int32_t* __restrict__ H, uint32_t iter_arg, const int32_t* iter_dev,
                                                 int ablation)
{
    const uint32_t iter = iter_dev ? (uint32_t)*iter_dev : iter_arg;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int red[33];
    __shared__ int goff[65];
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
    const int p = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    const int n = d.n, ld = d.ld;
    const int NP = next_pow2(n);
    const int32_t* Trow = d.T + (size_t)p * ld;
    int32_t* Arow = d.A + (size_t)p * ld;
    int32_t* Drow = d.delta + (size_t)p * ld;

    int mt = 0;
    for (int j = tid; j < n; j += NT) mt = max(mt, Trow[j]);
    mt = block_reduce_max(mt, red);

    for (int j = tid; j < NP || j < ld; j += NT) {
        unsigned long long key = ~0ull;
        if (j < n) {
            const int t = Trow[j];
            const int dl = mt > 0 ? (int)(((long long)(mt - t) * 65536) / mt) : 0;
            const long long v = w1 * (long long)d.etahat[j] + w2 * (long long)d.gamma[j] - w3 * (long long)dl;
            const int a = ablation == 2   // No_SM: a random ranking key instead of A
                              ? (int)(philox10((uint32_t)(j >> 2), kTagRank << 24, (uint32_t)(d.p0 + p), iter, d.k0,
                                               d.k1).v[j & 3] >> 1)
                              : (int)floor_div_65536(v);
            Arow[j] = a;
            Drow[j] = dl;
            key = ((unsigned long long)(~((unsigned)a ^ 0x80000000u)) << 32) | (unsigned)j;
        } else if (j < ld) {
            Arow[j] = 0;
            Drow[j] = 0;
        }
        if (j < NP) keys[j] = key;
    }
    __syncthreads();
    bitonic_sort(keys, NP);

    int32_t* orow = d.order + (size_t)p * ld;
    uint8_t* srow = d.sel + (size_t)p * ld;
    for (int r = tid; r < ld; r += NT) {
        orow[r] = r < n ? (int32_t)(keys[r] & 0xffffffffu) : 0;
        srow[r] = 0;
    }
    // Learned selection: S' ranked by (score desc, index asc) instead; the A
    // ranking above still orders the mutation candidates.  The score's bit
    // pattern maps to a signed integer with the float's order (-0 below +0).
    if (mode == 1 || (mode == 2 && (p & 1) == 0)) {
        __syncthreads();
        const float* sc = d.score + (size_t)p * ld;
        for (int j = tid; j < NP; j += NT) {
            unsigned long long key = ~0ull;
            if (j < n) {
                const unsigned b = __float_as_uint(sc[j]);
                const int a = b < 0x80000000u ? (int)b : -(int)(b & 0x7fffffffu) - 1;
                key = ((unsigned long long)(~((unsigned)a ^ 0x80000000u)) << 32) | (unsigned)j;
            }
            keys[j] = key;
        }
        __syncthreads();
        bitonic_sort(keys, NP);
    }
    const int base = off[p * K];
    if (tid <= K) goff[tid] = off[p * K + tid] - base;
    __syncthreads();
    const int M = goff[K];
    for (int r = tid; r < M; r += NT) {
        const int i = (int)(keys[r] & 0xffffffffu);
        srow[i] = 1;
        if (H) H[(size_t)p * ld + i] += 1;
    }
    const int NP2 = next_pow2(M > 0 ? M : 1);
    for (int r = tid; r < NP2; r += NT) {
        unsigned long long k2 = ~0ull;
        if (r < M) {
            int g = 0;
            while (g + 1 < K && goff[g + 1] <= r) ++g;
            k2 = ((unsigned long long)g << 32) | (keys[r] & 0xffffffffu);
        }
        keys[r] = k2;   // each thread rewrites only the entries it read
    }
    __syncthreads();
    bitonic_sort(keys, NP2);
    for (int r = tid; r < M; r += NT) idx[base + r] = (int32_t)(keys[r] & 0xffffffffu);
}

cudaError_t launch_select(const Dev& d, int64_t w1, int64_t w2, int64_t w3, int K, const int32_t* off,
                          int32_t* idx, int mode, bool count_hits, cudaStream_t s, uint32_t iter,
                          const int32_t* iter_dev, int ablation)
{
    const size_t sm = 8 * (size_t)next_pow2(d.n);
    cudaError_t e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_select<<<d.R, 1024, sm, s>>>(d, w1, w2, w3, K, off, idx, mode, count_hits ? d.H : nullptr, iter, iter_dev,
                                   ablation);
    note_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ __launch_bounds__(1024) void k_mutate(Dev d, int K, const int32_t* __restrict__ off, double rate_arg,
                                                 uint32_t iter_arg, const int32_t* iter_dev, const double* rates,
                                                 uint8_t* mask, int ldm, int half)
{
    __shared__ int red[33];
    __shared__ int wsum[32];
    const uint32_t iter = iter_dev ? (uint32_t)*iter_dev : iter_arg;
    const double rate = iter_dev ? rates[iter] : rate_arg;
    const int p = blockIdx.x, tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int n = d.n, ld = d.ld;
    const int32_t* Arow = d.A + (size_t)p * ld;
    const int32_t* orow = d.order + (size_t)p * ld;
    const uint8_t* srow = d.sel + (size_t)p * ld;
    const uint8_t* xrow = d.X + (size_t)p * ld;
    const int M = off[(p + 1) * K] - off[p * K];
    const int L = (int)floor((double)(n - M) * rate);
    if (L <= 0) return;

    int amin = INT_MAX, amax = INT_MIN;
    for (int j = tid; j < n; j += NT) { const int a = Arow[j]; amin = min(amin, a); amax = max(amax, a); }
    amin = block_reduce_min(amin, red);
    amax = block_reduce_max(amax, red);

    int taken = 0;  // candidates found before this chunk (uniform)
    for (int r0 = 0; r0 < n && taken < L; r0 += NT) {
        const int r = r0 + tid;
        int i = -1;
        bool pred = false;
        if (r < n) { i = orow[r]; pred = srow[i] == 0; }
        const unsigned bal = __ballot_sync(0xffffffffu, pred);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < (NT >> 5); ++w) { const int v = wsum[w]; before += w < warp ? v : 0; total += v; }
        const int rank = taken + before + __popc(bal & ((1u << lane) - 1u));
        if (pred && rank < L) {
            unsigned long long P;
            if (amax == amin || half) P = 2147483648ull;
            else P = ((unsigned long long)((long long)Arow[i] - amin) * 4294967295ull) /
                     (unsigned long long)((long long)amax - amin);
            const u32x4 w = philox10((uint32_t)(i >> 2), kTagMut << 24, (uint32_t)(d.p0 + p), iter, d.k0, d.k1);
            if ((unsigned long long)w.v[i & 3] < P) {
                const int slot = atomicAdd(&d.FCNT[p], 1);
                if (slot < ld) d.FL[(size_t)p * ld + slot] = i | (int)((unsigned)xrow[i] << 31);
                if (mask) mask[(size_t)p * ldm + i] = 1;
            }
        }
        taken += total;
        __syncthreads();
    }
}

cudaError_t launch_mutate(const Dev& d, int K, const int32_t* off, double rate, uint32_t iter,
                          const int32_t* iter_dev, const double* rates, uint8_t* mask, int ldm, cudaStream_t s,
                          bool half)
{
    k_mutate<<<d.R, 1024, 0, s>>>(d, K, off, rate, iter, iter_dev, rates, mask, ldm, half ? 1 : 0);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
