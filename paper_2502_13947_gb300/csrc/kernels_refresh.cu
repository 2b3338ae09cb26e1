// kernels_refresh.cu -- exact dense refresh of all gains on the tensor cores.
//
// H = Q X^T for every replica at once (H[p][j] = sum_k Q_jk x_pk), then
// g = (1 - 2x)(Q_jj + 2 (H - Q_jj x)) and E = sum_j x_j (Q_jj + H_j - Q_jj x_j):
// a from-scratch recompute of the state the other kernels update
// incrementally, used to check that the tracked gains and energies never
// drift (and to rebuild them).
//
// tcgen05 (5th-generation tensor cores) with BF16 operands and FP32
// accumulators in tensor memory.  Exact: |Q_ij| <= 128 and x in {0, 1} are
// BF16 integers, every product is exact, and every partial sum is an integer
// of magnitude <= 128 n <= 2^21 < 2^24, which FP32 represents exactly whatever the
// summation order.  (The int8 MMA kind is not available for sm_103a.)
//
// Tiles: 128 rows of Q (M) x BN replicas (N), K in chunks of 64 (128 bytes,
// one 128-byte-swizzled row per operand row), STAGES-deep TMA pipeline.
// Warp 0 lane 0 issues the TMA loads, warp 1 lane 0 issues the MMAs
// (M = 128, N = BN, K = 16 per instruction, 4 per chunk) and commits each
// stage back to the producer; after the last chunk all four warps read their
// 32 accumulator lanes (rows) from tensor memory and add them, as exact
// int32, into H (split-K CTAs over the same tile add into the same entries).
// Every mbarrier wait is bounded: on timeout the kernel raises an error flag,
// skips its output, releases its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace icd2s {

namespace {

constexpr int kBM = 128, kBK = 64;
constexpr uint32_t kStgBytes = 2 * 32 * kBM * 4;  // the persistent refresh's two epilogue tiles
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
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

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (iterations and wait_ns of wall time, 2 s unless a test asks
// for less); false, with the error flag raised, if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, uint64_t wait_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > wait_ns) break;
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (8-row groups of 1024 bytes): start address, stride
// between 8-row groups (1024 B), descriptor version 1, layout "128B swizzle".
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);        // start address
    d |= (uint64_t)1u << 16;                        // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset
    d |= (uint64_t)1u << 46;                        // version
    d |= (uint64_t)2u << 61;                        // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// element-wise add of a shared-memory tile into global memory by the TMA
// (the tensor map's type and box; elements outside the tensor are skipped)
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, int x, int y, uint32_t src)
{
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(map), "r"(x), "r"(y), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// named barrier that also returns whether `pred` holds in any of its threads
__device__ __forceinline__ bool named_bar_or(int id, int threads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// Persistent form: one CTA per SM walks a contiguous range of the work units
// (tile, K chunk), tiles of MS x 128 rows of Q by BN replicas taken in order
// and each tile's K chunks in order, so a CTA's range covers the end of one
// tile, whole tiles and the start of another ("stream-K"): every SM gets the
// same number of chunks, whatever the tile count.  Each run of chunks of one
// tile (a segment) accumulates in tensor memory and is added to H by the
// epilogue warps (exact int32 atomics: the segments of a tile may come from
// several CTAs).  With NACC = 2 accumulators the epilogue of one segment
// overlaps the MMAs of the next.  Warps: 0 = TMA producer (lane 0), 1 = MMA
// issuer (lane 0), 2..5 = epilogue (warp w reads accumulator lanes
// 32 (w mod 4) .. + 31).  Barriers: full/empty per stage, full/empty per
// accumulator, and `done` for the issuer's last MMAs.  Every wait is bounded
// by wait_ns; a timed-out wait raises the error flag and its role stops, so
// the others time out as well and the kernel ends with the flag set.
// skip_loads (fault injection for tests): the producer issues nothing.
// ---------------------------------------------------------------------------
template <int BN, int MS, int STAGES, int NACC>
__global__ __launch_bounds__(192, 1) void k_refresh_mma(const __grid_constant__ CUtensorMap tA,
                                                       const __grid_constant__ CUtensorMap tB,
                                                       const __grid_constant__ CUtensorMap tH, int n, int R,
                                                       int kc_total, int tiles_n, long long units, int* err,
                                                       unsigned long long wait_ns, int skip_loads)
{
    static_assert(MS * BN * NACC <= 512, "tensor memory holds 512 columns");
    constexpr uint32_t kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
    constexpr uint32_t kStage = MS * kABytes + kBBytes;
    constexpr uint32_t kIdesc = idesc_bf16_f32(kBM, BN);
    constexpr uint32_t kCols = MS * BN * NACC;  // a power of two >= 32
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    int32_t* stg = reinterpret_cast<int32_t*>(smem + STAGES * kStage);   // epilogue tiles [2][32][128]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * kStage + kStgBytes);
    // full[S], empty[S], afull[NACC], aempty[NACC], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2 * NACC + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES, afull0 = empty0 + 8 * STAGES,
                   aempty0 = afull0 + 8 * NACC, done = aempty0 + 8 * NACC;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(afull0 + 8 * a, 1);
            mbar_init(aempty0 + 8 * a, 128);   // every epilogue thread
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0 && !skip_loads) {
            // producer: A = Q[rows of the tile][chunk] (MS boxes of 128 rows), B = X[replicas of the tile][chunk]
            bool ok = true;
            long long issued = 0;
            for (long long u = u0; u < u1 && ok; ++u, ++issued) {
                const int s = (int)(issued % STAGES);
                const long long use = issued / STAGES;
                if (use > 0) ok = mbar_wait(empty0 + 8 * s, (uint32_t)((use - 1) & 1), err, wait_ns);
                if (!ok) break;
                const int tile = (int)(u / kc_total), kc = (int)(u % kc_total);
                const int tm = tile / tiles_n, tn = tile % tiles_n;
                const uint32_t fb = full0 + 8 * s;
                unsigned char* st = smem + (size_t)s * kStage;
                mbar_expect_tx(fb, kStage);
#pragma unroll
                for (int ms = 0; ms < MS; ++ms)
                    tma_load_2d(smem_u32(st + ms * kABytes), &tA, kc * kBK, (tm * MS + ms) * kBM, fb);
                tma_load_2d(smem_u32(st + MS * kABytes), &tB, kc * kBK, tn * BN, fb);
            }
            // every load issued has landed before the CTA can leave
            for (long long i = issued - STAGES > 0 ? issued - STAGES : 0; i < issued; ++i)
                mbar_wait(full0 + 8 * (int)(i % STAGES), (uint32_t)((i / STAGES) & 1), err, wait_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: per segment, accumulator a = segment mod NACC, freed by the epilogue
            bool ok = true;
            long long i = 0;
            int seg = 0;
            for (long long u = u0; u < u1 && ok; ++u, ++i) {
                const int kc = (int)(u % kc_total);
                const bool first = u == u0 || kc == 0, last = u + 1 == u1 || kc + 1 == kc_total;
                const int a = seg % NACC, ause = seg / NACC;
                if (first && ause > 0) {
                    ok = mbar_wait(aempty0 + 8 * a, (uint32_t)((ause - 1) & 1), err, wait_ns);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                const int s = (int)(i % STAGES);
                ok = mbar_wait(full0 + 8 * s, (uint32_t)((i / STAGES) & 1), err, wait_ns);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = smem_u32(smem + (size_t)s * kStage);
                const uint32_t b = st + MS * kABytes;
#pragma unroll
                for (int ms = 0; ms < MS; ++ms) {
                    const uint32_t d = tmem + (uint32_t)((a * MS + ms) * BN);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)  // K = 16 per instruction: 32 bytes along the row
                        mma_bf16(d, smem_desc_sw128(st + ms * kABytes + 32 * kk), smem_desc_sw128(b + 32 * kk),
                                 kIdesc, (!first || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);              // the stage is free once these MMAs have read it
                if (last) {
                    mma_commit(afull0 + 8 * a);          // the segment's sums are complete
                    ++seg;
                }
            }
            mma_commit(done);                            // tracks every MMA issued above
            mbar_wait(done, 0u, err, wait_ns);
        }
    } else {
        // epilogue: warp w owns accumulator lanes (rows) 32 (w mod 4) .. + 31.  Per
        // 32 replicas the 128 threads write the sums as int32 into a staging tile
        // [32 replicas][128 rows] (two tiles, alternating) and one thread adds the
        // tile into H with a TMA reduction; the tile is reused once that
        // reduction has read it.
        const int et = threadIdx.x - 64, quad = warp & 3;
        int seg = 0, chunk = 0;
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / kc_total), kc = (int)(u % kc_total);
            long long send = u + (kc_total - kc);        // the segment: to the tile's end or the range's
            if (send > u1) send = u1;
            const int tm = tile / tiles_n, tn = tile % tiles_n;
            const int a = seg % NACC, ause = seg / NACC;
            const bool got = mbar_wait(afull0 + 8 * a, (uint32_t)(ause & 1), err, wait_ns);
            // all 128 threads go on together (the loads below are warp-collective and
            // the tiles are shared), or all stop
            if (named_bar_or(1, 128, !got)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int ms = 0; ms < MS; ++ms) {
                const uint32_t tw = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((a * MS + ms) * BN);
#pragma unroll 1
                for (int c = 0; c < BN; c += 32, ++chunk) {
                    uint32_t v[32];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(tw + (uint32_t)c));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int b = chunk & 1;
                    if (chunk >= 2) {   // the reduction issued from this tile two chunks ago has read it
                        if (et == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                        named_bar_sync(1, 128);
                    }
                    int32_t* dst = stg + b * (32 * kBM) + quad * 32 + lane;
#pragma unroll
                    for (int t = 0; t < 32; ++t) dst[t * kBM] = __float2int_rn(__uint_as_float(v[t]));
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the TMA
                    named_bar_sync(1, 128);
                    if (et == 0)
                        tma_reduce_add_2d(&tH, (tm * MS + ms) * kBM, tn * BN + c, smem_u32(stg + b * (32 * kBM)));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(aempty0 + 8 * a);                // the accumulator may be overwritten
            ++seg;
            u = send;
        }
        if (et == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // every reduction is done
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// ---------------------------------------------------------------------------
// The same product with Q read as bytes: TMA brings int8 tiles of Q (half the
// bytes of BF16, and no BF16 copy of Q) beside BF16 tiles of X; four
// converter warps write the Q tiles as BF16 in the 128-byte-swizzled layout
// the MMA reads, and the MMA issuer takes them with the X tiles straight from
// the TMA stage.  Exact as above: every int8 value is a BF16 integer.  Warp 0
// lane 0 issues the TMA loads into SI stages, warp 1 lane 0 the MMAs from SC
// converted buffers, warps 2..5 convert and then run the epilogue (warp w
// reads accumulator lanes 32 (w mod 4) ..).  Every wait is bounded as above.
// ---------------------------------------------------------------------------
namespace {

// bf16 of 8 signed bytes (two words): b + 128 placed in the mantissa of 2^23
// and 2^23 + 128 subtracted gives the exact float b, whose top 16 bits are its bf16
__device__ __forceinline__ uint4 bf16x8_from_s8(uint2 w)
{
    const uint32_t u0 = w.x ^ 0x80808080u, u1 = w.y ^ 0x80808080u;
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = __float_as_uint(__uint_as_float(__byte_perm(u0, 0x4B000000u, 0x7540u + k)) - 8388736.0f);
        h[4 + k] = __float_as_uint(__uint_as_float(__byte_perm(u1, 0x4B000000u, 0x7540u + k)) - 8388736.0f);
    }
    return make_uint4(__byte_perm(h[0], h[1], 0x7632u), __byte_perm(h[2], h[3], 0x7632u),
                      __byte_perm(h[4], h[5], 0x7632u), __byte_perm(h[6], h[7], 0x7632u));
}

}  // namespace

template <int BN, int SI, int SC>
__global__ __launch_bounds__(192, 1) void k_refresh_i8(const __grid_constant__ CUtensorMap tA8,
                                                      const __grid_constant__ CUtensorMap tB, int n, int R,
                                                      int kc_total, int kc_per_split, int32_t* __restrict__ H,
                                                      int ldh, int* err, unsigned long long wait_ns, int skip_loads)
{
    constexpr uint32_t kA8 = kBM * kBK, kA16 = kBM * kBK * 2, kB16 = BN * kBK * 2;
    constexpr uint32_t kIdesc = idesc_bf16_f32(kBM, BN);
    constexpr int kConv = 128;  // converter threads (warps 2..5)
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* tB16 = smem;               // SI x kB16 (TMA stages of X, BF16, swizzled)
    unsigned char* cA = tB16 + SI * kB16;     // SC x kA16 (converted Q)
    unsigned char* tA8b = cA + SC * kA16;     // SI x kA8 (TMA stages of Q, bytes)
    uint64_t* bars = reinterpret_cast<uint64_t*>(tA8b + SI * kA8);  // ifull, iempty, cfull, cempty, done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SI + 2 * SC + 1);
    const uint32_t ifull0 = smem_u32(bars), iempty0 = ifull0 + 8 * SI, cfull0 = iempty0 + 8 * SI,
                   cempty0 = cfull0 + 8 * SC, done = cempty0 + 8 * SC;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kc0 = blockIdx.z * kc_per_split;
    const int kc1 = min(kc0 + kc_per_split, kc_total);
    const int nk = kc1 > kc0 ? kc1 - kc0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SI; ++s) {
            mbar_init(ifull0 + 8 * s, 1);
            mbar_init(iempty0 + 8 * s, kConv + 1);  // the converters (Q bytes) and the MMAs (X tile)
        }
        for (int s = 0; s < SC; ++s) {
            mbar_init(cfull0 + 8 * s, kConv);
            mbar_init(cempty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0 && nk > 0 && !skip_loads) {
        // producer: byte tiles of Q[m0 ..][k], BF16 tiles of X[n0 ..][k]
        int issued = 0;
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % SI, u = i / SI;
            if (u > 0) ok = mbar_wait(iempty0 + 8 * s, (uint32_t)((u - 1) & 1), err, wait_ns);
            if (!ok) break;
            const uint32_t fb = ifull0 + 8 * s;
            mbar_expect_tx(fb, kA8 + kB16);
            const int kx = (kc0 + i) * kBK;  // element column, a multiple of 64
            tma_load_2d(smem_u32(tA8b + s * kA8), &tA8, kx, m0, fb);
            tma_load_2d(smem_u32(tB16 + s * kB16), &tB, kx, n0, fb);
            ++issued;
        }
        for (int i = issued - SI > 0 ? issued - SI : 0; i < issued; ++i)
            mbar_wait(ifull0 + 8 * (i % SI), (uint32_t)((i / SI) & 1), err, wait_ns);
    } else if (warp == 1 && lane == 0 && nk > 0) {
        // MMA issuer: converted Q from buffer i mod SC (its stage's X tile has landed
        // before the converters released the buffer), X from TMA stage i mod SI
        for (int i = 0; i < nk && ok; ++i) {
            const int sc = i % SC, si = i % SI;
            ok = mbar_wait(cfull0 + 8 * sc, (uint32_t)((i / SC) & 1), err, wait_ns) &&
                 mbar_wait(ifull0 + 8 * si, (uint32_t)((i / SI) & 1), err, wait_ns);  // the X tile, observed directly
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = smem_u32(cA + sc * kA16), b = smem_u32(tB16 + si * kB16);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_bf16(tmem, smem_desc_sw128(a + 32 * kk), smem_desc_sw128(b + 32 * kk), kIdesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(cempty0 + 8 * sc);  // the converted buffer ...
            mma_commit(iempty0 + 8 * si);  // ... and the X tile of the stage are free again
        }
        mma_commit(done);
    } else if (warp >= 2 && nk > 0) {
        // converters: 8 bytes -> one 16-byte BF16 chunk, stored at its swizzled place
        // (chunk c of row r at c ^ (r mod 8) within the row's 128 bytes)
        const int c = threadIdx.x - 64;
        for (int i = 0; i < nk && ok; ++i) {
            const int si = i % SI, sc = i % SC, uc = i / SC;
            ok = mbar_wait(ifull0 + 8 * si, (uint32_t)((i / SI) & 1), err, wait_ns);
            if (ok && uc > 0) ok = mbar_wait(cempty0 + 8 * sc, (uint32_t)((uc - 1) & 1), err, wait_ns);
            if (!ok) break;
            const unsigned char* a8 = tA8b + si * kA8;
            unsigned char* a16 = cA + sc * kA16;
#pragma unroll
            for (int j = 0; j < kBM * 8 / kConv; ++j) {
                const int q = c + kConv * j, r = q >> 3, cc = q & 7;
                const uint2 w = *reinterpret_cast<const uint2*>(a8 + r * kBK + cc * 8);
                *reinterpret_cast<uint4*>(a16 + r * 128 + ((cc ^ (r & 7)) << 4)) = bf16x8_from_s8(w);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
            mbar_arrive(iempty0 + 8 * si);
            mbar_arrive(cfull0 + 8 * sc);
        }
    }
    __syncwarp();

    // epilogue: warps 2..5; warp w owns accumulator lanes (rows) 32 (w mod 4) ..
    // (a warp reads tensor memory only if every lane saw the sums complete)
    bool got = false;
    if (warp >= 2 && nk > 0) got = __all_sync(0xffffffffu, mbar_wait(done, 0u, err, wait_ns));
    if (got) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quad = warp & 3;
        const int row = m0 + quad * 32 + lane;
        const uint32_t tw = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < BN; cb += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tw + (uint32_t)cb));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < n) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int p = n0 + cb + t;
                    if (p < R) {
                        const int h = __float2int_rn(__uint_as_float(v[t]));
                        if (h != 0) atomicAdd(H + (size_t)p * ldh + row, h);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// int8 Q [n][ld] -> bf16 [n][ld]; uint8 X [R][ld] -> bf16 [R][ld]
__global__ void k_to_bf16_i8(const int8_t* __restrict__ src, size_t count, __nv_bfloat16_raw* __restrict__ dst)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        // integers in [-128, 127] are exact in bfloat16: the float's top 16 bits
        const float f = (float)src[i];
        __nv_bfloat16_raw r;
        r.x = (unsigned short)(__float_as_uint(f) >> 16);
        dst[i] = r;
    }
}

__global__ void k_to_bf16_u8(const uint8_t* __restrict__ src, size_t count, __nv_bfloat16_raw* __restrict__ dst)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        __nv_bfloat16_raw r;
        r.x = src[i] ? (unsigned short)0x3F80u : (unsigned short)0u;  // 1.0 or 0.0
        dst[i] = r;
    }
}

cudaError_t launch_to_bf16(const void* src, bool is_signed, size_t count, void* dst, cudaStream_t s)
{
    int blocks = (int)((count + 255) / 256);
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    if (blocks < 1) blocks = 1;
    if (is_signed)
        k_to_bf16_i8<<<blocks, 256, 0, s>>>(static_cast<const int8_t*>(src), count,
                                             static_cast<__nv_bfloat16_raw*>(dst));
    else
        k_to_bf16_u8<<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(src), count,
                                             static_cast<__nv_bfloat16_raw*>(dst));
    note_launch(1);
    return cudaGetLastError();
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// 2-D bf16 tensor [rows][ld] (ld elements per row), box = 64 columns x box_rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const void* base, int rows, int ld, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D byte tensor [rows][ld], box = 64 columns x box_rows, no swizzle
bool make_map_u8(CUtensorMap* m, const void* base, int rows, int ld, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int SI, int SC>
cudaError_t launch_i8(const CUtensorMap& tA, const CUtensorMap& tB, int n, int R, int ld, int splits, int32_t* H,
                      int* err, unsigned long long wait_ns, int skip_loads, cudaStream_t s)
{
    const size_t sm = 1024 + (size_t)SI * (kBM + 2 * BN) * kBK + (size_t)SC * kBM * kBK * 2 +
                      (2 * SI + 2 * SC + 1) * 8 + 16;
    auto kern = k_refresh_i8<BN, SI, SC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int kc_total = ld / kBK;
    const int kcps = (kc_total + splits - 1) / splits;
    dim3 grid((n + kBM - 1) / kBM, (R + BN - 1) / BN, (kc_total + kcps - 1) / kcps);
    kern<<<grid, 192, sm, s>>>(tA, tB, n, R, kc_total, kcps, H, ld, err, wait_ns, skip_loads);
    note_launch(1);
    return cudaGetLastError();
}

// 2-D int32 tensor [rows][ld] for the epilogue's TMA reductions, box = 128 x 32, no swizzle
bool make_map_h(CUtensorMap* m, const void* base, int rows, int ld)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kBM, 32u};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int MS, int STAGES, int NACC>
cudaError_t launch_mma(const CUtensorMap& tA, const CUtensorMap& tB, const CUtensorMap& tH, int n, int R, int ld,
                       int ctas, int* err, unsigned long long wait_ns, int skip_loads, cudaStream_t s)
{
    constexpr size_t kStage = (size_t)(MS * kBM + BN) * kBK * 2;
    const size_t sm = 1024 + STAGES * kStage + kStgBytes + (2 * STAGES + 2 * NACC + 1) * 8 + 16;
    auto kern = k_refresh_mma<BN, MS, STAGES, NACC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int kc_total = ld / kBK;
    const int tiles_m = (n + MS * kBM - 1) / (MS * kBM), tiles_n = (R + BN - 1) / BN;
    const long long units = (long long)tiles_m * tiles_n * kc_total;
    int grid = ctas > 0 ? ctas : device_sm_count();   // persistent: one CTA per SM
    if (grid > units) grid = (int)units;
    kern<<<grid, 192, sm, s>>>(tA, tB, tH, n, R, kc_total, tiles_n, units, err, wait_ns, skip_loads);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace

// H[R][ld] (int32, zeroed by the caller) += Q X^T on the tensor cores.  Qb: bf16 [n][ld];
// Xb: bf16 [R][ld]; ld a multiple of 128.  err: device flag raised on a
// timed-out wait.  bn: replicas per tile (128 / 256; 0 picks by R); rows: 128
// or 256 rows of Q per tile (0 = 128); ctas: persistent CTAs (0 = one per SM).
// wait_ns: bound of every pipeline wait; skip_loads: fault injection (no loads).
cudaError_t launch_refresh_mma(const void* Qb, const void* Xb, int n, int R, int ld, int32_t* H, int* err, int bn,
                               int ctas, int rows, unsigned long long wait_ns, int skip_loads, cudaStream_t s)
{
    CUtensorMap tA, tB, tH;
    const int BN = bn == 128 || bn == 256 ? bn : (R > 128 ? 256 : 128);
    if (!make_map(&tA, Qb, n, ld, kBM) || !make_map(&tB, Xb, R, ld, BN) || !make_map_h(&tH, H, R, ld))
        return cudaErrorInvalidValue;
    if (rows == 256) {  // two 128-row halves share each replica tile; one accumulator
        if (BN == 256) return launch_mma<256, 2, 3, 1>(tA, tB, tH, n, R, ld, ctas, err, wait_ns, skip_loads, s);
        return launch_mma<128, 2, 4, 2>(tA, tB, tH, n, R, ld, ctas, err, wait_ns, skip_loads, s);
    }
    if (BN == 256) return launch_mma<256, 1, 4, 2>(tA, tB, tH, n, R, ld, ctas, err, wait_ns, skip_loads, s);
    return launch_mma<128, 1, 6, 2>(tA, tB, tH, n, R, ld, ctas, err, wait_ns, skip_loads, s);
}

// H[R][ld] (int32, zeroed by the caller) += Q X^T with Q read as bytes:
// Q8 int8 [n][ld], Xb bf16 [R][ld]; ld a multiple of 128.
cudaError_t launch_refresh_i8(const void* Q8, const void* Xb, int n, int R, int ld, int32_t* H, int* err, int bn,
                              int splits, unsigned long long wait_ns, int skip_loads, cudaStream_t s)
{
    CUtensorMap tA, tB;
    const int BN = bn == 128 || bn == 256 ? bn : (R > 128 ? 256 : 128);
    if (!make_map_u8(&tA, Q8, n, ld, kBM) || !make_map(&tB, Xb, R, ld, BN)) return cudaErrorInvalidValue;
    const int tiles = ((n + kBM - 1) / kBM) * ((R + BN - 1) / BN);
    const int kc_total = ld / kBK;
    if (splits <= 0) splits = device_sm_count() / tiles;
    if (splits < 1) splits = 1;
    if (splits > kc_total) splits = kc_total;
    if (BN == 256) return launch_i8<256, 4, 3>(tA, tB, n, R, ld, splits, H, err, wait_ns, skip_loads, s);
    return launch_i8<128, 6, 3>(tA, tB, n, R, ld, splits, H, err, wait_ns, skip_loads, s);
}

// Counts entries where two gain/energy sets differ (the drift check).
__global__ void k_compare(const int32_t* __restrict__ G1, const int64_t* __restrict__ E1,
                          const int32_t* __restrict__ G2, const int64_t* __restrict__ E2, int n, int ld, int R,
                          int* mismatches)
{
    int bad = 0;
    const size_t total = (size_t)R * ld;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        if ((int)(i % ld) < n && G1[i] != G2[i]) ++bad;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < R; p += gridDim.x * blockDim.x)
        if (E1[p] != E2[p]) ++bad;
    bad = (int)__reduce_add_sync(0xffffffffu, (unsigned)bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

cudaError_t launch_compare(const int32_t* G1, const int64_t* E1, const int32_t* G2, const int64_t* E2, int n, int ld,
                           int R, int* mismatches, cudaStream_t s)
{
    int blocks = (int)(((size_t)R * ld + 255) / 256);
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    k_compare<<<blocks, 256, 0, s>>>(G1, E1, G2, E2, n, ld, R, mismatches);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace icd2s
