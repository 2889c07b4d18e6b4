// Helpers of the tcgen05 kernels (order-2 pairs and order-3 triples):
// tile constants, mbarrier waits with a time budget, TMA loads, shared-memory
// and instruction descriptors, MMA issue and commit, TMEM loads, and the
// epilogue's named barrier and bitonic sort.  Included by one translation
// unit per kernel; everything is internal to that unit.
#pragma once
#include <cuda.h>
#include <cfloat>
#include "fc_internal.cuh"

namespace fc {
namespace {

constexpr int TC_BM = 128;          // tile rows: 64 SNPs x genotype rows {0,1}
constexpr int TC_BN = 128;          // tile columns
constexpr int TC_BK = 128;          // K bytes (samples) per pipeline stage
constexpr int TC_SNPS = 64;         // SNPs per tile side
constexpr int TC_THREADS = 192;
// Kernels with several TMA producer warps: warp 0 and warps TC_PROD_WARP1 ..
// issue the copies (TMA copies issued from one thread complete about one
// stage at a time); producer p owns the stages s = p (mod producers).
constexpr int TC_PROD_WARP1 = 6;                              // after warp 1 (MMA) and the four epilogue warps
constexpr int TC_THREADS_MP = 32 * (TC_PROD_WARP1 + TC_MAX_PRODUCERS - 1);

// Producer index of warp w, or -1 (warp 0 -> 0, warp TC_PROD_WARP1 + q -> q + 1).
__device__ __forceinline__ int tc_producer_of(int w, int producers)
{
    const int p = w == 0 ? 0 : (w >= TC_PROD_WARP1 ? w - TC_PROD_WARP1 + 1 : -1);
    return p < producers ? p : -1;
}
constexpr int TC_SCHED = 4;         // depth of the tile-scheduling ring
constexpr int TC_LOOKAHEAD = 2;     // tiles the MMA thread publishes ahead of the one it consumes
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK;   // 16 KiB
constexpr uint32_t TC_B_BYTES = TC_BN * TC_BK;   // 16 KiB
constexpr unsigned FULL = 0xffffffffu;
constexpr long long WAIT_BUDGET = TC_WAIT_TICKS;  // clock64 ticks (~2 s) per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// The same test, letting the hardware suspend the thread until the phase
// completes or about 20 us pass (a waiting warp then issues nothing, which
// leaves the issue slots of its scheduler to the epilogue warps).
__device__ __forceinline__ bool mbar_try_suspend(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity.  On timeout it raises the
// CTA abort flag and the device error word; every role then leaves its loop.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t *err, long long budget = WAIT_BUDGET)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_suspend(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row (1024-byte) swizzle atoms.
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29,
// unused for swizzled K-major, set to 1), stride byte offset >> 4 (32-45:
// 1024 bytes between 8-row groups), fixed 0b001 at bits 46-48, swizzle mode
// 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fff);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both operands e4m3 or both e5m2 (A and B type fields,
// bits 7-9 and 10-12: 0 = E4M3, 1 = E5M2).
__host__ __device__ constexpr uint32_t idesc_f8_f32(int M, int N, bool e5m2)
{
    return idesc_e4m3_f32(M, N) | (e5m2 ? (1u << 7) | (1u << 10) : 0u);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Ties registers written by tcgen05.ld to a point after tcgen05.wait::ld:
// the compiler sees them redefined here, so no use can move above the wait.
template <int N>
__device__ __forceinline__ void tmem_regs_after_wait(uint32_t (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+r"(v[i]));
}

// Named barrier 1 over the NT epilogue threads.
template <int NT>
__device__ __forceinline__ void epi_bar_n() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }
__device__ __forceinline__ void epi_bar() { epi_bar_n<128>(); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr));
}

// Exact integer value of an FP32 accumulator holding an integer in [0, 2^23).
__device__ __forceinline__ uint32_t f2u_exact(uint32_t bits)
{
    return __float_as_uint(__uint_as_float(bits) + 8388608.0f) - 0x4B000000u;
}

__device__ __forceinline__ int ordered_int(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float from_ordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Descending bitonic sort of n = 2^p (score, rank) pairs by the NT
// epilogue threads (tid in [0, NT)).
template <int NT>
__device__ void epi_bitonic_desc_n(float *s, uint64_t *r, int n, int tid)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            epi_bar_n<NT>();
            for (int i = tid; i < (n >> 1); i += NT) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const float s1 = s[lo], s2 = s[hi];
                const uint64_t r1 = r[lo], r2 = r[hi];
                const bool sw = desc ? better(s2, r2, s1, r1) : better(s1, r1, s2, r2);
                if (sw) { s[lo] = s2; s[hi] = s1; r[lo] = r2; r[hi] = r1; }
            }
        }
    }
    epi_bar_n<NT>();
}
__device__ void epi_bitonic_desc(float *s, uint64_t *r, int n, int tid) { epi_bitonic_desc_n<128>(s, r, n, tid); }

}  // namespace
}  // namespace fc
