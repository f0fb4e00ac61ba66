// Shared tcgen05 building blocks of the tensor-core kernels: shared-memory matrix
// descriptors for K-major tiles with the 64-byte swizzle, the bf16 MMA and its commit,
// bounded mbarrier waits, tensor-memory allocation and loads, and the bf16 piece split
// of FP32 operands (one piece: bf16 rounding; three pieces: v = v0 + v1 + v2 exactly).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace qmc {
namespace tc {

constexpr int TM = 128;            // tile rows = MMA M = TMEM lanes
constexpr int KC = 32;             // K per chunk: two MMA K-steps of 16
constexpr uint32_t ROWB = KC * 2;  // bytes of one tile row (32 bf16)
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major tile with the 64-byte swizzle: 8-row
// groups 512 bytes apart (stride-dimension offset), K-step ks of 16 bf16 starts 32 * ks
// bytes into the rows (the swizzle is applied to the final address, so the start
// address moves inside the swizzle atom).  The leading-dimension offset is not used by
// swizzled K-major layouts and is set to 16 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);            // start address
    d |= (uint64_t)1 << 16;                              // leading-dimension byte offset 16 (unused)
    d |= (uint64_t)(512 >> 4) << 32;                     // stride-dimension byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                              // descriptor version for tcgen05
    d |= (uint64_t)4 << 61;                              // 64-byte swizzle
    return d;
}

// byte offset of the 16-byte group g (k = 8g..8g+7) of row r in a swizzled tile
__device__ __forceinline__ uint32_t sw64_off(int r, int g) {
    return (uint32_t)r * ROWB + ((uint32_t)(g ^ ((r >> 1) & 3)) << 4);
}

// instruction descriptor: D = F32, A = B = BF16, both K-major, dense, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
}

__device__ __forceinline__ void mbar_init2(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane (no wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Split 8 consecutive k of one row into P bf16 pieces and store each piece's 16 bytes
// (group g of row r) into the tiles tile0 + p * piece_stride.
// The bf16 pieces of two FP32 values (a in the low, b in the high half of each word).
// Piece 0 is the round-to-nearest bf16 (one conversion per pair); in the split tier the
// residual r1 = v - v0 (exact, |r1| <= 2^-9 |v|, at most 16 significant bits) is cut into
// its top 8 bits v1 (truncation: keep the upper half of the FP32 word) and the exact rest
// v2 = r1 - v1 (at most 8 significant bits), so v = v0 + v1 + v2 exactly with |v1| <=
// 2^-9 |v| and |v2| <= 2^-16 |v|.  The truncations are integer byte permutes, which keeps
// the conversion pipe to one instruction per pair.
template <int P>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t (&w)[P]) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b);
    const uint32_t p0 = *reinterpret_cast<const uint32_t*>(&h0);
    w[0] = p0;
    if constexpr (P == 3) {
        const float ra = a - __uint_as_float(p0 << 16), rb = b - __uint_as_float(p0 & 0xFFFF0000u);
        const uint32_t ua = __float_as_uint(ra), ub = __float_as_uint(rb);
        w[1] = __byte_perm(ua, ub, 0x7632);
        const float sa = ra - __uint_as_float(ua & 0xFFFF0000u), sb = rb - __uint_as_float(ub & 0xFFFF0000u);
        w[2] = __byte_perm(__float_as_uint(sa), __float_as_uint(sb), 0x7632);
    }
}

// Split 8 consecutive k of one row into P bf16 pieces and store each piece's 16 bytes
// (group g of row r) into the tiles tile0 + p * piece_stride.
template <int P>
__device__ __forceinline__ void store_group(unsigned char* tile0, uint32_t piece_stride, int r, int g,
                                            const float* v) {
    uint32_t w[P][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t q[P];
        split_pair<P>(v[2 * i], v[2 * i + 1], q);
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][i] = q[p];
    }
    const uint32_t off = sw64_off(r, g);
#pragma unroll
    for (int p = 0; p < P; ++p)
        *reinterpret_cast<uint4*>(tile0 + p * piece_stride + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// Descriptor arithmetic: the start address sits in the low 14 bits as address / 16, so a
// descriptor of addr + bytes is the descriptor of addr plus bytes / 16 (shared-memory
// addresses stay below 256 KB, so the field never carries).  The issuing thread then spends
// one add per MMA instead of building a descriptor: the MMA issue rate of a single thread is
// otherwise the bound of these kernels.
__device__ __forceinline__ uint64_t desc_add(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }

// The piece products of one K-step, smallest first: A piece i times B piece j; adesc, bdesc
// describe piece 0 of each operand at this K-step, the pieces A_PIECE / B_PIECE bytes apart.
template <int P, uint32_t A_PIECE, uint32_t B_PIECE>
__device__ __forceinline__ void issue_kstep(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            bool& first) {
    constexpr int NP = P == 3 ? 6 : 1;
    constexpr int pi[6] = {2, 1, 0, 1, 0, 0};
    constexpr int pj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = P == 3 ? pi[q] : 0, j = P == 3 ? pj[q] : 0;
        mma_bf16(tmem, desc_add(adesc, i * A_PIECE), desc_add(bdesc, j * B_PIECE), idesc, first ? 0u : 1u);
        first = false;
    }
}

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// one poll of phase `parity` of an mbarrier (true once that phase has completed)
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned char* align_1k(unsigned char* p) {
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

// ---------------------------------------------------------------------------------------------
// The warp-specialised kernels' building blocks: mbarrier phases (every wait bounded), TMA tile
// loads completing on an mbarrier, the MMA with A in tensor memory, tensor-memory stores and loads.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar) : "memory");
}
// Untiled bulk copy of `bytes` contiguous bytes (16-byte aligned addresses, a multiple of 16
// bytes) into this CTA's shared memory, completing on the mbarrier's transaction count
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// D (tensor memory) += A (tensor memory, M rows = lanes, two bf16 of consecutive K per 32-bit
// column) x B (shared memory, descriptor), or D = A x B when accumulate is 0
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        :: "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// 4 or 8 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&r)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
}
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                    "r"(r[7]) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

}  // namespace tc
}  // namespace qmc
