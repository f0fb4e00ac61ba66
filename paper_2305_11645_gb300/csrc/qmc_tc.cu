// Tensor-core block products for the split and bf16 tiers: the coarse block products
// B_e = X_e A_e of Algorithm 2 (X~_I A~_I on the b^(m-I) distinct rows of weight block I)
// and the block gradients dA_e = X_e^T F_e of the adjoint, on tcgen05.mma (kind::f16,
// bf16 operands, FP32 accumulation in tensor memory).  These compact kernels serve the
// problems below the level passes' and the fused adjoint's size thresholds, and the
// adjoint's levels that the TMA kernels do not take (fewer than 32 distinct rows, or
// folded from a materialised level on the fly); large problems run qmc_level_tc.cu,
// qmc_foldgrad_tc.cu and qmc_grad_tc.cu.
//
// Split tier.  Every FP32 operand v is written exactly as three bf16 pieces
//     v = v0 + v1 + v2,   v0 = bf16(v) (nearest), v1 = the top 8 bits of v - v0,
//     v2 = v - v0 - v1,   |v1| <= 2^-9 |v|, |v2| <= 2^-16 |v|
// (each difference is exact in FP32, so the three pieces hold all 24 bits of v), and a
// product keeps the six piece products with i + j <= 2:
//     v w ~ v0 w0 + v0 w1 + v1 w0 + v0 w2 + v1 w1 + v2 w0,
// the bf16x6 scheme of Henry, Tang and Heinecke (ARITH 2019).  The dropped terms are
// below 2^-24 |v w|.  All six products accumulate into one FP32 accumulator (bf16 keeps
// the FP32 exponent range, so no operand scaling is needed).
// Bf16 tier.  One piece, one product: v w ~ bf16(v) bf16(w).
//
// Structure of both kernels.  One CTA of 128 threads owns a 128-row tile of the MMA's M
// dimension.  K runs in chunks of 32 through two shared-memory stages.  Every thread
// loads its share of chunk c + 1 from global memory into registers (coalesced along
// the rows of the operand tiles) before it splits chunk c into bf16 pieces and stores
// them, so the loads of one chunk overlap the conversion of the previous one.  The
// pieces sit in K-major tiles with the 64-byte swizzle (rows of 32 bf16 = 64 bytes;
// the 16-byte group g of row r is stored at group g ^ ((r >> 1) & 3)), which keeps the
// threads' 16-byte stores and the tensor core's reads free of bank conflicts.  One
// thread issues a chunk's MMAs and commits them to the stage's mbarrier; the stage is
// refilled once that barrier has completed.  After the last chunk the threads read
// their rows of the accumulator (tcgen05.ld, TMEM lane = tile row) and store them.
// Every mbarrier wait is bounded; a wait that runs out sets the device error word, the
// tile's outputs are written as NaN and the kernel releases its tensor memory and returns.
#include <cuda_bf16.h>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

__device__ unsigned int g_tc_error;      // sticky: bit 0 = a bounded mbarrier wait ran out

using namespace tc;

namespace {

constexpr int NJ = 64;             // backward: block-gradient columns j per tile (MMA N <= 64)

__device__ __forceinline__ int entry_of(const Chain& ch, int bx) {
    int e = 0;
    while (e + 1 < ch.count && bx >= ch.tile0[e + 1]) ++e;
    return e;
}


// Thread-block prologue / epilogue shared by both kernels.
__device__ __forceinline__ uint32_t tc_setup(uint64_t* bar, uint32_t* tmem_slot, uint32_t ncols) {
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tmem_slot), ncols);
    if (threadIdx.x == 0) mbar_init2(bar);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    return *tmem_slot;
}
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t ncols) {
    fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, ncols);
    }
}

// After a wait ran out: one more bounded wait (by one thread, before the teardown's barrier) on
// the barrier of the last committed chunk.  A commit arrives once every MMA issued before it has
// completed, so when this wait succeeds no MMA still reads the stages or writes the tensor memory
// that the teardown releases.  If it runs out too, the CTA returns regardless (bounded).
__device__ __forceinline__ void drain_committed(uint64_t* bar, int committed) {
    if (committed >= 0) mbar_wait(smem_u32(&bar[committed & 1]), (committed >> 1) & 1);
}

// Publish the stage to the tensor core; returns false (in every thread) if any thread's
// wait ran out.
__device__ __forceinline__ bool publish_stage(bool ok) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before_sync();
    ok = __syncthreads_and(ok);
    fence_after_sync();
    return ok;
}

// 16-byte asynchronous copy global -> shared (zero-filled when !valid; src must still be a
// valid address), and the per-thread copy groups
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace

// ------------------------------------------------------------------------------------------
// Forward: B_e[r][t/4][rho][t%4] = sum_{k < tau_e} tab[r][tab_e + k n_e + rho] A[col0_e + k][t].
// Tile: 128 rows rho x 128 columns t; M = rho, N = t, K = k.  Both operands are contiguous
// along the tile's rows in global memory (rho for X, t for A), so thread i loads row i of
// X and row i (column t0 + i) of A for the 32 k of a chunk; every load instruction of a
// warp reads 128 contiguous bytes.
// Shared memory per stage: X and A tiles, P pieces x 128 rows x 64 B each.
// ------------------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) k_coarse_fwd_tc(const float* __restrict__ tab, long long tab_stride,
                                                       const float* __restrict__ A, int ldA, int tau_pad,
                                                       const __grid_constant__ Chain ch, float* __restrict__ B,
                                                       long long B_stride) {
    constexpr uint32_t TILE = TM * ROWB;              // one piece of one operand: 8 KB
    constexpr uint32_t OPND = P * TILE;
    constexpr uint32_t STAGE = 2 * OPND;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);          // the swizzle pattern follows address bits 7-8
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int e = entry_of(ch, blockIdx.x);
    const long long rho0 = (long long)(blockIdx.x - ch.tile0[e]) * TM;
    const int logn = ch.logn[e], tau_e = ch.tau[e];
    const long long n_e = 1LL << logn;
    const int t0 = blockIdx.y * TM;
    const int r = blockIdx.z;
    const int nchunks = (tau_e + KC - 1) / KC;
    const uint32_t tmem = tc_setup(bar, tmem_slot, TM);

    // 256 threads: thread tq = tid % 128 of warps 0-3 loads and converts row rho0 + tq of X (its
    // TMEM lane), of warps 4-7 row t0 + tq of A^T; the two halves store the accumulator's
    // columns 0-63 and 64-127 of their lanes
    const int tq = tid & (TM - 1);
    const bool lower = tid < TM;
    const long long rho = rho0 + tq;
    const int t = t0 + tq;
    const bool row_ok = rho < n_e, col_ok = t < tau_pad;
    const bool src_ok = lower ? row_ok : col_ok;
    const float* src = lower ? tab + (long long)r * tab_stride + ch.tab[e] + (row_ok ? rho : 0)
                             : A + (long long)ch.col0[e] * ldA + (col_ok ? t : 0);
    const long long kstride = lower ? n_e : (long long)ldA;
    float vv[KC];
    bool ok = true, first = true;
    int committed = -1;                                // last chunk whose MMAs were committed
    // Iteration it loads chunk it and converts chunk it - 1 (one load site keeps the code small).
    for (int it = 0; it <= nchunks; ++it) {
        float vc[KC];
#pragma unroll
        for (int i = 0; i < KC; ++i) vc[i] = vv[i];
        if (it < nchunks) {
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                const int k = it * KC + i;
                vv[i] = (k < tau_e && src_ok) ? __ldg(src + (long long)k * kstride) : 0.0f;
            }
        }
        if (it == 0) continue;
        const int c = it - 1;
        const int s = c & 1;
        unsigned char* Xs = smem + s * STAGE;
        unsigned char* As = Xs + OPND;
        const int ksteps = min(2, (tau_e - c * KC + 15) >> 4);
        if (c >= 2) ok = mbar_wait(smem_u32(&bar[s]), ((c - 2) >> 1) & 1);
        if (ok) {
            unsigned char* dst = lower ? Xs : As;
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (g < 2 * ksteps) store_group<P>(dst, TILE, tq, g, vc + 8 * g);
        }
        ok = publish_stage(ok);
        if (!ok) break;
        if (tid == 0) {
            const uint32_t idesc = idesc_bf16(TM);
            for (int ks = 0; ks < ksteps; ++ks)
                issue_kstep<P, TILE, TILE>(tmem, smem_desc_sw64(smem_u32(Xs) + 32 * ks),
                                           smem_desc_sw64(smem_u32(As) + 32 * ks), idesc, first);
            mma_commit(smem_u32(&bar[s]));
        }
        committed = c;
    }
    if (ok) ok = mbar_wait(smem_u32(&bar[(nchunks - 1) & 1]), ((nchunks - 1) >> 1) & 1);
    fence_after_sync();
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        atomicOr(&g_tc_error, 1u);
        drain_committed(bar, committed);
    }

    float* Be = B + (long long)r * B_stride + ch.boff[e];
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    {
        const int half = lower ? 0 : 1;
        uint32_t d[2][32];
        if (ok) {
            tmem_ld32(lane_addr + half * 64, d[0]);
            tmem_ld32(lane_addr + half * 64 + 32, d[1]);
            tmem_wait_ld();
        }
        if (row_ok) {
#pragma unroll
            for (int g = 0; g < 16; ++g) {
                const int tt = t0 + half * 64 + 4 * g;
                const uint32_t* q = &d[g >> 3][(g & 7) * 4];
                const float4 v = ok ? make_float4(__uint_as_float(q[0]), __uint_as_float(q[1]),
                                                  __uint_as_float(q[2]), __uint_as_float(q[3]))
                                    : make_float4(qnan(), qnan(), qnan(), qnan());
                if (tt < tau_pad) *reinterpret_cast<float4*>(Be + (((long long)(tt >> 2) << logn) << 2) + (rho << 2)) = v;
            }
        }
    }
    tc_teardown(tmem, TM);
}

// ------------------------------------------------------------------------------------------
// Backward: part[e][sp][j][t] = sum over k = (r, rho) in split sp of
//           tab[r][tab_e + j n_e + rho] * F_e[r][rho][t],
// F_e[rho] = sum_{q < 2^flog} Fsrc[rho + q n_e] (the adjoint of the periodic tiling).
// Computed transposed, D[t][j] = sum_k F_e[k][t] X[k][j]: M = t (128 rows), N = j (a tile
// of up to 64 columns of the entry), K = k.  F is contiguous along t, so thread i loads
// column t0 + i of F for the 32 k of a chunk (coalesced over the warp); X is contiguous
// along k, so each thread loads 16 consecutive k of one row j (float4 loads when the
// chunk lies inside one shift's rows, n_e >= 32).  A split covers a multiple of 32 rows.
// Shared memory per stage: F^T (P pieces x 128 rows x 64 B) and X (P x 64 rows x 64 B).
// ------------------------------------------------------------------------------------------
// Main path (levels with at least 32 distinct rows whose F is read without an on-the-fly fold):
// the raw FP32 chunks of F (32 rows x 128 columns t) and X (64 rows j x 32 k) are copied into
// RAWS shared-memory stages with 16-byte cp.async, RAWS - 1 chunks ahead of the one being
// converted, so the copies need no registers and their latency is hidden behind the
// conversion and the MMAs; each thread then converts its row of F^T and its half row of X from
// shared memory into the bf16 pieces.  Other levels take the register path below (one chunk of
// loads in flight).
constexpr int RAWS = 4;
// Chunk c accumulates into tensor-memory accumulator c % NACC (64 columns each), summed in FP32
// in a fixed order at the end: an FP32 accumulation chain inside the tensor core is then at
// most kper / NACC rows long, which keeps the split tier's gradient error near 2^-24 sqrt(64).
constexpr int NACC = 4;
constexpr uint32_t RAW_F = KC * TM * 4;              // F chunk: [k][t], 512 B rows
constexpr uint32_t RAW_XROW = (KC + 4) * 4;          // X chunk rows padded to 144 B (bank spread)
constexpr uint32_t RAW_X = NJ * RAW_XROW;
constexpr uint32_t RAW_STAGE = RAW_F + RAW_X;

template <int P>
__global__ void __launch_bounds__(256, 1) k_coarse_grad_tc(const float* __restrict__ tab, long long tab_stride,
                                                           const float* __restrict__ Froot, long long root_stride,
                                                           const float* __restrict__ Fchain, long long chain_stride,
                                                           int tau_pad, const __grid_constant__ Chain ch,
                                                           float* __restrict__ part, int reff, float xcen) {
    constexpr uint32_t TILEA = TM * ROWB, TILEB = NJ * ROWB;
    constexpr uint32_t OPA = P * TILEA, OPB = P * TILEB;
    constexpr uint32_t STAGE = OPA + OPB;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);          // the swizzle pattern follows address bits 7-8
    unsigned char* raw = smem + 2 * STAGE;             // RAWS raw FP32 stages (main path)
    uint64_t* bar = reinterpret_cast<uint64_t*>(raw + RAWS * RAW_STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(raw + RAWS * RAW_STAGE + 16);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int e = entry_of(ch, blockIdx.x);
    const int local = blockIdx.x - ch.tile0[e];
    const int tau_e = ch.tau[e], logn = ch.logn[e], nsplit = ch.split[e];
    const int jt = local / nsplit, sp = local - jt * nsplit;
    const int j0 = jt * NJ;
    const int nj = min(NJ, tau_e - j0);
    const uint32_t nmma = (uint32_t)((nj + 15) & ~15);
    const long long n_e = 1LL << logn;
    const int fold = 1 << ch.flog[e];
    const float* Fsrc = (ch.fsel[e] ? Fchain : Froot) + ch.foff[e];
    const long long F_stride = ch.fsel[e] ? chain_stride : root_stride;
    const long long rstep = n_e * tau_pad;
    const long long Ktot = (long long)reff * n_e;
    const long long kb = (long long)sp * ch.kper[e], ke = min(Ktot, kb + ch.kper[e]);
    const int nchunks = ke > kb ? (int)((ke - kb + KC - 1) / KC) : 0;
    const int t0 = blockIdx.y * TM;
    const uint32_t tmem = tc_setup(bar, tmem_slot, NACC * NJ);

    // 256 threads: thread tq = tid % 128 owns column t = t0 + tq (TMEM lane tq); in the main path
    // every thread converts half a row of F^T and a quarter row of X, and all share the copies
    // and the epilogue
    const int tq = tid & (TM - 1);
    const bool lower = tid < TM;
    const int t = t0 + tq;
    const bool col_ok = t < tau_pad;
    const int jrow = tq & (NJ - 1), khalf = tq >> 6;  // X: row j0 + jrow, one half of the chunk
    const bool jrow_ok = jrow < nj;
    const float* xcol = tab + ch.tab[e] + (long long)(j0 + (jrow_ok ? jrow : 0)) * n_e;
    const float* Fcol = Fsrc + (col_ok ? t : 0);
    const bool whole = n_e >= KC;                      // a chunk never crosses a shift boundary
    bool ok = true;
    int committed = -1;                                // last chunk whose MMAs were committed
    if (whole && fold == 1) {
        // ------------------------------------------------------------ main path
        const int lane = tid & 31;
        auto copy_chunk = [&](int c) {
            if (c < nchunks) {
                const long long k0 = kb + (long long)c * KC;
                const long long rr = k0 >> logn, rho0 = k0 & (n_e - 1);
                const uint32_t rs = smem_u32(raw + (c % RAWS) * RAW_STAGE);
                // F: warp w copies rows 4w .. 4w + 3, lane l the columns t0 + 4l .. + 3
                const bool tin = t0 + 4 * lane < tau_pad;
                const float* fsrc = Fsrc + rr * F_stride + rho0 * tau_pad + (tin ? t0 + 4 * lane : 0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int row = warp * 4 + i;
                    cp_async16(rs + row * (TM * 4) + lane * 16, fsrc + (long long)row * tau_pad, tin);
                }
                // X: 64 rows j x 8 groups of 4 k, two per thread
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int idx = tid + 256 * u, jr = idx >> 3, q = idx & 7;
                    const bool jin = jr < nj;
                    const float* xsrc = tab + ch.tab[e] + (long long)(j0 + (jin ? jr : 0)) * n_e + rr * tab_stride +
                                        rho0 + 4 * q;
                    cp_async16(rs + RAW_F + jr * RAW_XROW + q * 16, xsrc, jin);
                }
            }
            cp_async_commit();                          // (one group per chunk, possibly empty)
        };
#pragma unroll
        for (int c = 0; c < RAWS - 1; ++c) copy_chunk(c);
        for (int c = 0; c < nchunks; ++c) {
            copy_chunk(c + RAWS - 1);                   // into the stage chunk c - 1 was converted from
            cp_async_wait<RAWS - 1>();                  // this thread's copies of chunk c have landed
            __syncthreads();                            // and every thread's
            const unsigned char* rs = raw + (c % RAWS) * RAW_STAGE;
            const int s = c & 1;
            unsigned char* Fs = smem + s * STAGE;
            unsigned char* Xs = Fs + OPA;
            if (c >= 2) ok = mbar_wait(smem_u32(&bar[s]), ((c - 2) >> 1) & 1);
            if (ok) {
                // every thread: k 16h .. 16h + 15 of row tq of F^T (h = tid / 128), and k 8q .. 8q + 7
                // of row tid % 64 of X (q = tid / 64)
                const int h = tid >> 7;
                float fc[16];
                const float* fr = reinterpret_cast<const float*>(rs) + 16 * h * TM + tq;
#pragma unroll
                for (int i = 0; i < 16; ++i) fc[i] = fr[i * TM];
                store_group<P>(Fs, TILEA, tq, 2 * h, fc);
                store_group<P>(Fs, TILEA, tq, 2 * h + 1, fc + 8);
                const int xj = tid & (NJ - 1), xq = tid >> 6;
                if (xj < (int)nmma) {
                    const float4* xr = reinterpret_cast<const float4*>(rs + RAW_F + xj * RAW_XROW) + 2 * xq;
                    const float4 a = xr[0], b = xr[1];
                    const float d = xj < nj ? xcen : 0.0f;          // (padding rows stay zero)
                    const float xv[8] = {a.x - d, a.y - d, a.z - d, a.w - d, b.x - d, b.y - d, b.z - d, b.w - d};
                    store_group<P>(Xs, TILEB, xj, xq, xv);
                }
            }
            ok = publish_stage(ok);
            if (!ok) break;
            if (tid == 0) {
                const uint32_t idesc = idesc_bf16(nmma);
                bool fresh = c < NACC;                  // the accumulator's first chunk
                for (int ks = 0; ks < 2; ++ks)
                    issue_kstep<P, TILEA, TILEB>(tmem + (uint32_t)((c % NACC) * NJ),
                                                 smem_desc_sw64(smem_u32(Fs) + 32 * ks),
                                                 smem_desc_sw64(smem_u32(Xs) + 32 * ks), idesc, fresh);
                mma_commit(smem_u32(&bar[s]));
            }
            committed = c;
        }
        cp_async_wait<0>();
    } else {
    float fv[KC], xw[16];
    // Iteration it loads chunk it and converts chunk it - 1 (one load site keeps the code small).
    for (int it = 0; it <= nchunks; ++it) {
        float fc[KC], xc[16];
#pragma unroll
        for (int i = 0; i < KC; ++i) fc[i] = fv[i];
#pragma unroll
        for (int i = 0; i < 16; ++i) xc[i] = xw[i];
        if (it < nchunks && lower) {                   // (warps 4-7 only join the barriers here)
            const long long k0 = kb + (long long)it * KC;
            if (whole) {
                const long long rr = k0 >> logn, rho0 = k0 & (n_e - 1);
                const float* fp = Fcol + rr * F_stride + rho0 * tau_pad;
#pragma unroll
                for (int i = 0; i < KC; ++i) {
                    float v = 0.0f;
                    if (k0 + i < ke && col_ok) {
                        const float* q = fp + (long long)i * tau_pad;
                        v = __ldg(q);
#pragma unroll 1
                        for (int f = 1; f < fold; ++f) v += __ldg(q + f * rstep);
                    }
                    fv[i] = v;
                }
                const float* xp = xcol + rr * tab_stride + rho0 + 16 * khalf;
                const long long kx = k0 + 16 * khalf;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (jrow_ok && kx + 4 * i + 4 <= ke) v4 = __ldg(reinterpret_cast<const float4*>(xp) + i);
                    else if (jrow_ok) {
                        v4.x = kx + 4 * i + 0 < ke ? __ldg(xp + 4 * i + 0) : 0.f;
                        v4.y = kx + 4 * i + 1 < ke ? __ldg(xp + 4 * i + 1) : 0.f;
                        v4.z = kx + 4 * i + 2 < ke ? __ldg(xp + 4 * i + 2) : 0.f;
                    }
                    xw[4 * i] = v4.x; xw[4 * i + 1] = v4.y; xw[4 * i + 2] = v4.z; xw[4 * i + 3] = v4.w;
                }
            } else {
                // levels with fewer than 32 distinct rows: a chunk spans several shifts
                const long long r0 = k0 >> logn;
                const int rho0 = (int)(k0 & (n_e - 1));
#pragma unroll
                for (int i = 0; i < KC; ++i) {
                    const int q = rho0 + i;
                    float v = 0.0f;
                    if (k0 + i < ke && col_ok) {
                        const float* fq = Fcol + (r0 + (q >> logn)) * F_stride + (long long)(q & (n_e - 1)) * tau_pad;
                        v = __ldg(fq);
#pragma unroll 1
                        for (int f = 1; f < fold; ++f) v += __ldg(fq + f * rstep);
                    }
                    fv[i] = v;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int q = rho0 + 16 * khalf + i;
                    xw[i] = (k0 + 16 * khalf + i < ke && jrow_ok)
                                ? __ldg(xcol + (r0 + (q >> logn)) * tab_stride + (q & (n_e - 1))) : 0.0f;
                }
            }
        }
        if (it == 0) continue;
        const int c = it - 1;
        const int s = c & 1;
        unsigned char* Fs = smem + s * STAGE;
        unsigned char* Xs = Fs + OPA;
        const int ksteps = (int)min(2LL, (ke - kb - (long long)c * KC + 15) >> 4);
        if (c >= 2) ok = mbar_wait(smem_u32(&bar[s]), ((c - 2) >> 1) & 1);
        if (ok && lower) {
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (g < 2 * ksteps) store_group<P>(Fs, TILEA, tq, g, fc + 8 * g);
            if (khalf < ksteps) {
                // (centred rows; rows beyond the split's end meet F = 0, padding columns are not stored)
                const float d = jrow_ok ? xcen : 0.0f;
#pragma unroll
                for (int i = 0; i < 16; ++i) xc[i] -= d;
                store_group<P>(Xs, TILEB, jrow, 2 * khalf, xc);
                store_group<P>(Xs, TILEB, jrow, 2 * khalf + 1, xc + 8);
            }
        }
        ok = publish_stage(ok);
        if (!ok) break;
        if (tid == 0) {
            const uint32_t idesc = idesc_bf16(nmma);
            bool fresh = c < NACC;                      // the accumulator's first chunk
            for (int ks = 0; ks < ksteps; ++ks)
                issue_kstep<P, TILEA, TILEB>(tmem + (uint32_t)((c % NACC) * NJ),
                                             smem_desc_sw64(smem_u32(Fs) + 32 * ks),
                                             smem_desc_sw64(smem_u32(Xs) + 32 * ks), idesc, fresh);
            mma_commit(smem_u32(&bar[s]));
        }
        committed = c;
    }
    }
    if (ok && nchunks > 0) ok = mbar_wait(smem_u32(&bar[(nchunks - 1) & 1]), ((nchunks - 1) >> 1) & 1);
    fence_after_sync();
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        atomicOr(&g_tc_error, 1u);
        drain_committed(bar, committed);
    }

    // D[t][j]: TMEM lane = t - t0, column = j - j0; warps w and w + 4 share lanes 32 (w % 4) ..,
    // the lower ones store columns 0..31, the upper ones 32..63
    const int cb = lower ? 0 : 32;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb;
    float* pe = part + ch.poff[e] + ((long long)sp * tau_e + j0 + cb) * tau_pad + t;
    float sum[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) sum[i] = 0.0f;
    const bool have = ok && nchunks > 0;
    if (have && (int)nmma > cb) {
        for (int a = 0; a < NACC && a < nchunks; ++a) {   // accumulators in order
            uint32_t d[32];
            tmem_ld32(lane_addr + (uint32_t)(a * NJ), d);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) sum[i] += __uint_as_float(d[i]);
        }
    }
    if (col_ok) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (cb + i < nj) {
                const float v = have ? sum[i] : (ok ? 0.0f : qnan());
                pe[(long long)i * tau_pad] = v;
            }
        }
    }
    tc_teardown(tmem, NACC * NJ);
}

// ------------------------------------------------------------------------------------------
// launchers.  The forward's shared-memory request also caps its CTAs per SM so that their
// tensor memory (128 columns each) fits in the SM's 512 columns.
// ------------------------------------------------------------------------------------------
namespace {
template <int P> constexpr size_t fwd_smem() {
    const size_t need = 2 * (2 * P * TM * ROWB) + 1024 + 64;
    return need < 58 * 1024 ? 58 * 1024 : need;         // <= 3 CTAs per SM
}
template <int P> constexpr size_t bwd_smem() {
    return 2 * (P * TM * ROWB + P * NJ * ROWB) + RAWS * RAW_STAGE + 1024 + 64;   // one CTA per SM
}
}  // namespace

int tc_fwd_rows() { return TM; }
int tc_grad_cols() { return NJ; }

cudaError_t launch_coarse_fwd_tc(const float* tab, long long tab_stride, const float* A, int ldA, int tau_pad,
                                 const Chain& ch, float* B, long long B_stride, int reff, int pieces,
                                 cudaStream_t st) {
    if (ch.count == 0) return cudaSuccess;
    if (pieces != 1 && pieces != 3) return cudaErrorInvalidValue;
    dim3 grid(ch.tile0[ch.count], (tau_pad + TM - 1) / TM, reff);
    if (pieces == 3) {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_fwd_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fwd_smem<3>());
        if (e != cudaSuccess) return e;
        k_coarse_fwd_tc<3><<<grid, 256, fwd_smem<3>(), st>>>(tab, tab_stride, A, ldA, tau_pad, ch, B, B_stride);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_fwd_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fwd_smem<1>());
        if (e != cudaSuccess) return e;
        k_coarse_fwd_tc<1><<<grid, 256, fwd_smem<1>(), st>>>(tab, tab_stride, A, ldA, tau_pad, ch, B, B_stride);
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_grad_tc(const float* tab, long long tab_stride, const float* Froot, long long root_stride,
                                  const float* Fchain, long long chain_stride, int tau_pad, const Chain& ch,
                                  float* part, int reff, int ntiles, int pieces, float xc, cudaStream_t st) {
    if (ch.count == 0 || ntiles == 0) return cudaSuccess;
    if (pieces != 1 && pieces != 3) return cudaErrorInvalidValue;
    dim3 grid(ntiles, (tau_pad + TM - 1) / TM);
    if (pieces == 3) {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_grad_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bwd_smem<3>());
        if (e != cudaSuccess) return e;
        k_coarse_grad_tc<3><<<grid, 256, bwd_smem<3>(), st>>>(tab, tab_stride, Froot, root_stride, Fchain,
                                                              chain_stride, tau_pad, ch, part, reff, xc);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_grad_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bwd_smem<1>());
        if (e != cudaSuccess) return e;
        k_coarse_grad_tc<1><<<grid, 256, bwd_smem<1>(), st>>>(tab, tab_stride, Froot, root_stride, Fchain,
                                                              chain_stride, tau_pad, ch, part, reff, xc);
    }
    return cudaGetLastError();
}

// Self-test of the bounded waits: one thread polls, at most `polls` times, an mbarrier that nothing
// arrives at, then raises bit 31 of the error word as a tensor-core kernel whose wait ran out raises
// bit 0.  The kernel returns either way; the host reads the word through qmc_device_status.
__global__ void k_selftest_wait(uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t a = tc::smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool done = false;
    for (uint32_t it = 0; it < polls && !done; ++it) done = tc::mbar_try(a, 0);
    if (!done) atomicOr(&g_tc_error, 0x80000000u);
}

cudaError_t launch_selftest_wait(uint32_t polls, cudaStream_t st) {
    k_selftest_wait<<<1, 32, 0, st>>>(polls);
    return cudaGetLastError();
}

cudaError_t tc_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_tc_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(unsigned int));
}

}  // namespace qmc
