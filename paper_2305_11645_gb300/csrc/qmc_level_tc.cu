// Algorithm 2 on the tensor cores, from the coarsest level down (split and bf16 tiers).
//
// The coarse levels I >= JF (the levels the fine band does not expand) contribute to root row
// rho of the fine band the sum over I of X~_I[rho mod n_I] A~_I, X~_I the n_I = 2^(m-I)
// distinct rows of weight block I and A~_I its rows of A.  Algorithm 2 forms this top down,
//     P~_I = tile(P~_{I+1}, 2) + X~_I A~_I,
// each level's block product on its distinct rows only.  Here a pass does one such step (or
// several levels at once: the sum over its levels of X~_I[rho mod n_I] A~_I plus the previous
// pass's rows rho mod n_next), and the last pass writes the root values S.  The N x tau
// product never exists; each level's partial sum is written once at n_I rows.
//
// Operands.  Every FP32 operand v is written exactly as three bf16 pieces v0 + v1 + v2 (split
// tier; bf16x6: six piece products with i + j <= 2, see qmc_tc.cuh) or rounded to one (bf16
// tier), by k_split_x (the point table of the coarse levels) and k_split_a (A's coarse rows),
// in row-major blocks of 32 columns: a row is 64 bytes, which a TMA copy with the 64-byte
// swizzle places in shared memory exactly as the MMA's K-major descriptors read it.
//
// k_level_tc.  One persistent CTA per SM walks the pass's tiles of 128 rows x 256 columns:
//   warp 0      TMA producer: for each 32-column chunk of each level, the P pieces of the X tile
//               (128 x 32) and of the A tile (256 x 32) into a ring of shared-memory stages;
//   warp 1      allocates 512 tensor-memory columns (two 128 x 256 FP32 accumulators) and issues,
//               from one thread, the chunk's MMAs (M = 128, N = 256, K = 16, bf16 -> FP32), then
//               commits the stage back to the producer and, after a tile's last chunk, the
//               accumulator to the epilogue;
//   warps 2-13  epilogue: each reads its 32 rows x 96 or 64 columns of the accumulator, adds the
//               coarser pass's rows (rho mod n_next) and stores the tile, in the [t/4][rho][4]
//               layout of the root values, while the MMAs of the next tile fill the other
//               accumulator.
// Every wait is bounded: one that runs out sets the device error word and the role stops;
// the other roles' waits then run out in turn, the MMA thread waits (bounded) for its last
// commit, and the CTA releases its tensor memory and returns.  The call's outputs are then
// undefined and qmc_device_status reports QMC_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

// sticky: bit 0 = a bounded wait of a level pass ran out (read with level_error_word; each
// translation unit of the library has its own device symbols)
__device__ unsigned int g_level_error;

using namespace tc;

namespace {

constexpr int LT_M = 128;               // tile rows (MMA M, tensor-memory lanes)
constexpr int LT_N = 256;               // tile columns t (MMA N)
constexpr uint32_t XPIECE = LT_M * 64;  // one piece of the X tile: 128 rows x 64 bytes
constexpr uint32_t APIECE = LT_N * 64;  // one piece of the A tile: 256 rows x 64 bytes
constexpr int kEpi = 12;                // epilogue warps: 3 per tensor-memory lane quarter
constexpr int kThreads = 64 + 32 * kEpi;   // producer, MMA, epilogue

template <int P> constexpr int stages() { return P == 3 ? 3 : 6; }
template <int P> constexpr uint32_t stage_bytes() { return P * (XPIECE + APIECE); }
template <int P> constexpr size_t level_smem() {
    return 1024 + (size_t)stages<P>() * stage_bytes<P>() + 256;
}


// ------------------------------------------------------------------------------------------
// k_split_x: the coarse levels' point-table entries as bf16 pieces.  Thread (row, g) of block
// (level s, piece-chunk kc) writes the 8 columns 32 kc + 8 g .. + 7 of row rho of the level
// (zero beyond its tau_I columns) for every piece; row rho < n'_I reads table row rho mod n_I.
// Four consecutive threads take the four 16-byte groups of one row, so a warp writes 8 whole
// 64-byte rows of a piece (512 contiguous bytes) and reads 8 consecutive table rows (one 32-byte
// sector) of each of 4 columns per load (with consecutive rows per thread, each 16-byte store
// filled a quarter of a different row: 0.28 ms against 0.21 ms on the 2^20-point step).
// ------------------------------------------------------------------------------------------
struct SplitXArgs {
    int nlev;
    LevelSeg seg[kMaxPasses];        // every coarse level with columns (the passes' segments)
    long long blk0[kMaxPasses + 1];  // prefix sums of the (level, chunk) blocks' rows x 4 groups
};

template <int P>
__global__ void __launch_bounds__(256) k_split_x(const float* __restrict__ tab, long long tab_stride,
                                                 const __grid_constant__ SplitXArgs sa, long long rows_per_shift,
                                                 uint4* __restrict__ xp, float xc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= sa.blk0[sa.nlev]) return;
    int l = 0;
    while (l + 1 < sa.nlev && i >= sa.blk0[l + 1]) ++l;
    const LevelSeg& sg = sa.seg[l];
    const long long loc = i - sa.blk0[l];
    const long long nrep = 1LL << sg.logn_rep;
    const int g = (int)(loc & 3);
    const long long rho = (loc >> 2) & (nrep - 1);
    const int kc = (int)(loc >> (2 + sg.logn_rep));
    const float* src = tab + (long long)r * tab_stride + sg.tab + (rho & ((1LL << sg.logn) - 1));
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int jj = kc * 32 + g * 8 + q;
        v[q] = jj < sg.tau ? __ldg(src + ((long long)jj << sg.logn)) - xc : 0.0f;
    }
    uint32_t w[P][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t pc[P];
        split_pair<P>(v[2 * q], v[2 * q + 1], pc);
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][q] = pc[p];
    }
    uint4* base = xp + ((long long)r * rows_per_shift + sg.xrow) * 4 + g;
#pragma unroll
    for (int p = 0; p < P; ++p)
        base[(((long long)(p * sg.chunks + kc) << sg.logn_rep) + rho) * 4] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// k_split_a: A's coarse rows as bf16 pieces, one block of tA rows (columns t) per (level, piece,
// chunk).  Thread (t, g) of a level chunk reads 8 rows j of A at column t (consecutive threads,
// consecutive t: contiguous reads) and writes its 16 bytes of every piece.
template <int P>
__global__ void __launch_bounds__(256) k_split_a(const float* __restrict__ A, int ldA, int tau,
                                                 const __grid_constant__ SplitXArgs sa, int tA, uint4* __restrict__ ap) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // block (level l, chunk kc) holds tA x 4 threads
    long long acc = 0;
    int l = 0, kc = -1;
    for (; l < sa.nlev; ++l) {
        const long long n = (long long)sa.seg[l].chunks * tA * 4;
        if (i < acc + n) { kc = (int)((i - acc) / ((long long)tA * 4)); break; }
        acc += n;
    }
    if (kc < 0) return;
    const LevelSeg& sg = sa.seg[l];
    const long long loc = i - acc - (long long)kc * tA * 4;
    const int t = (int)(loc % tA), g = (int)(loc / tA);
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int jj = kc * 32 + g * 8 + q;
        v[q] = (jj < sg.tau && t < tau) ? __ldg(A + (long long)(sg.col0 + jj) * ldA + t) : 0.0f;
    }
    uint32_t w[P][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t pc[P];
        split_pair<P>(v[2 * q], v[2 * q + 1], pc);
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][q] = pc[p];
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        ap[(sg.arow + (long long)(p * sg.chunks + kc) * tA + t) * 4 + g] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ------------------------------------------------------------------------------------------
// k_level_tc: one pass of the top-down accumulation (see the file comment)
// ------------------------------------------------------------------------------------------
struct TileIdx {
    int r, t0;
    long long rho0;
};

// Tile order: the 256-column tiles of one row tile are consecutive (they share the X tiles),
// then the row tiles that read the same rows of the coarser pass (rho and rho + n_next), then
// the remaining row tiles and the shifts, so that data read twice is read close in time.
__device__ __forceinline__ TileIdx tile_of(const LevelPass& ps, long long id) {
    TileIdx ti;
    const int tt = (int)(id % ps.t_tiles);
    id /= ps.t_tiles;
    const int q = (int)(id % ps.reps);
    id /= ps.reps;
    const long long lo_tiles = ps.rho_tiles / ps.reps;
    const long long lo = id % lo_tiles;
    ti.r = (int)(id / lo_tiles);
    ti.rho0 = ((long long)q * lo_tiles + lo) * LT_M;
    ti.t0 = tt * LT_N;
    return ti;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) k_level_tc(const __grid_constant__ CUtensorMap xmap,
                                                          const __grid_constant__ CUtensorMap amap,
                                                          const __grid_constant__ LevelPass ps, float* __restrict__ wsf,
                                                          int tau_pad, int tA) {
    constexpr int ST = stages<P>();
    constexpr uint32_t SB = stage_bytes<P>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);            // the 64-byte swizzle follows address bits 7-8
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + ST * SB);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        tma_prefetch(&xmap);
        tma_prefetch(&amap);
        for (int s = 0; s < ST; ++s) { bar_init(&full[s], 1); bar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { bar_init(&tfull[a], 1); bar_init(&tempty[a], kEpi); }
        bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long it = 0;
            for (long long tile = blockIdx.x; tile < ps.ntiles && ok; tile += gridDim.x) {
                const TileIdx ti = tile_of(ps, tile);
                for (int sgi = 0; sgi < ps.nseg && ok; ++sgi) {
                    const LevelSeg& sg = ps.seg[sgi];
                    const long long nrep = 1LL << sg.logn_rep;
                    const int xr0 = (int)(sg.xrow + (ti.rho0 & (nrep - 1)));
                    for (int kc = 0; kc < sg.chunks; ++kc, ++it) {
                        const int s = (int)(it % ST);
                        const uint32_t ph = (uint32_t)((it / ST) & 1);
                        if (!bar_wait(smem_u32(&empty[s]), ph ^ 1)) { ok = false; break; }
                        const uint32_t fb = smem_u32(&full[s]);
                        bar_expect_tx(fb, SB);
                        unsigned char* st = smem + s * SB;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            tma_load_3d(smem_u32(st + p * XPIECE), &xmap, fb, 0,
                                        xr0 + (int)(((long long)(p * sg.chunks + kc)) << sg.logn_rep), ti.r);
                            tma_load_2d(smem_u32(st + P * XPIECE + p * APIECE), &amap, fb, 0,
                                        (int)(sg.arow + (long long)(p * sg.chunks + kc) * tA + ti.t0));
                        }
                    }
                }
            }
            if (!ok) {
                atomicOr(&g_level_error, 1u);
                // the copies already issued complete on their own: wait (bounded) for the last
                // fill of every stage before the CTA's shared memory goes away
                for (long long k = it - 1; k >= 0 && k >= it - ST; --k)
                    bar_wait(smem_u32(&full[k % ST]), (uint32_t)((k / ST) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(LT_N);
            long long it = 0, n = 0;
            for (long long tile = blockIdx.x; tile < ps.ntiles && ok; tile += gridDim.x, ++n) {
                const int a = (int)(n & 1);
                if (!bar_wait(smem_u32(&tempty[a]), (uint32_t)(((n >> 1) & 1) ^ 1))) { ok = false; break; }
                fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(a * LT_N);
                bool first = true;
                for (int sgi = 0; sgi < ps.nseg && ok; ++sgi) {
                    const LevelSeg& sg = ps.seg[sgi];
                    for (int kc = 0; kc < sg.chunks; ++kc, ++it) {
                        const int s = (int)(it % ST);
                        if (!bar_wait(smem_u32(&full[s]), (uint32_t)((it / ST) & 1))) { ok = false; break; }
                        fence_after_sync();
                        const uint32_t xs = smem_u32(smem + s * SB), as = xs + P * XPIECE;
                        const int ks_n = kc + 1 == sg.chunks ? sg.last_ksteps : 2;
                        for (int ks = 0; ks < ks_n; ++ks)
                            issue_kstep<P, XPIECE, APIECE>(acc, smem_desc_sw64(xs + 32 * ks), smem_desc_sw64(as + 32 * ks),
                                                           idesc, first);
                        mma_commit(smem_u32(&empty[s]));
                    }
                }
                if (ok) mma_commit(smem_u32(&tfull[a]));
            }
            if (!ok) atomicOr(&g_level_error, 1u);
            // every MMA issued by this thread has completed once this commit arrives
            mma_commit(smem_u32(drain));
            bar_wait(smem_u32(drain), 0);
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        // warp: lanes 32 quarter of the accumulator, its 32-column groups part, part + 3, ...
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        const int ng = (LT_N / 32 - part + kEpi / 4 - 1) / (kEpi / 4);
        const long long n_out = 1LL << ps.logn_out;
        const bool has_next = ps.logn_next >= 0;
        const long long nmask = has_next ? (1LL << ps.logn_next) - 1 : 0;
        long long n = 0;
        const float* cr = ps.const_off >= 0 ? wsf + ps.const_off : nullptr;
        // the coarser pass's rows (or the constant row) of one 32-column group of a tile
        auto load_group = [&](const TileIdx& ti, int cg, float4 (&pv)[8]) {
            const long long rho = ti.rho0 + quarter * 32 + lane;
            const bool row_ok = rho < n_out;
            const float* nx = has_next ? wsf + ps.next_off + (long long)ti.r * ps.next_stride + (rho & nmask) * 4
                                       : nullptr;
            const int tb = ti.t0 + (part + (kEpi / 4) * cg) * 32;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int t = tb + 4 * q;
                pv[q] = (has_next && row_ok && t < tau_pad)
                            ? __ldg(reinterpret_cast<const float4*>(nx + ((long long)(t >> 2) << ps.logn_next) * 4))
                            : (cr && t < tau_pad) ? __ldg(reinterpret_cast<const float4*>(cr + t))
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        float4 pn[8];                 // the next group's values, loaded one group ahead
        if (blockIdx.x < ps.ntiles) load_group(tile_of(ps, blockIdx.x), 0, pn);
        for (long long tile = blockIdx.x; tile < ps.ntiles; tile += gridDim.x, ++n) {
            const int a = (int)(n & 1);
            if (!bar_wait(smem_u32(&tfull[a]), (uint32_t)((n >> 1) & 1))) { ok = false; break; }
            fence_after_sync();
            const TileIdx ti = tile_of(ps, tile);
            const long long rho = ti.rho0 + quarter * 32 + lane;
            const bool row_ok = rho < n_out;
            float* out = wsf + ps.out_off + (long long)ti.r * ps.out_stride + rho * 4;
            const uint32_t lane_addr = tmem + (uint32_t)(a * LT_N) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int cg = 0; cg < ng; ++cg) {
                const int col = (part + (kEpi / 4) * cg) * 32;       // the group's first column in the tile
                const int tb = ti.t0 + col;
                float4 pv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) pv[q] = pn[q];
                if (cg + 1 < ng) load_group(ti, cg + 1, pn);
                else if (tile + gridDim.x < ps.ntiles) load_group(tile_of(ps, tile + gridDim.x), 0, pn);
                uint32_t d[32];
                tmem_ld32(lane_addr + col, d);
                tmem_wait_ld();
                if (row_ok) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int t = tb + 4 * q;
                        if (t < tau_pad) {
                            const float4 v = make_float4(pv[q].x + __uint_as_float(d[4 * q]),
                                                         pv[q].y + __uint_as_float(d[4 * q + 1]),
                                                         pv[q].z + __uint_as_float(d[4 * q + 2]),
                                                         pv[q].w + __uint_as_float(d[4 * q + 3]));
                            *reinterpret_cast<float4*>(out + ((long long)(t >> 2) << ps.logn_out) * 4) = v;
                        }
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) bar_arrive(smem_u32(&tempty[a]));
        }
        if (!ok && lane == 0) atomicOr(&g_level_error, 1u);
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// A tensor map over rows of 32 bf16 (64 bytes): dims {32, rows[, shifts]}, box {32, box_rows[, 1]},
// 64-byte swizzle.  Out-of-range rows read as zero.
cudaError_t make_map(CUtensorMap* m, void* base, long long rows, int shifts, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {32, (cuuint64_t)rows, (cuuint64_t)shifts};
    const cuuint64_t strides[2] = {64, (cuuint64_t)rows * 64};
    const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, shifts > 0 ? 3 : 2, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

SplitXArgs split_args(const LevelPlan& lp, bool a_side, int tA) {
    SplitXArgs sa{};
    for (int p = 0; p < lp.npass; ++p)
        for (int s = 0; s < lp.pass[p].nseg; ++s) sa.seg[sa.nlev++] = lp.pass[p].seg[s];
    sa.blk0[0] = 0;
    for (int l = 0; l < sa.nlev; ++l)
        sa.blk0[l + 1] = sa.blk0[l] + (long long)sa.seg[l].chunks * 4 *
                                          (a_side ? (long long)tA : (1LL << sa.seg[l].logn_rep));
    return sa;
}

}  // namespace

// Column sums of F (rows x tau_pad per shift) over every shift and row, in a fixed order: CTA (t
// block, chunk c) sums rows c, c + 64, ... of every shift into part[c][t] (double); the last kernel
// sums the 64 chunks in order.  A thread's chain is a compensated FP32 sum (Neumaier: the rounding
// error of every addition carried in a second float; error at most about 2 u |sum| + n u^2 sum |x|,
// u = 2^-24, n the chain length), at the FP32 rate: double additions, at GB300's FP64 rate, took
// 0.085 ms of the 2^20-point step for these sums.
constexpr int kColChunks = 64;
__global__ void __launch_bounds__(128) k_col_sums(const float* __restrict__ F, long long shift_stride, long long rows,
                                                  int reff, int tau_pad, double* __restrict__ part) {
    const int t = blockIdx.x * 128 + threadIdx.x;
    const int c = blockIdx.y;
    if (t >= tau_pad) return;
    float sum = 0.0f, comp = 0.0f;
    for (int r = 0; r < reff; ++r)
        for (long long k = c; k < rows; k += kColChunks) {
            const float x = __ldg(F + r * shift_stride + k * tau_pad + t);
            const float u = __fadd_rn(sum, x);
            comp = __fadd_rn(comp, fabsf(sum) >= fabsf(x) ? __fadd_rn(__fsub_rn(sum, u), x)
                                                            : __fadd_rn(__fsub_rn(x, u), sum));
            sum = u;
        }
    part[(long long)c * tau_pad + t] = (double)sum + (double)comp;
}
__global__ void __launch_bounds__(128) k_col_sums_final(const double* __restrict__ part, int tau_pad,
                                                        double* __restrict__ gsum) {
    const int t = blockIdx.x * 128 + threadIdx.x;
    if (t >= tau_pad) return;
    double acc = 0.0;
    for (int c = 0; c < kColChunks; ++c) acc += part[(long long)c * tau_pad + t];
    gsum[t] = acc;
}

cudaError_t launch_col_sums(const float* F, long long shift_stride, long long rows, int reff, int tau_pad,
                            double* part, double* gsum, cudaStream_t st) {
    k_col_sums<<<dim3((tau_pad + 127) / 128, kColChunks), 128, 0, st>>>(F, shift_stride, rows, reff, tau_pad, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_col_sums_final<<<(tau_pad + 127) / 128, 128, 0, st>>>(part, tau_pad, gsum);
    return cudaGetLastError();
}

// c[t] = xc * (sum of 64 chunk partials of the coarse rows of A), in double
__global__ void __launch_bounds__(128) k_const_final(const double* __restrict__ part, int tau, int tau_pad, float xc,
                                                     float* __restrict__ c) {
    const int t = blockIdx.x * 128 + threadIdx.x;
    if (t >= tau_pad) return;
    double acc = 0.0;
    for (int k = 0; k < 64; ++k) acc += part[(long long)k * tau_pad + t];
    c[t] = t < tau ? (float)((double)xc * acc) : 0.0f;
}

cudaError_t launch_const_row(const float* A, int ldA, int tau, int tau_pad, const LevelPlan& lp, unsigned char* ws,
                             cudaStream_t st) {
    // the coarse columns are the contiguous rows col0 .. s-1 of A (w is nondecreasing): their column
    // sums in 64 row chunks, then the chunks in order
    const SplitXArgs sa = split_args(lp, true, lp.tA);
    int j0 = 1 << 30, j1 = 0;
    for (int l = 0; l < sa.nlev; ++l) {
        j0 = std::min(j0, sa.seg[l].col0);
        j1 = std::max(j1, sa.seg[l].col0 + sa.seg[l].tau);
    }
    if (j1 <= j0) return cudaSuccess;
    double* part = reinterpret_cast<double*>(ws + lp.cpart_off);
    if (ldA != tau_pad) return cudaErrorInvalidValue;
    k_col_sums<<<dim3((tau_pad + 127) / 128, 64), 128, 0, st>>>(A + (long long)j0 * ldA, 0, j1 - j0, 1, tau_pad, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // (A's row stride is tau_pad: A is read in place only when tau is a multiple of 4)
    k_const_final<<<(tau_pad + 127) / 128, 128, 0, st>>>(part, tau, tau_pad, lp.xc, reinterpret_cast<float*>(ws + lp.c_off));
    return cudaGetLastError();
}

cudaError_t level_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_level_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_level_error, &zero, sizeof(unsigned int));
}

size_t level_tc_smem(int pieces) { return pieces == 3 ? level_smem<3>() : level_smem<1>(); }

cudaError_t launch_split_x(const float* tab, long long tab_stride, const LevelPlan& lp, int reff, unsigned char* ws,
                           cudaStream_t st) {
    const SplitXArgs sa = split_args(lp, false, lp.tA);
    const long long n = sa.blk0[sa.nlev];
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)reff);
    uint4* xp = reinterpret_cast<uint4*>(ws + lp.x_off);
    if (lp.pieces == 3) k_split_x<3><<<grid, 256, 0, st>>>(tab, tab_stride, sa, lp.x_rows_per_shift, xp, lp.xc);
    else k_split_x<1><<<grid, 256, 0, st>>>(tab, tab_stride, sa, lp.x_rows_per_shift, xp, lp.xc);
    return cudaGetLastError();
}

cudaError_t launch_split_a(const float* A, int ldA, int tau, const LevelPlan& lp, unsigned char* ws, cudaStream_t st) {
    const SplitXArgs sa = split_args(lp, true, lp.tA);
    const long long n = sa.blk0[sa.nlev];
    if (n == 0) return cudaSuccess;
    uint4* ap = reinterpret_cast<uint4*>(ws + lp.a_off);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (lp.pieces == 3) k_split_a<3><<<blocks, 256, 0, st>>>(A, ldA, tau, sa, lp.tA, ap);
    else k_split_a<1><<<blocks, 256, 0, st>>>(A, ldA, tau, sa, lp.tA, ap);
    return cudaGetLastError();
}

cudaError_t launch_level_pass(const LevelPlan& lp, int p, int reff, int tau_pad, unsigned char* ws, cudaStream_t st) {
    const LevelPass& ps = lp.pass[p];
    if (ps.ntiles == 0) return cudaSuccess;
    CUtensorMap xmap, amap;
    cudaError_t e = make_map(&xmap, ws + lp.x_off, lp.x_rows_per_shift, reff, LT_M);
    if (e != cudaSuccess) return e;
    e = make_map(&amap, ws + lp.a_off, lp.a_rows, 0, LT_N);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>(ps.ntiles, sms);
    float* wsf = reinterpret_cast<float*>(ws);
    if (lp.pieces == 3) {
        e = cudaFuncSetAttribute(k_level_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)level_smem<3>());
        if (e != cudaSuccess) return e;
        k_level_tc<3><<<grid, kThreads, level_smem<3>(), st>>>(xmap, amap, ps, wsf, tau_pad, lp.tA);
    } else {
        e = cudaFuncSetAttribute(k_level_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)level_smem<1>());
        if (e != cudaSuccess) return e;
        k_level_tc<1><<<grid, kThreads, level_smem<1>(), st>>>(xmap, amap, ps, wsf, tau_pad, lp.tA);
    }
    return cudaGetLastError();
}

}  // namespace qmc
