// The adjoint of Algorithm 2's lowest coarse levels in one pass over the root gradients (split and
// bf16 tiers).  The adjoint of the periodic tiling sends the root gradients F_JF to every coarser
// level: level I's block gradient is dA_I = sum_r sum_rho X_{r,I}[rho mod n_I]^T F_{r,JF}[rho] over
// the root rows rho (the same sum as over the folded gradient F_I[rho'] = sum_q F_JF[rho' + q n_I]
// of Algorithm 2's distinct rows, taken before the fold).  For the L lowest levels JF .. JF+L-1
// this kernel reads F_JF once: every root chunk goes to the tensor cores once, against the rows of
// all L levels' point tables stacked into one B operand, and only the fold F_{JF+L} (the input of
// the remaining levels) is written.
//
// Work item: (shift r, column tile t0 .. t0+127, residue block rho0 .. rho0+31 of the n_out =
// n_{JF+L} rows of level JF+L).  Its root rows are rho0 + k + q n_out (k < 32, q < 2^L); root chunk q
// meets level JF+d's rows rho0 + k + (q mod 2^(L-d)) n_out.  One chunk's product is D[t][j] += sum_k
// F[k][t] X[k][j] with M = 128 columns t, N = the levels' columns (each rounded up to 16, at most
// 128 in all), K = 32 rows; D's columns are the levels' gradient columns side by side.
//
// One CTA per SM, each on one column tile and a contiguous range of (shift, residue block) items:
//   warp 0      TMA producer: the FP32 root chunks (128 t x 32 rows, a 3-D box over (t, rows,
//               shifts)) into a ring of raw stages;
//   warp 2      TMA producer: for every root chunk the pre-split bf16 pieces (k_split_xt) of the
//               levels' rows into the chunk's operand slot, one box per level and piece;
//   warp 1      allocates the tensor memory and one thread issues every chunk's MMAs, with the
//               chunk's F^T pieces read from tensor memory;
//   warps 3-10  converters: split the chunk's F^T into bf16 pieces in tensor memory (lane = column
//               t, two rows per 32-bit column), sum the chunks of an item into F_{JF+L} and write
//               it; warps 3-10, after every group of items (chains of at most 1024 rows), add the
//               accumulator into a running total in shared memory, one group behind the MMAs, and
//               at the end store the CTA's partial gradient, which k_grad_reduce sums over the
//               CTAs of the column tile.
// Every wait is bounded; a run-out sets the error word (foldgrad_error_word) and the roles stop as
// in the other tensor-core kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

// sticky: bit 0 = a bounded wait of the fold-gradient kernel ran out
__device__ unsigned int g_foldgrad_error;

using namespace tc;

namespace {

constexpr int FG_M = 128;                      // columns t per item (MMA M)
constexpr int FG_K = 32;                       // rows per chunk
constexpr int FG_NMAX = 128;                   // gradient columns of all fused levels (MMA N), at most
constexpr int RS = 4;                          // raw root-chunk stages
constexpr int CS = 4;                          // chunk operand slots
constexpr uint32_t RAW = FG_K * FG_M * 4;      // [k][t] FP32, 16 KB
// converter warps, kConv / 4 per tensor-memory lane quarter (8 with 16 rows each measured 7% faster
// than 16 with 8 rows: fewer barrier round trips per chunk, more independent work per thread)
constexpr int kConv = 8;
constexpr int kRPT = FG_K * 4 / kConv;         // rows of a chunk per converter thread
constexpr int kThreads = 96 + 32 * kConv;
static_assert(kConv == 8 || kConv == 16, "converter warps");
// Tensor memory (512 columns): accumulator sets b = 0, 1 at columns 128 b, and the operand slots'
// F^T pieces from column 256: slot s, piece p, K-step ks at 256 + 16 (P s + p) + 8 ks (one 32-bit
// column holds two bf16 of consecutive rows k).
constexpr uint32_t TM_SLOT0 = 256;
static_assert(TM_SLOT0 + 16 * 3 * CS <= 512, "tensor-memory slots");

// shared memory: raw stages, X slots (P pieces of ntot rows x 64 bytes), the running total
// [ntot columns j][128 lanes] FP32, barriers
__host__ __device__ constexpr uint32_t slot_bytes(int P, int ntot) { return (uint32_t)(P * ntot * 64); }
__host__ __device__ constexpr size_t fg_smem(int P, int ntot) {
    return 1024 + RS * RAW + CS * slot_bytes(P, ntot) + (size_t)ntot * 128 * 4 + 256;
}




// the CTA's column tile, split index and item range
struct CtaWork {
    int tt, sp;
    long long i0, i1;
};
__device__ __forceinline__ CtaWork cta_work(const FoldGradArgs& ga) {
    CtaWork w;
    w.tt = blockIdx.x / ga.cpt;
    w.sp = blockIdx.x - w.tt * ga.cpt;
    w.i0 = ga.items * w.sp / ga.cpt;
    w.i1 = ga.items * (w.sp + 1) / ga.cpt;
    return w;
}

// ---------------------------------------------------------------------------------------------
// k_split_xt: the fused levels' point-table columns, centred, as bf16 pieces in [piece][shift][j]
// [row] order (rows contiguous), which a TMA box of 32 rows x N columns with the 64-byte swizzle
// places in shared memory as the MMA's K-major B operand.  Thread = 8 consecutive rows of one
// column of one level.
// ---------------------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) k_split_xt(const float* __restrict__ tab, long long tab_stride,
                                                  const __grid_constant__ SplitXtArgs sa, int reff,
                                                  __nv_bfloat16* __restrict__ xp, float xc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= sa.blk0[sa.n]) return;
    int l = 0;
    while (l + 1 < sa.n && i >= sa.blk0[l + 1]) ++l;
    const long long loc = i - sa.blk0[l];
    const long long n = 1LL << sa.logn[l];
    const long long row0 = (loc & ((n >> 3) - 1)) << 3;
    const int j = (int)(loc >> (sa.logn[l] - 3));
    const float4* src = reinterpret_cast<const float4*>(tab + (long long)r * tab_stride + sa.tab[l] +
                                                        (long long)j * n + row0);
    const float4 a = __ldg(src), b = __ldg(src + 1);
    const float v[8] = {a.x - xc, a.y - xc, a.z - xc, a.w - xc, b.x - xc, b.y - xc, b.z - xc, b.w - xc};
    uint32_t w[P][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t pc[P];
        split_pair<P>(v[2 * q], v[2 * q + 1], pc);
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][q] = pc[p];
    }
    const long long per_piece = (long long)reff * sa.tau[l] * n;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        __nv_bfloat16* dst = xp + sa.off[l] + p * per_piece + ((long long)r * sa.tau[l] + j) * n + row0;
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
}


// ---------------------------------------------------------------------------------------------
// k_fold_grad_tc<P, L>
// ---------------------------------------------------------------------------------------------
template <int P, int L>
__global__ void __launch_bounds__(kThreads, 1) k_fold_grad_tc(const __grid_constant__ FoldGradArgs ga) {
    constexpr int STEPS = 1 << L;
    const int ntot = ga.acc[L - 1] + ga.nd[L - 1];                // MMA N: every fused level's columns
    const uint32_t sb = slot_bytes(P, ntot);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    unsigned char* raw = smem;                                    // RS raw stages
    unsigned char* slots = smem + RS * RAW;                       // CS operand slots: X pieces
    float* tot = reinterpret_cast<float*>(slots + CS * sb);       // running total [j][t]
    uint64_t* rfull = reinterpret_cast<uint64_t*>(tot + ntot * 128);
    uint64_t* rempty = rfull + RS;
    uint64_t* sfull = rempty + RS;                                // F^T pieces written
    uint64_t* sempty = sfull + CS;
    uint64_t* xfull = sempty + CS;                                // X pieces landed
    uint64_t* tdone = xfull + CS;                                 // [2]
    uint64_t* tfree = tdone + 2;                                  // [2]
    uint64_t* drain = tfree + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CtaWork cw = cta_work(ga);
    const long long nrb = (1LL << ga.log_out) >> 5;               // residue blocks per shift
    const long long n_out = 1LL << ga.log_out;
    const long long ngroups = (cw.i1 - cw.i0 + ga.group - 1) / ga.group;
    if (warp == 0 && lane == 0) {
        tma_prefetch(&ga.fmap);
        for (int d = 0; d < L; ++d)
            if (ga.nd[d]) tma_prefetch(&ga.xmap[d]);
        for (int s = 0; s < RS; ++s) { bar_init(&rfull[s], 1); bar_init(&rempty[s], kConv); }
        for (int s = 0; s < CS; ++s) { bar_init(&sfull[s], kConv); bar_init(&sempty[s], 1); bar_init(&xfull[s], 1); }
        for (int b = 0; b < 2; ++b) { bar_init(&tdone[b], 1); bar_init(&tfree[b], 8); }
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
        // ------------------------------------------------------------------ TMA producer of F_JF
        if (lane == 0) {
            long long itr = 0;
            for (long long it = cw.i0; it < cw.i1 && ok; ++it) {
                const int r = (int)(it / nrb);
                const int rho0 = (int)((it - (long long)r * nrb) << 5);
                for (int q = 0; q < STEPS && ok; ++q, ++itr) {
                    const int rs = (int)(itr % RS);
                    if (!bar_wait(smem_u32(&rempty[rs]), (uint32_t)(((itr / RS) & 1) ^ 1))) { ok = false; break; }
                    bar_expect_tx(smem_u32(&rfull[rs]), RAW);
                    if (ga.froot_tiled)                       // 32 rows of one tile: 16 KB in one copy
                        bulk_load(smem_u32(raw + rs * RAW),
                                  ga.froot + (long long)r * ga.froot_stride +
                                      ((long long)cw.tt * ga.n_root + rho0 + (long long)q * n_out) * FG_M,
                                  RAW, smem_u32(&rfull[rs]));
                    else
                        tma_load_3d(smem_u32(raw + rs * RAW), &ga.fmap, smem_u32(&rfull[rs]), cw.tt * FG_M,
                               rho0 + q * (int)n_out, r);
                }
            }
            if (!ok) {                                            // the copies still in flight land first
                atomicOr(&g_foldgrad_error, 1u);
                for (long long k = itr - 1; k >= 0 && k >= itr - RS; --k)
                    bar_wait(smem_u32(&rfull[k % RS]), (uint32_t)((k / RS) & 1));
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------------ TMA producer of X pieces
        if (lane == 0) {
            long long slot = 0;
            for (long long it = cw.i0; it < cw.i1 && ok; ++it) {
                const int r = (int)(it / nrb);
                const int rho0 = (int)((it - (long long)r * nrb) << 5);
                for (int q = 0; q < STEPS && ok; ++q, ++slot) {
                    const int cs = (int)(slot % CS);
                    if (!bar_wait(smem_u32(&sempty[cs]), (uint32_t)(((slot / CS) & 1) ^ 1))) { ok = false; break; }
                    const uint32_t fb = smem_u32(&xfull[cs]);
                    bar_expect_tx(fb, sb);
                    const uint32_t xs = smem_u32(slots + cs * sb);
                    for (int d = 0; d < L; ++d) {
                        if (!ga.nd[d]) continue;
                        const int row = rho0 + (q & ((1 << (L - d)) - 1)) * (int)n_out;
                        for (int p = 0; p < P; ++p)
                            tma_load_4d(xs + (uint32_t)((p * ntot + ga.acc[d]) * 64), &ga.xmap[d], fb, row, 0, r, p);
                    }
                }
            }
            if (!ok) {
                atomicOr(&g_foldgrad_error, 1u);
                for (long long k = slot - 1; k >= 0 && k >= slot - CS; --k)
                    bar_wait(smem_u32(&xfull[k % CS]), (uint32_t)((k / CS) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            long long slot = 0;
            const uint32_t idesc = idesc_bf16((uint32_t)ntot);
            const uint32_t xpiece = (uint32_t)ntot * 64;
            for (long long g = 0; g < ngroups && ok; ++g) {
                const int b = (int)(g & 1);
                if (!bar_wait(smem_u32(&tfree[b]), (uint32_t)(((g >> 1) & 1) ^ 1))) { ok = false; break; }
                fence_after_sync();
                bool fresh = true;
                const uint32_t dst = tmem + (uint32_t)(b * 128);
                const long long ib = cw.i0 + g * ga.group, ie = min(cw.i1, ib + ga.group);
                for (long long n = (ie - ib) * STEPS; n > 0 && ok; --n, ++slot) {
                    const int cs = (int)(slot % CS);
                    if (!bar_wait(smem_u32(&sfull[cs]), (uint32_t)((slot / CS) & 1)) ||
                        !bar_wait(smem_u32(&xfull[cs]), (uint32_t)((slot / CS) & 1))) { ok = false; break; }
                    fence_after_sync();
                    const uint32_t xs = smem_u32(slots + cs * sb);
                    const uint32_t ta = tmem + TM_SLOT0 + (uint32_t)(16 * P * cs);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t bd = smem_desc_sw64(xs + 32 * ks);
                        constexpr int NP = P == 3 ? 6 : 1;
                        constexpr int pi[6] = {2, 1, 0, 1, 0, 0};
                        constexpr int pj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
                        for (int pq = 0; pq < NP; ++pq) {
                            const int ia = P == 3 ? pi[pq] : 0, jb = P == 3 ? pj[pq] : 0;
                            mma_bf16_ts(dst, ta + (uint32_t)(16 * ia + 8 * ks), desc_add(bd, jb * xpiece), idesc,
                                        fresh ? 0u : 1u);
                            fresh = false;
                        }
                    }
                    mma_commit(smem_u32(&sempty[cs]));
                }
                if (ok) mma_commit(smem_u32(&tdone[b]));
            }
            if (!ok) atomicOr(&g_foldgrad_error, 1u);
            mma_commit(smem_u32(drain));
            bar_wait(smem_u32(drain), 0);
        }
    } else {
        // ------------------------------------------------------------------ converters
        // warp w takes tensor-memory lanes 32 (w % 4) .. + 31 (fixed by warp) = columns t, and
        // kRPT rows of every chunk; warps 3-10 also move the accumulator into the running total,
        // column half (w - 3) / 4
        const int quarter = warp & 3, h = (warp - 3) >> 2;        // rows kRPT h .. kRPT (h + 1) - 1
        const int tl = quarter * 32 + lane;
        const int t = cw.tt * FG_M + tl;
        const bool drainer = warp < 11;
        const int hd = (warp - 3) >> 2;                           // a drainer's column half
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        long long itr = 0, slot = 0;
        bool have_total = false;
        const int nh = ntot >> 1, j0 = hd * nh;                   // a drainer's columns (ntot % 16 == 0)

        // add accumulator set b into the running total (or start it)
        auto drain_group = [&](long long g) -> bool {
            if (!drainer) return true;
            const int b = (int)(g & 1);
            // (the tensor-memory loads below are warp-collective: the whole warp takes one branch)
            if (!__all_sync(0xffffffffu, bar_wait(smem_u32(&tdone[b]), (uint32_t)((g >> 1) & 1)))) return false;
            fence_after_sync();
            for (int c = 0; c < nh; c += 8) {
                uint32_t a[8];
                tmem_ld8(lane_base + (uint32_t)(b * 128 + j0 + c), a);
                tmem_wait_ld();
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    float* o = tot + (j0 + c + x) * 128 + tl;
                    *o = have_total ? *o + __uint_as_float(a[x]) : __uint_as_float(a[x]);
                }
            }
            have_total = true;
            fence_before_sync();
            __syncwarp();
            if (lane == 0) bar_arrive(smem_u32(&tfree[b]));
            return true;
        };

        for (long long g = 0; g < ngroups && ok; ++g) {
            const long long ib = cw.i0 + g * ga.group, ie = min(cw.i1, ib + ga.group);
            for (long long it = ib; it < ie && ok; ++it) {
                const int r = (int)(it / nrb);
                const long long rho0 = (it - (long long)r * nrb) << 5;
                float fsum[kRPT];
#pragma unroll
                for (int k = 0; k < kRPT; ++k) fsum[k] = 0.0f;
                for (int q = 0; q < STEPS; ++q, ++itr, ++slot) {
                    const int rs = (int)(itr % RS), cs = (int)(slot % CS);
                    if (!bar_wait(smem_u32(&rfull[rs]), (uint32_t)((itr / RS) & 1))) { ok = false; break; }
                    float v[kRPT];
                    const float* rf = reinterpret_cast<const float*>(raw + rs * RAW);
#pragma unroll
                    for (int k = 0; k < kRPT; ++k) v[k] = rf[(kRPT * h + k) * FG_M + tl];
                    __syncwarp();
                    if (lane == 0) bar_arrive(smem_u32(&rempty[rs]));
#pragma unroll
                    for (int k = 0; k < kRPT; ++k) fsum[k] += v[k];
                    // the chunk's F^T rows as bf16 pieces in the slot's tensor memory
                    if (!bar_wait(smem_u32(&sempty[cs]), (uint32_t)(((slot / CS) & 1) ^ 1))) { ok = false; break; }
                    fence_after_sync();
                    uint32_t w[P][kRPT / 2];
#pragma unroll
                    for (int x = 0; x < kRPT / 2; ++x) {
                        uint32_t pc[P];
                        split_pair<P>(v[2 * x], v[2 * x + 1], pc);
#pragma unroll
                        for (int p = 0; p < P; ++p) w[p][x] = pc[p];
                    }
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        tmem_st(lane_base + TM_SLOT0 + (uint32_t)(16 * (P * cs + p) + (kRPT / 2) * h), w[p]);
                    tmem_wait_st();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) bar_arrive(smem_u32(&sfull[cs]));
                }
                if (!ok) break;
                if (t < ga.tau_pad) {
                    // F_{JF+L} rows rho0 + 8h + k: the sum of the item's root chunks
                    float* o = ga.fout + (long long)r * ga.fout_stride + (rho0 + kRPT * h) * ga.tau_pad + t;
#pragma unroll
                    for (int k = 0; k < kRPT; ++k) o[(long long)k * ga.tau_pad] = fsum[k];
                }
            }
            if (!ok) break;
            if (g > 0 && !drain_group(g - 1)) { ok = false; break; }
        }
        if (ok && ngroups > 0 && !drain_group(ngroups - 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicOr(&g_foldgrad_error, 1u);
        // the CTA's partial: level d, split sp, column j, t
        if (ok && drainer && t < ga.tau_pad) {
            for (int d = 0; d < L; ++d) {
                float* pe = ga.part + ga.poff[d] + ((long long)cw.sp * ga.tau[d]) * ga.tau_pad + t;
                for (int j = 0; j < ga.tau[d]; ++j) {
                    const int col = ga.acc[d] + j;
                    if (col >= j0 && col < j0 + nh)
                        pe[(long long)j * ga.tau_pad] = have_total ? tot[col * 128 + tl] : 0.0f;
                }
            }
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

}  // namespace

cudaError_t foldgrad_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_foldgrad_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_foldgrad_error, &zero, sizeof(unsigned int));
}

cudaError_t launch_split_xt(const float* tab, long long tab_stride, const SplitXtArgs& sa, int reff, int pieces,
                            __nv_bfloat16* xp, float xc, cudaStream_t st) {
    const long long n = sa.blk0[sa.n];
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), reff);
    if (pieces == 3) k_split_xt<3><<<grid, 256, 0, st>>>(tab, tab_stride, sa, reff, xp, xc);
    else k_split_xt<1><<<grid, 256, 0, st>>>(tab, tab_stride, sa, reff, xp, xc);
    return cudaGetLastError();
}

// The tensor maps of one call: F_JF (FP32, dims t, rows, shifts; box 128 x 32 x 1, no swizzle) and
// each level's pre-split pieces (bf16, dims rows, j, shifts, pieces; box 32 x N_d x 1 x 1, 64-byte
// swizzle); elements outside the arrays read as zero.
cudaError_t launch_fold_grad_tc(FoldGradArgs& ga, int L, const float* Froot, long long root_stride, long long n_root,
                                const __nv_bfloat16* xp, const SplitXtArgs& sa, int reff, int pieces, cudaStream_t st) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    ga.froot = Froot;
    ga.froot_stride = root_stride;
    ga.n_root = n_root;
    if (ga.froot_tiled && (reinterpret_cast<uintptr_t>(Froot) % 16 != 0 || root_stride % 4 != 0 || n_root % FG_K != 0))
        return cudaErrorInvalidValue;                     // (the bulk copies' alignment and whole chunks)
    if (ga.froot_tiled) {
        // [r][t / 128][rows][128]: dims (128 columns, rows, column tiles, shifts)
        const cuuint64_t dims[4] = {FG_M, (cuuint64_t)n_root, (cuuint64_t)ga.t_tiles, (cuuint64_t)reff};
        const cuuint64_t strides[3] = {FG_M * 4, (cuuint64_t)n_root * FG_M * 4, (cuuint64_t)root_stride * 4};
        const cuuint32_t box[4] = {FG_M, FG_K, 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (fn(&ga.fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(Froot), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)ga.tau_pad, (cuuint64_t)n_root, (cuuint64_t)reff};
        const cuuint64_t strides[2] = {(cuuint64_t)ga.tau_pad * 4, (cuuint64_t)root_stride * 4};
        const cuuint32_t box[3] = {FG_M, FG_K, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (fn(&ga.fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(Froot), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    for (int l = 0; l < sa.n; ++l) {
        const int d = sa.lev[l];
        if (d < 0) continue;                      // (a k_grad_tc entry)
        const cuuint64_t n = 1ULL << sa.logn[l];
        const cuuint64_t dims[4] = {n, (cuuint64_t)sa.tau[l], (cuuint64_t)reff, (cuuint64_t)pieces};
        const cuuint64_t strides[3] = {n * 2, n * 2 * sa.tau[l], n * 2 * sa.tau[l] * reff};
        const cuuint32_t box[4] = {FG_K, (cuuint32_t)ga.nd[d], 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (fn(&ga.xmap[d], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(xp + sa.off[l]), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    int ntot = 0;
    for (int d = 0; d < L; ++d) ntot = std::max(ntot, ga.acc[d] + ga.nd[d]);
    if (ntot == 0 || ntot > FG_NMAX || ntot % 16 != 0 || ga.acc[L - 1] + ga.nd[L - 1] != ntot)
        return cudaErrorInvalidValue;
    const size_t smem = fg_smem(pieces, ntot);
    const unsigned grid = (unsigned)(ga.t_tiles * ga.cpt);
#define QMC_FG_LAUNCH(PP, LL)                                                                                   \
    do {                                                                                                       \
        cudaError_t e = cudaFuncSetAttribute(k_fold_grad_tc<PP, LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                                       \
        if (e != cudaSuccess) return e;                                                                        \
        k_fold_grad_tc<PP, LL><<<grid, kThreads, smem, st>>>(ga);                                              \
    } while (0)
    if (pieces == 3) {
        if (L == 1) QMC_FG_LAUNCH(3, 1); else if (L == 2) QMC_FG_LAUNCH(3, 2); else if (L == 3) QMC_FG_LAUNCH(3, 3);
        else return cudaErrorInvalidValue;
    } else {
        if (L == 1) QMC_FG_LAUNCH(1, 1); else if (L == 2) QMC_FG_LAUNCH(1, 2); else if (L == 3) QMC_FG_LAUNCH(1, 3);
        else return cudaErrorInvalidValue;
    }
#undef QMC_FG_LAUNCH
    return cudaGetLastError();
}

}  // namespace qmc
