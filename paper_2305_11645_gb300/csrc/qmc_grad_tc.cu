// Block gradients of the coarse levels above the fused ones on the tensor cores (split and bf16
// tiers): the adjoint of Algorithm 2's block products, dA_e = sum_r X_{r,e}^T F_{r,e} over the
// level's distinct rows, with F_e the root gradients folded onto the level (k_fold_grad_tc and
// k_fold_tree).
//
// D[t][j] = sum_k F_e[k][t] (X_e[k][j] - xc): M = 128 columns t, N = 128 gradient columns j (an
// entry has at most 128), K = the level's rows over every shift, cut into splits of at most 1024
// rows (a work unit = entry x t tile x split).  One persistent CTA per SM, warp-specialised:
//   warp 0      TMA producer: the raw FP32 chunk of F (32 rows k x 128 columns t, a 3-D box over
//               (t, rows, shifts)) into a ring of raw stages;
//   warp 2      TMA producer: the chunk's pre-split bf16 pieces of X (k_split_xt; 32 rows x 128
//               columns, 64-byte swizzle, a 4-D box over (rows, j, shifts, pieces)) into its slot;
//   warp 1      allocates the tensor memory (two accumulators, the slots' F^T pieces) and one
//               thread issues every chunk's MMAs, with F^T read from tensor memory, into the
//               accumulator of the unit's parity;
//   warps 3-10  converters: split the chunk's F^T into bf16 pieces in tensor memory (lane = column
//               t, two rows per 32-bit column); one unit behind the MMAs, they store the
//               unit's accumulator as its partial, which k_grad_reduce sums over the splits.
// Every wait is bounded; a run-out sets the error word (grad_error_word) and the roles stop as in
// the other tensor-core kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

// sticky: bit 0 = a bounded wait of the block-gradient kernel ran out (read with grad_error_word)
__device__ unsigned int g_grad_error;

using namespace tc;

namespace {

constexpr int GT_M = 128;                    // columns t per unit (MMA M)
constexpr int GT_N = 128;                    // gradient columns j per unit (MMA N)
constexpr int GK = 32;                       // rows k per chunk
constexpr int RS = 4;                        // raw stages
constexpr int CS = 4;                        // chunk slots
constexpr uint32_t RAW = GK * GT_M * 4;      // [k][t] FP32, 16 KB
constexpr uint32_t PX = GT_N * 64;           // one bf16 piece of X: 128 rows x 64 bytes
constexpr int kConv = 8;                     // converter warps, two per tensor-memory lane quarter
constexpr int kRPT = GK * 4 / kConv;         // rows of a chunk per converter thread
constexpr int kThreads = 96 + 32 * kConv;
// tensor memory: accumulators b = 0, 1 at columns 128 b; slot s's F^T piece p, K-step ks at
// 256 + 16 (P s + p) + 8 ks
constexpr uint32_t TM_SLOT0 = 256;
static_assert(TM_SLOT0 + 16 * 3 * CS <= 512, "tensor-memory slots");

template <int P> constexpr uint32_t slot_bytes() { return P * PX; }
template <int P> constexpr size_t grad_smem() { return 1024 + RS * RAW + CS * slot_bytes<P>() + 256; }


struct UnitIdx {
    int e, sp, t0;
    long long kb, ke;
};

// unit u: entry e, then t tile fastest (concurrent CTAs share the entry's X chunks), then split
__device__ __forceinline__ UnitIdx unit_of(const GradTcArgs& ga, long long u) {
    int e = 0;
    while (e + 1 < ga.n && u >= ga.unit0[e + 1]) ++e;
    const long long loc = u - ga.unit0[e];
    const GradTcEntry& en = ga.ent[e];
    UnitIdx ui;
    ui.e = e;
    ui.t0 = (int)(loc % ga.t_tiles) * GT_M;
    ui.sp = (int)(loc / ga.t_tiles);
    ui.kb = (long long)ui.sp * en.kper;
    ui.ke = min((long long)ga.reff * en.n, ui.kb + en.kper);
    return ui;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) k_grad_tc(const __grid_constant__ GradTcArgs ga, float* __restrict__ part,
                                                         int tau_pad) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    unsigned char* raw = smem;                                   // RS raw stages
    unsigned char* slots = smem + RS * RAW;                      // CS X slots (1 KB aligned)
    uint64_t* rfull = reinterpret_cast<uint64_t*>(slots + CS * slot_bytes<P>());
    uint64_t* rempty = rfull + RS;
    uint64_t* sfull = rempty + RS;
    uint64_t* sempty = sfull + CS;
    uint64_t* xfull = sempty + CS;
    uint64_t* tdone = xfull + CS;                                // [2]
    uint64_t* tfree = tdone + 2;                                 // [2]
    uint64_t* drain = tfree + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        for (int e = 0; e < ga.n; ++e) {
            tma_prefetch(&ga.fmap[e]);
            tma_prefetch(&ga.xmap[e]);
        }
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
        // ------------------------------------------------------------------ TMA producer of F
        if (lane == 0) {
            long long itr = 0;
            for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x) {
                const UnitIdx ui = unit_of(ga, u);
                const long long n = ga.ent[ui.e].n;
                for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++itr) {
                    const int rs = (int)(itr % RS);
                    if (!bar_wait(smem_u32(&rempty[rs]), (uint32_t)(((itr / RS) & 1) ^ 1))) { ok = false; break; }
                    bar_expect_tx(smem_u32(&rfull[rs]), RAW);
                    const int r = (int)(k0 / n), rho = (int)(k0 - (long long)r * n);
                    tma_load_3d(smem_u32(raw + rs * RAW), &ga.fmap[ui.e], smem_u32(&rfull[rs]), ui.t0, rho, r);
                }
            }
            if (!ok) {                                            // the copies still in flight land first
                atomicOr(&g_grad_error, 1u);
                for (long long k = itr - 1; k >= 0 && k >= itr - RS; --k)
                    bar_wait(smem_u32(&rfull[k % RS]), (uint32_t)((k / RS) & 1));
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------------ TMA producer of X pieces
        if (lane == 0) {
            long long slot = 0;
            for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x) {
                const UnitIdx ui = unit_of(ga, u);
                const long long n = ga.ent[ui.e].n;
                for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++slot) {
                    const int cs = (int)(slot % CS);
                    if (!bar_wait(smem_u32(&sempty[cs]), (uint32_t)(((slot / CS) & 1) ^ 1))) { ok = false; break; }
                    bar_expect_tx(smem_u32(&xfull[cs]), slot_bytes<P>());
                    const int r = (int)(k0 / n), rho = (int)(k0 - (long long)r * n);
                    tma_load_4d(smem_u32(slots + cs * slot_bytes<P>()), &ga.xmap[ui.e], smem_u32(&xfull[cs]), rho, 0, r, 0);
                }
            }
            if (!ok) {
                atomicOr(&g_grad_error, 1u);
                for (long long k = slot - 1; k >= 0 && k >= slot - CS; --k)
                    bar_wait(smem_u32(&xfull[k % CS]), (uint32_t)((k / CS) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(GT_N);
            long long slot = 0, nu = 0;
            for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x, ++nu) {
                const UnitIdx ui = unit_of(ga, u);
                const int b = (int)(nu & 1);
                if (!bar_wait(smem_u32(&tfree[b]), (uint32_t)(((nu >> 1) & 1) ^ 1))) { ok = false; break; }
                fence_after_sync();
                const uint32_t dst = tmem + (uint32_t)(b * GT_N);
                bool fresh = true;
                for (long long k0 = ui.kb; k0 < ui.ke && ok; k0 += GK, ++slot) {
                    const int cs = (int)(slot % CS);
                    if (!bar_wait(smem_u32(&sfull[cs]), (uint32_t)((slot / CS) & 1)) ||
                        !bar_wait(smem_u32(&xfull[cs]), (uint32_t)((slot / CS) & 1))) { ok = false; break; }
                    fence_after_sync();
                    const uint32_t xs = smem_u32(slots + cs * slot_bytes<P>());
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
                            mma_bf16_ts(dst, ta + (uint32_t)(16 * ia + 8 * ks), desc_add(bd, jb * PX), idesc,
                                        fresh ? 0u : 1u);
                            fresh = false;
                        }
                    }
                    mma_commit(smem_u32(&sempty[cs]));
                }
                if (ok) mma_commit(smem_u32(&tdone[b]));
            }
            if (!ok) atomicOr(&g_grad_error, 1u);
            mma_commit(smem_u32(drain));
            bar_wait(smem_u32(drain), 0);
        }
    } else {
        // ------------------------------------------------------------------ converters
        // warp w: tensor-memory lanes 32 (w % 4) .. + 31 = columns t, rows 16h .. 16h+15 of every
        // chunk, h = (w - 3) / 4, which is also the column half of the partial it stores
        const int quarter = warp & 3, h = (warp - 3) >> 2;
        const int tl = quarter * 32 + lane;
        const bool drainer = warp < 11;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        long long itr = 0, slot = 0;

        // the partial of the CTA's nu-th unit u
        auto store_unit = [&](long long u, long long nu) -> bool {
            if (!drainer) return true;
            const UnitIdx ui = unit_of(ga, u);
            const GradTcEntry& en = ga.ent[ui.e];
            const int b = (int)(nu & 1);
            // (the tensor-memory loads below are warp-collective: the whole warp takes one branch)
            if (!__all_sync(0xffffffffu, bar_wait(smem_u32(&tdone[b]), (uint32_t)((nu >> 1) & 1)))) return false;
            fence_after_sync();
            const int t = ui.t0 + tl;
            float* pe = part + en.poff + (long long)ui.sp * en.tau * tau_pad + t;
            for (int c = 0; c < 64; c += 8) {
                const int j0 = h * 64 + c;
                if (j0 >= en.tau) break;
                uint32_t a[8];
                tmem_ld8(lane_base + (uint32_t)(b * GT_N + j0), a);
                tmem_wait_ld();
                if (t < tau_pad) {
#pragma unroll
                    for (int x = 0; x < 8; ++x)
                        if (j0 + x < en.tau) pe[(long long)(j0 + x) * tau_pad] = __uint_as_float(a[x]);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) bar_arrive(smem_u32(&tfree[b]));
            return true;
        };

        long long nu = 0, prev = -1;
        for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x, ++nu) {
            const UnitIdx ui = unit_of(ga, u);
            for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++itr, ++slot) {
                const int rs = (int)(itr % RS), cs = (int)(slot % CS);
                if (!bar_wait(smem_u32(&rfull[rs]), (uint32_t)((itr / RS) & 1))) { ok = false; break; }
                float v[kRPT];
                const float* rf = reinterpret_cast<const float*>(raw + rs * RAW);
#pragma unroll
                for (int k = 0; k < kRPT; ++k) v[k] = rf[(kRPT * h + k) * GT_M + tl];
                __syncwarp();
                if (lane == 0) bar_arrive(smem_u32(&rempty[rs]));
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
            if (prev >= 0 && !store_unit(prev, nu - 1)) { ok = false; break; }
            prev = u;
        }
        if (ok && prev >= 0 && !store_unit(prev, nu - 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicOr(&g_grad_error, 1u);
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

cudaError_t grad_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_grad_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_grad_error, &zero, sizeof(unsigned int));
}

// Tensor maps: F_e (FP32, dims t, rows, shifts; box 128 x 32 x 1, no swizzle) and the entry's
// pre-split pieces (bf16, dims rows, j, shifts, pieces; box 32 x 128 x 1 x P, 64-byte swizzle);
// elements outside the arrays (columns t >= tau_pad, j >= tau_e) read as zero.
cudaError_t launch_grad_tc(const __nv_bfloat16* xp, const float* Froot, long long root_stride, const float* Fchain,
                           long long chain_stride, int tau_pad, const Chain& ch, const int* sel, const long long* xoff,
                           int nsel, float* part, int reff, int pieces, cudaStream_t st) {
    if (nsel == 0) return cudaSuccess;
    if (nsel > kMaxGradTc || (pieces != 1 && pieces != 3)) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    GradTcArgs ga{};
    ga.n = nsel;
    ga.reff = reff;
    ga.t_tiles = (tau_pad + GT_M - 1) / GT_M;
    long long units = 0;
    for (int i = 0; i < nsel; ++i) {
        const int e = sel[i];
        GradTcEntry& en = ga.ent[i];
        en.n = 1LL << ch.logn[e];
        en.tau = ch.tau[e];
        en.split = ch.split[e];
        en.kper = ch.kper[e];
        en.poff = ch.poff[e];
        en.xoff = xoff[i];
        if (en.tau > GT_N || en.n < GK || en.kper % GK != 0) return cudaErrorInvalidValue;
        ga.unit0[i] = units;
        units += (long long)en.split * ga.t_tiles;
        const float* Fb = (ch.fsel[e] ? Fchain : Froot) + ch.foff[e];
        const long long Fs = ch.fsel[e] ? chain_stride : root_stride;
        {
            const cuuint64_t dims[3] = {(cuuint64_t)tau_pad, (cuuint64_t)en.n, (cuuint64_t)reff};
            const cuuint64_t strides[2] = {(cuuint64_t)tau_pad * 4, (cuuint64_t)Fs * 4};
            const cuuint32_t box[3] = {GT_M, GK, 1};
            const cuuint32_t estr[3] = {1, 1, 1};
            if (fn(&ga.fmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(Fb), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        {
            const cuuint64_t n = (cuuint64_t)en.n;
            const cuuint64_t dims[4] = {n, (cuuint64_t)en.tau, (cuuint64_t)reff, (cuuint64_t)pieces};
            const cuuint64_t strides[3] = {n * 2, n * 2 * en.tau, n * 2 * en.tau * reff};
            const cuuint32_t box[4] = {GK, GT_N, 1, (cuuint32_t)pieces};
            const cuuint32_t estr[4] = {1, 1, 1, 1};
            if (fn(&ga.xmap[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(xp + en.xoff), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
    }
    ga.unit0[nsel] = units;
    ga.units = units;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>(units, sms);
    if (pieces == 3) {
        cudaError_t e = cudaFuncSetAttribute(k_grad_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<3>());
        if (e != cudaSuccess) return e;
        k_grad_tc<3><<<grid, kThreads, grad_smem<3>(), st>>>(ga, part, tau_pad);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_grad_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<1>());
        if (e != cudaSuccess) return e;
        k_grad_tc<1><<<grid, kThreads, grad_smem<1>(), st>>>(ga, part, tau_pad);
    }
    return cudaGetLastError();
}

}  // namespace qmc
