// Block gradients of the coarse levels on the tensor cores (split and bf16 tiers): the adjoint of
// Algorithm 2's block products, dA_e = sum_r X_{r,e}^T F_{r,e} over the level's distinct rows, with
// F_e the root gradients folded onto the level (k_fold_tree).
//
// D[t][j] = sum_k F_e[k][t] (X_e[k][j] - xc): M = 128 columns t, N = 64 gradient columns j, K = the
// level's rows over every shift, cut into splits of at most 4096 rows (a work unit = entry x j tile x
// t tile x split).  One persistent CTA per SM, warp-specialised:
//   warp 0      TMA producer: the raw FP32 chunk of F (32 rows k x 128 columns t, a 3-D box over
//               (t, rows, shifts)) and of X (64 columns j x 32 rows k, from the point table) into a
//               ring of raw stages;
//   warp 1      allocates 256 tensor-memory columns (four 128 x 64 FP32 accumulators) and one thread
//               issues each converted chunk's MMAs (M = 128, N = 64, K = 16) into accumulator
//               chunk % 4, so that an FP32 accumulation chain in tensor memory is at most 1024 rows;
//   warps 2-9   converters: split the raw chunk into bf16 pieces in the MMA's K-major, 64-byte-
//               swizzled layout (F transposed to [t][k], X centred by xc, padding columns zero), and
//               after a unit's last chunk read the four accumulators, sum them in a fixed order and
//               store the unit's partial, which k_grad_reduce sums over the splits.
// Every wait is bounded; a run-out sets the level kernels' error word and the CTA stops as in
// k_level_tc (the MMA thread drains its commits before the tensor memory is released).
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
constexpr int GT_N = 64;                     // gradient columns j per unit (MMA N)
constexpr int GK = 32;                       // rows k per chunk
constexpr int NACC = 4;
constexpr int RS = 4;                        // raw stages
constexpr int CS = 3;                        // converted stages
constexpr uint32_t RAW_F = GK * GT_M * 4;    // [k][t] FP32, 16 KB
constexpr uint32_t RAW_X = GT_N * GK * 4;    // [j][k] FP32, 8 KB
constexpr uint32_t RAW_STAGE = RAW_F + RAW_X;
constexpr uint32_t PF = GT_M * 64;           // one bf16 piece of F^T: 128 rows x 64 bytes
constexpr uint32_t PX = GT_N * 64;           // one bf16 piece of X: 64 rows x 64 bytes
constexpr int kThreads = 320;

template <int P> constexpr uint32_t cstage() { return P * (PF + PX); }
template <int P> constexpr size_t grad_smem() { return 1024 + RS * RAW_STAGE + CS * cstage<P>() + 256; }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar) : "memory");
}

struct UnitIdx {
    int e, sp, j0, t0;
    long long kb, ke;
};

__device__ __forceinline__ UnitIdx unit_of(const GradTcArgs& ga, long long u) {
    int e = 0;
    while (e + 1 < ga.n && u >= ga.unit0[e + 1]) ++e;
    const long long loc = u - ga.unit0[e];
    const GradTcEntry& en = ga.ent[e];
    UnitIdx ui;
    ui.e = e;
    ui.t0 = (int)(loc % ga.t_tiles) * GT_M;
    const long long rest = loc / ga.t_tiles;
    ui.sp = (int)(rest % en.split);
    ui.j0 = (int)(rest / en.split) * GT_N;
    ui.kb = (long long)ui.sp * en.kper;
    ui.ke = min((long long)ga.reff * en.n, ui.kb + en.kper);
    return ui;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) k_grad_tc(const __grid_constant__ GradTcArgs ga, float* __restrict__ part,
                                                         int tau_pad, float xc) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    unsigned char* craw = smem;                                  // RS raw stages
    unsigned char* cconv = smem + RS * RAW_STAGE;                // CS converted stages (1 KB aligned)
    uint64_t* rfull = reinterpret_cast<uint64_t*>(cconv + CS * cstage<P>());
    uint64_t* rempty = rfull + RS;
    uint64_t* cfull = rempty + RS;
    uint64_t* cempty = cfull + CS;
    uint64_t* tdone = cempty + CS;
    uint64_t* tfree = tdone + 1;
    uint64_t* drain = tfree + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        for (int e = 0; e < ga.n; ++e) {
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&ga.fmap[e])) : "memory");
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&ga.xmap[e])) : "memory");
        }
        for (int s = 0; s < RS; ++s) { bar_init(&rfull[s], 1); bar_init(&rempty[s], 8); }
        for (int s = 0; s < CS; ++s) { bar_init(&cfull[s], 8); bar_init(&cempty[s], 1); }
        bar_init(tdone, 1);
        bar_init(tfree, 8);
        bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), NACC * GT_N);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long it = 0;
            for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x) {
                const UnitIdx ui = unit_of(ga, u);
                const GradTcEntry& en = ga.ent[ui.e];
                for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++it) {
                    const int s = (int)(it % RS);
                    if (!bar_wait(smem_u32(&rempty[s]), (uint32_t)(((it / RS) & 1) ^ 1))) { ok = false; break; }
                    const uint32_t fb = smem_u32(&rfull[s]);
                    bar_expect_tx(fb, RAW_STAGE);
                    const int r = (int)(k0 / en.n), rho = (int)(k0 - (long long)r * en.n);
                    unsigned char* st = craw + s * RAW_STAGE;
                    // rows beyond the split's end (or the last shift) read as zero (out of range) or are
                    // rows of the next split, whose F is multiplied by X rows that are zero-filled
                    tma_load_3d(smem_u32(st), &ga.fmap[ui.e], fb, ui.t0, rho, r);
                    tma_load_3d(smem_u32(st + RAW_F), &ga.xmap[ui.e], fb, rho, ui.j0, r);
                }
            }
            if (!ok) {
                atomicOr(&g_grad_error, 1u);
                for (long long k = it - 1; k >= 0 && k >= it - RS; --k)
                    bar_wait(smem_u32(&rfull[k % RS]), (uint32_t)((k / RS) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(GT_N);
            long long it = 0, n = 0;
            for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x, ++n) {
                const UnitIdx ui = unit_of(ga, u);
                if (!bar_wait(smem_u32(tfree), (uint32_t)((n & 1) ^ 1))) { ok = false; break; }
                fence_after_sync();
                int c = 0;
                for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++it, ++c) {
                    const int s = (int)(it % CS);
                    if (!bar_wait(smem_u32(&cfull[s]), (uint32_t)((it / CS) & 1))) { ok = false; break; }
                    fence_after_sync();
                    const uint32_t fs = smem_u32(cconv + s * cstage<P>()), xs = fs + P * PF;
                    bool fresh = c < NACC;
                    for (int ks = 0; ks < 2; ++ks)
                        issue_kstep<P, PF, PX>(tmem + (uint32_t)((c % NACC) * GT_N), smem_desc_sw64(fs + 32 * ks),
                                               smem_desc_sw64(xs + 32 * ks), idesc, fresh);
                    mma_commit(smem_u32(&cempty[s]));
                }
                if (ok) mma_commit(smem_u32(tdone));
            }
            if (!ok) atomicOr(&g_grad_error, 1u);
            mma_commit(smem_u32(drain));
            bar_wait(smem_u32(drain), 0);
        }
    } else {
        // ------------------------------------------------------------------ converters and epilogue
        const int ct = threadIdx.x - 64;                       // 0..255
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        long long itr = 0, itc = 0, n = 0;
        for (long long u = blockIdx.x; u < ga.units && ok; u += gridDim.x, ++n) {
            const UnitIdx ui = unit_of(ga, u);
            const GradTcEntry& en = ga.ent[ui.e];
            const int nj = min(GT_N, en.tau - ui.j0);
            for (long long k0 = ui.kb; k0 < ui.ke; k0 += GK, ++itr, ++itc) {
                const int rs = (int)(itr % RS), cs = (int)(itc % CS);
                if (!bar_wait(smem_u32(&rfull[rs]), (uint32_t)((itr / RS) & 1))) { ok = false; break; }
                if (!bar_wait(smem_u32(&cempty[cs]), (uint32_t)(((itc / CS) & 1) ^ 1))) { ok = false; break; }
                const float* rf = reinterpret_cast<const float*>(craw + rs * RAW_STAGE);
                const float* rx = reinterpret_cast<const float*>(craw + rs * RAW_STAGE + RAW_F);
                unsigned char* fs = cconv + cs * cstage<P>();
                unsigned char* xs = fs + P * PF;
                const long long nk = ui.ke - k0;               // valid rows of this chunk (may be < 32)
                {   // F^T: row t = ct % 128, k = 16 (ct / 128) .. + 15
                    const int t = ct & 127, h = ct >> 7;
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int k = 16 * h + i;
                        v[i] = k < nk ? rf[k * GT_M + t] : 0.0f;
                    }
                    store_group<P>(fs, PF, t, 2 * h, v);
                    store_group<P>(fs, PF, t, 2 * h + 1, v + 8);
                }
                {   // X: row j = ct / 4, k = 8 (ct % 4) .. + 7 (the k group fastest, so that a quarter warp's
                    // 16-byte loads span two rows), centred; padding rows j >= nj stay zero
                    const int j = ct >> 2, q = ct & 3;
                    const float4* xr = reinterpret_cast<const float4*>(rx + j * GK + 8 * q);
                    const float4 a = xr[0], b = xr[1];
                    const float d = j < nj ? xc : 0.0f;
                    float v[8] = {a.x - d, a.y - d, a.z - d, a.w - d, b.x - d, b.y - d, b.z - d, b.w - d};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (8 * q + i >= nk || j >= nj) v[i] = 0.0f;
                    store_group<P>(xs, PX, j, q, v);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    bar_arrive(smem_u32(&rempty[rs]));
                    bar_arrive(smem_u32(&cfull[cs]));
                }
            }
            if (!ok) break;
            // the unit's partial: D[t][j] summed over the four accumulators in a fixed order
            if (!bar_wait(smem_u32(tdone), (uint32_t)(n & 1))) { ok = false; break; }
            fence_after_sync();
            const int chunks = (int)((ui.ke - ui.kb + GK - 1) / GK);
            const int t = ui.t0 + quarter * 32 + lane;
            float sum[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) sum[i] = 0.0f;
            const uint32_t la = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
            for (int a = 0; a < NACC && a < chunks; ++a) {
                uint32_t d[32];
                tmem_ld32(la + (uint32_t)(a * GT_N), d);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) sum[i] += __uint_as_float(d[i]);
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) bar_arrive(smem_u32(tfree));
            if (t < tau_pad) {
                float* pe = part + en.poff + ((long long)ui.sp * en.tau + ui.j0 + half * 32) * tau_pad + t;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (half * 32 + i < nj) pe[(long long)i * tau_pad] = sum[i];
            }
        }
        if (!ok && lane == 0) atomicOr(&g_grad_error, 1u);
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, NACC * GT_N);
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

// FP32 3-D tensor map, no swizzle: dims {d0, d1, d2}, strides (bytes) {s1, s2}, box {b0, b1, 1};
// out-of-range elements read as zero
cudaError_t map3(CUtensorMap* m, const void* base, long long d0, long long d1, long long d2, long long s1,
                 long long s2, int b0, int b1) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
    const cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
    const cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t grad_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_grad_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_grad_error, &zero, sizeof(unsigned int));
}

size_t grad_tc_smem(int pieces) { return pieces == 3 ? grad_smem<3>() : grad_smem<1>(); }

cudaError_t launch_grad_tc(const float* tab, long long tab_stride, const float* Froot, long long root_stride,
                           const float* Fchain, long long chain_stride, int tau_pad, const Chain& ch, const int* sel,
                           int nsel, float* part, int reff, int pieces, float xc, cudaStream_t st) {
    if (nsel == 0) return cudaSuccess;
    if (nsel > kMaxGradTc) return cudaErrorInvalidValue;
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
        ga.unit0[i] = units;
        units += (long long)((en.tau + GT_N - 1) / GT_N) * en.split * ga.t_tiles;
        const float* Fb = (ch.fsel[e] ? Fchain : Froot) + ch.foff[e];
        const long long Fs = ch.fsel[e] ? chain_stride : root_stride;
        // F: (t, rows rho < n_e, shifts), row stride tau_pad floats, shift stride Fs floats
        cudaError_t err = map3(&ga.fmap[i], Fb, tau_pad, en.n, reff, 4LL * tau_pad, 4LL * Fs, GT_M, GK);
        if (err != cudaSuccess) return err;
        // X: (rows rho < n_e, columns j of the entry, shifts): the entry's table columns
        err = map3(&ga.xmap[i], tab + ch.tab[e], en.n, en.tau, reff, 4LL * en.n, 4LL * tab_stride, GK, GT_N);
        if (err != cudaSuccess) return err;
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
        k_grad_tc<3><<<grid, kThreads, grad_smem<3>(), st>>>(ga, part, tau_pad, xc);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_grad_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<1>());
        if (e != cudaSuccess) return e;
        k_grad_tc<1><<<grid, kThreads, grad_smem<1>(), st>>>(ga, part, tau_pad, xc);
    }
    return cudaGetLastError();
}

}  // namespace qmc
