// Fused forward of the fine band on tensor cores (split and bf16 tiers, dyadic band S4:
// levels 0..3 with at most 1, 2, 4, 8 columns).
//
// Every output row k = rho + q n_root (root rho < n_root = N/16, leaf q < 16) is
//     y_k = S_4[rho] + sum_{I<4} sum_{j in level I} x_{k mod n_I, j} a_j,
// the root value S_4 (the periodic sum of the coarse block products, Algorithm 2) plus the
// fine band's 15 columns.  A tile of 128 rows holds 8 roots x 16 leaves (TMEM lane
// l = 16 (rho - rho0) + q), so the whole row block is one MMA pair with K = 32:
//     D = [X_f | E] [A_f ; S],   X_f: 128 x 16 fine coordinates of the rows (15 used),
//                                E:   128 x 16 with E[l][i] = [l / 16 == i] (8 used),
//                                A_f: the 15 fine rows of kappa A, S: kappa S_4 of the 8 roots.
// The split tier keeps six piece products of X_f A_f and the three products E S_p (E is
// exact in bf16); the bf16 tier one product each.  The epilogue applies the integrand to
// D straight out of tensor memory and keeps per-row sums, so y never reaches memory.
//
// Warp roles of the persistent CTA (one per SM, a fixed column tile of 256 columns):
//   warps 0-7   epilogue: warp w reads TMEM lanes 32 (w % 4).. and columns 128 (w / 4)..;
//   warps 8-11  producers: gather the rows' fine coordinates and the roots' S values,
//               split them into bf16 pieces and fill one of two shared-memory stages;
//   warp 12     MMA issue (one thread).
// Two TMEM accumulators of 256 columns let the MMAs of tile i+1 run under the epilogue of
// tile i.  Every wait is bounded; a wait that runs out raises the CTA's abort flag, which
// ends every role's loop, and sets the device error word.
#include <algorithm>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

__device__ unsigned int g_fine_tc_error;

using namespace tc;

namespace {

constexpr int NT = 256;                 // columns per tile (MMA N)
constexpr int EPI_WARPS = 8, PROD_WARPS = 4;
constexpr int THREADS = (EPI_WARPS + PROD_WARPS + 1) * 32;
constexpr int kRootsPerTile = 8;        // x 16 leaves = 128 rows per tile

template <int P>
struct FineSmem {
    static constexpr uint32_t TILE_A = TM * ROWB;          // one piece of [X_f | E]: 8 KB
    static constexpr uint32_t TILE_B = NT * ROWB;          // one piece of [A_f ; S]^T: 16 KB
    static constexpr uint32_t STAGE = P * (TILE_A + TILE_B);
    static constexpr uint32_t XST = 2 * STAGE;                // fp32 staging: 64 fine nodes x 8 roots
    static constexpr uint32_t SST = XST + 64 * 8 * 4;         // fp32 staging: NT columns x 8 roots
    static constexpr uint32_t BARS = SST + NT * 8 * 4;
    // at least 120 KB so that one CTA (holding all 512 TMEM columns) runs per SM
    static constexpr size_t bytes = 1024 + BARS + 128 < 120 * 1024 ? 120 * 1024 : 1024 + BARS + 128;
};

}  // namespace

template <int P, int F>
__global__ void __launch_bounds__(THREADS, 1) k_fine_fwd_tc(const FineArgs<float> a, int ntn, long long units) {
    using L = FineSmem<P>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BARS);        // producers -> MMA   (count 128)
    uint64_t* empty = full + 2;                                           // MMA -> producers   (commit)
    uint64_t* accf = full + 4;                                            // MMA -> epilogue    (commit)
    uint64_t* acce = full + 6;                                            // epilogue -> MMA    (count 256)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 8);
    volatile int* abort = reinterpret_cast<volatile int*>(full + 9);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = blockIdx.x % ntn;                 // this CTA's column tile
    const long long u0 = blockIdx.x / ntn, ustep = gridDim.x / ntn;
    const int t0 = nt * NT;
    const int ncols = min(NT, a.tau_pad - t0);
    const uint32_t nmma = (uint32_t)((ncols + 15) & ~15);
    const long long n_root = 1LL << a.logn_root;
    const int lmt = a.logn_root - 3;                  // log2 of the row tiles per shift (8 roots each)

    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 512);
    if (tid == 0) {
        mbar_init(&full[0], PROD_WARPS * 32); mbar_init(&full[1], PROD_WARPS * 32);
        mbar_init(&empty[0], 1); mbar_init(&empty[1], 1);
        mbar_init(&accf[0], 1); mbar_init(&accf[1], 1);
        mbar_init(&acce[0], EPI_WARPS * 32); mbar_init(&acce[1], EPI_WARPS * 32);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp >= EPI_WARPS && warp < EPI_WARPS + PROD_WARPS) {
        // ---------------------------------------------------------------- producers
        // A tile's inputs are read with coalesced 16-byte loads into fp32 staging buffers:
        //   fine nodes: item (lev, jj, c) = 16 lev + jj (16 >> lev) + c holds x of column jj of
        //     level lev at row rho + c n_root for the tile's 8 consecutive roots rho (32 bytes);
        //   S: the 8 roots' values of every column (the [t/4][rho][t%4] layout gives 128
        //     contiguous bytes per 4 columns).
        // Then every thread converts its own rows: row p of [X_f | E] and rows p, p+128 of
        // [A_f ; S]^T.  The loads of tile i+1 are in flight while tile i is converted.
        const int p = tid - EPI_WARPS * 32;
        float* Xst = reinterpret_cast<float*>(smem + L::XST);
        float* Sst = reinterpret_cast<float*>(smem + L::SST);
        auto prod_sync = [] { asm volatile("bar.sync 1, %0;" :: "n"(PROD_WARPS * 32) : "memory"); };
        // the producers' barrier with an OR over the threads: every producer takes the same
        // decision to stop, so none is left waiting at a barrier the others have quit
        auto prod_sync_or = [](bool v) {
            uint32_t r;
            asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                         "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(r) : "r"((uint32_t)v), "n"(PROD_WARPS * 32) : "memory");
            return r != 0;
        };
        // this thread's coalesced loads: fine node item p >> 1, roots 4 (p & 1)..+3;
        // S float4s f = p + 128 i: column group t4 = f >> 3, root f & 7
        const int item = p >> 1, lev_i = item >> 4, rem = item & 15;
        const int nodes_i = 16 >> lev_i, jj_i = rem / nodes_i, c_i = rem - jj_i * nodes_i;
        const bool item_live = jj_i < a.lev_tau[lev_i];
        const long long item_off = a.lev_tab[lev_i] + ((long long)jj_i << a.lev_logn[lev_i]) +
                                   (long long)c_i * n_root + 4 * (p & 1);
        float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), sr[4];
        auto load_tile = [&](long long u) {
            const long long r = u >> lmt, rho0 = (u & ((1LL << lmt) - 1)) * kRootsPerTile;
            xr = item_live ? __ldg(reinterpret_cast<const float4*>(a.tab + r * a.tab_stride + item_off + rho0))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            const float* S = a.S + r * a.S_stride;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int f = p + 128 * i, t4 = f >> 3, ri = f & 7;
                sr[i] = (S && t0 + 4 * t4 < a.tau_pad)
                            ? __ldg(reinterpret_cast<const float4*>(S + ((((long long)(t0 / 4 + t4)) << a.logn_root) +
                                                                         rho0 + ri) * 4))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        if (u0 < units) load_tile(u0);                     // in flight while the constant parts are set up
        {   // constant parts of both stages: E (piece 0), the fine rows of kappa A, zero padding
            float av[2][16];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = t0 + p + 128 * h;
#pragma unroll
                for (int lev = 0, kk = 0; lev < 4; ++lev) {
#pragma unroll
                    for (int jj = 0; jj < (1 << lev); ++jj, ++kk)
                        av[h][kk] = (jj < a.lev_tau[lev] && t < a.tau_pad)
                                        ? a.kappa * __ldg(a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA + t) : 0.0f;
                }
                av[h][15] = 0.0f;
            }
            float e[8], z[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) { e[i] = (i == (p >> 4)) ? 1.0f : 0.0f; z[i] = 0.0f; }
            for (int s = 0; s < 2; ++s) {
                unsigned char* As_ = smem + s * L::STAGE;
                unsigned char* Bs_ = As_ + P * L::TILE_A;
                store_group<P>(As_, L::TILE_A, p, 2, e);
                store_group<P>(As_, L::TILE_A, p, 3, z);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    store_group<P>(Bs_, L::TILE_B, p + 128 * h, 0, av[h]);
                    store_group<P>(Bs_, L::TILE_B, p + 128 * h, 1, av[h] + 8);
                    store_group<P>(Bs_, L::TILE_B, p + 128 * h, 3, z);
                }
            }
        }
        const int rl = p >> 4, q = p & 15;
        bool ok = true;
        for (long long it = 0;; ++it) {
            const long long u = u0 + it * ustep;
            // the previous tile's staging has been read by every producer
            if (prod_sync_or(u >= units || *abort || !ok)) break;
            *reinterpret_cast<float4*>(Xst + item * 8 + 4 * (p & 1)) = xr;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int f = p + 128 * i, t4 = f >> 3, ri = f & 7;
                Sst[(4 * t4 + 0) * 8 + ri] = sr[i].x;
                Sst[(4 * t4 + 1) * 8 + ri] = sr[i].y;
                Sst[(4 * t4 + 2) * 8 + ri] = sr[i].z;
                Sst[(4 * t4 + 3) * 8 + ri] = sr[i].w;
            }
            prod_sync();                                   // staging complete
            if (u + ustep < units) load_tile(u + ustep);   // in flight during the conversion below
            float x[16], sv[2][8];
#pragma unroll
            for (int lev = 0, kk = 0; lev < 4; ++lev) {
                const int c = q & ((16 >> lev) - 1);
#pragma unroll
                for (int jj = 0; jj < (1 << lev); ++jj, ++kk)
                    x[kk] = Xst[(16 * lev + jj * (16 >> lev) + c) * 8 + rl];
            }
            x[15] = 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 lo = *reinterpret_cast<const float4*>(Sst + (p + 128 * h) * 8);
                const float4 hi = *reinterpret_cast<const float4*>(Sst + (p + 128 * h) * 8 + 4);
                sv[h][0] = a.kappa * lo.x; sv[h][1] = a.kappa * lo.y; sv[h][2] = a.kappa * lo.z; sv[h][3] = a.kappa * lo.w;
                sv[h][4] = a.kappa * hi.x; sv[h][5] = a.kappa * hi.y; sv[h][6] = a.kappa * hi.z; sv[h][7] = a.kappa * hi.w;
            }
            const int s = (int)(it & 1);
            if (it >= 2) ok = mbar_wait_abort(&empty[s], (uint32_t)(((it - 2) >> 1) & 1), abort);
            if (ok) {                                      // (a failed wait stops all producers at the loop top)
                unsigned char* As_ = smem + s * L::STAGE;
                unsigned char* Bs_ = As_ + P * L::TILE_A;
                store_group<P>(As_, L::TILE_A, p, 0, x);
                store_group<P>(As_, L::TILE_A, p, 1, x + 8);
                store_group<P>(Bs_, L::TILE_B, p, 2, sv[0]);
                store_group<P>(Bs_, L::TILE_B, p + 128, 2, sv[1]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&full[s]);
            }
        }
    } else if (warp == EPI_WARPS + PROD_WARPS) {
        // ---------------------------------------------------------------- MMA issue
        if ((tid & 31) == 0) {
            const uint32_t idesc = idesc_bf16(nmma);
            for (long long it = 0;; ++it) {
                const long long u = u0 + it * ustep;
                if (u >= units || *abort) break;
                const int s = (int)(it & 1), b = (int)(it & 1);
                if (!mbar_wait_abort(&full[s], (uint32_t)((it >> 1) & 1), abort)) break;
                if (it >= 2 && !mbar_wait_abort(&acce[b], (uint32_t)(((it - 2) >> 1) & 1), abort)) break;
                fence_after_sync();
                const uint32_t As_ = smem_u32(smem + s * L::STAGE);
                const uint32_t Bs_ = As_ + P * L::TILE_A;
                const uint32_t d = tmem + (uint32_t)(b * NT);
                bool first = true;
                issue_kstep<P>(d, As_, L::TILE_A, Bs_, L::TILE_B, idesc, first);          // X_f A_f
#pragma unroll
                for (int j = 0; j < P; ++j)                                               // E S_j
                    mma_bf16(d, smem_desc_sw64(As_ + 32), smem_desc_sw64(Bs_ + 32 + j * L::TILE_B), idesc, 1u);
                mma_commit(smem_u32(&empty[s]));
                mma_commit(smem_u32(&accf[b]));
            }
        }
    } else if (warp < EPI_WARPS) {
        // ---------------------------------------------------------------- epilogue
        const int quarter = warp & 3, half = warp >> 2;
        const int l = quarter * 32 + (tid & 31);
        const int rl = l >> 4, q = l & 15;
        const int c_beg = half * 128;
        const int cg = (t0 + c_beg) >> 7;            // column group of the row partials
        const bool group_live = t0 + c_beg < a.tau;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        for (long long it = 0;; ++it) {
            const long long u = u0 + it * ustep;
            if (u >= units || *abort) break;
            const int b = (int)(it & 1);
            if (!mbar_wait_abort(&accf[b], (uint32_t)((it >> 1) & 1), abort)) break;
            fence_after_sync();
            float racc = 0.0f, rmax = -INFINITY;
            if (group_live) {
                constexpr int CWD = F == F_LOGSUMEXP ? 32 : 64;     // columns per TMEM wait
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += CWD) {
                    uint32_t d[CWD];
                    tmem_ld32(tmem + lane_base + (uint32_t)(b * NT + c_beg + c0), *reinterpret_cast<uint32_t(*)[32]>(d));
                    if constexpr (CWD == 64)
                        tmem_ld32(tmem + lane_base + (uint32_t)(b * NT + c_beg + c0 + 32),
                                  *reinterpret_cast<uint32_t(*)[32]>(d + 32));
                    tmem_wait_ld();
                    const int tb = t0 + c_beg + c0;
                    if constexpr (F == F_LOGSUMEXP) {
                        float mx = rmax;
#pragma unroll
                        for (int i = 0; i < CWD; ++i)
                            if (tb + i < a.tau) mx = fmaxf(mx, __uint_as_float(d[i]));
                        float sacc = racc * ex2f(rmax - mx);
#pragma unroll
                        for (int i = 0; i < CWD; ++i)
                            if (tb + i < a.tau) sacc += ex2f(__uint_as_float(d[i]) - mx);
                        racc = sacc;
                        rmax = mx;
                    } else {
                        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
                        for (int i = 0; i < CWD; i += 2) {
                            if (tb + i < a.tau) acc0 += Fn<F, float>::h(__uint_as_float(d[i]), a.c0);
                            if (tb + i + 1 < a.tau) acc1 += Fn<F, float>::h(__uint_as_float(d[i + 1]), a.c0);
                        }
                        racc += acc0 + acc1;
                    }
                }
            }
            fence_before_sync();
            mbar_arrive(&acce[b]);
            if (group_live) {
                const long long r = u >> lmt, rho0 = (u & ((1LL << lmt) - 1)) * kRootsPerTile;
                const long long k = rho0 + rl + (long long)q * n_root;
                const long long o = (r * a.cg_count + cg) * a.N + k;
                a.rowpart[o] = racc;
                if constexpr (F == F_LOGSUMEXP) a.rowmax[o] = rmax;
            }
        }
    }
    if (*abort && tid == 0) atomicOr(&g_fine_tc_error, 1u);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------------------------------
// launcher: one CTA per SM, CTAs spread evenly over the column tiles
// ------------------------------------------------------------------------------------------
namespace {
template <int P, int F>
cudaError_t fwd_tc_launch(const FineArgs<float>& a, cudaStream_t st) {
    const int ntn = (a.tau_pad + NT - 1) / NT;
    const long long units = (long long)a.reff * ((1LL << a.logn_root) / kRootsPerTile);
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long per = std::max(1, sms / ntn);
    per = std::min<long long>(per, units);
    const size_t smem = FineSmem<P>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_fine_fwd_tc<P, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fine_fwd_tc<P, F><<<(unsigned)(per * ntn), THREADS, smem, st>>>(a, ntn, units);
    return cudaGetLastError();
}

template <int P>
cudaError_t fwd_tc_f(const FineArgs<float>& a, int F, cudaStream_t st) {
    switch (F) {
        case F_LINEAR_MEAN: return fwd_tc_launch<P, F_LINEAR_MEAN>(a, st);
        case F_MEAN_COS: return fwd_tc_launch<P, F_MEAN_COS>(a, st);
        case F_CALL_MEAN_EXP: return fwd_tc_launch<P, F_CALL_MEAN_EXP>(a, st);
        case F_GAUSS_NORM2: return fwd_tc_launch<P, F_GAUSS_NORM2>(a, st);
        case F_PDE_INV_SQ: return fwd_tc_launch<P, F_PDE_INV_SQ>(a, st);
        case F_LOGSUMEXP: return fwd_tc_launch<P, F_LOGSUMEXP>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int fine_tc_group_cols() { return 128; }

cudaError_t launch_fine_fwd_tc(const FineArgs<float>& a, int F, int pieces, cudaStream_t st) {
    if (a.logn_root < 3) return cudaErrorInvalidValue;        // 8 roots per tile
    if (pieces == 3) return fwd_tc_f<3>(a, F, st);
    if (pieces == 1) return fwd_tc_f<1>(a, F, st);
    return cudaErrorInvalidValue;
}

cudaError_t fine_tc_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_fine_tc_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_fine_tc_error, &zero, sizeof(unsigned int));
}

}  // namespace qmc
