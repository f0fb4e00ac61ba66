// The fine band on tensor cores (split and bf16 tiers, dyadic band S4: levels 0..3 with
// at most 1, 2, 4, 8 columns): the fused forward and its adjoint.
//
// Every output row k = rho + q n_root (root rho < n_root = N/16, leaf q < 16) is
//     y_k = S_4[rho] + sum_{I<4} sum_{j in level I} x_{k mod n_I, j} a_j,
// the root value S_4 (the periodic sum of the coarse block products, Algorithm 2) plus the
// fine band's 15 columns.  A tile of 128 rows holds 8 roots x 16 leaves (TMEM lane
// l = 16 (rho - rho0) + q), so the whole row block is one MMA pair with K = 32:
//     D = W [A_f ; S],   W = [X_f | E]:  X_f: 128 x 16 fine coordinates of the rows (15 used),
//                                        E:   128 x 16, E[l][i] = [l / 16 == i] (8 used),
//                        A_f: the 15 fine rows of kappa A, S: kappa S_4 of the tile's 8 roots.
// The split tier keeps six piece products of X_f A_f and the three products E S_p (E is
// exact in bf16); the bf16 tier one product each.
//
// Forward: the epilogue applies the integrand to D straight out of tensor memory and keeps
// per-row sums, so y never reaches memory.
// Adjoint: with G[l][t] = coef_l h'(v_lt) (eq. (2)'s chain rule, coef from the forward's
// row finalisation), one more MMA family D' = G^T W gives, per column t,
//     D'[t][m], m < 15:       sum_l G[l][t] x_{l,m}   (the fine-band gradient, accumulated),
//     D'[t][16 + i], i < 8:   sum_q G[rho0 + i + q n_root][t]   (the root gradient F_4),
// i.e. the adjoint of the band's broadcast and of the root tiling in one product.  G^T is
// written by the epilogue as an MN-major operand; W is read as MN-major from the forward
// operand tile (the same bytes).  In the split tier the three pieces of W sit side by side
// along N (N = 96) and each piece of G multiplies all of them, so the accumulator holds
// G W_j for j = 0, 1, 2 (all nine piece products) and the epilogue adds the three blocks.
//
// Warp roles of the persistent CTA (one per SM, a fixed column tile):
//   epilogue warps (8 forward, 16 adjoint): warp w reads TMEM lanes 32 (w % 4).. and a
//               share of the columns;
//   4 producer warps: stage the rows' fine coordinates and the roots' S values with
//               coalesced loads, split them into bf16 pieces, fill one of two stages;
//   1 MMA warp (one thread issues).
// Every wait is bounded; a wait that runs out raises the CTA's abort flag, which ends every
// role's loop, and sets the device error word.
#include <algorithm>

#include "qmc_internal.cuh"
#include "qmc_tc.cuh"

namespace qmc {

__device__ unsigned int g_fine_tc_error;

using namespace tc;

namespace {

constexpr int EPI_WARPS = 8, PROD_WARPS = 4;                 // forward
constexpr int THREADS = (EPI_WARPS + PROD_WARPS + 1) * 32;
constexpr int EPI_WARPS_B = 16;                               // adjoint: 4 warps per TMEM lane quarter
constexpr int DRAIN_WARPS = 4;                                // adjoint: one per lane quarter
constexpr int THREADS_B = (EPI_WARPS_B + DRAIN_WARPS + PROD_WARPS + 1) * 32;
constexpr int kRootsPerTile = 8;        // x 16 leaves = 128 rows per tile
constexpr int NT_FWD = 256, NT_BWD = 128;

// Shared-memory map of the producer stages: per stage, P pieces of W (128 rows x 64 B) and
// P pieces of [A_f ; S]^T (NTT rows x 64 B), NS stages; FP32 staging of the coalesced loads.
template <int P, int NTT, int NS = 2>
struct Stages {
    static constexpr int NSTAGE = NS;
    static constexpr uint32_t TILE_A = TM * ROWB;
    static constexpr uint32_t TILE_B = NTT * ROWB;
    static constexpr uint32_t STAGE = P * (TILE_A + TILE_B);
    static constexpr uint32_t XST = NS * STAGE;               // 64 fine nodes x 8 roots
    static constexpr uint32_t SST = XST + 64 * 8 * 4;         // NTT columns x 8 roots
    static constexpr uint32_t END = SST + NTT * 8 * 4;
};

// descriptor of a 64-byte-swizzled MN-major operand: atoms of 8 K-rows x 32 MN-elements
// (512 B), K-groups sbo bytes apart, MN-groups of 32 elements lbo bytes apart
__device__ __forceinline__ uint64_t smem_desc_sw64_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// MMA with the A operand in tensor memory (16-bit elements packed two per 32-bit column)
__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        :: "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                    "r"(r[7]) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// The producers' barrier (named barrier 1) with an OR over the threads: every producer takes
// the same decision to stop, so none is left waiting at a barrier the others have quit.
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, %0;" :: "n"(PROD_WARPS * 32) : "memory"); }

// The four epilogue warps of one TMEM lane quarter (named barriers 2..5) with an OR of a flag.
__device__ __forceinline__ bool quarter_sync_or(int quarter, bool v) {
    uint32_t r;
    const uint32_t x = (uint32_t)v;
    switch (quarter) {
#define QMC_QSYNC(Q) \
        case Q: asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t" \
                             "bar.red.or.pred q, " #Q " + 2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}" \
                             : "=r"(r) : "r"(x) : "memory"); break;
        QMC_QSYNC(0) QMC_QSYNC(1) QMC_QSYNC(2) QMC_QSYNC(3)
#undef QMC_QSYNC
        default: r = 1;
    }
    return r != 0;
}
__device__ __forceinline__ bool prod_sync_or(bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v), "n"(PROD_WARPS * 32) : "memory");
    return r != 0;
}

// ------------------------------------------------------------------------------------------
// Producer loop (128 threads, p = 0..127), shared by both kernels.
// A tile's inputs are read with coalesced 16-byte loads into FP32 staging buffers:
//   fine nodes: item (lev, jj, c) = 16 lev + jj (16 >> lev) + c holds x of column jj of
//     level lev at row rho + c n_root for the tile's 8 consecutive roots rho (32 bytes);
//   S: the 8 roots' values of every column (the [t/4][rho][t%4] layout gives 128
//     contiguous bytes per 4 columns).
// Then every thread converts its own rows: row p of W and rows p + 128 h of [A_f ; S]^T.
// The loads of tile i+1 are in flight while tile i is converted.  A stage is refilled
// after the MMA thread's commit on empty[s] (all MMAs that read it have completed).
// ------------------------------------------------------------------------------------------
template <int P, int NTT, int NS>
__device__ __forceinline__ void producer_loop(const FineArgs<float>& a, unsigned char* smem, uint64_t* full,
                                              uint64_t* empty, volatile int* abort, int p, long long u0,
                                              long long ustep, long long units, int t0, int lmt) {
    using L = Stages<P, NTT, NS>;
    constexpr int H = NTT / 128;                 // B rows per thread
    constexpr int NSL = NTT / 128 * 2;           // S float4 loads per thread
    const long long n_root = 1LL << a.logn_root;
    float* Xst = reinterpret_cast<float*>(smem + L::XST);
    float* Sst = reinterpret_cast<float*>(smem + L::SST);
    const int item = p >> 1, lev_i = item >> 4, rem = item & 15;
    const int nodes_i = 16 >> lev_i, jj_i = rem / nodes_i, c_i = rem - jj_i * nodes_i;
    const bool item_live = jj_i < a.lev_tau[lev_i];
    const long long item_off = a.lev_tab[lev_i] + ((long long)jj_i << a.lev_logn[lev_i]) +
                               (long long)c_i * n_root + 4 * (p & 1);
    float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), sr[NSL];
    auto load_tile = [&](long long u) {
        const long long r = u >> lmt, rho0 = (u & ((1LL << lmt) - 1)) * kRootsPerTile;
        xr = item_live ? __ldg(reinterpret_cast<const float4*>(a.tab + r * a.tab_stride + item_off + rho0))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        const float* S = a.S + r * a.S_stride;
#pragma unroll
        for (int i = 0; i < NSL; ++i) {
            const int f = p + 128 * i, t4 = f >> 3, ri = f & 7;
            sr[i] = (S && t0 + 4 * t4 < a.tau_pad)
                        ? __ldg(reinterpret_cast<const float4*>(
                              S + ((((long long)(t0 / 4 + t4)) << a.logn_root) + rho0 + ri) * 4))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (u0 < units) load_tile(u0);                     // in flight while the constant parts are set up
    {   // constant parts of both stages: E (piece 0), the fine rows of kappa A, zero padding
        float av[H][16];
#pragma unroll
        for (int h = 0; h < H; ++h) {
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
        for (int s = 0; s < NS; ++s) {
            unsigned char* As_ = smem + s * L::STAGE;
            unsigned char* Bs_ = As_ + P * L::TILE_A;
            store_group<P>(As_, L::TILE_A, p, 2, e);
            store_group<P>(As_, L::TILE_A, p, 3, z);
#pragma unroll
            for (int h = 0; h < H; ++h) {
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
        for (int i = 0; i < NSL; ++i) {
            const int f = p + 128 * i, t4 = f >> 3, ri = f & 7;
            Sst[(4 * t4 + 0) * 8 + ri] = sr[i].x;
            Sst[(4 * t4 + 1) * 8 + ri] = sr[i].y;
            Sst[(4 * t4 + 2) * 8 + ri] = sr[i].z;
            Sst[(4 * t4 + 3) * 8 + ri] = sr[i].w;
        }
        prod_sync();                                   // staging complete
        if (u + ustep < units) load_tile(u + ustep);   // in flight during the conversion below
        float x[16], sv[H][8];
#pragma unroll
        for (int lev = 0, kk = 0; lev < 4; ++lev) {
            const int c = q & ((16 >> lev) - 1);
#pragma unroll
            for (int jj = 0; jj < (1 << lev); ++jj, ++kk) x[kk] = Xst[(16 * lev + jj * (16 >> lev) + c) * 8 + rl];
        }
        x[15] = 0.0f;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float4 lo = *reinterpret_cast<const float4*>(Sst + (p + 128 * h) * 8);
            const float4 hi = *reinterpret_cast<const float4*>(Sst + (p + 128 * h) * 8 + 4);
            sv[h][0] = a.kappa * lo.x; sv[h][1] = a.kappa * lo.y; sv[h][2] = a.kappa * lo.z; sv[h][3] = a.kappa * lo.w;
            sv[h][4] = a.kappa * hi.x; sv[h][5] = a.kappa * hi.y; sv[h][6] = a.kappa * hi.z; sv[h][7] = a.kappa * hi.w;
        }
        const int s = (int)(it % NS);
        if (it >= NS) ok = mbar_wait_abort(&empty[s], (uint32_t)(((it - NS) / NS) & 1), abort);
        if (ok) {                                      // (a failed wait stops all producers at the loop top)
            unsigned char* As_ = smem + s * L::STAGE;
            unsigned char* Bs_ = As_ + P * L::TILE_A;
            store_group<P>(As_, L::TILE_A, p, 0, x);
            store_group<P>(As_, L::TILE_A, p, 1, x + 8);
#pragma unroll
            for (int h = 0; h < H; ++h) store_group<P>(Bs_, L::TILE_B, p + 128 * h, 2, sv[h]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
        }
    }
}

// the forward MMA pair of one tile into accumulator d
template <int P, int NTT>
__device__ __forceinline__ void issue_forward(uint32_t d, uint32_t As_, uint32_t idesc) {
    using L = Stages<P, NTT>;
    const uint32_t Bs_ = As_ + P * L::TILE_A;
    bool first = true;
    const uint64_t da = smem_desc_sw64(As_), db = smem_desc_sw64(Bs_);
    issue_kstep<P, L::TILE_A, L::TILE_B>(d, da, db, idesc, first);                         // X_f A_f
#pragma unroll
    for (int j = 0; j < P; ++j)                                                          // E S_j
        mma_bf16(d, desc_add(da, 32), desc_add(db, 32 + j * L::TILE_B), idesc, 1u);
}

}  // namespace

// ==========================================================================================
// Forward (fused with the integrand): 256 columns per tile, two TMEM accumulators of 256.
// Barriers: full (producers -> MMA, count 128), empty (MMA commit -> producers),
// accf (MMA commit -> epilogue), acce (epilogue -> MMA, count 256).
// ==========================================================================================
template <int P, int F>
__global__ void __launch_bounds__(THREADS, 1) k_fine_fwd_tc(const FineArgs<float> a, int ntn, long long units) {
    using L = Stages<P, NT_FWD>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::END);
    uint64_t* empty = full + 2;
    uint64_t* accf = full + 4;
    uint64_t* acce = full + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 8);
    volatile int* abort = reinterpret_cast<volatile int*>(full + 9);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = blockIdx.x % ntn;                 // this CTA's column tile
    const long long u0 = blockIdx.x / ntn, ustep = gridDim.x / ntn;
    const int t0 = nt * NT_FWD;
    const int ncols = min(NT_FWD, a.tau_pad - t0);
    const uint32_t nmma = (uint32_t)((ncols + 15) & ~15);
    const long long n_root = 1LL << a.logn_root;
    const int lmt = a.logn_root - 3;                  // log2 of the row tiles per shift

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
        producer_loop<P, NT_FWD, 2>(a, smem, full, empty, abort, tid - EPI_WARPS * 32, u0, ustep, units, t0, lmt);
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
                issue_forward<P, NT_FWD>(tmem + (uint32_t)(b * NT_FWD), smem_u32(smem + s * L::STAGE), idesc);
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
                    tmem_ld32(tmem + lane_base + (uint32_t)(b * NT_FWD + c_beg + c0),
                              *reinterpret_cast<uint32_t(*)[32]>(d));
                    if constexpr (CWD == 64)
                        tmem_ld32(tmem + lane_base + (uint32_t)(b * NT_FWD + c_beg + c0 + 32),
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

// ==========================================================================================
// Adjoint: 128 columns per tile, the recomputed product transposed and G kept in tensor memory.
// The forward pair is issued with the operands swapped, D^T[t][l] = [A_f ; S]^T W^T, so the
// accumulator's lanes are columns t and its columns are the tile's rows l.  The epilogue
// thread of lane t forms G[l][t] = coef_l h'(v_lt) for its rows, splits it into bf16 pieces
// and stores them back into the same tensor-memory buffer (piece p of row pair (2i, 2i+1)
// in column 64 p + i, low half the even row).  That buffer is the A operand of
//     D'[t][m] = sum_l G^T[t][l] [W_0 | W_1 | W_2][l][m]     (A from tensor memory, W MN-major),
// so G never passes through shared memory.
// TMEM: two buffers of 192 columns (y as FP32 in 0..127, then the P pieces of G in
// 64 p .. 64 p + 63) at 0 and 192, the backward accumulator (32 P columns) at 384.  In the
// split tier piece i of G multiplies W_0 .. W_{2-i} (N = 96, 64, 32): block j of the
// accumulator collects G_0 W_j + ... + G_{2-j} W_j, the six products with i + j <= 2.
// Barriers (phases per tile): full/empty (producer stages), accf[2] (forward product in
// buffer b), gready (G of the tile stored, count 512), bwdf (backward MMAs complete: the
// buffer's G consumed, the backward accumulator ready), bwde (accumulator drained, count 128).
// Roles: 16 epilogue warps form G; 4 drain warps (one per lane quarter) read the backward
// accumulator after bwdf, add the band gradient and store the root gradients, then arrive
// on bwde, which the next tile's backward MMAs wait for.  An epilogue thread signals gready
// of tile i only after gready of tile i-1 has completed (its next phase needs this thread),
// which keeps every phase count exact.  Buffer i & 1 last held G of tile i-2, consumed
// before the MMA thread issued the forward of tile i.
// ==========================================================================================
template <int P, int F>
__global__ void __launch_bounds__(THREADS_B, 1) k_fine_bwd_tc(const FineArgs<float> a, int ntn, long long units) {
    using L = Stages<P, NT_BWD, 3>;
    constexpr int NS = L::NSTAGE;
    constexpr uint32_t BUF = 192, BWD = 384;                            // TMEM columns
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = align_1k(smem_raw);
    float2* coefs = reinterpret_cast<float2*>(smem + L::END);            // [epilogue warp][32 rows]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::END + EPI_WARPS_B * 32 * sizeof(float2));
    uint64_t* empty = full + NS;
    uint64_t* accf = full + 2 * NS;
    uint64_t* gready = accf + 2;
    uint64_t* bwdf = accf + 3;
    uint64_t* bwde = accf + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 5);
    volatile int* abort = reinterpret_cast<volatile int*>(accf + 6);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = blockIdx.x % ntn;
    const long long u0 = blockIdx.x / ntn, ustep = gridDim.x / ntn;
    const long long ntiles = units > u0 ? (units - u0 + ustep - 1) / ustep : 0;   // tiles of this CTA
    const int t0 = nt * NT_BWD;
    const long long n_root = 1LL << a.logn_root;
    const int lmt = a.logn_root - 3;

    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 512);
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], PROD_WARPS * 32);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accf[0], 1); mbar_init(&accf[1], 1);
        mbar_init(gready, EPI_WARPS_B * 32);
        mbar_init(bwdf, 1);
        mbar_init(bwde, DRAIN_WARPS * 32);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    constexpr int PROD0 = EPI_WARPS_B + DRAIN_WARPS, MMAW = PROD0 + PROD_WARPS;
    if (warp >= PROD0 && warp < MMAW) {
        producer_loop<P, NT_BWD, NS>(a, smem, full, empty, abort, tid - PROD0 * 32, u0, ustep, units, t0, lmt);
    } else if (warp >= EPI_WARPS_B && warp < PROD0) {
        // ---------------------------------------------------------------- drain
        const int quarter = warp - EPI_WARPS_B;
        const int t = t0 + quarter * 32 + (tid & 31);
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + BWD;
        float gacc[15];
#pragma unroll
        for (int j = 0; j < 15; ++j) gacc[j] = 0.0f;
        for (long long it = 0; it < ntiles; ++it) {
            if (!__all_sync(0xffffffffu, mbar_wait_abort(bwdf, (uint32_t)(it & 1), abort))) break;
            fence_after_sync();
            uint32_t d[P][16], rr[8];
#pragma unroll
            for (int j = 0; j < P; ++j) tmem_ld16(ta + 32 * j, d[j]);
            tmem_ld8(ta + 16, rr);
            tmem_wait_ld();
            fence_before_sync();
            mbar_arrive(bwde);
#pragma unroll
            for (int m = 0; m < 15; ++m) {
                float v = 0.0f;
#pragma unroll
                for (int j = P - 1; j >= 0; --j) v += __uint_as_float(d[j][m]);     // small blocks first
                gacc[m] += v;
            }
            const long long u = u0 + it * ustep;
            const long long r = u >> lmt, rho0 = (u & ((1LL << lmt) - 1)) * kRootsPerTile;
            if (t < a.tau_pad) {
#pragma unroll
                for (int i = 0; i < 8; ++i) a.Froot[(r * n_root + rho0 + i) * a.tau_pad + t] = __uint_as_float(rr[i]);
            }
        }
        if (t < a.tau_pad) {
            // this CTA's partial of the band gradient: partial p = blockIdx.x / ntn
            float* out = a.gradpart + (long long)(blockIdx.x / ntn) * 15 * a.tau_pad + t;
#pragma unroll
            for (int j = 0; j < 15; ++j) out[(long long)j * a.tau_pad] = gacc[j];
        }
    } else if (warp == MMAW) {
        // ---------------------------------------------------------------- MMA issue
        if ((tid & 31) == 0) {
            const uint32_t idesc_f = idesc_bf16(TM);                      // D^T: M = t, N = l = 128
            uint32_t idesc_bwd[P];                                        // A in TMEM, B (W) MN-major
#pragma unroll
            for (int i = 0; i < P; ++i) idesc_bwd[i] = idesc_bf16(32u * (P - i)) | (1u << 16);
            auto forward = [&](long long it) -> bool {                    // D^T of tile it into buffer it & 1
                const int s = (int)(it % NS), b = (int)(it & 1);
                if (!mbar_wait_abort(&full[s], (uint32_t)((it / NS) & 1), abort)) return false;
                fence_after_sync();
                const uint32_t W = smem_u32(smem + s * L::STAGE);
                const uint32_t Bt = W + P * L::TILE_A;
                const uint32_t d = tmem + (uint32_t)(b * BUF);
                bool first = true;
                const uint64_t dbt = smem_desc_sw64(Bt), dw = smem_desc_sw64(W);
                issue_kstep<P, L::TILE_B, L::TILE_A>(d, dbt, dw, idesc_f, first);       // A_f^T X_f^T
#pragma unroll
                for (int j = 0; j < P; ++j)                                             // S_j^T E^T
                    mma_bf16(d, desc_add(dbt, 32 + j * L::TILE_B), desc_add(dw, 32), idesc_f, 1u);
                mma_commit(smem_u32(&accf[b]));
                return true;
            };
            if (ntiles > 0 && forward(0)) {
                for (long long it = 0; it < ntiles; ++it) {
                    if (it + 1 < ntiles) {
                        // buffer (it + 1) & 1 held G of tile it - 1: its backward MMAs must be done
                        if (it >= 1 && !mbar_wait_abort(bwdf, (uint32_t)((it - 1) & 1), abort)) break;
                        if (!forward(it + 1)) break;
                    }
                    const int s = (int)(it % NS), b = (int)(it & 1);
                    if (!mbar_wait_abort(gready, (uint32_t)(it & 1), abort)) break;
                    // the drain warps have read the backward accumulator of tile it - 1
                    if (it >= 1 && !mbar_wait_abort(bwde, (uint32_t)((it - 1) & 1), abort)) break;
                    fence_after_sync();
                    // D' = G^T [W_0 | W_1 | W_2]: 8 K-steps of 16 rows; piece i of G multiplies the
                    // pieces W_0 .. W_{P-1-i} (N = 32 (P - i)), the six products with i + j <= 2
                    const uint64_t dw = smem_desc_sw64_mn(smem_u32(smem + s * L::STAGE), L::TILE_A, 512);
                    const uint32_t gbuf = tmem + (uint32_t)(b * BUF);
#pragma unroll
                    for (int ks = 0; ks < TM / 16; ++ks) {
#pragma unroll
                        for (int i = 0; i < P; ++i)
                            mma_bf16_tmem_a(tmem + BWD, gbuf + 64u * i + 8u * ks, desc_add(dw, ks * 1024),
                                            idesc_bwd[i], (ks == 0 && i == 0) ? 0u : 1u);
                    }
                    mma_commit(smem_u32(bwdf));
                    mma_commit(smem_u32(&empty[s]));
                }
            }
        }
    } else if (warp < EPI_WARPS_B) {
        // ---------------------------------------------------------------- epilogue
        // warp w: lanes 32 (w % 4) + i = columns t0 + 32 (w % 4) + i, rows l = 32 (w / 4) .. + 31
        const int quarter = warp & 3, rq = warp >> 2;
        const int lt = quarter * 32 + (tid & 31);         // column of the tile = TMEM lane
        const int t = t0 + lt;
        const int lane = tid & 31;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const float upstream = (float)a.upstream[0];
        float2* wcoef = coefs + warp * 32;
        // the saved {g'(u) gfac / (R N), log2 e u} of row l = 32 rq + lane of tile jt
        auto row_coef = [&](long long jt) {
            const long long u = u0 + jt * ustep;
            const long long r = u >> lmt, rho0 = (u & ((1LL << lmt) - 1)) * kRootsPerTile;
            const int l = rq * 32 + lane;
            const long long k = rho0 + (l >> 4) + (long long)(l & 15) * n_root;
            return __ldg(reinterpret_cast<const float2*>(a.rowsave) + r * a.N + k);
        };
        float2 coef_next = ntiles > 0 ? row_coef(0) : make_float2(0.f, 0.f);
        bool ok = true;
        for (long long it = 0; it < ntiles; ++it) {
            const int b = (int)(it & 1);
            const float2 coef_mine = coef_next;
            if (it + 1 < ntiles) coef_next = row_coef(it + 1);
            // the waits' outcome is made uniform over the warp (for the aligned tensor-memory
            // accesses) and over the lane quarter (for its named barrier) before anything depends on it
            bool okl = mbar_wait_abort(&accf[b], (uint32_t)((it >> 1) & 1), abort);
            okl = __all_sync(0xffffffffu, okl);
            const uint32_t ybuf = tmem + lane_base + (uint32_t)(b * BUF);
            uint32_t y[32];
            if (okl) {
                fence_after_sync();
                __syncwarp();
                wcoef[lane] = make_float2(upstream * coef_mine.x, coef_mine.y);
                tmem_ld32(ybuf + 32 * rq, y);
                tmem_wait_ld();
                __syncwarp();
            }
            // every warp of this lane quarter has read its y before any G piece overwrites them
            if (quarter_sync_or(quarter, !okl)) { ok = false; break; }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[P][8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float g2[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int c = 16 * h + 2 * i + e;                // row l = 32 rq + c
                        const float2 cf = wcoef[c];
                        g2[e] = t < a.tau ? cf.x * Fn<F, float>::hp(__uint_as_float(y[c]), a.c0, cf.y) : 0.0f;
                    }
                    uint32_t qp[P];
                    split_pair<P>(g2[0], g2[1], qp);
#pragma unroll
                    for (int pp = 0; pp < P; ++pp) w[pp][i] = qp[pp];
                }
#pragma unroll
                for (int pp = 0; pp < P; ++pp) tmem_st8(ybuf + 64u * pp + 16u * rq + 8u * h, w[pp]);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before_sync();
            if (it >= 1 && !mbar_wait_abort(gready, (uint32_t)((it - 1) & 1), abort)) { ok = false; break; }
            mbar_arrive(gready);
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
// launchers: one CTA per SM (all 512 TMEM columns), CTAs spread evenly over the column tiles
// ------------------------------------------------------------------------------------------
namespace {
// The persistent grids are sized for the 152 SMs of a GB300 (also the workspace's count of
// gradient partials, so it may not depend on the device the plan is made on).
constexpr int kGridSMs = 152;
int sm_count() { return kGridSMs; }

size_t at_least_120k(size_t b) { return b < 120 * 1024 ? 120 * 1024 : b; }

template <int P, int F>
cudaError_t fwd_tc_launch(const FineArgs<float>& a, cudaStream_t st) {
    const int ntn = (a.tau_pad + NT_FWD - 1) / NT_FWD;
    const long long units = (long long)a.reff * ((1LL << a.logn_root) / kRootsPerTile);
    const long long per = std::min<long long>(std::max(1, sm_count() / ntn), units);
    const size_t smem = at_least_120k(1024 + Stages<P, NT_FWD>::END + 128);
    cudaError_t e = cudaFuncSetAttribute(k_fine_fwd_tc<P, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fine_fwd_tc<P, F><<<(unsigned)(per * ntn), THREADS, smem, st>>>(a, ntn, units);
    return cudaGetLastError();
}

template <int P, int F>
cudaError_t bwd_tc_launch(const FineArgs<float>& a, cudaStream_t st) {
    const int ntn = (a.tau_pad + NT_BWD - 1) / NT_BWD;
    const long long units = (long long)a.reff * ((1LL << a.logn_root) / kRootsPerTile);
    const long long per = bwd_tc_partials(a.tau_pad, a.reff, a.logn_root);
    const size_t smem = at_least_120k(1024 + Stages<P, NT_BWD, 3>::END + EPI_WARPS_B * 32 * sizeof(float2) + 128);
    cudaError_t e = cudaFuncSetAttribute(k_fine_bwd_tc<P, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fine_bwd_tc<P, F><<<(unsigned)(per * ntn), THREADS_B, smem, st>>>(a, ntn, units);
    return cudaGetLastError();
}

template <int P, bool FWD>
cudaError_t tc_f(const FineArgs<float>& a, int F, cudaStream_t st) {
    switch (F) {
#define QMC_FINE_TC_CASE(FK) \
        case FK: return FWD ? fwd_tc_launch<P, FK>(a, st) : bwd_tc_launch<P, FK>(a, st);
        QMC_FINE_TC_CASE(F_LINEAR_MEAN)
        QMC_FINE_TC_CASE(F_MEAN_COS)
        QMC_FINE_TC_CASE(F_CALL_MEAN_EXP)
        QMC_FINE_TC_CASE(F_GAUSS_NORM2)
        QMC_FINE_TC_CASE(F_PDE_INV_SQ)
        QMC_FINE_TC_CASE(F_LOGSUMEXP)
#undef QMC_FINE_TC_CASE
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int fine_tc_group_cols() { return 128; }

// partials of the band gradient written by the adjoint kernel (CTAs per column tile)
long long bwd_tc_partials(int tau_pad, int reff, int logn_root) {
    const int ntn = (tau_pad + NT_BWD - 1) / NT_BWD;
    const long long units = (long long)reff * ((1LL << logn_root) / kRootsPerTile);
    return std::min<long long>(std::max(1, sm_count() / ntn), units);
}

cudaError_t launch_fine_fwd_tc(const FineArgs<float>& a, int F, int pieces, cudaStream_t st) {
    if (a.logn_root < 3) return cudaErrorInvalidValue;        // 8 roots per tile
    if (pieces == 3) return tc_f<3, true>(a, F, st);
    if (pieces == 1) return tc_f<1, true>(a, F, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fine_bwd_tc(const FineArgs<float>& a, int F, int pieces, cudaStream_t st) {
    if (a.logn_root < 3) return cudaErrorInvalidValue;
    if (pieces == 3) return tc_f<3, false>(a, F, st);
    if (pieces == 1) return tc_f<1, false>(a, F, st);
    return cudaErrorInvalidValue;
}

cudaError_t fine_tc_error_word(unsigned int* value, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(value, g_fine_tc_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_fine_tc_error, &zero, sizeof(unsigned int));
}

}  // namespace qmc
