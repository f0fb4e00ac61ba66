// Fine band S4 in FP32 on the CUDA cores: the levels w = 0..3 (at most 1, 2, 4 and 8 columns)
// expanded as the binary tree of Sec. 3.2, fused with the integrand (forward) or with the
// folded adjoint (backward).
//
// Notation as in qmc_fine.cuh: a root rho < n_root = 2^(m-4) of level 4 has the descendants
// rho + c n_root at level I (c < 2^(4-I)); node c at level I has the children c and c + 2^(4-I)
// at level I - 1, and leaf q is the output row k = rho + q n_root.  A root costs 64 multiply-
// adds per column for its 16 outputs (Algorithm 1's count for these levels: sum_I 2^(4-I) tau_I),
// 4 per output, against the 15 + 1 a dense row would take.  That is why the band stays on the
// FP32 pipes in every float tier: a tensor-core tile of the band multiplies 16 padded columns
// plus the root per output, six times over in the three-piece split, and its adjoint is bounded
// by the tensor pipe well above the 11 FP32 operations per output the tree takes here.
//
// Forward: a thread owns the 8 leaves q = b + 2i under level-3 node b of a root (the tree
// splits there without shared work) for NB = 1 (a CTA of 64 roots x 2 branches), or both nodes'
// 16 leaves for NB = 2 (a CTA of 128 roots); it keeps their x values in registers (as pairs of
// sibling nodes) and walks the CTA's columns; the kappa-scaled fine columns of A are staged in
// shared memory and read as six broadcast 16-byte loads per column, which serve NB subtrees, and
// the paired FP32 instructions (FFMA2, FADD2) take two siblings per instruction.
//
// Backward: a CTA covers 256 columns (4 warps x 32 lanes x 2 columns) of a range of roots, in
// two halves of 4 warps that take alternate roots.  The x values and row coefficients of 8 roots
// at a time are staged in shared memory (double-buffered, coalesced along the roots, each value
// stored twice) and read as broadcast 16-byte loads; each lane holds its two columns of A and its
// gradient accumulators in registers for every root it visits, the paired FP32 instructions
// taking both columns at once, so the only reductions are the two halves' at the end.
#include "qmc_internal.cuh"

namespace qmc {
namespace {

constexpr int kFwdThreads = 128;
// forward roots per CTA with NB level-3 nodes per thread (NB = 1: a thread per node, two per root;
// NB = 2: a thread per root, both nodes, half the loads of A per operation and twice the
// independent work per thread, with more registers)
__host__ __device__ constexpr int fwd_roots(int NB) { return kFwdThreads * NB / 2; }
constexpr int kBwdThreads = 256;
constexpr int kBwdCols = 256;                // columns per CTA: 4 warps x 32 lanes x 2
constexpr int kRB = 8;                       // roots per staged batch (materialised product)
constexpr int kBRB = 16;                     // roots per staged batch (adjoint: fewer barriers than 8,
                                             // 7.52 -> 7.33 ms on the 2^20-point step)
constexpr int kSlots = 96;                   // staged floats per root
// forward CTAs resident per SM: 7 (72 registers) where the integrand's h fits without spilling,
// else 5 (cos, the inverse square's reciprocal and log-sum-exp's running maximum need more)
__host__ __device__ constexpr int fwd_min_blocks(int F, int NB) {
    return NB == 1 ? ((F == F_LINEAR_MEAN || F == F_CALL_MEAN_EXP || F == F_GAUSS_NORM2) ? 7 : 5)
                   : ((F == F_LINEAR_MEAN || F == F_CALL_MEAN_EXP || F == F_GAUSS_NORM2) ? 4 : 3);
}
constexpr int kMaxCRS4 = 512;                // forward columns per CTA (dynamic shared memory 56 KB with
                                             // the root-value ring: 4 CTAs fill an SM's 228 KB)

// ------------------------------------------------------------------------------------------
// Forward
// ------------------------------------------------------------------------------------------

// Shared-memory layout of the staged fine columns of A, 24 floats per column:
//   [a3 0..7 | a2 0, a2 0, a2 1, a2 1, a2 2, a2 2, a2 3, a2 3 | a1 0, a1 0, a1 1, a1 1 | a0, a0, 0, 0]
// The paired FP32 instructions (two lanes of one register pair per instruction) then take their
// operands straight from the 16-byte loads: the level-3 dot product runs as two interleaved
// partial sums over (a3 2k, a3 2k+1), and the two sibling nodes of each lower level share an a.
constexpr int kAQuads = 6;

// The forward's root values S_4 pass through a ring of kSRing slots of 16 bytes per thread in
// shared memory, copied kSDist quads of columns ahead of their use
constexpr int kSDist = 3;
constexpr int kSRing = kSDist + 1;           // the slot refilled is the one read a quad earlier
__host__ __device__ constexpr size_t fwd_smem_bytes(int cr) {
    return (size_t)cr * kAQuads * 16 + (size_t)kSRing * kFwdThreads * 16;
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// 16-byte asynchronous copy global -> shared (zero-filled when !valid; src must still be a
// valid address), and the per-thread copy groups
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Row accumulator of u = sum_t h(v_t); log-sum-exp keeps (max, sum 2^(v - max)) and takes one
// ex2 per output: with d = v - max, 2^-|d| is either the new term (d <= 0) or the rescale of
// the old sum when v becomes the maximum (d > 0, new term 2^0 = 1).
template <int F>
struct RowAcc {
    float s, mx;
    __device__ __forceinline__ void init() { s = 0.0f; mx = -INFINITY; }
    __device__ __forceinline__ void add(float v, float c0) {
        if constexpr (F == F_LOGSUMEXP) {
            const float d = v - mx;
            const float e = ex2f(-fabsf(d));
            const bool up = d > 0.0f;
            s = up ? fmaf(s, e, 1.0f) : s + e;
            mx = up ? v : mx;
        } else {
            s += Fn<F, float>::h(v, c0);
        }
    }
};

// The row accumulators of two sibling leaves; the row-sum integrands add their two terms with
// one paired add.
template <int F>
struct RowAcc2 {
    float2 s, mx;
    __device__ __forceinline__ void init() { s = f2(0.0f, 0.0f); mx = f2(-INFINITY, -INFINITY); }
    __device__ __forceinline__ void add(float2 v, float c0) {
        if constexpr (F == F_LOGSUMEXP) {
            RowAcc<F> a{s.x, mx.x}, b{s.y, mx.y};
            a.add(v.x, c0);
            b.add(v.y, c0);
            s = f2(a.s, b.s);
            mx = f2(a.mx, b.mx);
        } else if constexpr (F == F_GAUSS_NORM2) {
            s = __ffma2_rn(v, v, s);                  // h(v) = v^2 and the row sum in one paired FMA
        } else if constexpr (F == F_LINEAR_MEAN) {
            s = __fadd2_rn(s, v);
        } else {
            s = __fadd2_rn(s, f2(Fn<F, float>::h(v.x, c0), Fn<F, float>::h(v.y, c0)));
        }
    }
};

template <int F, int NB>
__global__ void __launch_bounds__(kFwdThreads, fwd_min_blocks(F, NB)) k_fine_fwd_s4(const __grid_constant__ FineArgs<float> a) {
    constexpr int kNB = NB;
    constexpr int kFwdRoots = fwd_roots(NB);
    extern __shared__ __align__(16) float4 As_dyn[];        // [a.cr][kAQuads], then [kSRing][threads]
    float4 (*As)[kAQuads] = reinterpret_cast<float4 (*)[kAQuads]>(As_dyn);
    float4* ring = As_dyn + (size_t)a.cr * kAQuads;
    const int tid = threadIdx.x;
    // thread: root rho and its level-3 nodes b0 .. b0 + kNB - 1
    const int b0 = kNB == 2 ? 0 : tid / kFwdRoots;
    const long long n_root = 1LL << a.logn_root;
    const long long rho = (long long)blockIdx.x * kFwdRoots + (kNB == 2 ? tid : tid % kFwdRoots);
    const int cg = blockIdx.y, r = blockIdx.z;
    const int t_beg = cg * a.cr, t_end = min(t_beg + a.cr, a.tau);
    const int ncol = (t_end - t_beg + 3) & ~3;

    // x of each subtree (level-3 node b, level-2 nodes b + 2 i2, level-1 nodes b + 2 i1, leaves
    // b + 2 i), as register pairs: the level-3 columns (2k, 2k+1), and for the lower levels the
    // sibling nodes (i2 = 0, 1), (i1 = 0, 1), (i1 = 2, 3), (i = 2k, 2k+1)
    // (the loads of x and of the first root values are issued before the staging of A, so that
    // their latency overlaps it)
    const bool valid = rho < n_root;
    const long long step2 = 2LL << a.logn_root;                  // from node c to node c + 2
    float2 x3p[kNB][4], x2p[kNB][4], x1p[kNB][2][2], x0p[kNB][4];
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb) {
        const int b = b0 + nb;
        const float* tab = a.tab + (long long)r * a.tab_stride + (valid ? rho : 0) + ((long long)b << a.logn_root);
        const float* p3 = tab + a.lev_tab[3];
        float x3[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) x3[jj] = jj < a.lev_tau[3] ? __ldg(p3 + ((long long)jj << a.lev_logn[3])) : 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) x3p[nb][k] = f2(x3[2 * k], x3[2 * k + 1]);
        const float* p2 = tab + a.lev_tab[2];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const bool on = jj < a.lev_tau[2];
            const float* q = p2 + ((long long)jj << a.lev_logn[2]);
            x2p[nb][jj] = on ? f2(__ldg(q), __ldg(q + step2)) : f2(0.0f, 0.0f);
        }
        const float* p1 = tab + a.lev_tab[1];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const bool on = jj < a.lev_tau[1];
            const float* q = p1 + ((long long)jj << a.lev_logn[1]);
#pragma unroll
            for (int p = 0; p < 2; ++p)
                x1p[nb][p][jj] = on ? f2(__ldg(q + (2 * p) * step2), __ldg(q + (2 * p + 1) * step2)) : f2(0.0f, 0.0f);
        }
        const float* p0 = tab + a.lev_tab[0];
        const bool on0 = a.lev_tau[0] > 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            x0p[nb][k] = on0 ? f2(__ldg(p0 + (2 * k) * step2), __ldg(p0 + (2 * k + 1) * step2)) : f2(0.0f, 0.0f);
    }

    RowAcc2<F> acc[kNB][4];                               // leaves (2k, 2k+1) of each subtree
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[nb][k].init();
    const float kap = a.kappa, c0 = a.c0;
    // one column: every subtree's 8 outputs and their row accumulators
    auto column = [&](const float4* ac, float vroot) {
        const float4 A0 = ac[0], A1 = ac[1], A2 = ac[2], A3 = ac[3], A4 = ac[4], A5 = ac[5];
#pragma unroll
        for (int nb = 0; nb < kNB; ++nb) {
            // (the root value joins the scalar sum: a {vroot, 0} pair cost register moves on every
            // column, 3.25 -> 3.17 ms on the 2^20-point step)
            float2 s3 = __fmul2_rn(x3p[nb][0], f2(A0.x, A0.y));
            s3 = ffma2(x3p[nb][1], f2(A0.z, A0.w), s3);
            s3 = ffma2(x3p[nb][2], f2(A1.x, A1.y), s3);
            s3 = ffma2(x3p[nb][3], f2(A1.z, A1.w), s3);
            const float v3 = (s3.x + vroot) + s3.y;
            float2 v2 = ffma2(x2p[nb][0], f2(A2.x, A2.y), f2(v3, v3));        // level-2 nodes i2 = 0, 1
            v2 = ffma2(x2p[nb][1], f2(A2.z, A2.w), v2);
            v2 = ffma2(x2p[nb][2], f2(A3.x, A3.y), v2);
            v2 = ffma2(x2p[nb][3], f2(A3.z, A3.w), v2);
            // level-1 nodes (0, 1) and (2, 3): parents (0, 1), i.e. v2 itself
            const float2 v1a = ffma2(x1p[nb][0][1], f2(A4.z, A4.w), ffma2(x1p[nb][0][0], f2(A4.x, A4.y), v2));
            const float2 v1b = ffma2(x1p[nb][1][1], f2(A4.z, A4.w), ffma2(x1p[nb][1][0], f2(A4.x, A4.y), v2));
            // leaves (0, 1), (4, 5) below (0, 1) and (2, 3), (6, 7) below (2, 3)
            const float2 a0 = f2(A5.x, A5.y);
            acc[nb][0].add(ffma2(x0p[nb][0], a0, v1a), c0);
            acc[nb][1].add(ffma2(x0p[nb][1], a0, v1b), c0);
            acc[nb][2].add(ffma2(x0p[nb][2], a0, v1a), c0);
            acc[nb][3].add(ffma2(x0p[nb][3], a0, v1b), c0);
        }
    };
    // root values S_4 (layout [t/4][rho][4]): quad q of the group (columns t_beg + 4q ..) into ring
    // slot q % kSRing, kSDist quads ahead (no registers held by the copies in flight; register loads
    // two quads ahead left 10% of the kernel's time waiting on them), zeros without root values
    const float* S = (a.S && valid) ? a.S + (long long)r * a.S_stride + rho * 4 : nullptr;
    const long long squad = 4LL << a.logn_root;
    auto issue_s = [&](int q) {
        const int t = t_beg + 4 * q;
        const bool on = S && t < t_end;
        cp_async16((uint32_t)__cvta_generic_to_shared(ring + (q % kSRing) * kFwdThreads + tid),
                   on ? S + (long long)(t >> 2) * squad : a.tab, on);
        cp_async_commit();                                    // (one group per quad, possibly empty)
    };
#pragma unroll
    for (int q = 0; q < kSDist; ++q) issue_s(q);
    {
        // threads tid < 120 stage position jp = tid % 24 of the columns tid / 24, tid / 24 + 5, ...
        constexpr int W = 4 * kAQuads, STEP = kFwdThreads / W;
        const int jp = tid % W;
        int lev = 0, jj = 0;
        bool on = tid < STEP * W;
        if (jp < 8) { lev = 3; jj = jp; }
        else if (jp < 16) { lev = 2; jj = (jp - 8) >> 1; }
        else if (jp < 20) { lev = 1; jj = (jp - 16) >> 1; }
        else if (jp < 22) { lev = 0; jj = 0; }
        else on = false;
        on = on && jj < a.lev_tau[lev];
        const float* arow = a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA;
        float* Asf = reinterpret_cast<float*>(As);
        if (tid < STEP * W)
            for (int c = tid / W; c < ncol; c += STEP)
                Asf[c * W + jp] = (on && t_beg + c < a.tau) ? a.kappa * __ldg(arow + t_beg + c) : 0.0f;
    }
    __syncthreads();
    const int nfull = (t_end - t_beg) >> 2;
    int q = 0;
    for (; valid && q < nfull; ++q) {                     // whole quads: four independent columns
        cp_async_wait<kSDist - 1>();                      // this thread's copy of quad q has landed
        const float4 sq = ring[(q % kSRing) * kFwdThreads + tid];
        issue_s(q + kSDist);
        const float4* ac = As[4 * q];
        column(ac, kap * sq.x);
        column(ac + kAQuads, kap * sq.y);
        asm volatile("" ::: "memory");                 // (caps the columns' loads held at once)
        column(ac + 2 * kAQuads, kap * sq.z);
        column(ac + 3 * kAQuads, kap * sq.w);
    }
    if (valid && t_beg + 4 * q < t_end) {                 // the ragged last quad
        cp_async_wait<kSDist - 1>();
        const float4 sq = ring[(q % kSRing) * kFwdThreads + tid];
        const float sv[4] = {sq.x, sq.y, sq.z, sq.w};
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (t_beg + 4 * q + c < t_end) column(As[4 * q + c], kap * sv[c]);
    }
    cp_async_wait<0>();                                   // (no copy outlives the CTA)

    // row partials of this column group: rowpart[r][cg][k] (log-sum-exp: also rowmax)
    if (valid) {
#pragma unroll
        for (int nb = 0; nb < kNB; ++nb)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const long long o = ((long long)r * gridDim.y + cg) * a.N + rho + ((long long)(b0 + nb + 2 * i) << a.logn_root);
                a.rowpart[o] = (i & 1) ? acc[nb][i >> 1].s.y : acc[nb][i >> 1].s.x;
                if constexpr (F == F_LOGSUMEXP) a.rowmax[o] = (i & 1) ? acc[nb][i >> 1].mx.y : acc[nb][i >> 1].mx.x;
            }
    }
}

// ------------------------------------------------------------------------------------------
// Backward
// ------------------------------------------------------------------------------------------

// Staged values of one root, each stored twice ({v, v}, one register pair for the paired
// instructions over the thread's two columns), in slot order:
//   slots  0..15   x of the level-3 nodes (c3 = 0: columns 0..7, c3 = 1: columns 0..7)
//   slots 16..31   x of the level-2 nodes c2 = 0..3 (columns 0..3)
//   slots 32..63   per level-1 node c1: x columns 0, 1 and the x of its leaves c1, c1 + 8
//   slots 64..79   per level-2 node c2: coefficients of the leaves c2, c2 + 8, c2 + 4, c2 + 12
//   slots 80..95   the same leaves' -aux (log-sum-exp only)
// A root's row is kRowPad floats long: consecutive roots of a batch then start 16 bytes apart
// modulo 128, so that the staging stores of 8 roots hit distinct banks, and the reads are
// 16-byte aligned at fixed offsets.
constexpr int kRowPad = 2 * kSlots + 4;

// Where slot s of every root comes from, as a 32-bit code: bit 31 set for no value (0), else
// bit 30 for the row coefficients (rowsave, float offset code & 0x3fffffff + 2 rho; the aux
// slots read the second float of the pair and are negated) or the point table (tab, offset
// code + rho).  Offsets are within one shift's table or one shift's rowsave.
template <int F>
__device__ __forceinline__ unsigned bwd_slot_code(const FineArgs<float>& a, int s) {
    int lev, c, jj;
    if (s < 16) { lev = 3; c = s >> 3; jj = s & 7; }
    else if (s < 32) { lev = 2; c = (s - 16) >> 2; jj = s & 3; }
    else if (s < 64) {
        const int u = s - 32, e = u & 3;
        c = u >> 2;
        if (e < 2) { lev = 1; jj = e; } else { lev = 0; jj = 0; c += (e - 2) * 8; }
    } else {
        if (F != F_LOGSUMEXP && s >= 80) return 1u << 31;
        const int u = (s - 64) & 15, c2 = u >> 2, e = u & 3;
        const int q = c2 + ((e & 1) ? 8 : 0) + ((e & 2) ? 4 : 0);
        return (1u << 30) | (unsigned)(2 * ((long long)q << a.logn_root) + (s < 80 ? 0 : 1));
    }
    if (jj >= a.lev_tau[lev]) return 1u << 31;
    return (unsigned)(a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + ((long long)c << a.logn_root));
}

// h'(v) / gfac for the two columns of a lane (log-sum-exp: nax = -aux)
template <int F>
__device__ __forceinline__ float2 hp2(float2 v, float c0, float2 nax) {
    if constexpr (F == F_LOGSUMEXP) {
        const float2 w = __fadd2_rn(v, nax);
        return f2(ex2f(w.x), ex2f(w.y));
    } else if constexpr (F == F_GAUSS_NORM2) {
        return v;                                    // h' = 2 v: the 2 is in the staged row coefficient
    } else {
        return f2(Fn<F, float>::hp(v.x, c0, 0.0f), Fn<F, float>::hp(v.y, c0, 0.0f));
    }
}

// Dynamic shared memory of the adjoint: the double-buffered staging of kBRB roots, reused after
// the last batch for the reduction of the two root halves' gradients (15 rows of 256 CPL columns)
__host__ __device__ constexpr size_t bwd_smem_bytes(int cpl) {
    return sizeof(float) * 2 * kBRB * kRowPad > sizeof(float2) * 15 * (kBwdCols * cpl / 2)
               ? sizeof(float) * 2 * kBRB * kRowPad
               : sizeof(float2) * 15 * (kBwdCols * cpl / 2);
}

// CPL column pairs per lane: a CTA covers 256 CPL columns; a lane's pair p holds columns
// pass * 256 CPL + 256 p + 2 colw, +1.  With CPL = 2 every broadcast load of a root's staged x
// values feeds twice the FP32 work, at one CTA of 8 warps per SM instead of two.
template <int F, int CPL>
__global__ void __launch_bounds__(kBwdThreads, CPL == 1 ? 2 : 1) k_fine_bwd_s4(const __grid_constant__ FineArgs<float> a) {
    constexpr int kCols = kBwdCols * CPL;
    // the staging buffers and, after the last batch's barrier, the halves' reduction share the
    // dynamic shared memory (bwd_smem_bytes)
    extern __shared__ __align__(16) unsigned char bwd_dyn[];
    float (*xs)[kBRB][kRowPad] = reinterpret_cast<float (*)[kBRB][kRowPad]>(bwd_dyn);
    float2 (*red)[kCols / 2] = reinterpret_cast<float2 (*)[kCols / 2]>(bwd_dyn);
    __shared__ unsigned codes[kSlots];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int half = warp >> 2, colw = (warp & 3) * 32 + lane;   // column pair of this lane
    const int grp = blockIdx.x, pass = blockIdx.y, r = blockIdx.z;
    const long long n_root = 1LL << a.logn_root;
    int t[CPL];
    bool active[CPL];
#pragma unroll
    for (int p = 0; p < CPL; ++p) {
        t[p] = pass * kCols + kBwdCols * p + 2 * colw;
        active[p] = t[p] < a.tau_pad;                          // then t + 1 < tau_pad too
    }
    const float* tab = a.tab + (long long)r * a.tab_stride;
    const float upstream = (float)a.upstream[0];
    // the row coefficients are staged times upstream (and times 2 for the Gaussian norm, whose
    // h'(v) = 2 v then costs one multiply with the coefficient)
    const float coef_scale = F == F_GAUSS_NORM2 ? 2.0f * upstream : upstream;
    const float kap = a.kappa, c0 = a.c0;

    // kappa * A of the thread's columns and the band-gradient accumulators, as column pairs
    float2 ah3[CPL][8], ah2[CPL][4], ah1[CPL][2], ah0[CPL];
    float2 g3[CPL][8], g2[CPL][4], g1[CPL][2], g0[CPL];
    auto lda = [&](int p, int lev, int jj) -> float2 {
        if (!active[p] || jj >= a.lev_tau[lev]) return f2(0.0f, 0.0f);
        const float* q = a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA + t[p];
        return f2(kap * __ldg(q), kap * __ldg(q + 1));
    };
#pragma unroll
    for (int p = 0; p < CPL; ++p) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) { ah3[p][jj] = lda(p, 3, jj); g3[p][jj] = f2(0.0f, 0.0f); }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) { ah2[p][jj] = lda(p, 2, jj); g2[p][jj] = f2(0.0f, 0.0f); }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) { ah1[p][jj] = lda(p, 1, jj); g1[p][jj] = f2(0.0f, 0.0f); }
        ah0[p] = lda(p, 0, 0);
        g0[p] = f2(0.0f, 0.0f);
    }

    const long long rho_beg = (long long)grp * a.roots_per_cta;
    const long long rho_end = min(rho_beg + (long long)a.roots_per_cta, n_root);
    const int nb = rho_end > rho_beg ? (int)((rho_end - rho_beg + kBRB - 1) / kBRB) : 0;
    // staging: thread tid fills slots tid / kBRB + (256 / kBRB) u of batch root tid % kBRB
    constexpr int PER = kBRB * kSlots / kBwdThreads;
    constexpr int SST = kBwdThreads / kBRB;
    const int jst = tid % kBRB;
    const float* rsave = a.rowsave + 2 * (long long)r * a.N;
    if (tid < kSlots) codes[tid] = bwd_slot_code<F>(a, tid);    // (read after the first barrier)
    float pre[PER];
    auto fetch = [&](long long rb0) {
        const long long rho = rb0 + jst;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const unsigned code = codes[tid / kBRB + SST * u];
            float v = 0.0f;
            if (!(code >> 31) && rho < rho_end) {
                if (code >> 30) {
                    v = __ldg(rsave + (code & 0x3fffffffu) + 2 * rho);
                    v = (code & 1u) ? -v : coef_scale * v;
                } else {
                    v = __ldg(tab + code + rho);
                }
            }
            pre[u] = v;
        }
    };
    auto put = [&](int buf) {
#pragma unroll
        for (int u = 0; u < PER; ++u)
            *reinterpret_cast<float2*>(&xs[buf][jst][2 * (tid / kBRB + SST * u)]) = f2(pre[u], pre[u]);
    };
    // root values S_4 (layout [t/4][rho][4]) of the thread's columns, and its root-gradient columns:
    // row-major [rho][tau_pad], or 128-column tiles [t / 128][rho][128] (then a 32-row TMA box of
    // one tile is contiguous for the fused fold-gradient kernel)
    const float* Sb[CPL];
    float* Fb[CPL];
#pragma unroll
    for (int p = 0; p < CPL; ++p) {
        Sb[p] = (a.S && active[p])
                    ? a.S + (long long)r * a.S_stride + ((long long)(t[p] >> 2) << a.logn_root) * 4 + (t[p] & 3)
                    : nullptr;
        Fb[p] = a.froot_tiled
                    ? a.Froot + (long long)r * a.froot_stride + (((long long)(t[p] >> 7) << a.logn_root) << 7) + (t[p] & 127)
                    : a.Froot + (long long)r * n_root * a.tau_pad + t[p];
    }
    const long long frow = a.froot_tiled ? 128 : a.tau_pad;
    auto lds2 = [&](int p, long long rho) -> float2 {
        return Sb[p] ? __ldg(reinterpret_cast<const float2*>(Sb[p] + rho * 4)) : make_float2(0.0f, 0.0f);
    };

    __syncthreads();                                            // the slot codes
    if (nb > 0) { fetch(rho_beg); put(0); }
    __syncthreads();
    float2 snext[CPL];
#pragma unroll
    for (int p = 0; p < CPL; ++p) snext[p] = rho_beg + half < rho_end ? lds2(p, rho_beg + half) : make_float2(0.0f, 0.0f);
    for (int kb = 0; kb < nb; ++kb) {
        const long long rb0 = rho_beg + (long long)kb * kBRB;
        if (kb + 1 < nb) fetch(rb0 + kBRB);                       // in flight during this batch
        for (int j = half; j < kBRB; j += 2) {
            const long long rho = rb0 + j;
            if (rho >= rho_end) break;
            float2 sr[CPL];
#pragma unroll
            for (int p = 0; p < CPL; ++p) {
                sr[p] = snext[p];
                if (rho + 2 < rho_end) snext[p] = lds2(p, rho + 2);
            }
            const float* xr = xs[kb & 1][j];
            // slots 2g and 2g + 1, each a {v, v} pair
            // (the gradients F of a node's children are summed without a zero start)
            auto pairs = [&](int g, float2& p0, float2& p1) {
                const float4 q = *reinterpret_cast<const float4*>(xr + 4 * g);
                p0 = f2(q.x, q.y);
                p1 = f2(q.z, q.w);
            };
            float2 Fr[CPL];
#pragma unroll
            for (int c3 = 0; c3 < 2; ++c3) {
                // (x of the level-3 and level-2 nodes is read again for the gradient updates
                // instead of being held in registers across the subtree)
                // (two interleaved partial sums shorten the dependent chain)
                float2 v3[CPL], w3[CPL], F3[CPL];
#pragma unroll
                for (int p = 0; p < CPL; ++p) {
                    v3[p] = f2(kap * sr[p].x, kap * sr[p].y);
                    w3[p] = f2(0.0f, 0.0f);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 xa, xb;
                    pairs(4 * c3 + k, xa, xb);
#pragma unroll
                    for (int p = 0; p < CPL; ++p) {
                        v3[p] = ffma2(xa, ah3[p][2 * k], v3[p]);
                        w3[p] = ffma2(xb, ah3[p][2 * k + 1], w3[p]);
                    }
                }
#pragma unroll
                for (int p = 0; p < CPL; ++p) v3[p] = __fadd2_rn(v3[p], w3[p]);
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int c2 = c3 + 2 * k2;
                    float2 v2[CPL], w2[CPL], F2[CPL];
#pragma unroll
                    for (int p = 0; p < CPL; ++p) {
                        v2[p] = v3[p];
                        w2[p] = f2(0.0f, 0.0f);
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        float2 xa, xb;
                        pairs(8 + 2 * c2 + k, xa, xb);
#pragma unroll
                        for (int p = 0; p < CPL; ++p) {
                            v2[p] = ffma2(xa, ah2[p][2 * k], v2[p]);
                            w2[p] = ffma2(xb, ah2[p][2 * k + 1], w2[p]);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < CPL; ++p) v2[p] = __fadd2_rn(v2[p], w2[p]);
#pragma unroll
                    for (int k1 = 0; k1 < 2; ++k1) {             // level-1 node c1 = c2 + 4 k1
                        const int c1 = c2 + 4 * k1;
                        float2 x10, x11, x0a, x0b;
                        pairs(16 + 2 * c1, x10, x11);
                        pairs(17 + 2 * c1, x0a, x0b);
                        // leaves c1 and c1 + 8: coefficients (and -aux) in slots 64 + 4 c2 + 2 k1 + (0, 1)
                        float2 cfa, cfb, naa = f2(0.0f, 0.0f), nab = f2(0.0f, 0.0f);
                        pairs(32 + 2 * c2 + k1, cfa, cfb);
                        if constexpr (F == F_LOGSUMEXP) pairs(40 + 2 * c2 + k1, naa, nab);
#pragma unroll
                        for (int p = 0; p < CPL; ++p) {
                            const float2 v1 = ffma2(x11, ah1[p][1], ffma2(x10, ah1[p][0], v2[p]));
                            const float2 Ga = __fmul2_rn(cfa, hp2<F>(ffma2(x0a, ah0[p], v1), c0, naa));
                            const float2 Gb = __fmul2_rn(cfb, hp2<F>(ffma2(x0b, ah0[p], v1), c0, nab));
                            g0[p] = ffma2(x0b, Gb, ffma2(x0a, Ga, g0[p]));
                            const float2 F1 = __fadd2_rn(Ga, Gb);
                            g1[p][0] = ffma2(x10, F1, g1[p][0]);
                            g1[p][1] = ffma2(x11, F1, g1[p][1]);
                            F2[p] = k1 == 0 ? F1 : __fadd2_rn(F2[p], F1);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        float2 xa, xb;
                        pairs(8 + 2 * c2 + k, xa, xb);
#pragma unroll
                        for (int p = 0; p < CPL; ++p) {
                            g2[p][2 * k] = ffma2(xa, F2[p], g2[p][2 * k]);
                            g2[p][2 * k + 1] = ffma2(xb, F2[p], g2[p][2 * k + 1]);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < CPL; ++p) F3[p] = k2 == 0 ? F2[p] : __fadd2_rn(F3[p], F2[p]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 xa, xb;
                    pairs(4 * c3 + k, xa, xb);
#pragma unroll
                    for (int p = 0; p < CPL; ++p) {
                        g3[p][2 * k] = ffma2(xa, F3[p], g3[p][2 * k]);
                        g3[p][2 * k + 1] = ffma2(xb, F3[p], g3[p][2 * k + 1]);
                    }
                }
#pragma unroll
                for (int p = 0; p < CPL; ++p) Fr[p] = c3 == 0 ? F3[p] : __fadd2_rn(Fr[p], F3[p]);
            }
#pragma unroll
            for (int p = 0; p < CPL; ++p) {
                if (active[p]) {
                    // columns at or beyond tau carry no gradient
                    *reinterpret_cast<float2*>(Fb[p] + rho * frow) =
                        make_float2(t[p] < a.tau ? Fr[p].x : 0.0f, t[p] + 1 < a.tau ? Fr[p].y : 0.0f);
                }
            }
        }
        if (kb + 1 < nb) put((kb + 1) & 1);
        __syncthreads();
    }

    // the two root halves' accumulators, in a fixed order; gradient rows in the band's column
    // order: level 0, level 1 (2), level 2 (4), level 3 (8)
    auto row = [&](int p, int j) -> float2 {
        return j == 0 ? g0[p] : j < 3 ? g1[p][j - 1] : j < 7 ? g2[p][j - 3] : g3[p][j - 7];
    };
    if (half == 1) {
#pragma unroll
        for (int p = 0; p < CPL; ++p)
#pragma unroll
            for (int j = 0; j < 15; ++j) red[j][colw + (kBwdCols / 2) * p] = row(p, j);
    }
    __syncthreads();
    if (half == 0) {
#pragma unroll
        for (int p = 0; p < CPL; ++p) {
            if (!active[p]) continue;
            float* out = a.gradpart + ((long long)r * a.groups + grp) * 15 * a.tau_pad + t[p];
#pragma unroll
            for (int j = 0; j < 15; ++j) {
                const float2 o = __fadd2_rn(row(p, j), red[j][colw + (kBwdCols / 2) * p]);
                *reinterpret_cast<float2*>(out + (long long)j * a.tau_pad) =
                    make_float2(t[p] < a.tau ? o.x : 0.0f, t[p] + 1 < a.tau ? o.y : 0.0f);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Materialised product P = X A (Algorithms 1-2's output, no integrand)
// ------------------------------------------------------------------------------------------
// The product is bound by its 4-byte output writes, so the layout is chosen for them: a CTA
// covers 256 columns (4 warps x 32 lanes x 2) of a range of roots, and every lane walks the
// same roots with its two columns of A in registers.  A leaf's two outputs per lane then make
// one 256-byte contiguous segment of output row k = rho + q n_root per warp store (a thread per
// root would write 32 rows 4 tau bytes apart).  The x values of 8 roots at a time are staged
// in shared memory (double-buffered, each value stored twice for the paired instructions).
constexpr int kMatThreads = 128;
constexpr int kMatCols = 2 * kMatThreads;
constexpr int kMatSlots = 64;                  // x values per root
constexpr int kMatRowPad = 2 * kMatSlots + 4;

// Slot s of a root: level 3 (s < 16: node s / 8, column s % 8), level 2 (node (s-16) / 4,
// column s % 4), level 1 (node (s-32) / 2, column s % 2), level 0 (s >= 48: leaf c1 + 8 k0 for
// u = s - 48 = 2 c1 + k0, so that the two leaves under level-1 node c1 are adjacent).  As a
// code: bit 31 for no value (0), else the point-table offset (+ rho).
__device__ __forceinline__ unsigned mat_slot_code(const FineArgs<float>& a, int s) {
    int lev, c, jj;
    if (s < 16) { lev = 3; c = s >> 3; jj = s & 7; }
    else if (s < 32) { lev = 2; c = (s - 16) >> 2; jj = s & 3; }
    else if (s < 48) { lev = 1; c = (s - 32) >> 1; jj = s & 1; }
    else { const int u = s - 48; lev = 0; c = (u >> 1) + 8 * (u & 1); jj = 0; }
    if (jj >= a.lev_tau[lev]) return 1u << 31;
    return (unsigned)(a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + ((long long)c << a.logn_root));
}

__global__ void __launch_bounds__(kMatThreads, 5) k_fine_mat_s4(const __grid_constant__ FineArgs<float> a) {
    __shared__ __align__(16) float xs[2][kRB][kMatRowPad];
    __shared__ unsigned codes[kMatSlots];
    const int tid = threadIdx.x;
    const int grp = blockIdx.x, pass = blockIdx.y, r = blockIdx.z;
    const long long n_root = 1LL << a.logn_root;
    const int t = pass * kMatCols + 2 * tid;
    const bool active = t < a.tau_pad;                          // then t + 1 < tau_pad too
    const bool on0 = t < a.tau, on1 = t + 1 < a.tau;            // the columns written
    const float* tab = a.tab + (long long)r * a.tab_stride;
    const float kap = a.kappa;

    float2 ah3[8], ah2[4], ah1[2], ah0;
    auto lda = [&](int lev, int jj) -> float2 {
        if (!active || jj >= a.lev_tau[lev]) return f2(0.0f, 0.0f);
        const float* p = a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA + t;
        return f2(kap * __ldg(p), kap * __ldg(p + 1));
    };
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) ah3[jj] = lda(3, jj);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) ah2[jj] = lda(2, jj);
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) ah1[jj] = lda(1, jj);
    ah0 = lda(0, 0);

    const long long rho_beg = (long long)grp * a.roots_per_cta;
    const long long rho_end = min(rho_beg + (long long)a.roots_per_cta, n_root);
    const int nb = rho_end > rho_beg ? (int)((rho_end - rho_beg + kRB - 1) / kRB) : 0;
    // staging: thread tid fills slots tid / 8 + 16 u of batch root tid % 8
    constexpr int PER = kRB * kMatSlots / kMatThreads;
    const int jst = tid & 7;
    if (tid < kMatSlots) codes[tid] = mat_slot_code(a, tid);    // (read after the first barrier)
    float pre[PER];
    auto fetch = [&](long long rb0) {
        const long long rho = rb0 + jst;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const unsigned code = codes[(tid >> 3) + 16 * u];
            pre[u] = (!(code >> 31) && rho < rho_end) ? __ldg(tab + code + rho) : 0.0f;
        }
    };
    auto put = [&](int buf) {
#pragma unroll
        for (int u = 0; u < PER; ++u)
            *reinterpret_cast<float2*>(&xs[buf][jst][2 * ((tid >> 3) + 16 * u)]) = f2(pre[u], pre[u]);
    };
    // root values S_4 (layout [t/4][rho][4]) of the thread's columns
    const float* Sb = (a.S && active) ? a.S + (long long)r * a.S_stride + ((long long)(t >> 2) << a.logn_root) * 4 + (t & 3)
                                      : nullptr;
    auto lds2 = [&](long long rho) -> float2 {
        return Sb ? __ldg(reinterpret_cast<const float2*>(Sb + rho * 4)) : f2(0.0f, 0.0f);
    };
    // output rows of shift r: P[r][k][t]; with tau even, (k tau + t) is even and a lane's two
    // columns are one aligned 8-byte store
    float* Pr = a.P + (long long)r * a.N * a.tau + t;
    const long long qstride = n_root * a.tau;
    const bool pair_store = (a.tau & 1) == 0;
    auto out = [&](float* p, float2 y) {
        if (pair_store) {
            if (on1) *reinterpret_cast<float2*>(p) = y;
        } else {
            if (on0) p[0] = y.x;
            if (on1) p[1] = y.y;
        }
    };

    __syncthreads();                                            // the slot codes
    if (nb > 0) { fetch(rho_beg); put(0); }
    __syncthreads();
    float2 snext = rho_beg < rho_end ? lds2(rho_beg) : f2(0.0f, 0.0f);
    for (int kb = 0; kb < nb; ++kb) {
        const long long rb0 = rho_beg + (long long)kb * kRB;
        if (kb + 1 < nb) fetch(rb0 + kRB);                        // in flight during this batch
        for (int j = 0; j < kRB; ++j) {
            const long long rho = rb0 + j;
            if (rho >= rho_end) break;
            const float2 sr = snext;
            if (rho + 1 < rho_end) snext = lds2(rho + 1);
            const float* xr = xs[kb & 1][j];
            auto pairs = [&](int g, float2& p0, float2& p1) {
                const float4 q = *reinterpret_cast<const float4*>(xr + 4 * g);
                p0 = f2(q.x, q.y);
                p1 = f2(q.z, q.w);
            };
            float* prow = Pr + rho * a.tau;
#pragma unroll
            for (int c3 = 0; c3 < 2; ++c3) {
                float2 v3 = f2(kap * sr.x, kap * sr.y), w3 = f2(0.0f, 0.0f);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 xa, xb;
                    pairs(4 * c3 + k, xa, xb);
                    v3 = ffma2(xa, ah3[2 * k], v3);
                    w3 = ffma2(xb, ah3[2 * k + 1], w3);
                }
                v3 = __fadd2_rn(v3, w3);
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int c2 = c3 + 2 * k2;
                    float2 v2 = v3, w2 = f2(0.0f, 0.0f);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        float2 xa, xb;
                        pairs(8 + 2 * c2 + k, xa, xb);
                        v2 = ffma2(xa, ah2[2 * k], v2);
                        w2 = ffma2(xb, ah2[2 * k + 1], w2);
                    }
                    v2 = __fadd2_rn(v2, w2);
#pragma unroll
                    for (int k1 = 0; k1 < 2; ++k1) {             // level-1 node c1 = c2 + 4 k1
                        const int c1 = c2 + 4 * k1;
                        float2 x10, x11, x0a, x0b;
                        pairs(16 + c1, x10, x11);
                        pairs(24 + c1, x0a, x0b);
                        const float2 v1 = ffma2(x11, ah1[1], ffma2(x10, ah1[0], v2));
                        out(prow + c1 * qstride, ffma2(x0a, ah0, v1));            // leaf c1
                        out(prow + (c1 + 8) * qstride, ffma2(x0b, ah0, v1));      // leaf c1 + 8
                    }
                }
            }
        }
        if (kb + 1 < nb) put((kb + 1) & 1);
        __syncthreads();
    }
}

}  // namespace

int fine_s4_fwd_roots(int nb) { return fwd_roots(nb); }
int fine_s4_fwd_resident(int F, int nb) { return fwd_min_blocks(F, nb); }
int fine_s4_bwd_cols(int cpl) { return kBwdCols * cpl; }
int fine_s4_bwd_batch() { return kBRB; }
int fine_s4_mat_cols() { return kMatCols; }

cudaError_t launch_fine_mat_s4(const FineArgs<float>& a, dim3 grid, cudaStream_t st) {
    if (a.roots_per_cta < 1 || !a.P) return cudaErrorInvalidValue;
    k_fine_mat_s4<<<grid, kMatThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <int F, int NB>
static cudaError_t fwd_s4(const FineArgs<float>& a, dim3 grid, cudaStream_t st) {
    const size_t smem = fwd_smem_bytes(a.cr);
    // dynamic + static shared memory may exceed 48 KB; the attribute belongs to the current device,
    // so it is set on every launch (as for the tensor-core kernels), not once per process
    const cudaError_t e = cudaFuncSetAttribute(k_fine_fwd_s4<F, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)fwd_smem_bytes(kMaxCRS4));
    if (e != cudaSuccess) return e;
    k_fine_fwd_s4<F, NB><<<grid, kFwdThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NB>
static cudaError_t fwd_s4_nb(const FineArgs<float>& a, int F, dim3 grid, cudaStream_t st) {
    switch (F) {
        case F_LINEAR_MEAN: return fwd_s4<F_LINEAR_MEAN, NB>(a, grid, st);
        case F_MEAN_COS: return fwd_s4<F_MEAN_COS, NB>(a, grid, st);
        case F_CALL_MEAN_EXP: return fwd_s4<F_CALL_MEAN_EXP, NB>(a, grid, st);
        case F_GAUSS_NORM2: return fwd_s4<F_GAUSS_NORM2, NB>(a, grid, st);
        case F_PDE_INV_SQ: return fwd_s4<F_PDE_INV_SQ, NB>(a, grid, st);
        case F_LOGSUMEXP: return fwd_s4<F_LOGSUMEXP, NB>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fine_fwd_s4(const FineArgs<float>& a, int F, int nb, dim3 grid, cudaStream_t st) {
    if (a.cr < 4 || a.cr > kMaxCRS4 || (a.cr & 3)) return cudaErrorInvalidValue;
    if (nb == 2) return fwd_s4_nb<2>(a, F, grid, st);
    if (nb == 1) return fwd_s4_nb<1>(a, F, grid, st);
    return cudaErrorInvalidValue;
}

template <int CPL>
static cudaError_t bwd_s4(const FineArgs<float>& a, int F, dim3 grid, cudaStream_t st) {
    switch (F) {
#define QMC_BWD_S4(FF)                                                                                     \
    do {                                                                                                   \
        constexpr size_t smem = bwd_smem_bytes(CPL);                                                       \
        if (smem > 48 * 1024) {                                                                            \
            const cudaError_t e = cudaFuncSetAttribute(k_fine_bwd_s4<FF, CPL>,                             \
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            if (e != cudaSuccess) return e;                                                                \
        }                                                                                                  \
        k_fine_bwd_s4<FF, CPL><<<grid, kBwdThreads, smem, st>>>(a);                                        \
    } while (0)
        case F_LINEAR_MEAN: QMC_BWD_S4(F_LINEAR_MEAN); break;
        case F_MEAN_COS: QMC_BWD_S4(F_MEAN_COS); break;
        case F_CALL_MEAN_EXP: QMC_BWD_S4(F_CALL_MEAN_EXP); break;
        case F_GAUSS_NORM2: QMC_BWD_S4(F_GAUSS_NORM2); break;
        case F_PDE_INV_SQ: QMC_BWD_S4(F_PDE_INV_SQ); break;
        case F_LOGSUMEXP: QMC_BWD_S4(F_LOGSUMEXP); break;
#undef QMC_BWD_S4
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fine_bwd_s4(const FineArgs<float>& a, int F, int cpl, dim3 grid, cudaStream_t st) {
    if (cpl == 2) return bwd_s4<2>(a, F, grid, st);
    if (cpl == 1) return bwd_s4<1>(a, F, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace qmc
