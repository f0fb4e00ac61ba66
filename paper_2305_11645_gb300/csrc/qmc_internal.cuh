// Internal declarations of the GB300 reduced-QMC library: kernel argument
// structs, the bit-exact point generator, coordinate transforms, integrand
// functors and the launchers the host planner calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qmc {

constexpr int kMaxLevels = 32;     // levels I = 0..m (level m holds the constant columns, w_j >= m)
constexpr int kMaxChain = 48;      // coarse entries (levels, cut into column ranges); Chain stays ~4 KB

// Kinds, transforms and integrands mirror include/qmc.h.
enum { KIND_LATTICE = 0, KIND_NET = 1, KIND_MC = 2, KIND_POLY = 3 };
enum { T_IDENTITY = 0, T_CENTER = 1, T_INV_NORMAL = 2, T_TENT = 3 };
enum { F_NONE = 0, F_LINEAR_MEAN, F_MEAN_COS, F_CALL_MEAN_EXP, F_GAUSS_NORM2, F_PDE_INV_SQ, F_LOGSUMEXP };
enum { SHAPE_S0 = 0, SHAPE_S1 = 1, SHAPE_S4 = 4 };
enum { MODE_FUSED = 0, MODE_MATERIALIZE = 1 };

// The rule as the kernels see it.  Per-level data describe Algorithm 2's
// weight blocks: level I holds the columns j with min(w_j, m) = I, contiguous
// because w is nondecreasing, each with n_I = 2^(m-I) distinct rows.
struct DevRule {
    int kind, m, s, transform;
    int R;                          // shifts present in `shift` (0 = unshifted)
    const uint32_t* gen;            // lattice: z[s]; net: C[s*m] column masks; reduced MC: the samples
                                    // of every replica, [r][T_tot] in the distinct-row table's layout
    const uint32_t* shift;          // R*s or nullptr
    long long T_tot;                // distinct-row table entries per shift / replica
    int nlev;                       // m + 1
    int lev_tau[kMaxLevels];
    int lev_col0[kMaxLevels];
    long long lev_tab[kMaxLevels + 1];   // offset of level I in the distinct-row table (prefix sums)
    // A non-periodic reduced net (Sec. 4, Algorithm 4's case): every column is on level 0 with all
    // N rows, its points use every digit of the row index, and column j's last min(w_j, m) rows of
    // C^(j) are zeroed by its own w: the columns wcol0[g] .. wcol0[g+1]-1 have min(w, m) = wval[g].
    int nonper;
    int nw;
    int wcol0[kMaxLevels + 1], wval[kMaxLevels];
    // a prime base b > 2 (Sec. 1.3, Sec. 5): level I has n_I = b^(m-I) distinct rows
    int b;
    long long lev_n[kMaxLevels];
};

// min(w_j, m) of column j of a non-periodic net
__device__ __forceinline__ int wcl_of(const DevRule& R, int j) {
    int v = 0;
    for (int g = 0; g < R.nw; ++g)
        if (j >= R.wcol0[g]) v = R.wval[g];
    return v;
}

// ---------------------------------------------------------------------------------------------
// Point generator (bit-exact integer arithmetic).
//   lattice (Sec. 1.3): u = (row * z_j) mod 2^q, X32 = u * 2^(32-q)
//   net (Sec. 4, Algorithm 3): y = XOR of the column masks selected by the digits of row
//        (least significant first), with the last min(w_j,m) rows zeroed
//        (eq. reduced_genmat_net2), X32 = y * 2^(32-m)
//   q = m - min(w_j, m); row < 2^q is the row index within one period.  A non-periodic net
//   passes q = m (every digit of the point index) and zeroes column j's own last rows.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t unshifted_x32(const DevRule& R, int j, uint32_t row, int q) {
    if (R.kind == KIND_LATTICE) {
        if (q == 0) return 0u;
        const uint32_t mask = (q >= 32) ? 0xFFFFFFFFu : ((1u << q) - 1u);
        const uint32_t u = (row * R.gen[j]) & mask;     // mod 2^q needs only the low 32 bits
        return (q >= 32) ? u : (u << (32 - q));
    }
    if (R.kind == KIND_POLY) {
        // k(x) x^w gt(x) mod x^m over F_2: the coefficients of x^w .. x^(m-1) are those of
        // k(x) gt(x) mod x^q, q = m - w, and the coefficient of x^(w+i) is the digit of 2^(i-q)
        // (nu of Sec. 1.3).  So u = (row carry-less-times gt) mod 2^q, x = u 2^-q.
        if (q == 0) return 0u;
        const uint32_t g = R.gen[j];
        uint32_t u = 0;
        for (int b = 0; b < q; ++b)
            if ((row >> b) & 1u) u ^= g << b;
        const uint32_t mask = (q >= 32) ? 0xFFFFFFFFu : ((1u << q) - 1u);
        u &= mask;
        return (q >= 32) ? u : (u << (32 - q));
    }
    const uint32_t* Cj = R.gen + (size_t)j * (size_t)R.m;
    uint32_t y = 0;
    for (int b = 0; b < q; ++b)
        if ((row >> b) & 1u) y ^= Cj[b];
    const int wcl = R.nonper ? wcl_of(R, j) : R.m - q;
    y &= (wcl >= 32) ? 0u : ~((1u << wcl) - 1u);
    return y << (32 - R.m);
}

__device__ __forceinline__ uint32_t apply_shift(int kind, uint32_t x, uint32_t d) {
    return kind == KIND_LATTICE ? (x + d) : (x ^ d);   // {x + Delta} mod 1, or the digital shift (nets,
                                                        // polynomial lattices)
}

// ---------------------------------------------------------------------------------------------
// Coordinate transforms phi (Sec. 2.3) of x = X32 * 2^-32, rounded once to T.
// The 32-bit integer conversions are explicit cvt instructions: the unsigned value
// 2^32 - X32 must be converted as unsigned (2^31 included), never folded into -X32.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float u32_to_f32(uint32_t v) {
    float r;
    asm("cvt.rn.f32.u32 %0, %1;" : "=f"(r) : "r"(v));
    return r;
}
__device__ __forceinline__ float i32_to_f32(int v) {
    float r;
    asm("cvt.rn.f32.s32 %0, %1;" : "=f"(r) : "r"(v));
    return r;
}
__device__ __forceinline__ double u32_to_f64(uint32_t v) {
    double r;
    asm("cvt.rn.f64.u32 %0, %1;" : "=d"(r) : "r"(v));
    return r;
}
__device__ __forceinline__ double i32_to_f64(int v) {
    double r;
    asm("cvt.rn.f64.s32 %0, %1;" : "=d"(r) : "r"(v));
    return r;
}

template <class T> struct Tr;

template <> struct Tr<float> {
    static __device__ __forceinline__ float apply(uint32_t x, int tr) {
        const float two_m32 = 2.3283064365386963e-10f, two_m31 = 4.656612873077393e-10f;
        // 1 - x for x >= 1/2 is (2^32 - X32) 2^-32 <= 1/2; 2^32 - X32 <= 2^31 fits a uint32
        const uint32_t cmp = 0u - x;
        switch (tr) {
            case T_CENTER: return i32_to_f32((int)(x ^ 0x80000000u)) * two_m32;
            case T_TENT: return (x < 0x80000000u) ? u32_to_f32(x) * two_m31 : u32_to_f32(cmp) * two_m31;
            case T_INV_NORMAL: {      // one quantile call on the half nearer 0, then the sign
                const bool low = x < 0x80000000u;
                const float z = normcdfinvf(u32_to_f32(low ? x : cmp) * two_m32);
                return low ? z : -z;
            }
            default: return u32_to_f32(x) * two_m32;
        }
    }
};

template <> struct Tr<double> {
    static __device__ __forceinline__ double apply(uint32_t x, int tr) {
        const double two_m32 = 2.3283064365386962890625e-10, two_m31 = 4.656612873077392578125e-10;
        const uint32_t cmp = 0u - x;
        switch (tr) {
            case T_CENTER: return i32_to_f64((int)(x ^ 0x80000000u)) * two_m32;
            case T_TENT: return (x < 0x80000000u) ? u32_to_f64(x) * two_m31 : u32_to_f64(cmp) * two_m31;
            case T_INV_NORMAL: {
                const bool low = x < 0x80000000u;
                const double z = normcdfinv(u32_to_f64(low ? x : cmp) * two_m32);
                return low ? z : -z;
            }
            default: return u32_to_f64(x) * two_m32;
        }
    }
};

// ---------------------------------------------------------------------------------------------
// Integrands, row-separable: f(y) = g(u), u = sum_t h(y_t)   (eq. (2)'s f).
// The kernels carry v = kappa * y instead of y: kappa multiplies A's staged
// columns and the coarse root values once, so that exp(c y) = 2^v costs one
// ex2 per output (kappa = c log2 e); log-sum-exp works in base 2 (kappa = log2 e).
// G = dQ/dy_t = coef_k * gfac * hp(v, aux) with coef_k = upstream g'(u_k)/(R N).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float ex2f(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2(float x) { return ex2f(x); }
__device__ __forceinline__ double ex2(double x) { return exp2(x); }

constexpr double kLog2e = 1.4426950408889634;
constexpr double kLn2 = 0.6931471805599453;

template <int F, class T> struct Fn {
    static __host__ __device__ double kappa(double c) {
        return F == F_CALL_MEAN_EXP ? c * kLog2e : F == F_LOGSUMEXP ? kLog2e : 1.0;
    }
    static __host__ __device__ double gfac(double c) { return F == F_CALL_MEAN_EXP ? c : 1.0; }
    // contribution of one output to the row sum u (not used for LOGSUMEXP)
    static __device__ __forceinline__ T h(T v, T c) {
        if constexpr (F == F_LINEAR_MEAN) return v;
        else if constexpr (F == F_MEAN_COS) return cos(v);
        else if constexpr (F == F_CALL_MEAN_EXP) return ex2(v);
        else if constexpr (F == F_GAUSS_NORM2) return v * v;
        else if constexpr (F == F_PDE_INV_SQ) { T r = T(1) / (T(1) + c * v); return r * r; }
        else return v;
    }
    // h'(y) / gfac in terms of v (LOGSUMEXP: 2^(v - aux), aux = log2 e * log sum exp(y))
    static __device__ __forceinline__ T hp(T v, T c, T aux) {
        if constexpr (F == F_LINEAR_MEAN) return T(1);
        else if constexpr (F == F_MEAN_COS) return -sin(v);
        else if constexpr (F == F_CALL_MEAN_EXP) return ex2(v);
        else if constexpr (F == F_GAUSS_NORM2) return T(2) * v;
        else if constexpr (F == F_PDE_INV_SQ) { T r = T(1) / (T(1) + c * v); return T(-2) * c * r * r * r; }
        else return ex2(v - aux);
    }
};

// ---------------------------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------------------------

// Coarse chain: the weight blocks at levels >= JF that are not expanded by the
// register tree.  Entry e is level lev[e] with n = 2^logn[e] distinct rows.
struct Chain {
    int count;
    int lev[kMaxChain], logn[kMaxChain], tau[kMaxChain], col0[kMaxChain];
    long long tab[kMaxChain];        // table offset of the level's first column
    long long boff[kMaxChain];       // element offset of B_e inside a shift's area
    int tile0[kMaxChain + 1];        // prefix sums of work tiles (per kernel)
    int split[kMaxChain];            // k-splits (backward grad GEMM)
    long long kper[kMaxChain];       // K rows per split (tensor-core backward: a multiple of 32)
    long long poff[kMaxChain];       // partial-buffer offsets (backward grad GEMM)
    // backward: where level e's folded gradient F_e comes from -- the root folds (fsel 0) or a
    // folded level (fsel 1) at offset foff, still to be folded 2^flog times on the fly
    int fsel[kMaxChain], flog[kMaxChain];
    long long foff[kMaxChain];
};

// Levels folded by k_fold_tree: F_{JF+d} for d = 1..depth from the root folds, each written at
// off[d] when want[d] (a coarse level with columns).  Top nodes: 2^logn_top of level JF+depth.
struct FoldLevels {
    int depth, logn_top;
    int want[8];
    long long off[8];
};

constexpr int kMaxCR = 256;          // columns per CTA of the fine forward kernel

// ---------------------------------------------------------------------------------------------
// Block gradients on the tensor cores (qmc_grad_tc.cu): the coarse entries with at least 32
// distinct rows whose folded gradient is materialised, each with a TMA map of F (t, rows, shifts)
// and of its table columns (rows, columns, shifts).
// ---------------------------------------------------------------------------------------------
}  // namespace qmc
#include <cuda.h>
#include <cuda_bf16.h>
namespace qmc {
constexpr int kMaxGradTc = 24;
struct GradTcEntry {
    long long n, kper, poff;
    long long xoff;                  // bf16 element offset of the entry's pre-split table columns
    int tau, split;
};
struct GradTcArgs {
    CUtensorMap fmap[kMaxGradTc];    // F_e: (t, rows, shifts) FP32
    CUtensorMap xmap[kMaxGradTc];    // the entry's pieces: (rows, j, shifts, pieces) bf16
    GradTcEntry ent[kMaxGradTc];
    long long unit0[kMaxGradTc + 1];
    long long units;
    int n, reff, t_tiles;
};
cudaError_t launch_grad_tc(const __nv_bfloat16* xp, const float* Froot, long long root_stride, const float* Fchain,
                           long long chain_stride, int tau_pad, const Chain& ch, const int* sel, const long long* xoff,
                           int nsel, float* part, int reff, int pieces, cudaStream_t st);
cudaError_t grad_error_word(unsigned int* value, bool clear);

// ---------------------------------------------------------------------------------------------
// Fold and block gradients of the lowest L <= 3 coarse levels in one pass over the root gradients
// (qmc_foldgrad_tc.cu), with the levels' table columns pre-split into bf16 pieces (k_split_xt).
// ---------------------------------------------------------------------------------------------
constexpr int kMaxFoldLv = 3;
constexpr int kMaxSplitXt = kMaxGradTc + kMaxFoldLv;
struct SplitXtArgs {
    int n;                           // table column ranges pre-split (fused levels, then k_grad_tc entries)
    int lev[kMaxSplitXt];            // d of a fused level JF + d, or -1
    int logn[kMaxSplitXt], tau[kMaxSplitXt];
    long long tab[kMaxSplitXt];      // table offset of the range's first column
    long long off[kMaxSplitXt];      // bf16 element offset of its pieces in the split buffer
    long long blk0[kMaxSplitXt + 1]; // prefix sums of tau x n / 8 threads
};
struct FoldGradArgs {
    CUtensorMap fmap;                // F_JF: (t, rows, shifts)
    CUtensorMap xmap[kMaxFoldLv];    // level JF + d pieces: (rows, j, shifts, pieces)
    float* fout;                     // F_{JF+L}: n_out rows x tau_pad per shift, fout_stride apart
    long long fout_stride;
    float* part;
    long long poff[kMaxFoldLv];      // partial offsets: [split][j][tau_pad] per level
    long long items;                 // shifts x n_out / 32 (shift, residue block) items
    int nd[kMaxFoldLv];              // MMA N of each level (0: no columns)
    int tau[kMaxFoldLv];
    int acc[kMaxFoldLv];             // accumulator column offsets
    int nt;                          // columns of one accumulator set
    int log_out;                     // log2 n_out
    int tau_pad, cpt, t_tiles, group;
    int froot_tiled;                 // F_JF in 128-column tiles, [r][t / 128][rows][128]
    const float* froot;              // F_JF (the tiled layout: a chunk of 32 rows is 16 KB contiguous)
    long long froot_stride;          // floats per shift
    long long n_root;
};
cudaError_t launch_split_xt(const float* tab, long long tab_stride, const SplitXtArgs& sa, int reff, int pieces,
                            __nv_bfloat16* xp, float xc, cudaStream_t st);
cudaError_t launch_fold_grad_tc(FoldGradArgs& ga, int L, const float* Froot, long long root_stride, long long n_root,
                                const __nv_bfloat16* xp, const SplitXtArgs& sa, int reff, int pieces, cudaStream_t st);
cudaError_t foldgrad_error_word(unsigned int* value, bool clear);

// ---------------------------------------------------------------------------------------------
// Base b > 2: one weight level of the top-down sum (qmc_base_b.cu).  Level I's n = b^(m-I)
// distinct rows of its tau columns (A's rows col0 ..), written at n_out rows (n, or N for the
// last level) on top of the coarser level's n_next rows.
// ---------------------------------------------------------------------------------------------
struct LevelB {
    int level, tau, col0;
    long long n, tab, n_out, n_next;
};
template <class T>
cudaError_t launch_table_b(const DevRule& R, T* tab, long long T_tot, long long stride, int reff, unsigned int* ticket,
                           cudaStream_t st);
cudaError_t launch_points_b(const DevRule& R, uint32_t* out, long long total, bool full, int shift_idx,
                            cudaStream_t st);
template <class T>
cudaError_t launch_level_b(const T* tab, long long tab_stride, const T* A, int ldA, int tau_pad, const LevelB& lv,
                           T* out, long long out_stride, const T* next, long long next_stride, bool rowmajor, int tau,
                           int reff, cudaStream_t st);
template <class T>
cudaError_t launch_rows_b(const T* S, long long S_stride, long long N, int tau, int F, double kappa, double c0,
                          T* rowpart, T* rowmax, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_grad_rows_b(const T* S, long long S_stride, long long N, int tau, int tau_pad, int F, double kappa,
                               double c0, const T* rowsave, const double* upstream, T* G, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_fold_b(const T* src, long long n_src, T* dst, long long n_dst, int tau_pad, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_grad_b(const T* tab, long long tab_stride, const T* F, const LevelB& lv, long long kper, int splits,
                          int reff, int tau_pad, T* part, cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// Algorithm 2 on the tensor cores, top down: a pass computes, for rho < n_out,
//   Pt_out[rho] = sum over its levels I of X~_I[rho mod n_I] A~_I + Pt_next[rho mod n_next],
// where Pt_next is the previous (coarser) pass's output (none for the first pass).  One level
// per pass is Algorithm 2's step P~_I = tile(P~_{I+1}) + X~_I A~_I; the last pass writes the
// root values S of the fine band.  The operands come as bf16 pieces in global memory, in
// blocks of 32 columns (64-byte rows) that a TMA box of 32 x 128 (X) or 32 x 256 (A) copies:
//   X pieces: per shift, per level I, per piece p, per chunk kc: n'_I = max(n_I, 128) rows of
//             columns 32 kc .. 32 kc + 31 of the level (row rho holds X~_I[rho mod n_I]);
//   A pieces: per level I, per piece p, per chunk kc: tA rows (columns t of A, tA a multiple
//             of 256) of the same 32 columns j.
// ---------------------------------------------------------------------------------------------
constexpr int kMaxPassSeg = 4;       // levels summed by one pass
constexpr int kMaxPasses = 40;

struct LevelSeg {
    int level;                       // I
    int chunks;                      // K chunks of 32 columns
    int last_ksteps;                 // 16-column K-steps of the last chunk (1 or 2)
    int logn;                        // log2 n_I (n_I = 2^(m-I) distinct rows)
    int logn_rep;                    // log2 n'_I, n'_I = max(n_I, 128)
    int col0, tau;                   // the level's columns of A (first, count)
    long long tab;                   // the level's offset in the FP32 point table
    long long xrow;                  // X-pieces row of (piece 0, chunk 0, row 0) within a shift
    long long arow;                  // A-pieces row of (piece 0, chunk 0, t 0)
};

struct LevelPass {
    int nseg;
    LevelSeg seg[kMaxPassSeg];
    int logn_out;                    // rows written: n_out = 2^logn_out
    long long out_off, out_stride;   // float offsets of the output area and of one shift's part
    int logn_next;                   // log2 n_next, or -1 (no coarser pass)
    long long next_off, next_stride;
    int rho_tiles, t_tiles, reps;    // 128-row tiles, 256-column tiles, row tiles per next-pass tile
    long long ntiles;                // rho_tiles * t_tiles * shifts
    long long const_off;             // first pass of centred points: float offset of the constant row
                                     // xc sum_j a_j (added in place of a coarser pass), else -1
};

struct LevelPlan {
    int npass;
    LevelPass pass[kMaxPasses];
    int pieces;                      // 3 (split tier) or 1 (bf16 tier)
    long long x_rows_per_shift;      // rows of 32 bf16 of one shift's X pieces
    long long a_rows;                // rows of 32 bf16 of the A pieces
    int tA;                          // A-piece rows per chunk block (columns t, a multiple of 256)
    size_t x_off, a_off;             // byte offsets of the piece areas in the workspace
    size_t c_off;                    // byte offset of the constant row (tau_pad floats)
    size_t cpart_off;                // byte offset of its 64 x tau_pad double partial sums
    float xc;                        // centring of the points (x - xc is split; 0 or 1/2)
};

cudaError_t launch_split_a(const float* A, int ldA, int tau, const LevelPlan& lp, unsigned char* ws,
                           cudaStream_t st);
cudaError_t launch_split_x(const float* tab, long long tab_stride, const LevelPlan& lp, int reff, unsigned char* ws,
                           cudaStream_t st);
cudaError_t launch_level_pass(const LevelPlan& lp, int p, int reff, int tau_pad, unsigned char* ws, cudaStream_t st);
cudaError_t level_error_word(unsigned int* value, bool clear);
// the constant row xc sum_{coarse j} A[j][t] of centred points, summed in double
cudaError_t launch_const_row(const float* A, int ldA, int tau, int tau_pad, const LevelPlan& lp, unsigned char* ws,
                             cudaStream_t st);
// column sums of the top folded gradient level over every shift and row, in double: gsum[t]
cudaError_t launch_col_sums(const float* F, long long shift_stride, long long rows, int reff, int tau_pad,
                            double* part, double* gsum, cudaStream_t st);

template <class T> struct FineArgs {
    const T* tab; long long tab_stride;       // distinct-row table, per shift
    const T* A; int ldA;                      // A (or its padded copy), row stride ldA
    int tau, tau_pad;
    int logn_root;                            // root level JF: n_root = 2^(m-JF)
    int lev_tau[4], lev_col0[4], lev_logn[4];
    long long lev_tab[4];
    const T* S; long long S_stride;           // root values S_JF = sum of the coarse block products, per shift
    int cr, cg_count, reff, r0;
    long long N;
    T* rowpart; T* rowmax;                     // FUSED: [r][cg][N]
    T* P;                                      // MATERIALIZE: [r][N][tau]
    T c0, c1;                                  // integrand parameters
    T kappa;                                   // v = kappa * y
    // backward
    const T* rowsave;        // per row: {g'(u_k) gfac/(R_eff N), log2 e * u_k} from the forward finalisation
    const double* upstream;
    double tau_d, K_d;
    T* Froot;                                  // [r][n_root][tau_pad], or with froot_tiled
                                               // [r][t / 128][n_root][128] (froot_stride per shift)
    int froot_tiled;
    long long froot_stride;
    T* gradpart;                               // [r][group][KF][tau_pad]
    int roots_per_cta, groups, kf_actual;
    int fkind;
};

// ---------------------------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
template <class T>
cudaError_t launch_table(const DevRule& R, T* tab, long long T_tot, long long stride, int reff, unsigned int* ticket,
                         cudaStream_t st);
cudaError_t launch_points_full(const DevRule& R, uint32_t* out, int shift_idx, cudaStream_t st);
cudaError_t launch_points_distinct(const DevRule& R, uint32_t* out, long long T_tot, int shift_idx,
                                   cudaStream_t st);
template <class T>
cudaError_t launch_pad_A(const T* A, T* Ap, int s, int tau, int tau_pad, cudaStream_t st);
template <class T>
cudaError_t launch_coarse_fwd(const T* tab, long long tab_stride, const T* A, int ldA, int tau_pad,
                              const Chain& ch, T* B, long long B_stride, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_chain_sum(const T* B, long long B_stride, const Chain& ch, T* S, long long S_stride,
                             int logn_root, int tau_pad, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_fine_fwd(const FineArgs<T>& a, int shape, bool exact, int F, int mode, dim3 grid,
                            cudaStream_t st);
template <class T>
cudaError_t launch_rows_finalize(const T* rowpart, const T* rowmax, int cg_count, long long N, int reff,
                                 int F, double tau, double c, double K, double coef_scale, T* rowsave, T* rowf_out,
                                 double* fpart, int nblk, unsigned int* ticket, double* est, cudaStream_t st);
template <class T>
cudaError_t launch_fine_bwd(const FineArgs<T>& a, int shape, bool exact, int F, dim3 grid, cudaStream_t st);
template <class T>
cudaError_t launch_fold_tree(const T* Froot, long long root_stride, T* Fchain, long long chain_stride,
                             const FoldLevels& fl, int tau_pad, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_coarse_grad(const T* tab, long long tab_stride, const T* Froot, long long root_stride,
                               const T* Fchain, long long chain_stride, int tau_pad, const Chain& ch, T* part,
                               int reff, int ntiles, cudaStream_t st);
template <class T>
cudaError_t launch_grad_reduce(const T* gradpart_f, int nfine_part, int kf_width, const int* koff_lev,
                               const int* col0_lev, const int* tau_lev, int jf, const T* part_c,
                               const Chain& ch, int tau, int tau_pad, int s, T* grad, const double* gsum,
                               double xc, cudaStream_t st);

// tensor-core block products (split tier: pieces = 3, bf16 tier: pieces = 1); FP32 data
int tc_fwd_rows();        // rows of a forward tile (the chain's tile0 counts tiles of this many rows)
int tc_grad_cols();       // block-gradient columns of a backward tile
cudaError_t launch_coarse_fwd_tc(const float* tab, long long tab_stride, const float* A, int ldA, int tau_pad,
                                 const Chain& ch, float* B, long long B_stride, int reff, int pieces,
                                 cudaStream_t st);
cudaError_t launch_coarse_grad_tc(const float* tab, long long tab_stride, const float* Froot, long long root_stride,
                                  const float* Fchain, long long chain_stride, int tau_pad, const Chain& ch,
                                  float* part, int reff, int ntiles, int pieces, float xc, cudaStream_t st);
cudaError_t tc_error_word(unsigned int* value, bool clear);
// one CTA whose bounded wait on an mbarrier that nothing completes runs out after `polls` polls
cudaError_t launch_selftest_wait(uint32_t polls, cudaStream_t st);
// the S4 fine band in FP32 on the CUDA cores: forward CTAs of fine_s4_fwd_roots(nb) roots, nb = 1
// or 2 level-3 nodes per thread (grid: root blocks x column groups of a.cr <= 512 columns x
// shifts), adjoint CTAs of fine_s4_bwd_cols(cpl) columns, cpl = 1 or 2 column pairs per lane
// (grid: root groups of a.roots_per_cta roots,
// a multiple of fine_s4_bwd_batch() x column passes x shifts)
int fine_s4_fwd_roots(int nb);
int fine_s4_fwd_resident(int F, int nb);   // forward CTAs resident per SM for integrand F
int fine_s4_bwd_cols(int cpl);
int fine_s4_bwd_batch();
cudaError_t launch_fine_fwd_s4(const FineArgs<float>& a, int F, int nb, dim3 grid, cudaStream_t st);
cudaError_t launch_fine_bwd_s4(const FineArgs<float>& a, int F, int cpl, dim3 grid, cudaStream_t st);
// the materialised S4 band (P = X A, float tiers): CTAs of fine_s4_mat_cols() columns over
// a.roots_per_cta roots (grid: root groups x column passes x shifts)
int fine_s4_mat_cols();
cudaError_t launch_fine_mat_s4(const FineArgs<float>& a, dim3 grid, cudaStream_t st);

}  // namespace qmc
