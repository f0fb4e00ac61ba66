// Internal declarations of the GB300 reduced-QMC library: kernel argument
// structs, the bit-exact point generator, coordinate transforms, integrand
// functors and the launchers the host planner calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qmc {

constexpr int kMaxLevels = 32;     // levels I = 0..m (level m holds the constant columns, w_j >= m)
constexpr int kMaxChain = 32;

// Kinds, transforms and integrands mirror include/qmc.h.
enum { KIND_LATTICE = 0, KIND_NET = 1 };
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
    const uint32_t* gen;            // lattice: z[s]; net: C[s*m] column masks
    const uint32_t* shift;          // R*s or nullptr
    int nlev;                       // m + 1
    int lev_tau[kMaxLevels];
    int lev_col0[kMaxLevels];
    long long lev_tab[kMaxLevels + 1];   // offset of level I in the distinct-row table (prefix sums)
};

// ---------------------------------------------------------------------------------------------
// Point generator (bit-exact integer arithmetic).
//   lattice (Sec. 1.3): u = (row * z_j) mod 2^q, X32 = u * 2^(32-q)
//   net (Sec. 4, Algorithm 3): y = XOR of the column masks selected by the digits of row
//        (least significant first), with the last min(w_j,m) rows zeroed
//        (eq. reduced_genmat_net2), X32 = y * 2^(32-m)
//   q = m - min(w_j, m); row < 2^q is the row index within one period.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t unshifted_x32(const DevRule& R, int j, uint32_t row, int q) {
    if (R.kind == KIND_LATTICE) {
        if (q == 0) return 0u;
        const uint32_t mask = (q >= 32) ? 0xFFFFFFFFu : ((1u << q) - 1u);
        const uint32_t u = (row * R.gen[j]) & mask;     // mod 2^q needs only the low 32 bits
        return (q >= 32) ? u : (u << (32 - q));
    }
    const uint32_t* Cj = R.gen + (size_t)j * (size_t)R.m;
    uint32_t y = 0;
    for (int b = 0; b < q; ++b)
        if ((row >> b) & 1u) y ^= Cj[b];
    const int wcl = R.m - q;
    y &= (wcl >= 32) ? 0u : ~((1u << wcl) - 1u);
    return y << (32 - R.m);
}

__device__ __forceinline__ uint32_t apply_shift(int kind, uint32_t x, uint32_t d) {
    return kind == KIND_LATTICE ? (x + d) : (x ^ d);   // {x + Delta} mod 1, or the digital shift
}

// ---------------------------------------------------------------------------------------------
// Coordinate transforms phi (Sec. 2.3) of x = X32 * 2^-32, rounded once to T.
// ---------------------------------------------------------------------------------------------
template <class T> struct Tr;

template <> struct Tr<float> {
    static __device__ __forceinline__ float apply(uint32_t x, int tr) {
        const float two_m32 = 2.3283064365386963e-10f, two_m31 = 4.656612873077393e-10f;
        // 1 - x for x >= 1/2 is (2^32 - X32) 2^-32 <= 1/2, held exactly in 64 bits
        const unsigned long long cmp = 0x100000000ull - (unsigned long long)x;
        switch (tr) {
            case T_CENTER: return (float)((long long)x - 0x80000000ll) * two_m32;
            case T_TENT: return (x < 0x80000000u) ? (float)x * two_m31 : (float)cmp * two_m31;
            case T_INV_NORMAL:
                return (x < 0x80000000u) ? normcdfinvf((float)x * two_m32) : -normcdfinvf((float)cmp * two_m32);
            default: return (float)x * two_m32;
        }
    }
};

template <> struct Tr<double> {
    static __device__ __forceinline__ double apply(uint32_t x, int tr) {
        const double two_m32 = 2.3283064365386962890625e-10, two_m31 = 4.656612873077392578125e-10;
        const unsigned long long cmp = 0x100000000ull - (unsigned long long)x;
        switch (tr) {
            case T_CENTER: return (double)((long long)x - 0x80000000ll) * two_m32;
            case T_TENT: return (x < 0x80000000u) ? (double)x * two_m31 : (double)cmp * two_m31;
            case T_INV_NORMAL:
                return (x < 0x80000000u) ? normcdfinv((double)x * two_m32) : -normcdfinv((double)cmp * two_m32);
            default: return (double)x * two_m32;
        }
    }
};

// ---------------------------------------------------------------------------------------------
// Integrands, row-separable: f(y) = g(u), u = sum_t h(y_t)   (eq. (2)'s f)
// For LOGSUMEXP the row state is (max, sum exp(y - max)).
// ---------------------------------------------------------------------------------------------
template <int F, class T> struct Fn {
    static __device__ __forceinline__ T h(T y, T c) {
        if constexpr (F == F_LINEAR_MEAN) return y;
        else if constexpr (F == F_MEAN_COS) return cos(y);
        else if constexpr (F == F_CALL_MEAN_EXP) return exp(c * y);
        else if constexpr (F == F_GAUSS_NORM2) return y * y;
        else if constexpr (F == F_PDE_INV_SQ) { T r = T(1) / (T(1) + c * y); return r * r; }
        else return y;
    }
    // h'(y) (LOGSUMEXP: exp(y - L) with L = log sum exp(y) passed as `aux`)
    static __device__ __forceinline__ T hprime(T y, T c, T aux) {
        if constexpr (F == F_LINEAR_MEAN) return T(1);
        else if constexpr (F == F_MEAN_COS) return -sin(y);
        else if constexpr (F == F_CALL_MEAN_EXP) return c * exp(c * y);
        else if constexpr (F == F_GAUSS_NORM2) return T(2) * y;
        else if constexpr (F == F_PDE_INV_SQ) { T r = T(1) / (T(1) + c * y); return T(-2) * c * r * r * r; }
        else return exp(y - aux);
    }
};

// float specialisations use the fast single-precision intrinsics where their
// error (a few ulp over the ranges of these integrands) is inside the FP32 tier.
template <> __device__ __forceinline__ float Fn<F_CALL_MEAN_EXP, float>::h(float y, float c) { return __expf(c * y); }
template <> __device__ __forceinline__ float Fn<F_CALL_MEAN_EXP, float>::hprime(float y, float c, float) {
    return c * __expf(c * y);
}
template <> __device__ __forceinline__ float Fn<F_LOGSUMEXP, float>::hprime(float y, float, float aux) {
    return __expf(y - aux);
}

// g(u) and g'(u) in double (tau, params as given)
__device__ __forceinline__ double g_of(int F, double u, double tau, double c, double K) {
    switch (F) {
        case F_LINEAR_MEAN: case F_MEAN_COS: case F_PDE_INV_SQ: return u / tau;
        case F_CALL_MEAN_EXP: return fmax(u / tau - K, 0.0);
        case F_GAUSS_NORM2: return exp(-u / (2.0 * tau));
        default: return u;   // LOGSUMEXP: u already is log sum exp
    }
}
__device__ __forceinline__ double gprime_of(int F, double u, double tau, double c, double K) {
    switch (F) {
        case F_LINEAR_MEAN: case F_MEAN_COS: case F_PDE_INV_SQ: return 1.0 / tau;
        case F_CALL_MEAN_EXP: return (u / tau - K > 0.0) ? 1.0 / tau : 0.0;
        case F_GAUSS_NORM2: return -exp(-u / (2.0 * tau)) / (2.0 * tau);
        default: return 1.0;
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------------------------

// Coarse chain: the weight blocks at levels >= JF that are not expanded by the
// register tree.  Entry e is level lev[e] with n = 2^logn[e] distinct rows.
struct Chain {
    int count;
    int lev[kMaxChain], logn[kMaxChain], tau[kMaxChain], col0[kMaxChain];
    long long tab[kMaxChain];        // table offset of the level's first column
    long long boff[kMaxChain];       // element offset of B_e / F_e inside a shift's area
    int tile0[kMaxChain + 1];        // prefix sums of work tiles (per kernel)
    int split[kMaxChain];            // k-splits (backward grad GEMM)
    long long poff[kMaxChain];       // partial-buffer offsets (backward grad GEMM)
};

template <class T> struct FineArgs {
    const T* tab; long long tab_stride;       // distinct-row table, per shift
    const T* A; int ldA;                      // A (or its padded copy), row stride ldA
    int tau, tau_pad;
    int logn_root;                            // root level JF: n_root = 2^(m-JF)
    int lev_tau[4], lev_col0[4], lev_logn[4];
    long long lev_tab[4];
    const T* B; long long B_stride;           // coarse block products, per shift
    Chain chain;                               // (only count/logn/boff used here)
    int cr, cg_count, reff, r0;
    long long N;
    T* rowpart; T* rowmax;                     // FUSED: [r][cg][N]
    T* P;                                      // MATERIALIZE: [r][N][tau]
    T c0, c1;                                  // integrand parameters
    // backward
    const double* rowsave; const double* upstream; double coef_scale;   // 1/(R_eff N)
    double tau_d, K_d;
    T* Froot;                                  // [r][n_root][tau_pad]
    T* gradpart;                               // [r][group][KF][tau_pad]
    int roots_per_cta, groups, kf_actual;
    int fkind;
};

// ---------------------------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
template <class T>
cudaError_t launch_table(const DevRule& R, T* tab, long long T_tot, int reff, cudaStream_t st);
cudaError_t launch_points_full(const DevRule& R, uint32_t* out, int shift_idx, cudaStream_t st);
cudaError_t launch_points_distinct(const DevRule& R, uint32_t* out, long long T_tot, int shift_idx,
                                   cudaStream_t st);
template <class T>
cudaError_t launch_pad_A(const T* A, T* Ap, int s, int tau, int tau_pad, cudaStream_t st);
template <class T>
cudaError_t launch_coarse_fwd(const T* tab, long long tab_stride, const T* A, int ldA, int tau_pad,
                              const Chain& ch, T* B, long long B_stride, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_fine_fwd(const FineArgs<T>& a, int shape, int F, int mode, dim3 grid, cudaStream_t st);
template <class T>
cudaError_t launch_rows_finalize(const T* rowpart, const T* rowmax, int cg_count, long long N, int reff,
                                 int F, double tau, double c, double K, double* rowsave, T* rowf_out,
                                 double* fpart, int nblk, cudaStream_t st);
cudaError_t launch_est_finalize(const double* fpart, int nblk, int reff, long long N, double* est,
                                cudaStream_t st);
template <class T>
cudaError_t launch_fine_bwd(const FineArgs<T>& a, int shape, int F, dim3 grid, cudaStream_t st);
template <class T>
cudaError_t launch_fold(const T* src, long long src_stride, int logn_src, T* dst, long long dst_stride,
                        int logn_dst, int tau_pad, int reff, cudaStream_t st);
template <class T>
cudaError_t launch_coarse_grad(const T* tab, long long tab_stride, const T* Froot, long long root_stride,
                               const T* Fchain, long long chain_stride, int jf, int tau_pad, const Chain& ch,
                               T* part, int reff, int ntiles, cudaStream_t st);
template <class T>
cudaError_t launch_grad_reduce(const T* gradpart_f, int nfine_part, int kf_width, const int* koff_lev,
                               const int* col0_lev, const int* tau_lev, int jf, const T* part_c,
                               const Chain& ch, int tau, int tau_pad, int s, T* grad, cudaStream_t st);

}  // namespace qmc
