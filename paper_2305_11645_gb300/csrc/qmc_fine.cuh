// Fine-band kernels: the last JF levels of Algorithm 2 expanded as a binary
// tree in registers, fused with the integrand (forward) or with the folded
// adjoint (backward).
//
// Notation (Sec. 3.2): level I holds the tau_I columns with min(w_j,m) = I,
// each with n_I = 2^(m-I) distinct rows; S_I = tile(S_{I+1}) + X_I A_I.
// A thread (forward) or a warp (backward) owns one root row rho < n_JF of
// S_JF.  The root's descendants are the rows rho + c*n_JF of level I < JF,
// c < 2^(JF-I); the children of node c at level I are c and c + 2^(JF-I) at
// level I-1, and the leaves (level 0) are the output rows k = rho + c*n_JF.
// Every node adds its level's block product x_{row,j} a_j to its parent's
// value, so one root costs sum_I 2^(JF-I) tau_I multiply-adds per column --
// Algorithm 1's count, with no value recomputed and nothing written to memory.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

// Compile-time shape of the fine band: JF levels with at most K(I) columns at level I.
template <int JF_, int K0, int K1, int K2, int K3>
struct Band {
    static constexpr int JF = JF_;
    __host__ __device__ static constexpr int K(int lev) {
        return lev == 0 ? K0 : lev == 1 ? K1 : lev == 2 ? K2 : lev == 3 ? K3 : 0;
    }
    __host__ __device__ static constexpr int nodes(int lev) { return 1 << (JF - lev); }
    __host__ __device__ static constexpr int xoff(int lev) {
        int o = 0;
        for (int i = 0; i < lev; ++i) o += nodes(i) * K(i);
        return o;
    }
    __host__ __device__ static constexpr int koff(int lev) {
        int o = 0;
        for (int i = 0; i < lev; ++i) o += K(i);
        return o;
    }
    static constexpr int NX = xoff(JF);     // x values held per root
    static constexpr int KF = koff(JF);     // fine columns (upper bound)
    static constexpr int NL = 1 << JF;      // leaves per root
};

using BandS0 = Band<0, 0, 0, 0, 0>;
using BandS1 = Band<1, 16, 0, 0, 0>;
using BandS4 = Band<4, 1, 2, 4, 8>;

template <class T, int CW> struct Vec;
template <> struct Vec<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) {
        float4 q = __ldg(reinterpret_cast<const float4*>(p)); v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[2]) {
        float2 q = __ldg(reinterpret_cast<const float2*>(p)); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <> struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double (&v)[2]) {
        double2 q = __ldg(reinterpret_cast<const double2*>(p)); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};
template <class T> struct Vec<T, 1> {
    static __device__ __forceinline__ void ld(const T* p, T (&v)[1]) { v[0] = __ldg(p); }
    static __device__ __forceinline__ void st(T* p, const T (&v)[1]) { *p = v[0]; }
};

// Sum of the coarse block products B_e[rho mod n_e] over the chain: the value
// of the root S_JF[rho] for CW columns starting at t0 (B layout [t/4][row][4]).
template <class T, int CW>
__device__ __forceinline__ void root_value(const FineArgs<T>& a, const T* B, long long rho, int t0, T (&v)[CW]) {
#pragma unroll
    for (int c = 0; c < CW; ++c) v[c] = T(0);
    for (int e = 0; e < a.chain.count; ++e) {
        const long long ne = 1LL << a.chain.logn[e];
        const T* p = B + a.chain.boff[e] + ((((long long)(t0 >> 2)) << a.chain.logn[e]) << 2) +
                     ((rho & (ne - 1)) << 2) + (t0 & 3);
        T u[CW];
        Vec<T, CW>::ld(p, u);
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] += u[c];
    }
}

// ------------------------------------------------------------------------------------------
// Forward: one thread per root, x of the whole subtree in registers, a broadcast.
// ------------------------------------------------------------------------------------------
template <class T, class BandT, int F, int MODE, int CW>
struct FwdThread {
    static constexpr int JF = BandT::JF, NX = BandT::NX, NL = BandT::NL, KF = BandT::KF;
    // a values of levels with at least 4 nodes per root are loaded once per chunk
    __host__ __device__ static constexpr bool hoisted(int lev) { return BandT::nodes(lev) >= 4; }

    const FineArgs<T>& a;
    long long rho;
    int t0, nvalid;
    T x[NX > 0 ? NX : 1];
    T ah[KF > 0 ? KF : 1][CW];
    T racc[NL], rmax[NL];

    __device__ __forceinline__ FwdThread(const FineArgs<T>& args, long long rho_) : a(args), rho(rho_) {}

    __device__ __forceinline__ void load_x(const T* tab) {
#pragma unroll
        for (int lev = 0; lev < JF; ++lev)
#pragma unroll
            for (int c = 0; c < BandT::nodes(lev); ++c)
#pragma unroll
                for (int jj = 0; jj < BandT::K(lev); ++jj) {
                    T v = T(0);
                    if (jj < a.lev_tau[lev])
                        v = __ldg(tab + a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + rho +
                                  ((long long)c << a.logn_root));
                    x[BandT::xoff(lev) + c * BandT::K(lev) + jj] = v;
                }
    }

    __device__ __forceinline__ void load_a(int lev, int jj, T (&av)[CW]) const {
        Vec<T, CW>::ld(a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA + t0, av);
    }

    __device__ __forceinline__ void hoist() {
#pragma unroll
        for (int lev = 0; lev < JF; ++lev)
            if (hoisted(lev))
#pragma unroll
                for (int jj = 0; jj < BandT::K(lev); ++jj) {
                    T av[CW];
                    if (jj < a.lev_tau[lev]) load_a(lev, jj, av);
                    else {
#pragma unroll
                        for (int c = 0; c < CW; ++c) av[c] = T(0);
                    }
#pragma unroll
                    for (int c = 0; c < CW; ++c) ah[BandT::koff(lev) + jj][c] = av[c];
                }
    }

    template <int C>
    __device__ __forceinline__ void leaf(const T (&v)[CW]) {
        if constexpr (MODE == MODE_MATERIALIZE) {
            const long long k = rho + ((long long)C << a.logn_root);
            T* p = a.P + ((long long)blockIdx.z * a.N + k) * a.tau + t0;
            if (nvalid == CW && (a.tau % CW) == 0) {
                Vec<T, CW>::st(p, v);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    if (c < nvalid) p[c] = v[c];
            }
        } else if constexpr (F == F_LOGSUMEXP) {
            T mx = rmax[C];
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c < nvalid) mx = fmax(mx, v[c]);
            T sacc = racc[C] * Fn<F_CALL_MEAN_EXP, T>::h(rmax[C] - mx, T(1));
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c < nvalid) sacc += Fn<F_CALL_MEAN_EXP, T>::h(v[c] - mx, T(1));
            racc[C] = sacc;
            rmax[C] = mx;
        } else {
            T acc = T(0);
            if (nvalid == CW) {
#pragma unroll
                for (int c = 0; c < CW; ++c) acc += Fn<F, T>::h(v[c], a.c0);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    if (c < nvalid) acc += Fn<F, T>::h(v[c], a.c0);
            }
            racc[C] += acc;
        }
    }

    template <int LEV, int C>
    __device__ __forceinline__ void node(const T (&vp)[CW]) {
        T v[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = vp[c];
#pragma unroll
        for (int jj = 0; jj < BandT::K(LEV); ++jj) {
            if (jj < a.lev_tau[LEV]) {
                T av[CW];
                if constexpr (hoisted(LEV)) {
#pragma unroll
                    for (int c = 0; c < CW; ++c) av[c] = ah[BandT::koff(LEV) + jj][c];
                } else {
                    load_a(LEV, jj, av);
                }
                const T xv = x[BandT::xoff(LEV) + C * BandT::K(LEV) + jj];
#pragma unroll
                for (int c = 0; c < CW; ++c) v[c] = fma(xv, av[c], v[c]);
            }
        }
        if constexpr (LEV == 0) {
            leaf<C>(v);
        } else {
            node<LEV - 1, C>(v);
            node<LEV - 1, C + (1 << (JF - LEV))>(v);
        }
    }

    __device__ __forceinline__ void expand(const T (&vroot)[CW]) {
        if constexpr (JF == 0) {
            leaf<0>(vroot);
        } else {
            node<JF - 1, 0>(vroot);
            node<JF - 1, 1>(vroot);
        }
    }
};

template <class T, class BandT, int F, int MODE, int CW>
__global__ void __launch_bounds__(128) k_fine_fwd(const __grid_constant__ FineArgs<T> a) {
    using Th = FwdThread<T, BandT, F, MODE, CW>;
    const long long n_root = 1LL << a.logn_root;
    const long long rho = (long long)blockIdx.x * 128 + threadIdx.x;
    if (rho >= n_root) return;
    const int cg = blockIdx.y, r = blockIdx.z;
    Th th(a, rho);
    th.load_x(a.tab + (long long)r * a.tab_stride);
#pragma unroll
    for (int l = 0; l < Th::NL; ++l) {
        th.racc[l] = T(0);
        th.rmax[l] = -INFINITY;
    }
    const T* B = a.B ? a.B + (long long)r * a.B_stride : nullptr;
    const int t_beg = cg * a.cr;
    const int t_end = min(t_beg + a.cr, a.tau_pad);
    for (int t0 = t_beg; t0 < t_end; t0 += CW) {
        th.t0 = t0;
        th.nvalid = min(CW, a.tau - t0);
        if (th.nvalid <= 0) break;
        T vroot[CW];
        if (B) root_value<T, CW>(a, B, rho, t0, vroot);
        else {
#pragma unroll
            for (int c = 0; c < CW; ++c) vroot[c] = T(0);
        }
        th.hoist();
        th.expand(vroot);
    }
    if constexpr (MODE == MODE_FUSED) {
#pragma unroll
        for (int l = 0; l < Th::NL; ++l) {
            const long long k = rho + ((long long)l << a.logn_root);
            const long long o = ((long long)r * a.cg_count + cg) * a.N + k;
            a.rowpart[o] = th.racc[l];
            if constexpr (F == F_LOGSUMEXP) a.rowmax[o] = th.rmax[l];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Backward: one warp per root (x and the per-leaf coefficients in shared memory,
// broadcast), each lane owns CW columns.  The leaves give G = coef_k h'(y);
// folding G back up the same tree (the adjoint of the periodic tiling) gives at
// every node F = sum of G over its leaves, and the fine-column gradient is
// sum over nodes of x_{node,j} F_node.  The root's F is written for the coarse levels.
// ------------------------------------------------------------------------------------------
template <class T, class BandT, int F, int CW>
struct BwdLane {
    static constexpr int JF = BandT::JF, NX = BandT::NX, NL = BandT::NL, KF = BandT::KF;
    const FineArgs<T>& a;
    const T* xs;      // this warp's x values (shared)
    const T* cf;      // coef per leaf
    const T* ax;      // aux per leaf (log-sum-exp of the row)
    int t0, nvalid;
    T gacc[KF > 0 ? KF : 1][CW];

    __device__ __forceinline__ BwdLane(const FineArgs<T>& args) : a(args) {}

    template <int C>
    __device__ __forceinline__ void leaf(const T (&v)[CW], T (&Fo)[CW]) {
        const T coef = cf[C], aux = ax[C];
#pragma unroll
        for (int c = 0; c < CW; ++c) Fo[c] = (c < nvalid) ? coef * Fn<F, T>::hprime(v[c], a.c0, aux) : T(0);
    }

    template <int LEV, int C>
    __device__ __forceinline__ void node(const T (&vp)[CW], T (&Fp)[CW]) {
        T v[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = vp[c];
#pragma unroll
        for (int jj = 0; jj < BandT::K(LEV); ++jj) {
            if (jj < a.lev_tau[LEV]) {
                T av[CW];
                Vec<T, CW>::ld(a.A + (long long)(a.lev_col0[LEV] + jj) * a.ldA + t0, av);
                const T xv = xs[BandT::xoff(LEV) + C * BandT::K(LEV) + jj];
#pragma unroll
                for (int c = 0; c < CW; ++c) v[c] = fma(xv, av[c], v[c]);
            }
        }
        T Fn_[CW];
        if constexpr (LEV == 0) {
            leaf<C>(v, Fn_);
        } else {
#pragma unroll
            for (int c = 0; c < CW; ++c) Fn_[c] = T(0);
            node<LEV - 1, C>(v, Fn_);
            node<LEV - 1, C + (1 << (JF - LEV))>(v, Fn_);
        }
#pragma unroll
        for (int jj = 0; jj < BandT::K(LEV); ++jj) {
            if (jj < a.lev_tau[LEV]) {
                const T xv = xs[BandT::xoff(LEV) + C * BandT::K(LEV) + jj];
#pragma unroll
                for (int c = 0; c < CW; ++c) gacc[BandT::koff(LEV) + jj][c] = fma(xv, Fn_[c], gacc[BandT::koff(LEV) + jj][c]);
            }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) Fp[c] += Fn_[c];
    }

    __device__ __forceinline__ void expand(const T (&vroot)[CW], T (&Froot)[CW]) {
#pragma unroll
        for (int c = 0; c < CW; ++c) Froot[c] = T(0);
        if constexpr (JF == 0) {
            leaf<0>(vroot, Froot);
        } else {
            node<JF - 1, 0>(vroot, Froot);
            node<JF - 1, 1>(vroot, Froot);
        }
    }
};

// decode x index -> (lev, node, column) with the band's compile-time layout
template <class BandT>
__device__ __forceinline__ void decode_x(int idx, int& lev, int& c, int& jj) {
    lev = 0;
#pragma unroll
    for (int l = 1; l < BandT::JF; ++l)
        if (idx >= BandT::xoff(l)) lev = l;
    int off = 0, K = 1;
#pragma unroll
    for (int l = 0; l < BandT::JF; ++l)
        if (l == lev) { off = BandT::xoff(l); K = BandT::K(l); }
    const int rel = idx - off;
    c = rel / K;
    jj = rel - c * K;
}

template <class T, class BandT, int F, int CW>
__global__ void __launch_bounds__(256) k_fine_bwd(const __grid_constant__ FineArgs<T> a) {
    using L = BwdLane<T, BandT, F, CW>;
    constexpr int NX = BandT::NX, NL = BandT::NL, KF = BandT::KF, JF = BandT::JF;
    constexpr int COLS = 32 * CW;
    __shared__ T xs[8][NX > 0 ? NX : 1];
    __shared__ T cfs[8][NL];
    __shared__ T axs[8][NL];
    __shared__ T red[KF > 0 ? KF : 1][COLS];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, pass = blockIdx.y, r = blockIdx.z;
    const long long n_root = 1LL << a.logn_root;
    const T* tab = a.tab + (long long)r * a.tab_stride;
    const T* B = a.B ? a.B + (long long)r * a.B_stride : nullptr;
    const int t0 = pass * COLS + lane * CW;
    const bool active = t0 < a.tau_pad;
    const double upstream = a.upstream[0];

    L ln(a);
    ln.xs = xs[warp];
    ln.cf = cfs[warp];
    ln.ax = axs[warp];
    ln.t0 = t0;
    ln.nvalid = min(CW, a.tau - t0);
#pragma unroll
    for (int j = 0; j < (KF > 0 ? KF : 1); ++j)
#pragma unroll
        for (int c = 0; c < CW; ++c) ln.gacc[j][c] = T(0);

    for (int i = warp; i < a.roots_per_cta; i += 8) {
        const long long rho = (long long)g * a.roots_per_cta + i;
        if (rho >= n_root) break;
        for (int idx = lane; idx < NX; idx += 32) {
            int lev, c, jj;
            decode_x<BandT>(idx, lev, c, jj);
            T v = T(0);
            if (jj < a.lev_tau[lev])
                v = tab[a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + rho + ((long long)c << a.logn_root)];
            xs[warp][idx] = v;
        }
        if (lane < NL) {
            const long long k = rho + ((long long)lane << a.logn_root);
            const double u = a.rowsave[(long long)r * a.N + k];
            cfs[warp][lane] = (T)(upstream * gprime_of(F, u, a.tau_d, (double)a.c0, a.K_d) * a.coef_scale);
            axs[warp][lane] = (T)u;
        }
        __syncwarp();
        if (active && ln.nvalid > 0) {
            T vroot[CW], Froot[CW];
            if (B) root_value<T, CW>(a, B, rho, t0, vroot);
            else {
#pragma unroll
                for (int c = 0; c < CW; ++c) vroot[c] = T(0);
            }
            ln.expand(vroot, Froot);
            Vec<T, CW>::st(a.Froot + ((long long)r * n_root + rho) * a.tau_pad + t0, Froot);
        } else if (active) {
            T z[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) z[c] = T(0);
            Vec<T, CW>::st(a.Froot + ((long long)r * n_root + rho) * a.tau_pad + t0, z);
        }
        __syncwarp();
    }

    if constexpr (KF > 0) {
        // fixed-order reduction of the per-warp gradient partials
        for (int w = 0; w < 8; ++w) {
            if (warp == w) {
#pragma unroll
                for (int j = 0; j < KF; ++j)
#pragma unroll
                    for (int c = 0; c < CW; ++c)
                        red[j][lane * CW + c] = (w == 0 ? T(0) : red[j][lane * CW + c]) + ln.gacc[j][c];
            }
            __syncthreads();
        }
        T* out = a.gradpart + ((long long)r * a.groups + g) * KF * a.tau_pad;
        for (int idx = threadIdx.x; idx < KF * COLS; idx += blockDim.x) {
            const int j = idx / COLS, col = idx - j * COLS;
            const int t = pass * COLS + col;
            if (t < a.tau_pad) out[(long long)j * a.tau_pad + t] = red[j][col];
        }
    }
    (void)JF;
}

}  // namespace qmc
