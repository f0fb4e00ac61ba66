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
//
// The fine columns of A (pre-scaled by the integrand's kappa) are staged in
// shared memory once per CTA; the root values S_JF come from one coarse buffer
// and are prefetched a chunk (forward) or a root (backward) ahead.
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
    static __device__ __forceinline__ void lds(const float* p, float (&v)[4]) {
        float4 q = *reinterpret_cast<const float4*>(p); v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[2]) {
        float2 q = __ldg(reinterpret_cast<const float2*>(p)); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void lds(const float* p, float (&v)[2]) {
        float2 q = *reinterpret_cast<const float2*>(p); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <> struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double (&v)[2]) {
        double2 q = __ldg(reinterpret_cast<const double2*>(p)); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void lds(const double* p, double (&v)[2]) {
        double2 q = *reinterpret_cast<const double2*>(p); v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};
template <class T> struct Vec<T, 1> {
    static __device__ __forceinline__ void ld(const T* p, T (&v)[1]) { v[0] = __ldg(p); }
    static __device__ __forceinline__ void lds(const T* p, T (&v)[1]) { v[0] = *p; }
    static __device__ __forceinline__ void st(T* p, const T (&v)[1]) { *p = v[0]; }
};

// root value S_JF[rho] for CW columns from t0 (layout [t/4][row][4]); zero without coarse levels
template <class T, int CW>
__device__ __forceinline__ void load_root(const T* S, int logn_root, long long rho, int t0, T (&v)[CW]) {
    if (S) {
        Vec<T, CW>::ld(S + ((((long long)(t0 >> 2)) << logn_root) << 2) + (rho << 2) + (t0 & 3), v);
    } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = T(0);
    }
}

// Stage kappa * A[col0_I + jj][t_beg + c] for the fine columns into shared memory As[KF][W].
template <class T, class BandT, int W>
__device__ __forceinline__ void stage_A(const FineArgs<T>& a, T* As, int t_beg) {
    constexpr int KF = BandT::KF;
    for (int idx = threadIdx.x; idx < KF * W; idx += blockDim.x) {
        const int j = idx / W, c = idx - j * W;
        int lev = 0;
#pragma unroll
        for (int l = 1; l < BandT::JF; ++l)
            if (j >= BandT::koff(l)) lev = l;
        const int jj = j - BandT::koff(lev);
        const int t = t_beg + c;
        T v = T(0);
        if (jj < a.lev_tau[lev] && t < a.tau_pad) v = a.kappa * a.A[(long long)(a.lev_col0[lev] + jj) * a.ldA + t];
        As[idx] = v;
    }
}

// ------------------------------------------------------------------------------------------
// Forward: one thread per root, x of the whole subtree in registers, a broadcast from smem.
// ------------------------------------------------------------------------------------------
template <class T, class BandT, int F, int MODE, int CW, bool EXACT>
struct FwdThread {
    static constexpr int JF = BandT::JF, NX = BandT::NX, NL = BandT::NL, KF = BandT::KF;
    // a values of levels with at least 8 nodes per root are read once per chunk
    __host__ __device__ static constexpr bool hoisted(int lev) { return BandT::nodes(lev) >= 8; }

    const FineArgs<T>& a;
    const T* As;      // shared: kappa * A fine columns of this CTA's column range, [KF][kMaxCR]
    long long rho;
    int t0, ac, nvalid;
    T x[NX > 0 ? NX : 1];
    T ah[KF > 0 ? KF : 1][CW];
    T racc[NL], rmax[NL];

    __device__ __forceinline__ FwdThread(const FineArgs<T>& args, const T* as, long long rho_)
        : a(args), As(as), rho(rho_) {}

    __device__ __forceinline__ bool has(int lev, int jj) const { return EXACT || jj < a.lev_tau[lev]; }

    __device__ __forceinline__ void load_x(const T* tab) {
#pragma unroll
        for (int lev = 0; lev < JF; ++lev)
#pragma unroll
            for (int c = 0; c < BandT::nodes(lev); ++c)
#pragma unroll
                for (int jj = 0; jj < BandT::K(lev); ++jj) {
                    T v = T(0);
                    if (has(lev, jj))
                        v = __ldg(tab + a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + rho +
                                  ((long long)c << a.logn_root));
                    x[BandT::xoff(lev) + c * BandT::K(lev) + jj] = v;
                }
    }

    __device__ __forceinline__ void load_a(int lev, int jj, T (&av)[CW]) const {
        Vec<T, CW>::lds(As + (BandT::koff(lev) + jj) * kMaxCR + ac, av);
    }

    __device__ __forceinline__ void hoist() {
#pragma unroll
        for (int lev = 0; lev < JF; ++lev)
            if (hoisted(lev))
#pragma unroll
                for (int jj = 0; jj < BandT::K(lev); ++jj) {
                    T av[CW];
                    load_a(lev, jj, av);
#pragma unroll
                    for (int c = 0; c < CW; ++c) ah[BandT::koff(lev) + jj][c] = av[c];
                }
    }

    // FULL: all CW columns of the chunk are < tau (no masking); otherwise only nvalid are.
    template <int C, bool FULL>
    __device__ __forceinline__ void leaf(const T (&v)[CW]) {
        if constexpr (MODE == MODE_MATERIALIZE) {
            const long long k = rho + ((long long)C << a.logn_root);
            T* p = a.P + ((long long)blockIdx.z * a.N + k) * a.tau + t0;
            if (FULL && (a.tau % CW) == 0) {
                Vec<T, CW>::st(p, v);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    if (FULL || c < nvalid) p[c] = v[c];
            }
        } else if constexpr (F == F_LOGSUMEXP) {
            // online log-sum-exp in base 2: state (max, sum 2^(v - max))
            T mx = rmax[C];
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (FULL || c < nvalid) mx = fmax(mx, v[c]);
            T sacc = racc[C] * ex2(rmax[C] - mx);
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (FULL || c < nvalid) sacc += ex2(v[c] - mx);
            racc[C] = sacc;
            rmax[C] = mx;
        } else {
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (FULL || c < nvalid) acc += Fn<F, T>::h(v[c], a.c0);
            racc[C] += acc;
        }
    }

    template <int LEV, int C, bool FULL>
    __device__ __forceinline__ void node(const T (&vp)[CW]) {
        T v[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = vp[c];
#pragma unroll
        for (int jj = 0; jj < BandT::K(LEV); ++jj) {
            if (has(LEV, jj)) {
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
            leaf<C, FULL>(v);
        } else {
            node<LEV - 1, C, FULL>(v);
            node<LEV - 1, C + (1 << (JF - LEV)), FULL>(v);
        }
    }

    template <bool FULL>
    __device__ __forceinline__ void expand(const T (&vroot)[CW]) {
        if constexpr (JF == 0) {
            leaf<0, FULL>(vroot);
        } else {
            node<JF - 1, 0, FULL>(vroot);
            node<JF - 1, 1, FULL>(vroot);
        }
    }
};

template <class T, class BandT, int F, int MODE, int CW, bool EXACT>
__global__ void __launch_bounds__(128, 4) k_fine_fwd(const __grid_constant__ FineArgs<T> a) {
    using Th = FwdThread<T, BandT, F, MODE, CW, EXACT>;
    __shared__ __align__(16) T As[(BandT::KF > 0 ? BandT::KF : 1) * kMaxCR];
    const long long n_root = 1LL << a.logn_root;
    const long long rho = (long long)blockIdx.x * 128 + threadIdx.x;
    const int cg = blockIdx.y, r = blockIdx.z;
    const int t_beg = cg * a.cr;
    const int t_end = min(t_beg + a.cr, a.tau_pad);
    if constexpr (BandT::KF > 0) {
        stage_A<T, BandT, kMaxCR>(a, As, t_beg);
        __syncthreads();
    }
    if (rho >= n_root) return;
    Th th(a, As, rho);
    th.load_x(a.tab + (long long)r * a.tab_stride);
#pragma unroll
    for (int l = 0; l < Th::NL; ++l) {
        th.racc[l] = T(0);
        th.rmax[l] = -INFINITY;
    }
    const T* S = a.S ? a.S + (long long)r * a.S_stride : nullptr;
    T vnext[CW];
    load_root<T, CW>(S, a.logn_root, rho, t_beg, vnext);
    // chunks whose CW columns all lie below tau, then at most one ragged chunk
    const int t_full = max(t_beg, min(t_end, t_beg + ((a.tau - t_beg) / CW) * CW));
    int t0 = t_beg;
    for (; t0 < t_full; t0 += CW) {
        th.t0 = t0;
        th.ac = t0 - t_beg;
        T vroot[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) vroot[c] = a.kappa * vnext[c];
        if (t0 + CW < t_end) load_root<T, CW>(S, a.logn_root, rho, t0 + CW, vnext);
        th.hoist();
        th.template expand<true>(vroot);
    }
    if (t0 < t_end && t0 < a.tau) {
        th.t0 = t0;
        th.ac = t0 - t_beg;
        th.nvalid = a.tau - t0;
        T vroot[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) vroot[c] = a.kappa * vnext[c];
        th.hoist();
        th.template expand<false>(vroot);
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
// broadcast), each lane owns CW columns and holds their fine columns of A in
// registers for every root it visits.  The leaves give G = coef_k h'(y);
// folding G back up the same tree (the adjoint of the periodic tiling) gives at
// every node F = sum of G over its leaves, and the fine-column gradient is
// sum over nodes of x_{node,j} F_node.  The root's F is written for the coarse levels.
// ------------------------------------------------------------------------------------------
template <class T, class BandT, int F, int CW, bool EXACT>
struct BwdLane {
    static constexpr int JF = BandT::JF, NX = BandT::NX, NL = BandT::NL, KF = BandT::KF;
    static constexpr int COLS = 32 * CW;
    const FineArgs<T>& a;
    const T* xs;      // this warp's x values (shared)
    const T* cf;      // coef per leaf
    const T* ax;      // aux per leaf (log2 e * log-sum-exp of the row)
    int nvalid;
    T ah[KF > 0 ? KF : 1][CW];      // kappa * A fine columns of this lane, the same for every root
    T gacc[KF > 0 ? KF : 1][CW];

    __device__ __forceinline__ BwdLane(const FineArgs<T>& args) : a(args) {}

    __device__ __forceinline__ bool has(int lev, int jj) const { return EXACT || jj < a.lev_tau[lev]; }

    __device__ __forceinline__ void load_a(int t0, bool active) {
#pragma unroll
        for (int lev = 0; lev < JF; ++lev)
#pragma unroll
            for (int jj = 0; jj < BandT::K(lev); ++jj) {
                T av[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) av[c] = T(0);
                if (active && has(lev, jj)) Vec<T, CW>::ld(a.A + (long long)(a.lev_col0[lev] + jj) * a.ldA + t0, av);
#pragma unroll
                for (int c = 0; c < CW; ++c) ah[BandT::koff(lev) + jj][c] = a.kappa * av[c];
            }
    }

    template <int C>
    __device__ __forceinline__ void leaf(const T (&v)[CW], T (&Fo)[CW]) {
        const T coef = cf[C], aux = ax[C];
#pragma unroll
        for (int c = 0; c < CW; ++c) Fo[c] = (c < nvalid) ? coef * Fn<F, T>::hp(v[c], a.c0, aux) : T(0);
    }

    template <int LEV, int C>
    __device__ __forceinline__ void node(const T (&vp)[CW], T (&Fp)[CW]) {
        constexpr int K = BandT::K(LEV);
        T xv[K];
#pragma unroll
        for (int jj = 0; jj < K; ++jj) xv[jj] = xs[BandT::xoff(LEV) + C * K + jj];
        T v[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = vp[c];
#pragma unroll
        for (int jj = 0; jj < K; ++jj) {
            if (has(LEV, jj)) {
#pragma unroll
                for (int c = 0; c < CW; ++c) v[c] = fma(xv[jj], ah[BandT::koff(LEV) + jj][c], v[c]);
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
        for (int jj = 0; jj < K; ++jj) {
            if (has(LEV, jj)) {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    gacc[BandT::koff(LEV) + jj][c] = fma(xv[jj], Fn_[c], gacc[BandT::koff(LEV) + jj][c]);
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

template <class T, class BandT, int F, int CW, bool EXACT>
__global__ void __launch_bounds__(256, 2) k_fine_bwd(const __grid_constant__ FineArgs<T> a) {
    using L = BwdLane<T, BandT, F, CW, EXACT>;
    constexpr int NX = BandT::NX, NL = BandT::NL, KF = BandT::KF;
    constexpr int COLS = L::COLS;
    __shared__ T xs[8][NX > 0 ? NX : 1];
    __shared__ T cfs[8][NL];
    __shared__ T axs[8][NL];
    __shared__ T red[KF > 0 ? KF : 1][COLS];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, pass = blockIdx.y, r = blockIdx.z;
    const long long n_root = 1LL << a.logn_root;
    const T* tab = a.tab + (long long)r * a.tab_stride;
    const T* S = a.S ? a.S + (long long)r * a.S_stride : nullptr;
    const int t_pass = pass * COLS;
    const int t0 = t_pass + lane * CW;
    const bool active = t0 < a.tau_pad;
    const T upstream = (T)a.upstream[0];

    L ln(a);
    ln.xs = xs[warp];
    ln.cf = cfs[warp];
    ln.ax = axs[warp];
    ln.nvalid = min(CW, a.tau - t0);
    ln.load_a(t0, active);
#pragma unroll
    for (int j = 0; j < (KF > 0 ? KF : 1); ++j)
#pragma unroll
        for (int c = 0; c < CW; ++c) ln.gacc[j][c] = T(0);

    const long long rho0 = (long long)g * a.roots_per_cta;
    T vnext[CW];
    if (active && rho0 + warp < n_root) load_root<T, CW>(S, a.logn_root, rho0 + warp, t0, vnext);
    for (int i = warp; i < a.roots_per_cta; i += 8) {
        const long long rho = rho0 + i;
        if (rho >= n_root) break;
        for (int idx = lane; idx < NX; idx += 32) {
            int lev, c, jj;
            decode_x<BandT>(idx, lev, c, jj);
            T v = T(0);
            if (EXACT || jj < a.lev_tau[lev])
                v = tab[a.lev_tab[lev] + ((long long)jj << a.lev_logn[lev]) + rho + ((long long)c << a.logn_root)];
            xs[warp][idx] = v;
        }
        if (lane < NL) {
            const long long k = rho + ((long long)lane << a.logn_root);
            cfs[warp][lane] = upstream * a.rowsave[2 * ((long long)r * a.N + k)];
            axs[warp][lane] = a.rowsave[2 * ((long long)r * a.N + k) + 1];
        }
        __syncwarp();
        if (active) {
            T vroot[CW], Froot[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) vroot[c] = a.kappa * vnext[c];
            if (rho + 8 < n_root && i + 8 < a.roots_per_cta) load_root<T, CW>(S, a.logn_root, rho + 8, t0, vnext);
            if (ln.nvalid > 0) {
                ln.expand(vroot, Froot);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c) Froot[c] = T(0);
            }
            Vec<T, CW>::st(a.Froot + ((long long)r * n_root + rho) * a.tau_pad + t0, Froot);
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
            const int t = t_pass + col;
            if (t < a.tau_pad) out[(long long)j * a.tau_pad + t] = red[j][col];
        }
    }
}

}  // namespace qmc
