// Coarse-level kernels and reductions.
//
//  k_coarse_fwd    B_e = X_e A_e for every coarse weight block e (Algorithm 2's
//                  X~_I A~_I on the b^(m-I) distinct rows only), all blocks and
//                  shifts in one launch.  The fine kernels add B_e[k mod n_e]
//                  periodically (the tiling of Algorithm 2).
//  k_rows_finalize f(x_k^T A) = g(u_k) per row from the column-group partials,
//                  and fixed-order block sums of f for the mean (eq. (2)).
//                  The last block to finish forms Q_r = N^-1 sum_k f and the
//                  mean over shifts.
//  k_fold_tree     the root gradients (or, after the fused adjoint, the fold it
//                  wrote) folded level by level onto the distinct rows of every
//                  coarse level.
//  k_chain_sum     S_JF[rho] = sum_e B_e[rho mod n_e]: the root values of the
//                  fine band (Algorithm 2's tiling of the coarse levels).
//  k_coarse_grad   dA_e = sum_r X_{r,e}^T F_{r,e}, with F_e[rho] = sum_q
//                  F_JF[rho + q n_e] folded on the fly from the root gradients
//                  (the adjoint of the periodic tiling), split over K = R n_e.
//  k_grad_reduce   fixed-order sum of all gradient partials into dA.
#include "qmc_internal.cuh"
#include "qmc_finalize.cuh"

namespace qmc {

__device__ __forceinline__ int chain_entry(const Chain& ch, int bx) {
    int e = 0;
    while (e + 1 < ch.count && bx >= ch.tile0[e + 1]) ++e;
    return e;
}

// ------------------------------------------------------------------------------------------
// B_e[r][t/4][rho][t%4] = sum_{jj < tau_e} tab[r][tab_e + jj n_e + rho] * A[col0_e + jj][t]
// 64 x 64 output tile per CTA, 16-deep K steps staged in shared memory.
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_coarse_fwd(const T* __restrict__ tab, long long tab_stride,
                                                    const T* __restrict__ A, int ldA, int tau_pad,
                                                    const __grid_constant__ Chain ch, T* __restrict__ B,
                                                    long long B_stride) {
    __shared__ T Xs[16][64];
    __shared__ T As[16][64];
    const int e = chain_entry(ch, blockIdx.x);
    const int mt = blockIdx.x - ch.tile0[e];
    const int logn = ch.logn[e], tau_e = ch.tau[e];
    const long long n_e = 1LL << logn;
    const long long rho0 = (long long)mt * 64;
    const int t0 = blockIdx.y * 64;
    const int r = blockIdx.z;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const T* tabr = tab + (long long)r * tab_stride + ch.tab[e];

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = T(0);

    for (int k0 = 0; k0 < tau_e; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + 256 * q, kk = idx >> 6, rr = idx & 63;
            const bool kv = (k0 + kk) < tau_e;
            Xs[kk][rr] = (kv && rho0 + rr < n_e) ? tabr[(long long)(k0 + kk) * n_e + rho0 + rr] : T(0);
            As[kk][rr] = (kv && t0 + rr < tau_pad) ? A[(long long)(ch.col0[e] + k0 + kk) * ldA + t0 + rr] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T xv[4], av[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][tx + 16 * i];
#pragma unroll
            for (int c = 0; c < 4; ++c) av[c] = As[kk][4 * ty + c];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][c] = fma(xv[i], av[c], acc[i][c]);
        }
        __syncthreads();
    }
    const int t = t0 + 4 * ty;
    if (t >= tau_pad) return;
    T* Br = B + (long long)r * B_stride + ch.boff[e] + (((long long)(t >> 2) << logn) << 2);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long rho = rho0 + tx + 16 * i;
        if (rho < n_e) {
#pragma unroll
            for (int c = 0; c < 4; ++c) Br[(rho << 2) + c] = acc[i][c];
        }
    }
}

template <class T>
cudaError_t launch_coarse_fwd(const T* tab, long long tab_stride, const T* A, int ldA, int tau_pad,
                              const Chain& ch, T* B, long long B_stride, int reff, cudaStream_t st) {
    if (ch.count == 0) return cudaSuccess;
    dim3 grid(ch.tile0[ch.count], (tau_pad + 63) / 64, reff);
    k_coarse_fwd<T><<<grid, 256, 0, st>>>(tab, tab_stride, A, ldA, tau_pad, ch, B, B_stride);
    return cudaGetLastError();
}
template cudaError_t launch_coarse_fwd<float>(const float*, long long, const float*, int, int, const Chain&,
                                              float*, long long, int, cudaStream_t);
template cudaError_t launch_coarse_fwd<double>(const double*, long long, const double*, int, int, const Chain&,
                                               double*, long long, int, cudaStream_t);

// S[r][t/4][rho][t%4] = sum_e B_e[r][t/4][rho mod n_e][t%4], rho < n_root (Algorithm 2's
// periodic tiling of the coarse block products onto the root rows).
// A thread owns one group of four columns and the 2^D root rows rho' + q n_top of the subtree
// of node rho' < n_top = n_root / 2^D.  An entry of level JF + d (n_e = n_root / 2^d) has
// 2^(D-d) distinct rows among the thread's 2^D (root row q uses row q mod 2^(D-d)) and one row
// for d >= D, so every distinct block row is loaded once per thread, not once per root row.
// The entries at or above the subtree's top go into one sum (batches of 8 loads, all issued
// before their adds), which every root row adds at the end; the first batch's loads are in
// flight while the entries below the top (the chain's first ones: it comes in ascending level
// order) add their rows into the root rows.  Consecutive threads take consecutive rho', so
// every load and store of a warp is contiguous.
template <class T> struct V4 { T x, y, z, w; };

template <class T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        return {v.x, v.y, v.z, v.w};
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        return {a.x, a.y, b.x, b.y};
    }
}
template <class T>
__device__ __forceinline__ void st4(T* p, const V4<T>& v) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
        reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
    }
}
template <class T>
__device__ __forceinline__ void add4(V4<T>& a, const V4<T>& b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }

template <class T, int D>
__global__ void __launch_bounds__(128) k_chain_sum(const T* __restrict__ B, long long B_stride,
                                                   const __grid_constant__ Chain ch, T* __restrict__ S,
                                                   long long S_stride, int logn_root, int tau_pad) {
    constexpr int NQ = 1 << D;
    const int logn_top = logn_root - D;
    const long long rho = (long long)blockIdx.x * 128 + threadIdx.x;
    const long long t4 = blockIdx.y;
    const int r = blockIdx.z;
    if (rho >= (1LL << logn_top)) return;
    const T* Br = B + (long long)r * B_stride;
    const V4<T> zero = {T(0), T(0), T(0), T(0)};
    auto ent = [&](int e, long long row) { return ld4<T>(Br + ch.boff[e] + ((t4 << ch.logn[e]) << 2) + (row << 2)); };
    auto is_top = [&](int e) { return logn_root - ch.logn[e] >= D; };
    // up to 8 entries at or above the top, from the last one down (their rows rho' mod n_e)
    V4<T> w[8];
    int e = ch.count - 1;
    auto batch = [&]() {
        int n = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ei = e - i;
            const bool on = ei >= 0 && is_top(ei);
            w[i] = on ? ent(ei, rho & ((1LL << ch.logn[ei]) - 1)) : zero;
            n += on ? 1 : 0;
        }
        return n;
    };
    int n = batch();
    // the entries below the top, level JF + d for d = 0 .. D - 1: rows rho' + q n_top, q < 2^(D-d)
    V4<T> v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = zero;
    int f = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        for (; f < ch.count && logn_root - ch.logn[f] == d; ++f) {
            V4<T> x[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < (1 << (D - d))) x[q] = ent(f, rho + ((long long)q << logn_top));
#pragma unroll
            for (int q = 0; q < NQ; ++q) add4(v[q], x[q & ((1 << (D - d)) - 1)]);
        }
    }
    V4<T> top = zero;
    for (;;) {
#pragma unroll
        for (int i = 0; i < 8; ++i) add4(top, w[i]);
        e -= n;
        if (n < 8 || e < 0 || !is_top(e)) break;
        n = batch();
    }
    T* o = S + (long long)r * S_stride + ((t4 << logn_root) << 2) + (rho << 2);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        add4(v[q], top);
        st4<T>(o + ((long long)q << logn_top << 2), v[q]);
    }
}

template <class T>
cudaError_t launch_chain_sum(const T* B, long long B_stride, const Chain& ch, T* S, long long S_stride, int logn_root,
                             int tau_pad, int reff, cudaStream_t st) {
    // 2^D groups of 4 values per thread in registers: the deepest subtree that still leaves
    // about 512 threads per SM to hide the loads' latency, at most 8 rows (at 16 the registers
    // allow 4 CTAs per SM: the 2^20 x 1024, 16-shift sum took 3.11 ms against 2.58 at 8)
    constexpr int DMAX = 3;
    int D = logn_root < DMAX ? logn_root : DMAX;
    while (D > 0 && ((1LL << (logn_root - D)) * (tau_pad / 4) * reff) < 152LL * 512) --D;
    const long long n_top = 1LL << (logn_root - D);
    dim3 grid((unsigned)((n_top + 127) / 128), (unsigned)(tau_pad / 4), (unsigned)reff);
    switch (D) {
        case 0: k_chain_sum<T, 0><<<grid, 128, 0, st>>>(B, B_stride, ch, S, S_stride, logn_root, tau_pad); break;
        case 1: k_chain_sum<T, 1><<<grid, 128, 0, st>>>(B, B_stride, ch, S, S_stride, logn_root, tau_pad); break;
        case 2: k_chain_sum<T, 2><<<grid, 128, 0, st>>>(B, B_stride, ch, S, S_stride, logn_root, tau_pad); break;
        case 3: k_chain_sum<T, 3><<<grid, 128, 0, st>>>(B, B_stride, ch, S, S_stride, logn_root, tau_pad); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template cudaError_t launch_chain_sum<float>(const float*, long long, const Chain&, float*, long long, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_chain_sum<double>(const double*, long long, const Chain&, double*, long long, int, int,
                                              int, cudaStream_t);

// ------------------------------------------------------------------------------------------
// row finalisation and the mean
// ------------------------------------------------------------------------------------------
// A CTA of 256 threads takes rpt rows per thread (consecutive threads, consecutive rows), so
// that large problems run in a few waves instead of one CTA per 256 rows; with rpt > 1 rows are
// taken two at a time, the loads of both rows' partials issued before their sums.
template <class T>
__global__ void __launch_bounds__(256) k_rows_finalize(const T* __restrict__ rowpart, const T* __restrict__ rowmax,
                                                       int cg_count, long long N, int F, double tau, double c,
                                                       double K, double coef_scale, T* __restrict__ rowsave,
                                                       T* __restrict__ rowf, double* __restrict__ fpart, int nblk,
                                                       int rpt, unsigned int* ticket, double* __restrict__ est) {
    // Per-row arithmetic in T (the row sums are T partials).  The CTA's rows are summed with
    // warp shuffles in T and the warp sums in double; the mean over the CTAs is in double.
    __shared__ double sh[32];
    const int r = blockIdx.y;
    const T inv_tau = (T)(1.0 / tau);
    const T* rp0 = rowpart + (long long)r * cg_count * N;
    const T* rm0 = rowmax ? rowmax + (long long)r * cg_count * N : nullptr;
    T fsum = T(0);
    if (rpt == 1) {
        // one row per thread (problems of up to about four waves)
        const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (k < N) {
            T u;
            if (F == F_LOGSUMEXP) {
                T M = -INFINITY;
#pragma unroll 8
                for (int g = 0; g < cg_count; ++g) M = fmax(M, rm0[(long long)g * N + k]);
                T S = T(0);
#pragma unroll 8
                for (int g = 0; g < cg_count; ++g) S += rp0[(long long)g * N + k] * exp2(rm0[(long long)g * N + k] - M);
                u = lse_row(M, S);
            } else {
                u = T(0);
#pragma unroll 8
                for (int g = 0; g < cg_count; ++g) u += rp0[(long long)g * N + k];
            }
            fsum = finalize_row<T>(F, u, inv_tau, tau, K, coef_scale, rowsave, rowf, (long long)r * N + k);
        }
    }
    for (int i = 0; rpt > 1 && i < rpt; i += 2) {
        const long long k0 = ((long long)blockIdx.x * rpt + i) * blockDim.x + threadIdx.x;
        const long long k1 = k0 + blockDim.x;
        const bool on0 = k0 < N, on1 = i + 1 < rpt && k1 < N;
        if (!on0) break;
        T u0, u1 = T(0);
        if (F == F_LOGSUMEXP) {
            // the partials hold (max, sum 2^(v - max)) of v = y log2 e
            T M0 = -INFINITY, M1 = -INFINITY;
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) {
                M0 = fmax(M0, rm0[(long long)g * N + k0]);
                if (on1) M1 = fmax(M1, rm0[(long long)g * N + k1]);
            }
            T S0 = T(0), S1 = T(0);
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) {
                S0 += rp0[(long long)g * N + k0] * exp2(rm0[(long long)g * N + k0] - M0);
                if (on1) S1 += rp0[(long long)g * N + k1] * exp2(rm0[(long long)g * N + k1] - M1);
            }
            u0 = lse_row(M0, S0);
            if (on1) u1 = lse_row(M1, S1);
        } else {
            u0 = T(0);
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) {
                u0 += rp0[(long long)g * N + k0];
                if (on1) u1 += rp0[(long long)g * N + k1];
            }
        }
        fsum += finalize_row<T>(F, u0, inv_tau, tau, K, coef_scale, rowsave, rowf, (long long)r * N + k0);
        if (on1) fsum += finalize_row<T>(F, u1, inv_tau, tau, K, coef_scale, rowsave, rowf, (long long)r * N + k1);
    }
    const double s = block_sum_t<T>(fsum, sh);
    finalize_estimate(s, r, blockIdx.x, nblk, gridDim.y, N, gridDim.x * gridDim.y, ticket, fpart, est, sh);
}

template <class T>
cudaError_t launch_rows_finalize(const T* rowpart, const T* rowmax, int cg_count, long long N, int reff, int F,
                                 double tau, double c, double K, double coef_scale, T* rowsave, T* rowf_out,
                                 double* fpart, int nblk, unsigned int* ticket, double* est, cudaStream_t st) {
    if (nblk < 1) return cudaErrorInvalidValue;
    const long long rpt = (N + 256LL * nblk - 1) / (256LL * nblk);       // rows per thread
    dim3 grid(nblk, reff);
    k_rows_finalize<T><<<grid, 256, 0, st>>>(rowpart, rowmax, cg_count, N, F, tau, c, K, coef_scale, rowsave,
                                             rowf_out, fpart, nblk, (int)rpt, ticket, est);
    return cudaGetLastError();
}
template cudaError_t launch_rows_finalize<float>(const float*, const float*, int, long long, int, int, double, double,
                                                 double, double, float*, float*, double*, int, unsigned int*, double*,
                                                 cudaStream_t);
template cudaError_t launch_rows_finalize<double>(const double*, const double*, int, long long, int, int, double,
                                                  double, double, double, double*, double*, double*, int, unsigned int*,
                                                  double*, cudaStream_t);

// ------------------------------------------------------------------------------------------
// backward: folds, coarse gradient GEMMs, final reduction
// ------------------------------------------------------------------------------------------
// part[e][split][jj][t] = sum over (r, rho) in the split of tab[r][tab_e + jj n_e + rho] * F_e[r][rho][t]
// CTA: 8 warps x 32 lanes x 4 columns; the warps share a 16-column j tile and
// interleave the K range independently (each row's x values are warp-uniform
// loads, two rows in flight per iteration), and the eight warp partials are
// summed in a fixed order at the end.
template <class T>
__device__ __forceinline__ void fold_row(const T* fp, long long fold, long long rstep, T (&fv)[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) fv[c] = fp[c];
    for (long long q = 1; q < fold; ++q) {
        const T* f4 = fp + q * rstep;
#pragma unroll
        for (int c = 0; c < 4; ++c) fv[c] += f4[c];
    }
}

template <class T>
__global__ void __launch_bounds__(256, 2) k_coarse_grad(const T* __restrict__ tab, long long tab_stride,
                                                     const T* __restrict__ Froot, long long root_stride,
                                                     const T* __restrict__ Fchain, long long chain_stride,
                                                     int tau_pad, const __grid_constant__ Chain ch,
                                                     T* __restrict__ part, int reff) {
    __shared__ T red[16][128];
    const int e = chain_entry(ch, blockIdx.x);
    const int local = blockIdx.x - ch.tile0[e];
    const int tau_e = ch.tau[e], logn = ch.logn[e], nsplit = ch.split[e];
    const int jt = local / nsplit, sp = local - jt * nsplit;
    const int j0 = jt * 16;
    const long long n_e = 1LL << logn;
    const long long fold = 1LL << ch.flog[e];
    const T* Froot_e = (ch.fsel[e] ? Fchain : Froot) + ch.foff[e];
    const long long F_stride = ch.fsel[e] ? chain_stride : root_stride;
    const long long Ktot = (long long)reff * n_e;
    const long long kper = (Ktot + nsplit - 1) / nsplit;
    const long long kb = (long long)sp * kper, ke = min(Ktot, kb + kper);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.y * 128 + lane * 4;
    const bool active = t < tau_pad;

    T acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[j][c] = T(0);

    // each warp takes a contiguous share of the K range; 32 rows of x at a time are loaded
    // coalesced (lane = row) into the warp's own shared-memory slice
    __shared__ __align__(16) T xw[8][16][32];      // [warp][column][row]: conflict-free row stores
    const long long wper = (ke - kb + 7) / 8;
    const long long wb = kb + warp * wper, we = min(ke, wb + wper);
    const long long rstep = n_e * tau_pad;
    const T* tab_e = tab + ch.tab[e] + (long long)j0 * n_e;      // column j0, row 0, shift 0
    const int jn = min(16, tau_e - j0);
    for (long long k0 = wb; k0 < we; k0 += 32) {
        {
            const long long k = k0 + lane;
            const long long r = k >> logn, rho = k & (n_e - 1);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
                xw[warp][jj][lane] = (k < we && jj < jn) ? __ldg(tab_e + r * tab_stride + (long long)jj * n_e + rho) : T(0);
        }
        __syncwarp();
        if (active) {
            const int kn = (int)min((long long)32, we - k0);
            for (int i = 0; i < kn; i += 2) {
                const long long ka = k0 + i, kb2 = ka + 1;
                const bool has_b = i + 1 < kn;
                T fa[4], fb[4];
                fold_row<T>(Froot_e + (ka >> logn) * F_stride + (ka & (n_e - 1)) * tau_pad + t, fold, rstep, fa);
                if (has_b) {
                    fold_row<T>(Froot_e + (kb2 >> logn) * F_stride + (kb2 & (n_e - 1)) * tau_pad + t, fold, rstep, fb);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) fb[c] = T(0);
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const T xa = xw[warp][jj][i];
                    const T xb = xw[warp][jj][i + 1 < 32 ? i + 1 : i];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[jj][c] = fma(xb, fb[c], fma(xa, fa[c], acc[jj][c]));
                }
            }
        }
        __syncwarp();
    }
    for (int w = 0; w < 8; ++w) {
        if (warp == w) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
#pragma unroll
                for (int c = 0; c < 4; ++c) red[jj][lane * 4 + c] = (w == 0 ? T(0) : red[jj][lane * 4 + c]) + acc[jj][c];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < 16 * 128; idx += 256) {
        const int jj = idx >> 7, col = idx & 127;
        const int tt = blockIdx.y * 128 + col;
        if (j0 + jj < tau_e && tt < tau_pad)
            part[ch.poff[e] + ((long long)sp * tau_e + j0 + jj) * tau_pad + tt] = red[jj][col];
    }
}

template <class T>
cudaError_t launch_coarse_grad(const T* tab, long long tab_stride, const T* Froot, long long root_stride,
                               const T* Fchain, long long chain_stride, int tau_pad, const Chain& ch, T* part,
                               int reff, int ntiles, cudaStream_t st) {
    if (ch.count == 0) return cudaSuccess;
    dim3 grid(ntiles, (tau_pad + 127) / 128);
    k_coarse_grad<T><<<grid, 256, 0, st>>>(tab, tab_stride, Froot, root_stride, Fchain, chain_stride, tau_pad, ch,
                                           part, reff);
    return cudaGetLastError();
}
template cudaError_t launch_coarse_grad<float>(const float*, long long, const float*, long long, const float*,
                                               long long, int, const Chain&, float*, int, int, cudaStream_t);
template cudaError_t launch_coarse_grad<double>(const double*, long long, const double*, long long, const double*,
                                                long long, int, const Chain&, double*, int, int, cudaStream_t);

// Hierarchical fold of the root gradients (the adjoint of Algorithm 2's tiling):
// F_{I+1}[rho] = F_I[rho] + F_I[rho + n_{I+1}].  A thread owns one column t and one top
// node rho' < n_top of level JF+D: it loads the 2^D root rows rho' + q n_top of its subtree
// (coalesced over the warp's consecutive columns, all loads in flight at once), folds them
// level by level in registers and writes the folded rows of every wanted level.
// one level of the fold, d = 1..D (a compile-time recursion keeps every index static)
template <class T, int D, int d>
struct FoldStep {
    static __device__ __forceinline__ void run(T (&v)[1 << D], T* Fchain, const FoldLevels& fl, long long base,
                                               long long rstep) {
        constexpr int half = 1 << (D - d);
        T* dst = Fchain + fl.off[d] + base;
        const bool want = fl.want[d] != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            v[q] += v[q + half];
            if (want) dst[q * rstep] = v[q];
        }
        FoldStep<T, D, d + 1>::run(v, Fchain, fl, base, rstep);
    }
};
template <class T, int D>
struct FoldStep<T, D, D + 1> {
    static __device__ __forceinline__ void run(T (&)[1 << D], T*, const FoldLevels&, long long, long long) {}
};

template <class T, int D>
__global__ void __launch_bounds__(128) k_fold_tree(const T* __restrict__ Froot, long long root_stride,
                                                   T* __restrict__ Fchain, long long chain_stride,
                                                   const FoldLevels fl, int tau_pad) {
    const long long rho = blockIdx.x;
    const int t = blockIdx.y * 128 + threadIdx.x;
    const int r = blockIdx.z;
    if (t >= tau_pad) return;
    const long long rstep = ((long long)1 << fl.logn_top) * tau_pad;     // row stride of the subtree
    const T* src = Froot + (long long)r * root_stride + rho * tau_pad + t;
    T v[1 << D];
#pragma unroll
    for (int q = 0; q < (1 << D); ++q) v[q] = __ldg(src + q * rstep);
    FoldStep<T, D, 1>::run(v, Fchain, fl, (long long)r * chain_stride + rho * tau_pad + t, rstep);
}

template <class T>
cudaError_t launch_fold_tree(const T* Froot, long long root_stride, T* Fchain, long long chain_stride,
                             const FoldLevels& fl, int tau_pad, int reff, cudaStream_t st) {
    if (fl.depth <= 0) return cudaSuccess;
    dim3 grid((unsigned)(1LL << fl.logn_top), (tau_pad + 127) / 128, reff);
    switch (fl.depth) {
        case 1: k_fold_tree<T, 1><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad); break;
        case 2: k_fold_tree<T, 2><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad); break;
        case 3: k_fold_tree<T, 3><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad); break;
        case 4: k_fold_tree<T, 4><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad); break;
        case 5: k_fold_tree<T, 5><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad); break;
        case 6:
            if constexpr (sizeof(T) == 4) {
                k_fold_tree<T, 6><<<grid, 128, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad);
                break;
            }
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template cudaError_t launch_fold_tree<float>(const float*, long long, float*, long long, const FoldLevels&, int, int,
                                             cudaStream_t);
template cudaError_t launch_fold_tree<double>(const double*, long long, double*, long long, const FoldLevels&, int,
                                              int, cudaStream_t);

struct FineCols {
    int jf, kf_width, nfine_part;
    int koff[4], col0[4], tau[4];
};

// dA[j][t] = sum of column j's gradient partials (the fine band's, or the coarse entry's
// k-splits).  A CTA owns column j and kGradCols columns t: warp w sums the partials
// p = w, w + 8, ... (8 columns per lane, coalesced, four partials' loads in flight together),
// and the eight warp sums are added in a fixed order.
constexpr int kGradCols = 256;

template <class T>
__global__ void __launch_bounds__(256) k_grad_reduce(const T* __restrict__ gradpart_f, const FineCols fc,
                                                     const T* __restrict__ part_c, const __grid_constant__ Chain ch,
                                                     int tau, int tau_pad, int s, T* __restrict__ grad,
                                                     const double* __restrict__ gsum, double xc) {
    __shared__ double red[8][kGradCols];        // (partials summed in double whatever T is)
    const int j = blockIdx.x, t0 = blockIdx.y * kGradCols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // where column j's partials are: base + p * stride, p < count
    const T* base = nullptr;
    long long stride = 0;
    int count = 0;
    bool coarse = false;
    for (int I = 0; I < fc.jf; ++I)
        if (fc.tau[I] > 0 && j >= fc.col0[I] && j < fc.col0[I] + fc.tau[I]) {
            base = gradpart_f + (long long)(fc.koff[I] + (j - fc.col0[I])) * tau_pad;
            stride = (long long)fc.kf_width * tau_pad;
            count = fc.nfine_part;
        }
    for (int q = 0; q < ch.count; ++q)
        if (j >= ch.col0[q] && j < ch.col0[q] + ch.tau[q]) {
            base = part_c + ch.poff[q] + (long long)(j - ch.col0[q]) * tau_pad;
            stride = (long long)ch.tau[q] * tau_pad;
            count = ch.split[q];
            coarse = true;
        }
    constexpr int C = kGradCols / 32;
    T v[C];                                      // (a warp's partials in T, the 8 warp sums in double)
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = T(0);
    int p = warp;
    for (; p + 24 < count; p += 32) {
        T w[4][C];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const T* bp = base + (long long)(p + 8 * h) * stride + t0 + lane;
#pragma unroll
            for (int c = 0; c < C; ++c) w[h][c] = t0 + 32 * c + lane < tau ? __ldg(bp + 32 * c) : T(0);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] += (w[0][c] + w[1][c]) + (w[2][c] + w[3][c]);
    }
    for (; p < count; p += 8) {
        const T* bp = base + (long long)p * stride + t0 + lane;
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (t0 + 32 * c + lane < tau) v[c] += __ldg(bp + 32 * c);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) red[warp][32 * c + lane] = (double)v[c];
    __syncthreads();
    for (int i = threadIdx.x; i < kGradCols; i += 256) {
        if (t0 + i < tau) {
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) acc += red[w][i];
            // centred block products: X^T G = (X - xc)^T G + xc 1 (1^T G), 1^T G summed in double
            if (coarse && gsum) acc += xc * gsum[t0 + i];
            grad[(long long)j * tau + t0 + i] = (T)acc;
        }
    }
}

template <class T>
cudaError_t launch_grad_reduce(const T* gradpart_f, int nfine_part, int kf_width, const int* koff_lev,
                               const int* col0_lev, const int* tau_lev, int jf, const T* part_c, const Chain& ch,
                               int tau, int tau_pad, int s, T* grad, const double* gsum, double xc, cudaStream_t st) {
    FineCols fc;
    fc.jf = jf;
    fc.kf_width = kf_width;
    fc.nfine_part = nfine_part;
    for (int i = 0; i < 4; ++i) {
        fc.koff[i] = i < jf ? koff_lev[i] : 0;
        fc.col0[i] = i < jf ? col0_lev[i] : 0;
        fc.tau[i] = i < jf ? tau_lev[i] : 0;
    }
    const dim3 grid((unsigned)s, (unsigned)((tau + kGradCols - 1) / kGradCols));
    k_grad_reduce<T><<<grid, 256, 0, st>>>(gradpart_f, fc, part_c, ch, tau, tau_pad, s, grad, gsum, xc);
    return cudaGetLastError();
}
template cudaError_t launch_grad_reduce<float>(const float*, int, int, const int*, const int*, const int*, int,
                                               const float*, const Chain&, int, int, int, float*, const double*, double,
                                               cudaStream_t);
template cudaError_t launch_grad_reduce<double>(const double*, int, int, const int*, const int*, const int*, int,
                                                const double*, const Chain&, int, int, int, double*, const double*,
                                                double, cudaStream_t);

}  // namespace qmc
