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
//  k_fold_tree     the root gradients folded level by level onto the distinct
//                  rows of every coarse level.
//  k_chain_sum     S_JF[rho] = sum_e B_e[rho mod n_e]: the root values of the
//                  fine band (Algorithm 2's tiling of the coarse levels).
//  k_coarse_grad   dA_e = sum_r X_{r,e}^T F_{r,e}, with F_e[rho] = sum_q
//                  F_JF[rho + q n_e] folded on the fly from the root gradients
//                  (the adjoint of the periodic tiling), split over K = R n_e.
//  k_grad_reduce   fixed-order sum of all gradient partials into dA.
#include "qmc_internal.cuh"

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

// S[r][t/4][rho][t%4] = sum_e B_e[r][t/4][rho mod n_e][t%4], rho < n_root
template <class T>
__global__ void k_chain_sum(const T* __restrict__ B, long long B_stride, const __grid_constant__ Chain ch,
                            T* __restrict__ S, long long S_stride, int logn_root, int tau_pad) {
    // one group of four columns of one root row per thread; the entries' loads are independent
    const int r = blockIdx.y;
    const long long n_root = 1LL << logn_root;
    const long long total = n_root * (tau_pad >> 2);
    const long long e4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e4 >= total) return;
    const T* Br = B + (long long)r * B_stride;
    const long long t4 = e4 >> logn_root, rho = e4 & (n_root - 1);
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
    for (int e = 0; e < ch.count; ++e) {
        const T* p = Br + ch.boff[e] + ((t4 << ch.logn[e]) << 2) + ((rho & ((1LL << ch.logn[e]) - 1)) << 2);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += __ldg(p + c);
    }
    T* o = S + (long long)r * S_stride + (e4 << 2);
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = acc[c];
}

template <class T>
cudaError_t launch_chain_sum(const T* B, long long B_stride, const Chain& ch, T* S, long long S_stride, int logn_root,
                             int tau_pad, int reff, cudaStream_t st) {
    const long long total = (1LL << logn_root) * (tau_pad / 4);
    const long long blocks = (total + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks, reff);
    k_chain_sum<T><<<grid, 256, 0, st>>>(B, B_stride, ch, S, S_stride, logn_root, tau_pad);
    return cudaGetLastError();
}
template cudaError_t launch_chain_sum<float>(const float*, long long, const Chain&, float*, long long, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_chain_sum<double>(const double*, long long, const Chain&, double*, long long, int, int,
                                              int, cudaStream_t);

// ------------------------------------------------------------------------------------------
// row finalisation and the mean
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

template <class T>
__global__ void __launch_bounds__(256) k_rows_finalize(const T* __restrict__ rowpart, const T* __restrict__ rowmax,
                                                       int cg_count, long long N, int F, double tau, double c,
                                                       double K, double coef_scale, T* __restrict__ rowsave,
                                                       T* __restrict__ rowf, double* __restrict__ fpart, int nblk,
                                                       unsigned int* ticket, double* __restrict__ est) {
    // Per-row arithmetic in T (the row sums are T partials); only the sum over rows is kept in
    // double.  The call payoff's kink test u/tau > K is taken in double, without a division.
    __shared__ double sh[32];
    const int r = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T inv_tau = (T)(1.0 / tau);
    double f = 0.0;
    if (k < N) {
        T u;
        const T* rp = rowpart + (long long)r * cg_count * N + k;
        if (F == F_LOGSUMEXP) {
            // the partials hold (max, sum 2^(v - max)) of v = y log2 e
            const T* rm = rowmax + (long long)r * cg_count * N + k;
            T M = -INFINITY;
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) M = fmax(M, rm[(long long)g * N]);
            T S = T(0);
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) S += rp[(long long)g * N] * exp2(rm[(long long)g * N] - M);
            u = (M + log2(S)) * (T)kLn2;
        } else {
            u = T(0);
#pragma unroll 8
            for (int g = 0; g < cg_count; ++g) u += rp[(long long)g * N];
        }
        T fv, gp;
        switch (F) {
            case F_LINEAR_MEAN: case F_MEAN_COS: case F_PDE_INV_SQ: fv = u * inv_tau; gp = inv_tau; break;
            case F_CALL_MEAN_EXP: {
                const bool active = (double)u * (1.0 / tau) - K > 0.0;
                fv = active ? u * inv_tau - (T)K : T(0);
                gp = active ? inv_tau : T(0);
                break;
            }
            case F_GAUSS_NORM2: fv = exp(T(-0.5) * u * inv_tau); gp = T(-0.5) * inv_tau * fv; break;
            default: fv = u; gp = T(1); break;     // log-sum-exp: u is log sum exp(y)
        }
        f = (double)fv;
        if (rowsave) {
            // what the backward needs of this row: g'(u) gfac/(R N) and log2 e * u
            rowsave[2 * ((long long)r * N + k)] = gp * (T)coef_scale;
            rowsave[2 * ((long long)r * N + k) + 1] = u * (T)kLog2e;
        }
        if (rowf) rowf[(long long)r * N + k] = fv;
    }
    const double s = block_sum(f, sh);
    if (!est) {
        if (threadIdx.x == 0) fpart[(long long)r * nblk + blockIdx.x] = s;
        return;
    }
    // the last block to finish forms Q_r = N^-1 sum_k f for every shift and their mean,
    // summing the block partials in a fixed order (deterministic whichever block is last)
    __shared__ bool last;
    if (threadIdx.x == 0) {
        fpart[(long long)r * nblk + blockIdx.x] = s;
        __threadfence();
        const unsigned int total = gridDim.x * gridDim.y;
        last = atomicAdd(ticket, 1u) == total - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double mean = 0.0;
    const int reff = gridDim.y;
    for (int rr = 0; rr < reff; ++rr) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += __ldcg(fpart + (long long)rr * nblk + b);
        const double sr = block_sum(v, sh);
        if (threadIdx.x == 0) {
            est[rr] = sr / (double)N;
            mean += sr / (double)N;
        }
    }
    if (threadIdx.x == 0) est[reff] = mean / reff;
}

template <class T>
cudaError_t launch_rows_finalize(const T* rowpart, const T* rowmax, int cg_count, long long N, int reff, int F,
                                 double tau, double c, double K, double coef_scale, T* rowsave, T* rowf_out,
                                 double* fpart, int nblk, unsigned int* ticket, double* est, cudaStream_t st) {
    dim3 grid(nblk, reff);
    k_rows_finalize<T><<<grid, 256, 0, st>>>(rowpart, rowmax, cg_count, N, F, tau, c, K, coef_scale, rowsave,
                                             rowf_out, fpart, nblk, ticket, est);
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
// F_{I+1}[rho] = F_I[rho] + F_I[rho + n_{I+1}].  A CTA (one warp) owns a top node
// rho' < n_top of level JF+depth and 128 columns; the 2^depth root rows
// rho' + q n_top of its subtree are held in shared memory, each lane folds its own
// four columns level by level and writes the folded rows of every coarse level.
template <class T>
__global__ void __launch_bounds__(32) k_fold_tree(const T* __restrict__ Froot, long long root_stride,
                                                  T* __restrict__ Fchain, long long chain_stride,
                                                  const FoldLevels fl, int tau_pad) {
    constexpr int kMaxDepth = sizeof(T) == 8 ? 5 : 6;     // 32 KB of shared memory either way
    __shared__ __align__(16) T S[(1 << kMaxDepth) * 32 * 4];
    const int lane = threadIdx.x;
    const long long rho = blockIdx.x;
    const int t = blockIdx.y * 128 + lane * 4;
    const int r = blockIdx.z;
    if (t >= tau_pad) return;
    const int rows = 1 << fl.depth;
    T* Sl = S + lane * 4;
    const T* src = Froot + (long long)r * root_stride + rho * tau_pad + t;
#pragma unroll 8
    for (int q = 0; q < rows; ++q) {
        const T* p = src + (((long long)q << fl.logn_top) * tau_pad);
#pragma unroll
        for (int c = 0; c < 4; ++c) Sl[q * 128 + c] = p[c];
    }
    int cur = rows;
    for (int d = 1; d <= fl.depth; ++d) {
        const int half = cur >> 1;
        T* dst = Fchain + fl.off[d] + (long long)r * chain_stride + rho * tau_pad + t;
        for (int q = 0; q < half; ++q) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const T v = Sl[q * 128 + c] + Sl[(q + half) * 128 + c];
                Sl[q * 128 + c] = v;
                if (fl.want[d]) dst[(((long long)q << fl.logn_top) * tau_pad) + c] = v;
            }
        }
        cur = half;
    }
}

template <class T>
cudaError_t launch_fold_tree(const T* Froot, long long root_stride, T* Fchain, long long chain_stride,
                             const FoldLevels& fl, int tau_pad, int reff, cudaStream_t st) {
    if (fl.depth <= 0) return cudaSuccess;
    dim3 grid((unsigned)(1LL << fl.logn_top), (tau_pad + 127) / 128, reff);
    k_fold_tree<T><<<grid, 32, 0, st>>>(Froot, root_stride, Fchain, chain_stride, fl, tau_pad);
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

template <class T>
__global__ void k_grad_reduce(const T* __restrict__ gradpart_f, const FineCols fc, const T* __restrict__ part_c,
                              const __grid_constant__ Chain ch, int tau, int tau_pad, int s, T* __restrict__ grad) {
    const long long total = (long long)s * tau;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / tau);
        const int t = (int)(e - (long long)j * tau);
        T v = T(0);
        bool done = false;
        for (int I = 0; I < fc.jf && !done; ++I) {
            if (fc.tau[I] > 0 && j >= fc.col0[I] && j < fc.col0[I] + fc.tau[I]) {
                const int jl = fc.koff[I] + (j - fc.col0[I]);
#pragma unroll 8
                for (int p = 0; p < fc.nfine_part; ++p)
                    v += gradpart_f[((long long)p * fc.kf_width + jl) * tau_pad + t];
                done = true;
            }
        }
        for (int q = 0; q < ch.count && !done; ++q) {
            if (j >= ch.col0[q] && j < ch.col0[q] + ch.tau[q]) {
                const int jj = j - ch.col0[q];
#pragma unroll 8
                for (int sp = 0; sp < ch.split[q]; ++sp)
                    v += part_c[ch.poff[q] + ((long long)sp * ch.tau[q] + jj) * tau_pad + t];
                done = true;
            }
        }
        grad[e] = v;
    }
}

template <class T>
cudaError_t launch_grad_reduce(const T* gradpart_f, int nfine_part, int kf_width, const int* koff_lev,
                               const int* col0_lev, const int* tau_lev, int jf, const T* part_c, const Chain& ch,
                               int tau, int tau_pad, int s, T* grad, cudaStream_t st) {
    FineCols fc;
    fc.jf = jf;
    fc.kf_width = kf_width;
    fc.nfine_part = nfine_part;
    for (int i = 0; i < 4; ++i) {
        fc.koff[i] = i < jf ? koff_lev[i] : 0;
        fc.col0[i] = i < jf ? col0_lev[i] : 0;
        fc.tau[i] = i < jf ? tau_lev[i] : 0;
    }
    long long total = (long long)s * tau;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_grad_reduce<T><<<(unsigned)blocks, 256, 0, st>>>(gradpart_f, fc, part_c, ch, tau, tau_pad, s, grad);
    return cudaGetLastError();
}
template cudaError_t launch_grad_reduce<float>(const float*, int, int, const int*, const int*, const int*, int,
                                               const float*, const Chain&, int, int, int, float*, cudaStream_t);
template cudaError_t launch_grad_reduce<double>(const double*, int, int, const int*, const int*, const int*, int,
                                                const double*, const Chain&, int, int, int, double*, cudaStream_t);

}  // namespace qmc
