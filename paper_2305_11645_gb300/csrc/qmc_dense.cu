// Coarse-level kernels and reductions.
//
//  k_coarse_fwd    B_e = X_e A_e for every coarse weight block e (Algorithm 2's
//                  X~_I A~_I on the b^(m-I) distinct rows only), all blocks and
//                  shifts in one launch.  The fine kernels add B_e[k mod n_e]
//                  periodically (the tiling of Algorithm 2).
//  k_rows_finalize f(x_k^T A) = g(u_k) per row from the column-group partials,
//                  and fixed-order block sums of f for the mean (eq. (2)).
//  k_est_finalize  Q_r = N^-1 sum_k f, and the mean over shifts.
//  k_fold          F_I[rho] = sum_q F_I'[rho + q n_I]: the adjoint of the
//                  periodic tiling (folds the output-row gradient onto the
//                  distinct rows of a coarser level).
//  k_coarse_grad   dA_e = sum_r X_{r,e}^T F_{r,e} (split over K = R * n_e).
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
                                                       double K, double* __restrict__ rowsave, T* __restrict__ rowf,
                                                       double* __restrict__ fpart, int nblk) {
    __shared__ double sh[32];
    const int r = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double f = 0.0;
    if (k < N) {
        double u;
        if (F == F_LOGSUMEXP) {
            double M = -INFINITY;
            for (int g = 0; g < cg_count; ++g) M = fmax(M, (double)rowmax[((long long)r * cg_count + g) * N + k]);
            double S = 0.0;
            for (int g = 0; g < cg_count; ++g) {
                const long long o = ((long long)r * cg_count + g) * N + k;
                S += (double)rowpart[o] * exp((double)rowmax[o] - M);
            }
            u = M + log(S);
        } else {
            u = 0.0;
            for (int g = 0; g < cg_count; ++g) u += (double)rowpart[((long long)r * cg_count + g) * N + k];
        }
        f = g_of(F, u, tau, c, K);
        if (rowsave) rowsave[(long long)r * N + k] = u;
        if (rowf) rowf[(long long)r * N + k] = (T)f;
    }
    const double s = block_sum(f, sh);
    if (threadIdx.x == 0) fpart[(long long)r * nblk + blockIdx.x] = s;
}

template <class T>
cudaError_t launch_rows_finalize(const T* rowpart, const T* rowmax, int cg_count, long long N, int reff, int F,
                                 double tau, double c, double K, double* rowsave, T* rowf_out, double* fpart,
                                 int nblk, cudaStream_t st) {
    dim3 grid(nblk, reff);
    k_rows_finalize<T><<<grid, 256, 0, st>>>(rowpart, rowmax, cg_count, N, F, tau, c, K, rowsave, rowf_out, fpart,
                                             nblk);
    return cudaGetLastError();
}
template cudaError_t launch_rows_finalize<float>(const float*, const float*, int, long long, int, int, double, double,
                                                 double, double*, float*, double*, int, cudaStream_t);
template cudaError_t launch_rows_finalize<double>(const double*, const double*, int, long long, int, int, double,
                                                  double, double, double*, double*, double*, int, cudaStream_t);

__global__ void __launch_bounds__(256) k_est_finalize(const double* __restrict__ fpart, int nblk, int reff,
                                                      long long N, double* __restrict__ est) {
    __shared__ double sh[32];
    double mean = 0.0;
    for (int r = 0; r < reff; ++r) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += fpart[(long long)r * nblk + b];
        const double s = block_sum(v, sh);
        if (threadIdx.x == 0) {
            est[r] = s / (double)N;
            mean += s / (double)N;
        }
    }
    if (threadIdx.x == 0) est[reff] = mean / reff;
}

cudaError_t launch_est_finalize(const double* fpart, int nblk, int reff, long long N, double* est, cudaStream_t st) {
    k_est_finalize<<<1, 256, 0, st>>>(fpart, nblk, reff, N, est);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// backward: folds, coarse gradient GEMMs, final reduction
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_fold(const T* __restrict__ src, long long src_stride, int logn_src, T* __restrict__ dst,
                       long long dst_stride, int logn_dst, int tau_pad) {
    const int r = blockIdx.y;
    const long long n_dst = 1LL << logn_dst;
    const long long reps = 1LL << (logn_src - logn_dst);
    const long long total = n_dst * tau_pad;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long rho = e / tau_pad;
        const int t = (int)(e - rho * tau_pad);
        T acc = T(0);
        for (long long q = 0; q < reps; ++q) acc += src[(long long)r * src_stride + (rho + q * n_dst) * tau_pad + t];
        dst[(long long)r * dst_stride + rho * tau_pad + t] = acc;
    }
}

template <class T>
cudaError_t launch_fold(const T* src, long long src_stride, int logn_src, T* dst, long long dst_stride, int logn_dst,
                        int tau_pad, int reff, cudaStream_t st) {
    long long total = (1LL << logn_dst) * tau_pad;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    dim3 grid((unsigned)blocks, reff);
    k_fold<T><<<grid, 256, 0, st>>>(src, src_stride, logn_src, dst, dst_stride, logn_dst, tau_pad);
    return cudaGetLastError();
}
template cudaError_t launch_fold<float>(const float*, long long, int, float*, long long, int, int, int, cudaStream_t);
template cudaError_t launch_fold<double>(const double*, long long, int, double*, long long, int, int, int,
                                         cudaStream_t);

// part[e][split][jj][t] = sum over (r, rho) in the split of tab[r][tab_e + jj n_e + rho] * F_e[r][rho][t]
// CTA: 128 threads x 4 columns, 16 columns j of the level; x staged in shared memory 64 rows at a time.
template <class T>
__global__ void __launch_bounds__(128) k_coarse_grad(const T* __restrict__ tab, long long tab_stride,
                                                     const T* __restrict__ Froot, long long root_stride,
                                                     const T* __restrict__ Fchain, long long chain_stride, int jf,
                                                     int tau_pad, const __grid_constant__ Chain ch,
                                                     T* __restrict__ part, int reff) {
    __shared__ T xs[64][16];
    const int e = chain_entry(ch, blockIdx.x);
    const int local = blockIdx.x - ch.tile0[e];
    const int tau_e = ch.tau[e], logn = ch.logn[e], nsplit = ch.split[e];
    const int jt = local / nsplit, sp = local - jt * nsplit;
    const int j0 = jt * 16;
    const long long n_e = 1LL << logn;
    const long long Ktot = (long long)reff * n_e;
    const long long kper = (Ktot + nsplit - 1) / nsplit;
    const long long kb = (long long)sp * kper, ke = min(Ktot, kb + kper);
    const int t = blockIdx.y * 512 + threadIdx.x * 4;
    const bool active = t < tau_pad;
    const bool at_root = ch.lev[e] == jf;
    const T* F = at_root ? Froot : Fchain + ch.boff[e];
    const long long F_stride = at_root ? root_stride : chain_stride;

    T acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[j][c] = T(0);

    for (long long k0 = kb; k0 < ke; k0 += 64) {
        for (int idx = threadIdx.x; idx < 64 * 16; idx += 128) {
            const int kk = idx >> 4, jj = idx & 15;
            const long long k = k0 + kk;
            T v = T(0);
            if (k < ke && j0 + jj < tau_e) {
                const long long r = k >> logn, rho = k & (n_e - 1);
                v = tab[r * tab_stride + ch.tab[e] + (long long)(j0 + jj) * n_e + rho];
            }
            xs[kk][jj] = v;
        }
        __syncthreads();
        if (active) {
            const int kn = (int)min((long long)64, ke - k0);
            for (int kk = 0; kk < kn; ++kk) {
                const long long k = k0 + kk;
                const long long r = k >> logn, rho = k & (n_e - 1);
                const T* fp = F + r * F_stride + rho * tau_pad + t;
                T fv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) fv[c] = fp[c];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const T xv = xs[kk][jj];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[jj][c] = fma(xv, fv[c], acc[jj][c]);
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
        if (j0 + jj < tau_e) {
            T* o = part + ch.poff[e] + ((long long)sp * tau_e + j0 + jj) * tau_pad + t;
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = acc[jj][c];
        }
    }
}

template <class T>
cudaError_t launch_coarse_grad(const T* tab, long long tab_stride, const T* Froot, long long root_stride,
                               const T* Fchain, long long chain_stride, int jf, int tau_pad, const Chain& ch,
                               T* part, int reff, int ntiles, cudaStream_t st) {
    if (ch.count == 0) return cudaSuccess;
    dim3 grid(ntiles, (tau_pad + 511) / 512);
    k_coarse_grad<T><<<grid, 128, 0, st>>>(tab, tab_stride, Froot, root_stride, Fchain, chain_stride, jf, tau_pad,
                                           ch, part, reff);
    return cudaGetLastError();
}
template cudaError_t launch_coarse_grad<float>(const float*, long long, const float*, long long, const float*,
                                               long long, int, int, const Chain&, float*, int, int, cudaStream_t);
template cudaError_t launch_coarse_grad<double>(const double*, long long, const double*, long long, const double*,
                                                long long, int, int, const Chain&, double*, int, int, cudaStream_t);

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
                for (int p = 0; p < fc.nfine_part; ++p)
                    v += gradpart_f[((long long)p * fc.kf_width + jl) * tau_pad + t];
                done = true;
            }
        }
        for (int q = 0; q < ch.count && !done; ++q) {
            if (j >= ch.col0[q] && j < ch.col0[q] + ch.tau[q]) {
                const int jj = j - ch.col0[q];
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
