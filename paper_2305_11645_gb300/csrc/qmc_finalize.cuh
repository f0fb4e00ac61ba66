// Row finalisation shared by the finalisation kernel and the fused fine-band forward: the
// integrand's g(u) and g'(u) of a row from its row sum (eq. (2)), and the mean over N.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

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

// sum over the CTA in a fixed order: warp shuffles in T, then the warp sums in double
template <class T>
__device__ __forceinline__ double block_sum_t(T v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

// log-sum-exp row sum u = log sum_t exp(y_t) from the combined partial (max M, sum S of 2^(v - M))
// of v = y log2 e
template <class T>
__device__ __forceinline__ T lse_row(T M, T S) { return (M + log2(S)) * (T)kLn2; }

// f = g(u) of row k, and what the backward needs of it, g'(u) gfac/(R N) and log2 e * u, at
// rowsave[2 idx], rowsave[2 idx + 1] (idx = r N + k); f also at rowf[idx] when asked for.
// The call payoff's kink test u/tau > K is taken in double, without a division.
template <class T>
__device__ __forceinline__ T finalize_row(int F, T u, T inv_tau, double tau, double K, double coef_scale,
                                          T* __restrict__ rowsave, T* __restrict__ rowf, long long idx) {
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
    if (rowsave) {
        rowsave[2 * idx] = gp * (T)coef_scale;
        rowsave[2 * idx + 1] = u * (T)kLog2e;
    }
    if (rowf) rowf[idx] = fv;
    return fv;
}

// CTA partial s of sum_k f for shift r goes to fpart[r * nblk + slot].  With est, the last CTA
// to take the ticket (total CTAs in all) forms Q_r = N^-1 sum_slot fpart[r][slot] for every
// shift and their mean est[reff], summing in a fixed order (deterministic whichever CTA is last).
// Every thread of the CTA calls it.
__device__ __forceinline__ void finalize_estimate(double s, int r, int slot, int nblk, int reff, long long N,
                                                  unsigned int total, unsigned int* ticket, double* fpart,
                                                  double* est, double* sh) {
    __shared__ bool last;
    if (!est) {
        if (threadIdx.x == 0) fpart[(long long)r * nblk + slot] = s;
        return;
    }
    if (threadIdx.x == 0) {
        fpart[(long long)r * nblk + slot] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == total - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double mean = 0.0;
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

}  // namespace qmc
