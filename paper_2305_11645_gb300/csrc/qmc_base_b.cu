// Reduced lattices and reduced Monte Carlo in a prime base b > 2 (Sec. 1.3: N = b^m; Sec. 5:
// N_j = b^(m - w_j)), on the CUDA cores in the precision's type (double for QMC_FP64, float for
// the others).
//
// The structure is Algorithm 2's with b-fold repetition: weight block I has n_I = b^(m-I)
// distinct rows, and P~_I = tile(P~_{I+1}, b) + X~_I A~_I from the coarsest level down, each
// level's block product on its distinct rows only.  With no binary fine band, the last level's
// sum is the product at all N rows; the integrand and its row sums, and the adjoint's
// G = f'(Y) / (R N), are then formed row by row, and the adjoint folds G back level by level,
// F_{I'}[rho] = sum_q F_I[rho + q n_{I'}], before each level's block gradient X~_I^T F_I.
//
// Points: a lattice coordinate is u / b^q, u = (k z_j) mod b^q, q = m - min(w_j, m), which has
// no 32-bit fixed-point form; it is formed in double as u / b^q (one rounded division) and the
// shift D_j 2^-32 as {x + D_j 2^-32}, the rounded sum less 1 when it reaches 1, then transformed
// in double and rounded once to the precision's type.  Reduced MC samples are the caller's
// 32-bit words, x = y 2^-32, as in base 2.
#include "qmc_internal.cuh"

namespace qmc {
namespace {

// transform of a point given in double (Sec. 2.3), rounded once to T
template <class T>
__device__ __forceinline__ T tr_double(double x, int tr) {
    switch (tr) {
        case T_CENTER: return (T)(x - 0.5);
        case T_TENT: return (T)(1.0 - fabs(1.0 - 2.0 * x));
        case T_INV_NORMAL: return (T)(x < 0.5 ? normcdfinv(x) : -normcdfinv(1.0 - x));
        default: return (T)x;
    }
}

__device__ __forceinline__ int level_b(const DevRule& R, long long g) {
    int lo = 0, hi = R.nlev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g >= R.lev_tab[mid]) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// x of table entry g (lattice: unshifted numerator and level period, returned in u / n)
__device__ __forceinline__ void entry_b(const DevRule& R, long long g, int& j, long long& u, long long& n) {
    const int I = level_b(R, g);
    n = R.lev_n[I];
    const long long idx = g - R.lev_tab[I];
    j = R.lev_col0[I] + (int)(idx / n);
    const long long row = idx - (idx / n) * n;
    u = (long long)(((unsigned long long)row * (unsigned long long)R.gen[j]) % (unsigned long long)n);
}

template <class T>
__global__ void k_table_b(const __grid_constant__ DevRule R, T* __restrict__ tab, long long T_tot, long long stride,
                          int reff, unsigned int* ticket) {
    if (ticket && blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0u;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < T_tot;
         g += (long long)gridDim.x * blockDim.x) {
        if (R.kind == KIND_MC) {
            for (int r = 0; r < reff; ++r)
                tab[(long long)r * stride + g] =
                    tr_double<T>((double)__ldg(R.gen + (long long)r * T_tot + g) * 2.3283064365386962890625e-10,
                                 R.transform);
            continue;
        }
        int j;
        long long u, n;
        entry_b(R, g, j, u, n);
        const double x0 = (double)u / (double)n;
        for (int r = 0; r < reff; ++r) {
            double x = x0;
            if (R.shift) {
                x = x0 + (double)R.shift[(size_t)r * R.s + j] * 2.3283064365386962890625e-10;
                if (x >= 1.0) x -= 1.0;
            }
            tab[(long long)r * stride + g] = tr_double<T>(x, R.transform);
        }
    }
}

// the unshifted numerators u (lattice) or the sample words (reduced MC), full or distinct layout
__global__ void k_points_b(const __grid_constant__ DevRule R, uint32_t* __restrict__ out, long long total, int full,
                           int shift_idx) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long g = e;
        if (full) {                    // e = k s + j: table entry of column j, row k mod n_j
            const long long k = e / R.s;
            const int j = (int)(e - k * R.s);
            int I = 0;
            for (int L = 0; L < R.nlev; ++L)
                if (R.lev_tau[L] > 0 && R.lev_col0[L] <= j) I = L;
            g = R.lev_tab[I] + (long long)(j - R.lev_col0[I]) * R.lev_n[I] + k % R.lev_n[I];
        }
        if (R.kind == KIND_MC) {
            out[e] = R.gen[(long long)shift_idx * R.T_tot + g];
        } else {
            int j;
            long long u, n;
            entry_b(R, g, j, u, n);
            out[e] = (uint32_t)u;
        }
    }
}

// ------------------------------------------------------------------------------------------
// one level of the top-down sum: out[r][rho][t] for rho < n_out,
//   = next[r][rho mod n_next][t] + sum_{jj < tau_I} tab[r][tab_I + jj n_I + rho mod n_I] A[col0 + jj][t]
// (rows n_out = n_I, or N for the last level), in the [t/4][rho][4] layout (or row-major P[r][rho][t]
// for a materialised last level).  64 x 64 tiles, 16-deep K steps staged in shared memory.
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_level_b(const T* __restrict__ tab, long long tab_stride, const T* __restrict__ A,
                                                 int ldA, int tau_pad, LevelB lv, T* __restrict__ out,
                                                 long long out_stride, const T* __restrict__ next, long long next_stride,
                                                 int rowmajor, int tau) {
    __shared__ T Xs[16][64];
    __shared__ T As[16][64];
    const long long rho0 = (long long)blockIdx.x * 64;
    const int t0 = blockIdx.y * 64;
    const int r = blockIdx.z;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const T* tabr = tab + (long long)r * tab_stride + lv.tab;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
    for (int k0 = 0; k0 < lv.tau; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + 256 * q, kk = idx >> 6, rr = idx & 63;
            const bool kv = (k0 + kk) < lv.tau;
            const long long rho = rho0 + rr;
            Xs[kk][rr] = (kv && rho < lv.n_out) ? tabr[(long long)(k0 + kk) * lv.n + rho % lv.n] : T(0);
            As[kk][rr] = (kv && t0 + rr < tau_pad) ? A[(long long)(lv.col0 + k0 + kk) * ldA + t0 + rr] : T(0);
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
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long rho = rho0 + tx + 16 * i;
        if (rho >= lv.n_out) continue;
        T v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = acc[i][c];
        if (next) {
            const T* nx = next + (long long)r * next_stride + (long long)(t >> 2) * lv.n_next * 4 + (rho % lv.n_next) * 4;
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] += nx[c];
        }
        if (rowmajor) {
            T* o = out + (long long)r * out_stride + rho * tau;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (t + c < tau) o[t + c] = v[c];
        } else {
            T* o = out + (long long)r * out_stride + (long long)(t >> 2) * lv.n_out * 4 + rho * 4;
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = v[c];
        }
    }
}

// ------------------------------------------------------------------------------------------
// the integrand's row sums over the root values S (all N rows, [t/4][rho][4]): one thread per row
// of one shift; rowpart[r][0][k] = u_k (log-sum-exp: the maximum in rowmax and sum 2^(v - max))
// ------------------------------------------------------------------------------------------
template <class T, int F>
__global__ void __launch_bounds__(256) k_rows_b(const T* __restrict__ S, long long S_stride, long long N, int tau,
                                                T kappa, T c0, T* __restrict__ rowpart, T* __restrict__ rowmax) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (k >= N) return;
    const T* s = S + (long long)r * S_stride + k * 4;
    T u = T(0), mx = -INFINITY;
    for (int t = 0; t < tau; ++t) {
        const T v = kappa * s[(long long)(t >> 2) * N * 4 + (t & 3)];
        if constexpr (F == F_LOGSUMEXP) {
            const T d = v - mx;
            if (d > T(0)) { u = u * ex2(-d) + T(1); mx = v; }
            else u += ex2(d);
        } else {
            u += Fn<F, T>::h(v, c0);
        }
    }
    rowpart[(long long)r * N + k] = u;
    if constexpr (F == F_LOGSUMEXP) rowmax[(long long)r * N + k] = mx;
}

// G[r][k][t] = upstream g'(u_k) gfac/(R N) h'(y_kt) (rowsave from the finalisation) over all N rows
template <class T, int F>
__global__ void __launch_bounds__(256) k_grad_rows_b(const T* __restrict__ S, long long S_stride, long long N, int tau,
                                                     int tau_pad, T kappa, T c0, const T* __restrict__ rowsave,
                                                     const double* __restrict__ upstream, T* __restrict__ G) {
    const int t = blockIdx.y * 64 + (threadIdx.x & 63);
    const long long k = (long long)blockIdx.x * 4 + (threadIdx.x >> 6);
    const int r = blockIdx.z;
    if (k >= N || t >= tau_pad) return;
    T g = T(0);
    if (t < tau) {
        const T v = kappa * S[(long long)r * S_stride + (long long)(t >> 2) * N * 4 + k * 4 + (t & 3)];
        const long long idx = (long long)r * N + k;
        const T coef = (T)upstream[0] * rowsave[2 * idx];
        g = coef * Fn<F, T>::hp(v, c0, rowsave[2 * idx + 1]);
    }
    G[((long long)r * N + k) * tau_pad + t] = g;
}

// F_dst[r][rho][t] = sum_{q < n_src / n_dst} F_src[r][rho + q n_dst][t], rho < n_dst
template <class T>
__global__ void __launch_bounds__(256) k_fold_b(const T* __restrict__ src, long long n_src, T* __restrict__ dst,
                                                long long n_dst, int tau_pad) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (e >= n_dst * tau_pad) return;
    const long long rho = e / tau_pad;
    const int t = (int)(e - rho * tau_pad);
    const T* sp = src + (long long)r * n_src * tau_pad + rho * tau_pad + t;
    T acc = T(0);
    for (long long q = 0; q < n_src / n_dst; ++q) acc += sp[q * n_dst * tau_pad];
    dst[((long long)r * n_dst + rho) * tau_pad + t] = acc;
}

// block gradient partials of one level: part[sp][jj][t] = sum over rows (r, rho) of split sp of
// tab[r][tab_I + jj n_I + rho] F_I[r][rho][t]; a CTA takes 64 columns t and 4 rows jj per thread
// group (256 threads = 64 t x 4 jj groups of 4 rows), the X values of 32 rows staged in shared memory
template <class T>
__global__ void __launch_bounds__(256) k_grad_b(const T* __restrict__ tab, long long tab_stride, const T* __restrict__ F,
                                                LevelB lv, long long kper, int reff, int tau_pad, T* __restrict__ part) {
    __shared__ T Xs[32][17];
    const int t = blockIdx.y * 64 + (threadIdx.x & 63);
    const int jg = threadIdx.x >> 6;               // rows 4 jg .. 4 jg + 3 of the 16-row j tile
    const int j0 = blockIdx.z * 16;
    const int sp = blockIdx.x;
    const long long K = (long long)reff * lv.n;
    const long long kb = (long long)sp * kper, ke = min(K, kb + kper);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (long long k0 = kb; k0 < ke; k0 += 32) {
        for (int i = threadIdx.x; i < 32 * 16; i += 256) {
            const int kk = i >> 4, jj = i & 15;
            const long long k = k0 + kk;
            T v = T(0);
            if (k < ke && j0 + jj < lv.tau) {
                const long long rr = k / lv.n, rho = k - rr * lv.n;
                v = tab[rr * tab_stride + lv.tab + (long long)(j0 + jj) * lv.n + rho];
            }
            Xs[kk][jj] = v;
        }
        __syncthreads();
        if (t < tau_pad) {
            for (int kk = 0; kk < 32 && k0 + kk < ke; ++kk) {
                const long long k = k0 + kk;
                const long long rr = k / lv.n, rho = k - rr * lv.n;
                const T f = F[(rr * lv.n + rho) * tau_pad + t];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fma(Xs[kk][4 * jg + q], f, acc[q]);
            }
        }
        __syncthreads();
    }
    if (t < tau_pad) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = j0 + 4 * jg + q;
            if (jj < lv.tau) part[((long long)sp * lv.tau + jj) * tau_pad + t] = acc[q];
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <class T>
cudaError_t launch_table_b(const DevRule& R, T* tab, long long T_tot, long long stride, int reff, unsigned int* ticket,
                           cudaStream_t st) {
    long long blocks = std::min<long long>((T_tot + 255) / 256, 152 * 32);
    k_table_b<T><<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(R, tab, T_tot, stride, reff, ticket);
    return cudaGetLastError();
}
template cudaError_t launch_table_b<float>(const DevRule&, float*, long long, long long, int, unsigned int*, cudaStream_t);
template cudaError_t launch_table_b<double>(const DevRule&, double*, long long, long long, int, unsigned int*,
                                            cudaStream_t);

cudaError_t launch_points_b(const DevRule& R, uint32_t* out, long long total, bool full, int shift_idx,
                            cudaStream_t st) {
    long long blocks = std::min<long long>((total + 255) / 256, 152 * 64);
    k_points_b<<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(R, out, total, full ? 1 : 0, shift_idx);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_level_b(const T* tab, long long tab_stride, const T* A, int ldA, int tau_pad, const LevelB& lv,
                           T* out, long long out_stride, const T* next, long long next_stride, bool rowmajor, int tau,
                           int reff, cudaStream_t st) {
    dim3 grid((unsigned)((lv.n_out + 63) / 64), (unsigned)((tau_pad + 63) / 64), (unsigned)reff);
    k_level_b<T><<<grid, 256, 0, st>>>(tab, tab_stride, A, ldA, tau_pad, lv, out, out_stride, next, next_stride,
                                       rowmajor ? 1 : 0, tau);
    return cudaGetLastError();
}
template cudaError_t launch_level_b<float>(const float*, long long, const float*, int, int, const LevelB&, float*,
                                           long long, const float*, long long, bool, int, int, cudaStream_t);
template cudaError_t launch_level_b<double>(const double*, long long, const double*, int, int, const LevelB&, double*,
                                            long long, const double*, long long, bool, int, int, cudaStream_t);

template <class T>
cudaError_t launch_rows_b(const T* S, long long S_stride, long long N, int tau, int F, double kappa, double c0,
                          T* rowpart, T* rowmax, int reff, cudaStream_t st) {
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)reff);
    switch (F) {
        case F_LINEAR_MEAN: k_rows_b<T, F_LINEAR_MEAN><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        case F_MEAN_COS: k_rows_b<T, F_MEAN_COS><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        case F_CALL_MEAN_EXP: k_rows_b<T, F_CALL_MEAN_EXP><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        case F_GAUSS_NORM2: k_rows_b<T, F_GAUSS_NORM2><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        case F_PDE_INV_SQ: k_rows_b<T, F_PDE_INV_SQ><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        case F_LOGSUMEXP: k_rows_b<T, F_LOGSUMEXP><<<grid, 256, 0, st>>>(S, S_stride, N, tau, (T)kappa, (T)c0, rowpart, rowmax); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template cudaError_t launch_rows_b<float>(const float*, long long, long long, int, int, double, double, float*, float*,
                                          int, cudaStream_t);
template cudaError_t launch_rows_b<double>(const double*, long long, long long, int, int, double, double, double*,
                                           double*, int, cudaStream_t);

template <class T>
cudaError_t launch_grad_rows_b(const T* S, long long S_stride, long long N, int tau, int tau_pad, int F, double kappa,
                               double c0, const T* rowsave, const double* upstream, T* G, int reff, cudaStream_t st) {
    dim3 grid((unsigned)((N + 3) / 4), (unsigned)((tau_pad + 63) / 64), (unsigned)reff);
#define QMC_GRB(FK) k_grad_rows_b<T, FK><<<grid, 256, 0, st>>>(S, S_stride, N, tau, tau_pad, (T)kappa, (T)c0, rowsave, upstream, G)
    switch (F) {
        case F_LINEAR_MEAN: QMC_GRB(F_LINEAR_MEAN); break;
        case F_MEAN_COS: QMC_GRB(F_MEAN_COS); break;
        case F_CALL_MEAN_EXP: QMC_GRB(F_CALL_MEAN_EXP); break;
        case F_GAUSS_NORM2: QMC_GRB(F_GAUSS_NORM2); break;
        case F_PDE_INV_SQ: QMC_GRB(F_PDE_INV_SQ); break;
        case F_LOGSUMEXP: QMC_GRB(F_LOGSUMEXP); break;
        default: return cudaErrorInvalidValue;
    }
#undef QMC_GRB
    return cudaGetLastError();
}
template cudaError_t launch_grad_rows_b<float>(const float*, long long, long long, int, int, int, double, double,
                                               const float*, const double*, float*, int, cudaStream_t);
template cudaError_t launch_grad_rows_b<double>(const double*, long long, long long, int, int, int, double, double,
                                                const double*, const double*, double*, int, cudaStream_t);

template <class T>
cudaError_t launch_fold_b(const T* src, long long n_src, T* dst, long long n_dst, int tau_pad, int reff, cudaStream_t st) {
    dim3 grid((unsigned)((n_dst * tau_pad + 255) / 256), (unsigned)reff);
    k_fold_b<T><<<grid, 256, 0, st>>>(src, n_src, dst, n_dst, tau_pad);
    return cudaGetLastError();
}
template cudaError_t launch_fold_b<float>(const float*, long long, float*, long long, int, int, cudaStream_t);
template cudaError_t launch_fold_b<double>(const double*, long long, double*, long long, int, int, cudaStream_t);

template <class T>
cudaError_t launch_grad_b(const T* tab, long long tab_stride, const T* F, const LevelB& lv, long long kper, int splits,
                          int reff, int tau_pad, T* part, cudaStream_t st) {
    dim3 grid((unsigned)splits, (unsigned)((tau_pad + 63) / 64), (unsigned)((lv.tau + 15) / 16));
    k_grad_b<T><<<grid, 256, 0, st>>>(tab, tab_stride, F, lv, kper, reff, tau_pad, part);
    return cudaGetLastError();
}
template cudaError_t launch_grad_b<float>(const float*, long long, const float*, const LevelB&, long long, int, int, int,
                                          float*, cudaStream_t);
template cudaError_t launch_grad_b<double>(const double*, long long, const double*, const LevelB&, long long, int, int,
                                           int, double*, cudaStream_t);

}  // namespace qmc
