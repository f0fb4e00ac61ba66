// Point generation kernels: the distinct-row table that every product kernel
// reads (one period of every column, shifted and transformed), and the
// user-facing bit-exact point dumps of qmc_gen_points.
#include "qmc_internal.cuh"

namespace qmc {

// Level of table index g (levels are few; linear scan over the prefix sums).
// the level I with lev_tab[I] <= g < lev_tab[I + 1] (binary search; empty levels have
// lev_tab[I] == lev_tab[I + 1] and are never returned for a valid g)
__device__ __forceinline__ int level_of(const DevRule& R, long long g) {
    int lo = 0, hi = R.nlev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g >= R.lev_tab[mid]) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Column j's level: the largest I with lev_col0[I] <= j among non-empty levels.
__device__ __forceinline__ int level_of_col(const DevRule& R, int j) {
    int lvl = 0;
    for (int I = 0; I < R.nlev; ++I)
        if (R.lev_tau[I] > 0 && R.lev_col0[I] <= j) lvl = I;
    return lvl;
}

// Distinct-row table: tab[r*T_tot + lev_tab[I] + (j - col0_I) * n_I + row] = phi(X32 of x_{row,j}, shift r).
// It is the first kernel of every forward pass and also clears the ticket that the
// row finalisation uses to elect the block that forms the estimates.
template <class T>
__global__ void k_table(const __grid_constant__ DevRule R, T* __restrict__ tab, long long T_tot, long long stride,
                        int reff, unsigned int* ticket) {
    if (ticket && blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0u;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < T_tot;
         g += (long long)gridDim.x * blockDim.x) {
        if (R.kind == KIND_MC) {        // reduced MC (Sec. 5): replica r's samples are in the table's layout
            for (int r = 0; r < reff; ++r)
                tab[(long long)r * stride + g] = Tr<T>::apply(__ldg(R.gen + (long long)r * T_tot + g), R.transform);
            continue;
        }
        const int I = level_of(R, g);
        const int q = R.m - I;                              // 2^q rows per column at this level
        const long long idx = g - R.lev_tab[I];
        const int j = R.lev_col0[I] + (int)(idx >> q);
        const uint32_t row = (uint32_t)(idx & ((1LL << q) - 1));
        const uint32_t x0 = unshifted_x32(R, j, row, q);
#pragma unroll 4
        for (int r = 0; r < reff; ++r) {
            const uint32_t x = R.shift ? apply_shift(R.kind, x0, R.shift[(size_t)r * R.s + j]) : x0;
            tab[(long long)r * stride + g] = Tr<T>::apply(x, R.transform);
        }
    }
}

template <class T>
cudaError_t launch_table(const DevRule& R, T* tab, long long T_tot, long long stride, int reff, unsigned int* ticket,
                         cudaStream_t st) {
    long long blocks = (T_tot + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_table<T><<<(unsigned)blocks, 256, 0, st>>>(R, tab, T_tot, stride, reff, ticket);
    return cudaGetLastError();
}
template cudaError_t launch_table<float>(const DevRule&, float*, long long, long long, int, unsigned int*, cudaStream_t);
template cudaError_t launch_table<double>(const DevRule&, double*, long long, long long, int, unsigned int*,
                                          cudaStream_t);

// Full layout: out[k*s + j] = X32 of x_{k,j}, row k mod 2^q of column j.
__global__ void k_points_full(DevRule R, uint32_t* __restrict__ out, int shift_idx) {
    const long long total = (1LL << R.m) * R.s;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long k = e / R.s;
        const int j = (int)(e - k * R.s);
        const int I = level_of_col(R, j);
        const int q = R.m - I;
        const uint32_t row = (uint32_t)(k & ((1LL << q) - 1));
        if (R.kind == KIND_MC) {        // eq. randpts: x_{j,k} = y_{j, k mod N_j}
            out[e] = R.gen[(long long)shift_idx * R.T_tot + R.lev_tab[I] + ((long long)(j - R.lev_col0[I]) << q) + row];
            continue;
        }
        uint32_t x = unshifted_x32(R, j, row, q);
        if (R.shift) x = apply_shift(R.kind, x, R.shift[(size_t)shift_idx * R.s + j]);
        out[e] = x;
    }
}

cudaError_t launch_points_full(const DevRule& R, uint32_t* out, int shift_idx, cudaStream_t st) {
    long long total = (1LL << R.m) * R.s;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_points_full<<<(unsigned)blocks, 256, 0, st>>>(R, out, shift_idx);
    return cudaGetLastError();
}

__global__ void k_points_distinct(DevRule R, uint32_t* __restrict__ out, long long T_tot, int shift_idx) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < T_tot;
         g += (long long)gridDim.x * blockDim.x) {
        if (R.kind == KIND_MC) {        // the samples already are one period of every column
            out[g] = R.gen[(long long)shift_idx * T_tot + g];
            continue;
        }
        const int I = level_of(R, g);
        const int q = R.m - I;
        const long long idx = g - R.lev_tab[I];
        const int j = R.lev_col0[I] + (int)(idx >> q);
        const uint32_t row = (uint32_t)(idx & ((1LL << q) - 1));
        uint32_t x = unshifted_x32(R, j, row, q);
        if (R.shift) x = apply_shift(R.kind, x, R.shift[(size_t)shift_idx * R.s + j]);
        out[g] = x;
    }
}

cudaError_t launch_points_distinct(const DevRule& R, uint32_t* out, long long T_tot, int shift_idx,
                                   cudaStream_t st) {
    long long blocks = (T_tot + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_points_distinct<<<(unsigned)blocks, 256, 0, st>>>(R, out, T_tot, shift_idx);
    return cudaGetLastError();
}

// Copy A (s x tau) into a zero-padded s x tau_pad buffer (tau_pad a multiple of 4).
template <class T>
__global__ void k_pad_A(const T* __restrict__ A, T* __restrict__ Ap, int s, int tau, int tau_pad) {
    const long long total = (long long)s * tau_pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / tau_pad;
        const int t = (int)(e - j * tau_pad);
        Ap[e] = (t < tau) ? A[j * tau + t] : T(0);
    }
}

template <class T>
cudaError_t launch_pad_A(const T* A, T* Ap, int s, int tau, int tau_pad, cudaStream_t st) {
    long long total = (long long)s * tau_pad;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_pad_A<T><<<(unsigned)blocks, 256, 0, st>>>(A, Ap, s, tau, tau_pad);
    return cudaGetLastError();
}
template cudaError_t launch_pad_A<float>(const float*, float*, int, int, int, cudaStream_t);
template cudaError_t launch_pad_A<double>(const double*, double*, int, int, int, cudaStream_t);

}  // namespace qmc
