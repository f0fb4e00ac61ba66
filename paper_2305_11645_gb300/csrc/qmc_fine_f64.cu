// FP64 instantiations of the fine-band kernels (see qmc_fine.cuh): the FP64 tier
// uses the single-level band (S1) or no band (S0).
#include "qmc_fine.cuh"

namespace qmc {

template <class BandT, int CW>
static cudaError_t fwd_d(const FineArgs<double>& a, int F, int mode, dim3 grid, cudaStream_t st) {
    if (mode == MODE_MATERIALIZE) {
        k_fine_fwd<double, BandT, F_NONE, MODE_MATERIALIZE, CW, false><<<grid, 128, 0, st>>>(a);
        return cudaGetLastError();
    }
    switch (F) {
        case F_LINEAR_MEAN: k_fine_fwd<double, BandT, F_LINEAR_MEAN, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        case F_MEAN_COS: k_fine_fwd<double, BandT, F_MEAN_COS, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        case F_CALL_MEAN_EXP: k_fine_fwd<double, BandT, F_CALL_MEAN_EXP, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        case F_GAUSS_NORM2: k_fine_fwd<double, BandT, F_GAUSS_NORM2, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        case F_PDE_INV_SQ: k_fine_fwd<double, BandT, F_PDE_INV_SQ, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        case F_LOGSUMEXP: k_fine_fwd<double, BandT, F_LOGSUMEXP, MODE_FUSED, CW, false><<<grid, 128, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class BandT, int CW>
static cudaError_t bwd_d(const FineArgs<double>& a, int F, dim3 grid, cudaStream_t st) {
    switch (F) {
        case F_LINEAR_MEAN: k_fine_bwd<double, BandT, F_LINEAR_MEAN, CW, false><<<grid, 256, 0, st>>>(a); break;
        case F_MEAN_COS: k_fine_bwd<double, BandT, F_MEAN_COS, CW, false><<<grid, 256, 0, st>>>(a); break;
        case F_CALL_MEAN_EXP: k_fine_bwd<double, BandT, F_CALL_MEAN_EXP, CW, false><<<grid, 256, 0, st>>>(a); break;
        case F_GAUSS_NORM2: k_fine_bwd<double, BandT, F_GAUSS_NORM2, CW, false><<<grid, 256, 0, st>>>(a); break;
        case F_PDE_INV_SQ: k_fine_bwd<double, BandT, F_PDE_INV_SQ, CW, false><<<grid, 256, 0, st>>>(a); break;
        case F_LOGSUMEXP: k_fine_bwd<double, BandT, F_LOGSUMEXP, CW, false><<<grid, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
cudaError_t launch_fine_fwd<double>(const FineArgs<double>& a, int shape, bool, int F, int mode, dim3 grid,
                                    cudaStream_t st) {
    switch (shape) {
        case SHAPE_S1: return fwd_d<BandS1, 2>(a, F, mode, grid, st);
        case SHAPE_S0: return fwd_d<BandS0, 2>(a, F, mode, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_fine_bwd<double>(const FineArgs<double>& a, int shape, bool, int F, dim3 grid, cudaStream_t st) {
    switch (shape) {
        case SHAPE_S1: return bwd_d<BandS1, 1>(a, F, grid, st);
        case SHAPE_S0: return bwd_d<BandS0, 2>(a, F, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
