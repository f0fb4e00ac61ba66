// FP32 instantiations of the fine-band kernels (see qmc_fine.cuh).
#include "qmc_fine.cuh"

namespace qmc {

template <class BandT, int CW, bool EXACT>
static cudaError_t fwd_f(const FineArgs<float>& a, int F, int mode, dim3 grid, cudaStream_t st) {
    if (mode == MODE_MATERIALIZE) {
        k_fine_fwd<float, BandT, F_NONE, MODE_MATERIALIZE, CW, EXACT><<<grid, 128, 0, st>>>(a);
        return cudaGetLastError();
    }
    switch (F) {
        case F_LINEAR_MEAN: k_fine_fwd<float, BandT, F_LINEAR_MEAN, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        case F_MEAN_COS: k_fine_fwd<float, BandT, F_MEAN_COS, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        case F_CALL_MEAN_EXP: k_fine_fwd<float, BandT, F_CALL_MEAN_EXP, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        case F_GAUSS_NORM2: k_fine_fwd<float, BandT, F_GAUSS_NORM2, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        case F_PDE_INV_SQ: k_fine_fwd<float, BandT, F_PDE_INV_SQ, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        case F_LOGSUMEXP: k_fine_fwd<float, BandT, F_LOGSUMEXP, MODE_FUSED, CW, EXACT><<<grid, 128, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class BandT, int CW, bool EXACT>
static cudaError_t bwd_f(const FineArgs<float>& a, int F, dim3 grid, cudaStream_t st) {
    switch (F) {
        case F_LINEAR_MEAN: k_fine_bwd<float, BandT, F_LINEAR_MEAN, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        case F_MEAN_COS: k_fine_bwd<float, BandT, F_MEAN_COS, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        case F_CALL_MEAN_EXP: k_fine_bwd<float, BandT, F_CALL_MEAN_EXP, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        case F_GAUSS_NORM2: k_fine_bwd<float, BandT, F_GAUSS_NORM2, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        case F_PDE_INV_SQ: k_fine_bwd<float, BandT, F_PDE_INV_SQ, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        case F_LOGSUMEXP: k_fine_bwd<float, BandT, F_LOGSUMEXP, CW, EXACT><<<grid, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
cudaError_t launch_fine_fwd<float>(const FineArgs<float>& a, int shape, bool exact, int F, int mode, dim3 grid,
                                   cudaStream_t st) {
    switch (shape) {
        case SHAPE_S4:
            return exact ? fwd_f<BandS4, 4, true>(a, F, mode, grid, st) : fwd_f<BandS4, 4, false>(a, F, mode, grid, st);
        case SHAPE_S1: return fwd_f<BandS1, 4, false>(a, F, mode, grid, st);
        case SHAPE_S0: return fwd_f<BandS0, 4, false>(a, F, mode, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_fine_bwd<float>(const FineArgs<float>& a, int shape, bool exact, int F, dim3 grid,
                                   cudaStream_t st) {
    switch (shape) {
        case SHAPE_S4: return exact ? bwd_f<BandS4, 2, true>(a, F, grid, st) : bwd_f<BandS4, 2, false>(a, F, grid, st);
        case SHAPE_S1: return bwd_f<BandS1, 2, false>(a, F, grid, st);
        case SHAPE_S0: return bwd_f<BandS0, 4, false>(a, F, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
