// search_inst.cuh -- instantiations of the search kernel and its launch helpers.
//
// CH = float4 chunks of the raw vector per lane (d <= 128*CH); NB = R/32
// neighbours per lane; lean = the 64-register build (CH <= 2 only).  One
// unit per NB keeps the builds parallel.
#include "search.cuh"

#ifndef SQG_NB
#error "define SQG_NB (1 or 2) before including search_inst.cuh"
#endif

namespace sqg {

template <int CH, bool LEAN>
static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
    auto fn = search_kernel<CH, SQG_NB, LEAN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CH, bool LEAN>
static cudaError_t occ_one(int block, size_t smem, int *nb) {
    auto fn = search_kernel<CH, SQG_NB, LEAN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, fn, block, smem);
}

#if SQG_NB == 1
#define SQG_LAUNCH_NAME launch_search_nb1
#define SQG_OCC_NAME search_occupancy_nb1
#else
#define SQG_LAUNCH_NAME launch_search_nb2
#define SQG_OCC_NAME search_occupancy_nb2
#endif

// ch < 0 selects the lean build of |ch| (1 or 2).
cudaError_t SQG_LAUNCH_NAME(int ch, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
#define CALL(X, L) launch_one<X, L>(grid, block, smem, s, a)
    switch (ch) {
        case -1: return CALL(1, true);
        case -2: return CALL(2, true);
        case 1: return CALL(1, false);
        case 2: return CALL(2, false);
        case 4: return CALL(4, false);
        case 8: return CALL(8, false);
        case 12: return CALL(12, false);
        case 16: return CALL(16, false);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t SQG_OCC_NAME(int ch, int block, size_t smem, int *nb) {
#define CALL(X, L) occ_one<X, L>(block, smem, nb)
    switch (ch) {
        case -1: return CALL(1, true);
        case -2: return CALL(2, true);
        case 1: return CALL(1, false);
        case 2: return CALL(2, false);
        case 4: return CALL(4, false);
        case 8: return CALL(8, false);
        case 12: return CALL(12, false);
        case 16: return CALL(16, false);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace sqg
