// search_inst.cuh -- instantiations of the search kernel and its launch helpers.
//
// CH = float4 chunks of the raw vector per lane (d <= 128*CH); NB = R/32
// neighbours per lane.  One unit per NB keeps the builds parallel.
#include "search.cuh"

#ifndef SQG_NB
#error "define SQG_NB (1 or 2) before including search_inst.cuh"
#endif

namespace sqg {

template <int CH>
static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
    auto fn = search_kernel<CH, SQG_NB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CH>
static cudaError_t occ_one(int block, size_t smem, int *nb) {
    auto fn = search_kernel<CH, SQG_NB>;
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

cudaError_t SQG_LAUNCH_NAME(int ch, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
#define CALL(X) launch_one<X>(grid, block, smem, s, a)
    switch (ch) {
        case 1: return CALL(1);
        case 2: return CALL(2);
        case 4: return CALL(4);
        case 8: return CALL(8);
        case 12: return CALL(12);
        case 16: return CALL(16);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t SQG_OCC_NAME(int ch, int block, size_t smem, int *nb) {
#define CALL(X) occ_one<X>(block, smem, nb)
    switch (ch) {
        case 1: return CALL(1);
        case 2: return CALL(2);
        case 4: return CALL(4);
        case 8: return CALL(8);
        case 12: return CALL(12);
        case 16: return CALL(16);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace sqg
