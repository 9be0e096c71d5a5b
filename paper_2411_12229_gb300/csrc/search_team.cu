// search_team.cu -- search kernels with teams of 16 or 8 lanes per query (2 or
// 4 queries per warp), for d <= 256 (CH 1, 2) and out-degree 32 or 64.
#include "search.cuh"

namespace sqg {

template <int CH, int NB, int T>
static cudaError_t team_launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
    auto fn = search_kernel<CH, NB, false, T>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CH, int NB, int T>
static cudaError_t team_occ_one(int block, size_t smem, int *nb) {
    auto fn = search_kernel<CH, NB, false, T>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, fn, block, smem);
}

#define SQG_TEAM_SWITCH(CALL)                                 \
    switch (ch * 100 + nb * 10 + (team == 16 ? 1 : team == 8 ? 2 : 0)) { \
        case 111: return CALL(1, 1, 16);                      \
        case 112: return CALL(1, 1, 8);                       \
        case 121: return CALL(1, 2, 16);                      \
        case 122: return CALL(1, 2, 8);                       \
        case 211: return CALL(2, 1, 16);                      \
        case 212: return CALL(2, 1, 8);                       \
        case 221: return CALL(2, 2, 16);                      \
        case 222: return CALL(2, 2, 8);                       \
        default: return cudaErrorInvalidValue;                \
    }

cudaError_t launch_search_team(int ch, int nb, int team, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               const SearchArgs &a) {
#define CALL(C, N, T) team_launch_one<C, N, T>(grid, block, smem, s, a)
    SQG_TEAM_SWITCH(CALL)
#undef CALL
}

cudaError_t search_occupancy_team(int ch, int nb, int team, int block, size_t smem, int *blocks_per_sm) {
#define CALL(C, N, T) team_occ_one<C, N, T>(block, smem, blocks_per_sm)
    SQG_TEAM_SWITCH(CALL)
#undef CALL
}

}  // namespace sqg
