// search_compact_wide.cu -- the compact search kernel (search_compact.cuh)
// for 256 < d <= 1024 (CH = 4, 8): a few resident blocks per SM, bounded by
// the vertex blocks in shared memory (12.8 KB at d = 960, out-degree 64),
// so every build may use many registers.
#include "search_compact.cuh"

namespace sqg {

#define SQG_COMPACT_WIDE_SWITCH(CALL)                  \
    switch (ch * 100 + nr * 10 + bnb) {                \
        case 412: return CALL(4, 1, 2, 4);             \
        case 414: return CALL(4, 1, 4, 4);             \
        case 422: return CALL(4, 2, 2, 4);             \
        case 424: return CALL(4, 2, 4, 4);             \
        case 812: return CALL(8, 1, 2, 3);             \
        case 814: return CALL(8, 1, 4, 3);             \
        case 822: return CALL(8, 2, 2, 3);             \
        case 824: return CALL(8, 2, 4, 3);             \
        default: return cudaErrorInvalidValue;         \
    }

cudaError_t launch_search_compact_wide(int ch, int nr, int bnb, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                       const SearchArgs &a) {
#define CALL(C, R, N, M) compact_launch_one<C, R, N, M>(grid, block, smem, s, a)
    SQG_COMPACT_WIDE_SWITCH(CALL)
#undef CALL
}

cudaError_t search_occupancy_compact_wide(int ch, int nr, int bnb, int block, size_t smem, int *blocks_per_sm) {
#define CALL(C, R, N, M) compact_occ_one<C, R, N, M>(block, smem, blocks_per_sm)
    SQG_COMPACT_WIDE_SWITCH(CALL)
#undef CALL
}

}  // namespace sqg
