// search_compact_stop.cu -- the compact search kernel (search_compact.cuh)
// with the learned early stop fused, for every d and out-degree it serves.
// The stop keeps its hop-to-hop state and (d <= 256) its features in shared
// memory, so the builds run at the plain build's resident blocks per SM or
// one fewer: at d <= 256 with out-degree 32 and NB = 2 the plain build's 64
// registers hold the stop too, but measured 7 % slower than 72 registers
// and one block fewer (the search loop compiled around the stop's state).
#include "search_compact.cuh"

namespace sqg {

#define SQG_COMPACT_STOP_SWITCH(CALL)                  \
    switch (ch * 100 + nr * 10 + bnb) {                \
        case 112: return CALL(1, 1, 2, 7);             \
        case 114: return CALL(1, 1, 4, 7);             \
        case 122: return CALL(1, 2, 2, 6);             \
        case 124: return CALL(1, 2, 4, 6);             \
        case 212: return CALL(2, 1, 2, 7);             \
        case 214: return CALL(2, 1, 4, 6);             \
        case 222: return CALL(2, 2, 2, 6);             \
        case 224: return CALL(2, 2, 4, 5);             \
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

cudaError_t launch_search_compact_stop(int ch, int nr, int bnb, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                       const SearchArgs &a) {
#define CALL(C, R, N, M) compact_launch_one<C, R, N, M, true>(grid, block, smem, s, a)
    SQG_COMPACT_STOP_SWITCH(CALL)
#undef CALL
}

cudaError_t search_occupancy_compact_stop(int ch, int nr, int bnb, int block, size_t smem, int *blocks_per_sm) {
#define CALL(C, R, N, M) compact_occ_one<C, R, N, M, true>(block, smem, blocks_per_sm)
    SQG_COMPACT_STOP_SWITCH(CALL)
#undef CALL
}

}  // namespace sqg
