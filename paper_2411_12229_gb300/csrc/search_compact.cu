// search_compact.cu -- the compact search kernel (search_compact.cuh) for
// d <= 256 (CH = 1, 2), and the dispatch to the instantiations for larger d
// (search_compact_wide.cu).
#include "search_compact.cuh"

namespace sqg {

// (d chunks CH, neighbours per lane NR, beam slots per lane NB, lean build)
// -> the instantiation; lean 1 is the build for one more resident block
// per SM (out-degree 32 only)
#define SQG_COMPACT_SWITCH(CALL)                                            \
    switch (ch * 1000 + nr * 100 + bnb * 10 + (lean == 1 && nr == 1 ? 1 : 0)) { \
        case 1120: return CALL(1, 1, 2, 8);                                 \
        case 1121: return CALL(1, 1, 2, 9);                                 \
        case 2120: return CALL(2, 1, 2, 8);                                 \
        case 2121: return CALL(2, 1, 2, 9);                                 \
        case 1140: return CALL(1, 1, 4, 7);                                 \
        case 1141: return CALL(1, 1, 4, 8);                                 \
        case 2140: return CALL(2, 1, 4, 7);                                 \
        case 2141: return CALL(2, 1, 4, 8);                                 \
        case 1220: return CALL(1, 2, 2, 6);                                 \
        case 2220: return CALL(2, 2, 2, 6);                                 \
        case 1240: return CALL(1, 2, 4, 6);                                 \
        case 2240: return CALL(2, 2, 4, 6);                                 \
        default: return cudaErrorInvalidValue;                              \
    }

cudaError_t launch_search_compact(int ch, int nr, int bnb, int lean, dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, const SearchArgs &a) {
    if (ch > 2) return launch_search_compact_wide(ch, nr, bnb, grid, block, smem, s, a);
#define CALL(C, R, N, M) compact_launch_one<C, R, N, M>(grid, block, smem, s, a)
    SQG_COMPACT_SWITCH(CALL)
#undef CALL
}

cudaError_t search_occupancy_compact(int ch, int nr, int bnb, int lean, int block, size_t smem, int *blocks_per_sm) {
    if (ch > 2) return search_occupancy_compact_wide(ch, nr, bnb, block, smem, blocks_per_sm);
#define CALL(C, R, N, M) compact_occ_one<C, R, N, M>(block, smem, blocks_per_sm)
    SQG_COMPACT_SWITCH(CALL)
#undef CALL
}

}  // namespace sqg
