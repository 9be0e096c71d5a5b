// search_compact_big.cu -- the compact search kernel (search_compact.cuh)
// for d <= 256 with beams of 129-256 entries (NB = 8 slots per lane) or
// with 33-128 results (RK = 4 slots per lane), plain and with the learned
// stop fused.  Resident blocks of 4 warps per SM: the most at which the
// build does not spill (80 registers for 6 blocks, 96 for 5).
#include "search_compact.cuh"

namespace sqg {

// (d chunks CH, neighbours per lane NR, beam slots per lane NB, result
// slots per lane RK) -> (resident blocks of the plain build, of the stop build)
#define SQG_COMPACT_BIG_SWITCH(CALL)                                   \
    switch (ch * 1000 + nr * 100 + bnb * 10 + rk) {                   \
        case 1181: return stop ? CALL(1, 1, 8, 6, true, 1) : CALL(1, 1, 8, 7, false, 1); \
        case 1124: return stop ? CALL(1, 1, 2, 6, true, 4) : CALL(1, 1, 2, 7, false, 4); \
        case 1144: return stop ? CALL(1, 1, 4, 5, true, 4) : CALL(1, 1, 4, 6, false, 4); \
        case 1184: return stop ? CALL(1, 1, 8, 5, true, 4) : CALL(1, 1, 8, 6, false, 4); \
        case 1281: return stop ? CALL(1, 2, 8, 5, true, 1) : CALL(1, 2, 8, 6, false, 1); \
        case 1224: return stop ? CALL(1, 2, 2, 5, true, 4) : CALL(1, 2, 2, 6, false, 4); \
        case 1244: return stop ? CALL(1, 2, 4, 5, true, 4) : CALL(1, 2, 4, 6, false, 4); \
        case 1284: return stop ? CALL(1, 2, 8, 4, true, 4) : CALL(1, 2, 8, 5, false, 4); \
        case 2181: return stop ? CALL(2, 1, 8, 5, true, 1) : CALL(2, 1, 8, 6, false, 1); \
        case 2124: return stop ? CALL(2, 1, 2, 5, true, 4) : CALL(2, 1, 2, 6, false, 4); \
        case 2144: return stop ? CALL(2, 1, 4, 5, true, 4) : CALL(2, 1, 4, 6, false, 4); \
        case 2184: return stop ? CALL(2, 1, 8, 5, true, 4) : CALL(2, 1, 8, 5, false, 4); \
        case 2281: return stop ? CALL(2, 2, 8, 5, true, 1) : CALL(2, 2, 8, 5, false, 1); \
        case 2224: return stop ? CALL(2, 2, 2, 5, true, 4) : CALL(2, 2, 2, 5, false, 4); \
        case 2244: return stop ? CALL(2, 2, 4, 5, true, 4) : CALL(2, 2, 4, 5, false, 4); \
        case 2284: return stop ? CALL(2, 2, 8, 4, true, 4) : CALL(2, 2, 8, 5, false, 4); \
        default: return cudaErrorInvalidValue;                        \
    }

cudaError_t launch_search_compact_big(int ch, int nr, int bnb, int rk, bool stop, dim3 grid, dim3 block, size_t smem,
                                      cudaStream_t s, const SearchArgs &a) {
#define CALL(C, R, N, M, S, K) compact_launch_one<C, R, N, M, S, K>(grid, block, smem, s, a)
    SQG_COMPACT_BIG_SWITCH(CALL)
#undef CALL
}

cudaError_t search_occupancy_compact_big(int ch, int nr, int bnb, int rk, bool stop, int block, size_t smem,
                                         int *blocks_per_sm) {
#define CALL(C, R, N, M, S, K) compact_occ_one<C, R, N, M, S, K>(block, smem, blocks_per_sm)
    SQG_COMPACT_BIG_SWITCH(CALL)
#undef CALL
}

}  // namespace sqg
