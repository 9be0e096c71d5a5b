// search_nb1.cu -- search kernels for out-degree 32 (one neighbour per lane).
#define SQG_NB 1
#include "search_inst.cuh"
