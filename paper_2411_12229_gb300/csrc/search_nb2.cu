// search_nb2.cu -- search kernels for out-degree 64 (two neighbours per lane).
#define SQG_NB 2
#include "search_inst.cuh"
