// Order-4 MHD predictor + face kernel in F32 (see step_inst.cuh): the dispatch; each
// kernel variant is compiled in its own unit, step_o4_mhd_f32_<form>_<source>.cu.
#define ADER_ORDER 4
#define ADER_NV 8
#define ADER_REAL float
#define ADER_SPLIT_VARIANTS 1
#include "step_inst.cuh"
