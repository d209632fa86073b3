// Batched order-3 mhd phases in FP32 bulk (see batch_inst.cuh).
#define ADER_BORDER 3
#define ADER_BNV 8
#include "batch_inst.cuh"
