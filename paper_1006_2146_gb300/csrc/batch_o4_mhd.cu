// Batched order-4 mhd phases in FP32 bulk (see batch_inst.cuh).
#define ADER_BORDER 4
#define ADER_BNV 8
#include "batch_inst.cuh"
