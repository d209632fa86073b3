// Batched order-4 euler phases in FP32 bulk (see batch_inst.cuh).
#define ADER_BORDER 4
#define ADER_BNV 5
#include "batch_inst.cuh"
