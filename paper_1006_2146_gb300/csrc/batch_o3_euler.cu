// Batched order-3 euler phases in FP32 bulk (see batch_inst.cuh).
#define ADER_BORDER 3
#define ADER_BNV 5
#include "batch_inst.cuh"
