// Instantiates the batched phases for one (order, variable count) in FP32
// bulk; included by the small batch_o*_*.cu translation units.  Expects
// ADER_BORDER and ADER_BNV.
#include "batch.cuh"
#include "step_inst.cuh"

namespace ader {

template <int ORDER, int NV>
int batch_phase(int ph, const BatchGroupDev& g, int form, int solver, int threads, int blocks, cudaStream_t st,
                bool launch, const void** fn) {
    using R = float;
    const void* k = nullptr;
    switch (ph) {
        case PH_TO_F32: k = (const void*)kb_to_f32; break;
        case PH_FACE_B:
            if constexpr (NV == 8) k = (const void*)kb_face_b<ORDER, R>;
            break;
        case PH_WENO1D: k = (const void*)kb_weno1d<ORDER, NV, R>; break;
        case PH_CROSS1:
            if constexpr (ORDER >= 3) k = (const void*)kb_cross1<ORDER, NV, R>;
            break;
        case PH_CROSS2:
            if constexpr (ORDER == 4) k = (const void*)kb_cross2<NV, R>;
            break;
        case PH_PREDICT:
            k = form == FORM_NODAL ? (const void*)kb_predict_faces<ORDER, FORM_NODAL, NV, R>
                                   : (const void*)kb_predict_faces<ORDER, FORM_MODAL, NV, R>;
            break;
        case PH_UPDATE:
            k = solver == SOLVER_LINEARIZED ? (const void*)kb_flux_update<SOLVER_LINEARIZED, NV, R>
                                            : (const void*)kb_flux_update<SOLVER_HLL, NV, R>;
            break;
        case PH_EMF:
            if constexpr (NV == 8) k = (const void*)kb_emf<R>;
            break;
        case PH_CT:
            if constexpr (NV == 8) k = (const void*)kb_ct<R>;
            break;
        default: break;
    }
    if (fn) *fn = k;
    if (!k || !launch) return k ? 1 : 0;
    void* args[] = {(void*)&g};
    return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3((unsigned)threads), args, 0, st) == cudaSuccess ? 1 : -1;
}

template int batch_phase<ADER_BORDER, ADER_BNV>(int, const BatchGroupDev&, int, int, int, int, cudaStream_t, bool,
                                                const void**);

}  // namespace ader
