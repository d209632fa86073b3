// Order-4 instantiation of the predictor + face kernel (see step_kernels.cuh).
#include "step_kernels.cuh"
#include "zone_o4.cuh"

namespace ader {

template <> struct ZoneOps<4> {
    template <class R> static ADER_DEV void predict_modal(Vec<5, R>* m, R gm1, R cx, R cy, R cz, int n) {
        o4::predict_modal(m, gm1, cx, cy, cz, n);
    }
    template <class R> static ADER_DEV void predict_nodal(Vec<5, R>* m, R gm1, R cx, R cy, R cz, int n) {
        o4::predict_nodal(m, gm1, cx, cy, cz, n);
    }
    template <int D, class R> static ADER_DEV void face(const Vec<5, R>* p, R gm1, Vec<5, R>& ub, Vec<5, R>& avg, Vec<5, R>& Fa) {
        o4::face<D>(p, gm1, ub, avg, Fa);
    }
};

template int launch_predict_faces_order<4, double>(const StepArgs&, const double*, cudaStream_t);
template int launch_predict_faces_order<4, float>(const StepArgs&, const double*, cudaStream_t);

}  // namespace ader
