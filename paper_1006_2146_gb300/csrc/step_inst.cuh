// Instantiates the predictor + face kernel for one (order, variable count,
// precision); included by the small step_o*_*.cu translation units so that
// the build compiles them in parallel.  Expects ADER_ORDER, ADER_NV, ADER_REAL;
// with ADER_SPLIT_VARIANTS the unit holds only the dispatch and the kernel
// variants come from units that also define ADER_FORM and ADER_SRC.
#include "step_kernels.cuh"
#include "zone_o2.cuh"
#include "zone_o3.cuh"
#include "zone_o4.cuh"

namespace ader {

#define ADER_ZONEOPS(O)                                                                                              \
    template <> struct ZoneOps<O> {                                                                                  \
        template <int NV, class R> static ADER_DEV void predict_modal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& n) { \
            o##O::predict_modal(m, gm1, cx, cy, cz, n);                                                              \
        }                                                                                                            \
        template <int NV, class R> static ADER_DEV void predict_nodal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& n) { \
            o##O::predict_nodal(m, gm1, cx, cy, cz, n);                                                              \
        }                                                                                                            \
        template <int D, int NV, class R>                                                                            \
        static ADER_DEV void face(const Vec<NV, R>* p, R gm1, Vec<NV, R>& ub, Vec<NV, R>& avg, Vec<NV, R>& Fa) {     \
            o##O::face<D>(p, gm1, ub, avg, Fa);                                                                       \
        }                                                                                                            \
        template <int D, class R>                                                                                    \
        static ADER_DEV void face_mhd(const Vec<8, R>* p, R gm1, Vec<8, R>& ub, Vec<8, R>& avg, Vec<8, R>& Fa, R* eu, \
                                      R* ef) {                                                                       \
            o##O::face_mhd<D>(p, gm1, ub, avg, Fa, eu, ef);                                                           \
        }                                                                                                            \
        static constexpr bool HAS_SOURCE = o##O::HAS_SOURCE;                                                         \
        static constexpr bool HAS_SOURCE_MODAL = o##O::HAS_SOURCE_MODAL;                                             \
        template <int NV, class R>                                                                                   \
        static ADER_DEV void predict_modal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& n, const Src<R>& s,  \
                                               Vec<NV, R>& sdt) {                                                    \
            o##O::predict_modal_src(m, gm1, cx, cy, cz, n, s, sdt);                                                  \
        }                                                                                                            \
        template <int NV, class R>                                                                                   \
        static ADER_DEV void predict_nodal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& n, const Src<R>& s,  \
                                               Vec<NV, R>& sdt) {                                                    \
            o##O::predict_nodal_src(m, gm1, cx, cy, cz, n, s, sdt);                                                  \
        }                                                                                                            \
        static constexpr bool HAS_FACE_PAIR = o##O::HAS_FACE_PAIR;                                                   \
        template <int D, int NV, class R>                                                                            \
        static ADER_DEV void face_pair(const Vec<NV, R>* p, R gm1, Vec<NV, R>* ub, Vec<NV, R>* avg, Vec<NV, R>* Fa) {  \
            o##O::face_pair<D>(p, gm1, ub, avg, Fa);                                                                  \
        }                                                                                                            \
        template <int D, class R>                                                                                    \
        static ADER_DEV void edge_states(const Vec<8, R>* p, const Vec<8, R>& ub, const Vec<8, R>& avg, Vec<8, R>* e) { \
            o##O::edge_states<D>(p, ub, avg, e);                                                                      \
        }                                                                                                            \
    };

#ifndef ADER_ZONEOPS_DEFINED
#define ADER_ZONEOPS_DEFINED
ADER_ZONEOPS(2)
ADER_ZONEOPS(3)
ADER_ZONEOPS(4)
#endif

#ifdef ADER_ORDER
#ifdef ADER_FORM
// a translation unit of one kernel variant (ADER_FORM, ADER_SRC)
template void launch_pf_variant<ADER_ORDER, ADER_FORM, ADER_NV, ADER_REAL, ADER_SRC>(const StepArgs&, const double*,
                                                                                     cudaStream_t);
#else
#ifdef ADER_SPLIT_VARIANTS
// the variants are compiled in their own translation units (step_o*_*_<form>_<src>.cu)
extern template void launch_pf_variant<ADER_ORDER, FORM_MODAL, ADER_NV, ADER_REAL, false>(const StepArgs&,
                                                                                          const double*, cudaStream_t);
extern template void launch_pf_variant<ADER_ORDER, FORM_NODAL, ADER_NV, ADER_REAL, false>(const StepArgs&,
                                                                                          const double*, cudaStream_t);
extern template void launch_pf_variant<ADER_ORDER, FORM_MODAL, ADER_NV, ADER_REAL, true>(const StepArgs&,
                                                                                         const double*, cudaStream_t);
extern template void launch_pf_variant<ADER_ORDER, FORM_NODAL, ADER_NV, ADER_REAL, true>(const StepArgs&,
                                                                                         const double*, cudaStream_t);
#endif
template int launch_predict_faces_nv<ADER_ORDER, ADER_NV, ADER_REAL>(const StepArgs&, const double*, cudaStream_t);
#endif
#endif

}  // namespace ader
