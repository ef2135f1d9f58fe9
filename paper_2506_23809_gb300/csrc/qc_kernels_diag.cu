// qc_kernels_diag.cu -- the local-energy kernel's diagnostic instantiations: the same kernels as
// qc_kernels.cu with the pair-by-pair hit lists and the work counters compiled in.  An
// evaluation that asks for either (qc_eloc_out.hit_list, QC_OPT_COUNT_WORK) runs these; timed
// evaluations run the others, which carry none of the checks.
#include "qc_main_kernel.cuh"

namespace qc {

cudaError_t launch_eloc_main_diag(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                                  const LaunchCfg& c, cudaStream_t s) {
    return launch_main_variant<true>(sp, tp, ep, c, s);
}

cudaError_t prepare_kernels_diag(size_t max_smem) { return prepare_variant<true>(max_smem); }

}  // namespace qc
