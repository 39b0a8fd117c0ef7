// The register-resident solver with FP32 K^T rows (one K precision per
// translation unit, so the instantiations compile in parallel).
#include "resident_regs.cuh"

namespace swmd {

cudaError_t launch_regs_fp32(const ResidentArgs &a, int vrp, const TaskSet &ts, int sms, cudaStream_t s,
                              int nq, const ResidentArgs *batch) {
    return dispatch_regs<float>(a, vrp, ts, sms, s, nq, batch);
}

}  // namespace swmd
