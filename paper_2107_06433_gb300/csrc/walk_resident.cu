// a3 x t + a4 in one launch: the iteration-resident form of the fused walk.
#include "walk.cuh"

namespace swmd {

cudaError_t launch_resident(const ResidentArgs &a, Mapping m, int kprec, int sms,
                            cudaStream_t s) {
    switch (kprec) {
        case 0: return dispatch_resident<float>(a, m, sms, s);
        case 1: return dispatch_resident<__nv_bfloat16>(a, m, sms, s);
        case 2: return dispatch_resident<__half>(a, m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
