// a3: the fused SDDMM-SpMM iteration (Section III-C, SDDMM_SpMM type 1).
#include "walk3.cuh"

namespace swmd {

cudaError_t launch_fused(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk_prec<Kind::Fused>(a, m, kprec, sms, s);
}


cudaError_t launch_fused3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk3_prec<Kind::Fused>(a, vrp, kprec, sms, s);
}

}  // namespace swmd
