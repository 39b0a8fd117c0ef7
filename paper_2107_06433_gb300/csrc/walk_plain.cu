// The unfused iteration: SDDMM (Algorithm 2) writing v, then SpMM (Algorithm 3)
// reading it back -- the separate-kernel formulation Section III-C improves on.
#include "walk3.cuh"

namespace swmd {

cudaError_t launch_sddmm(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk_prec<Kind::Sddmm>(a, m, kprec, sms, s);
}

cudaError_t launch_spmm(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk_prec<Kind::Spmm>(a, m, kprec, sms, s);
}


cudaError_t launch_sddmm3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk3_prec<Kind::Sddmm>(a, vrp, kprec, sms, s);
}

cudaError_t launch_spmm3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk3_prec<Kind::Spmm>(a, vrp, kprec, sms, s);
}

}  // namespace swmd
