// a4: the final step of Algorithm 1 (SDDMM_SpMM type 2) and the distance.
#include "walk3.cuh"

namespace swmd {

cudaError_t launch_final(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk_prec<Kind::Final>(a, m, kprec, sms, s);
}

bool mapping_supported(Mapping m) {
    const int key = m.vrp * 10000 + m.q * 100 + m.p;
    switch (key) {
#define SWMD_CASE(V, QQ, PP) \
    case V * 10000 + QQ * 100 + PP: return true;
        SWMD_WALK_MAPPINGS(SWMD_CASE)
#undef SWMD_CASE
        default: return false;
    }
}

// VRP for v_r query words and Q lanes per nonzero: a multiple of 4Q that the
// cost kernel also supports (steps of 4 up to 32, of 8 up to 64, of 16 up to 128).
int vrp_for(int vr, int q) {
    int g = 4;
    if (vr > 32) g = 8;
    if (vr > 64) g = 16;
    if (g < 4 * q) g = 4 * q;
    int v = (vr + g - 1) / g * g;
    if (v > 32 && v % 8) v = (v + 7) / 8 * 8;
    if (v > 64 && v % 16) v = (v + 15) / 16 * 16;
    return v;
}


cudaError_t launch_final3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    return dispatch_walk3_prec<Kind::Final>(a, vrp, kprec, sms, s);
}

}  // namespace swmd
