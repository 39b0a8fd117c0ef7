// The register-resident solver (resident_regs.cuh): the (VRP, rows per lane)
// pairs it is compiled for, and the dispatch to one translation unit per K precision.
#include "common.cuh"

namespace swmd {

int regs_rows_per_lane(int vrp, int want) {
    if (vrp > 32) return 0;   // not supported: the shared-memory tiled solver takes over
    const int def = vrp <= 8 ? 8 : (vrp <= 20 ? 4 : 2);
    if (want <= 0) return def;
    // the (VRP, rows per lane) pairs compiled in resident_regs.cuh
    static const int ok[][2] = {{4, 8}, {8, 8}, {12, 4}, {16, 4}, {20, 4}, {24, 2}, {28, 2},
                                {32, 2}, {12, 8}, {16, 2}, {20, 2}, {20, 3}, {24, 3}, {32, 1},
                                {24, 4}};
    for (auto &e : ok)
        if (e[0] == vrp && e[1] == want) return want;
    return def;
}

cudaError_t launch_resident_regs(const ResidentArgs &a, int vrp, int kprec, const TaskSet &ts,
                                 int sms, cudaStream_t s, int nq, const ResidentArgs *batch) {
    switch (kprec) {
        case 0: return launch_regs_fp32(a, vrp, ts, sms, s, nq, batch);
        case 1: return launch_regs_bf16(a, vrp, ts, sms, s, nq, batch);
        case 2: return launch_regs_fp16(a, vrp, ts, sms, s, nq, batch);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
