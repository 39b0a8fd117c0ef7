// The column-split solver's kernels for task lists that hold the buckets of 48, 64
// and 96 rows (layouts of 16 and 32 columns), in a translation unit of their own.
#include "resident_cols.cuh"

namespace swmd {

cudaError_t launch_resident_cols_long(const ColArgs &a, int vrp, int sms, cudaStream_t s, int nq) {
    switch (vrp) {
        case 16: return run_cols<16, true>(a, sms, nq, s);
        case 32: return run_cols<32, true>(a, sms, nq, s);
        default: return cudaErrorInvalidValue;   // no bucket above 32 rows in the wider layouts
    }
}

}  // namespace swmd
