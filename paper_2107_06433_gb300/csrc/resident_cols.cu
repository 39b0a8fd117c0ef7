// The column-split solver's host side: buckets, layouts and launches (the kernels
// are in resident_cols.cuh; the instantiations with the buckets of 48 to 96 rows
// are compiled in resident_cols_long.cu).
#include "resident_cols.cuh"

namespace swmd {

int cols_bucket(int len, int vrp) {
    for (int lmax : {8, 16, 24, 32, 48, 64, 96})
        if (cols_fits(lmax, vrp) && lmax >= len) return lmax;
    return 0;
}

int cols_max_len(int vrp) {
    int best = 0;
    for (int lmax : {8, 16, 24, 32, 48, 64, 96})
        if (cols_fits(lmax, vrp)) best = lmax;
    return best;
}

int cols_docs_per_task(int lmax, int vrp) { return 32 / cols_team(lmax, vrp); }

// Layouts of 16 to 128 columns (teams of 4 to 32 lanes).  Narrower queries are
// padded to 16 columns: with teams of one or two lanes a lane would hold the
// tau of up to 32 rows besides the rows themselves, more than its registers.
bool cols_supported(int vrp) { return vrp == 16 || vrp == 32 || vrp == 64 || vrp == 128; }

int cols_vrp(int vr) {
    int v = 16;
    while (v < vr) v *= 2;
    return v;
}

cudaError_t launch_resident_cols(const ColArgs &a, int vrp, int sms, cudaStream_t s, int nq) {
    if (a.long_docs) return launch_resident_cols_long(a, vrp, sms, s, nq);
    switch (vrp) {
        case 16: return run_cols<16, false>(a, sms, nq, s);
        case 32: return run_cols<32, false>(a, sms, nq, s);
        case 64: return run_cols<64, false>(a, sms, nq, s);
        case 128: return run_cols<128, false>(a, sms, nq, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
