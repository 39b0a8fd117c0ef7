// swmd_query_noalloc: the whole query without any allocation in the call.
//
// Some callers cannot allocate device memory when they run a query: a server
// whose memory pool already owns the device's free memory (a cudaMalloc would
// fail or fragment that pool), or a latency-critical request path where
// cudaMalloc / cudaFree would add their implicit device synchronisation.  This
// entry point serves them.  It runs the same kernels as swmd_query_device on the
// resident path, but keeps the query's scratch -- the parameter block, the padded
// query ids and weights, K^T and KM^T -- in one fixed device array defined below,
// instead of the corpus's workspace.  The corpus itself is still created once,
// beforehand, by swmd_create_corpus.
//
// The array is a file-scope __device__ variable: every GPU on which this library
// is loaded holds its kScratchBytes until the process exits.  Host code cannot
// use the array's name as a device address (on the host it names a stand-in), so
// the device address is looked up with cudaGetSymbolAddress, once per device,
// with that device current, the first time the entry point runs on it.
#include <mutex>

#include "corpus.h"

namespace {

// 16 MiB: K^T and KM^T of up to 2M (word, query word) pairs in FP32 (for example
// 100,000 used words x 20 padded query words), or twice as many in BF16/FP16.
constexpr size_t kScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

using swmd::kMaxDevices;
std::mutex g_lookup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

using namespace swmd;

extern "C" int swmd_query_noalloc(swmd_corpus *c, const int32_t *d_ids, const float *d_r,
                                  int32_t v_r, float lambda, int32_t max_iter, double *d_out,
                                  int32_t *d_status, void *stream) {
    if (c && c->opt.tol > 0.f)
        return set_error(SWMD_EINVAL, "swmd_query_noalloc runs the resident path: tol > 0 is not available");
    if (!c) return set_error(SWMD_EINVAL, "swmd_query_noalloc: NULL corpus");
    if (v_r < 1 || v_r > c->opt.max_vr)
        return set_error(SWMD_EINVAL, "swmd_query_noalloc: %d query words; allowed 1..%d", v_r,
                         c->opt.max_vr);
    if (!(lambda > 0.f) || !(lambda < INFINITY) || max_iter < 0)
        return set_error(SWMD_EINVAL, "swmd_query_noalloc: lambda must be finite > 0, max_iter >= 0");
    if (!d_ids || !d_r || (c->Nl > 0 && !d_out))
        return set_error(SWMD_EINVAL, "swmd_query_noalloc: NULL device pointer");
    if (c->device < 0 || c->device >= kMaxDevices)
        return set_error(SWMD_EINVAL, "swmd_query_noalloc: device ordinal %d unsupported", c->device);
    if (c->Nl == 0) return SWMD_OK;

    std::lock_guard<std::mutex> lk(c->mu);
    const int kprec = c->opt.k_precision;
    const Mapping m = choose_mapping(c, v_r, SWMD_PATH_RESIDENT);
    const int vrp_cap = m.vrp;
    const size_t kbytes = (size_t)c->Vu * m.vrp * kprec_bytes(kprec);
    const size_t off_ids = align256(sizeof(QParams));
    const size_t off_r = off_ids + align256(sizeof(int32_t) * vrp_cap);
    const size_t off_status = off_r + align256(sizeof(float) * vrp_cap);
    const size_t off_kt = off_status + 256;
    const size_t off_kmt = off_kt + align256(kbytes);
    const size_t need = off_kmt + align256(kbytes);
    if (need > kScratchBytes)
        return set_error(SWMD_EINVAL,
                         "swmd_query_noalloc: this query needs %zu bytes of scratch (K^T and KM^T "
                         "of %d used words x %d padded query words) but the fixed array holds %zu; "
                         "use swmd_query_device",
                         need, c->Vu, m.vrp, kScratchBytes);

    DeviceGuard guard(c->device);
    void *base;
    {
        std::lock_guard<std::mutex> g(g_lookup_mu);
        if (!g_scratch_ptr[c->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "swmd_query_noalloc: cudaGetSymbolAddress");
            g_scratch_ptr[c->device] = p;
        }
        base = g_scratch_ptr[c->device];
    }
    char *b = static_cast<char *>(base);
    QParams *qp = reinterpret_cast<QParams *>(b);
    int *q_ids = reinterpret_cast<int *>(b + off_ids);
    float *r = reinterpret_cast<float *>(b + off_r);
    int *status = d_status ? d_status : reinterpret_cast<int *>(b + off_status);
    void *KT = b + off_kt;
    void *KMT = b + off_kmt;
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;

    // The prep kernel rewrites the parameter block, the zero-padded ids and
    // weights and clears the status word, so nothing left by an earlier call is
    // read; the cost kernel then writes every entry of K^T and KM^T.
    SWMD_CK(launch_prep(qp, lambda, v_r, c->V, d_ids, d_r, q_ids, r, vrp_cap, d_out, status, st));
    CostArgs ca{};
    ca.E = c->E;
    ca.d4 = c->d4;
    ca.used = c->used;
    ca.Vu = c->Vu;
    ca.q_ids = q_ids;
    ca.qp = qp;
    ca.V = c->V;
    ca.shift = c->opt.column_shift ? 1 : 0;
    {
        int s_ = 0, n_ = 0, cs_ = 0;
        resident_settings(c, v_r, kprec, &s_, &n_, &cs_);
        ca.split = cs_;
    }
    ca.KT = KT;
    ca.KMT = KMT;
    SWMD_CK(launch_cost(ca, m.vrp, kprec, st));
    IterArgs ia{};
    ia.doc_ptr = c->doc_ptr;
    ia.nz = c->nz;
    ia.KT = KT;
    ia.KMT = KMT;
    ia.r = r;
    ia.doc_orig = c->doc_orig;
    ia.qp = qp;
    ia.doc0 = 0;
    ia.N = c->Nl;
    ia.Vu = c->Vu;
    ia.first = 1;
    ResidentArgs ra{ia, max_iter};
    return run_resident(c, ra, m, kprec, v_r, st);
}
